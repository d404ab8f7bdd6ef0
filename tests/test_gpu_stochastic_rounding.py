"""Stochastic rounding of the half storage formats, end to end on the GPU.

A uniform state at rest collides to post_i = W_i rho at every node (no
stress, no velocity), so one step writes the same exact value v_i into every
node's direction i, and the stored half-format element must be one of the
two grid values around v_i.  Rounded stochastically, the fraction of nodes
that round up must be (v_i - lo) / (hi - lo): the mean over N nodes must
equal v_i within the binomial sampling error.  Rounded to nearest, every
node holds the nearer grid value."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_16000_gb300 import build
    build.build()


# theta = 0.35 and rho = 1.0217 put every v_i strictly between two grid values
# of both formats (at 0.2-0.8 of the spacing).  At theta = 1/3 the weights are
# 4/9, 1/9, 1/36 (ratios of powers of two), and the rounded initial state
# makes every v_i land exactly on the grid.
THETA, RHO = 0.35, 1.0217


def _one_step(storage, layout, sr, side=512, rho=RHO):
    from paper_2501_16000_gb300 import binding as B
    from paper_2501_16000_gb300.engine import Lattice
    with Lattice(side, side, 0.8, THETA, "guided", "oreg", storage, layout) as lat:
        lat.set_option(B.OLB_OPT_STOCHASTIC_ROUNDING, sr)
        lat.init_fields(np.full((side, side), rho), np.zeros((side, side)),
                        np.zeros((side, side)))
        f0 = lat.populations()
        lat.step(1)
        return f0, lat.populations()


# rest weights of the guided equilibrium (Eq. 11 at u = 0): Psi_a(0) Psi_b(0)
_P0, _P1 = 1 - THETA, THETA / 2
W_REST = np.array([_P0 * _P0] + [_P0 * _P1] * 4 + [_P1 * _P1] * 4)


@pytest.mark.parametrize("layout", ["ab", "aa"])
@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_stochastic_rounding_is_unbiased(storage, layout):
    f0, f1 = _one_step(storage, layout, sr=1)
    # the initial (round-to-nearest) state is uniform; its density sets v_i
    assert all(np.unique(f0[i]).size == 1 for i in range(9))
    rho = f0[:, 0, 0].sum()
    n = f1[0].size
    up_fractions = []
    for i in range(9):
        v = W_REST[i] * rho
        vals = np.unique(f1[i])
        assert 1 <= vals.size <= 2, (i, vals)
        lo, hi = vals.min(), vals.max()
        assert lo <= v + 1e-12 and v - 1e-12 <= hi, (i, lo, v, hi)
        if vals.size == 1:
            continue
        p = (v - lo) / (hi - lo)
        sigma = (hi - lo) * np.sqrt(p * (1 - p) / n)
        err = f1[i].mean() - v
        assert abs(err) <= 6 * sigma + 1e-15, (i, err, sigma)
        up_fractions.append(p)
    # the check means something: values fall strictly between grid points
    assert len(up_fractions) == 9 and min(up_fractions) > 0.1 and max(up_fractions) < 0.9


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_round_to_nearest_holds_the_nearer_grid_value(storage):
    f0, f1 = _one_step(storage, "ab", sr=0)
    rho = f0[:, 0, 0].sum()
    for i in range(9):
        vals = np.unique(f1[i])
        assert vals.size == 1, (i, vals)
    _, f1_sr = _one_step(storage, "ab", sr=1)
    biased = 0
    for i in range(9):
        v = W_REST[i] * rho
        lo, hi = f1_sr[i].min(), f1_sr[i].max()
        if hi > lo:
            assert abs(f1[i, 0, 0] - v) <= 0.5 * (hi - lo) + 1e-15
            # nearest rounding keeps a bias the stochastic mean does not have
            biased += abs(f1[i, 0, 0] - v) > 10 * abs(f1_sr[i].mean() - v)
    assert biased >= 7
