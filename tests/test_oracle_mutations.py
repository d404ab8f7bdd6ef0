"""The pins are strong enough: every plausible slip planted in a copy of the
oracle (wrong sign, dropped term, wrong index, transposed operand, the
equilibrium exactly as printed) fails at least one pin.

Mutations are applied to a temporary copy of ``oracle/oreg_oracle.c`` on the
CPU; the committed oracle is never modified."""
import os

import pytest

from oracle import oracle as O

from . import pins

SRC = os.path.join(os.path.dirname(O.__file__), "oreg_oracle.c")

# (name, exact text in the oracle, replacement[, text, replacement ...])
MUTATIONS = [
    ("velocity table entry", "{-1, 1}, {-1, -1}", "{-1, 1}, {1, 1}"),
    ("guided sign of c.u", "c2 - 1.0 + c * u[a]", "c2 - 1.0 - c * u[a]"),
    ("guided normalisation", "/ pow(2.0, c2)", "/ 2.0"),
    ("guided theta term", "u[a] * u[a] + theta)", "u[a] * u[a] + 1.0 / 3.0)"),
    ("polynomial as printed", " - uu / (2.0 * t0));", ");"),
    ("polynomial weight", "(1.0 - t0) : (t0 / 2.0)", "(1.0 - t0) : (t0 / 4.0)"),
    ("velocity not divided by rho", "*ux = jx / r;", "*ux = jx;"),
    ("predictor sign", "fneq[k] = f[k] - feq[k]", "fneq[k] = feq[k] - f[k]"),
    # Either delta term alone is harmless (the other factor is trace-free);
    # dropping both changes the scheme.
    ("both delta terms dropped", "(ca * cb - ck2 * delta / (double)ORA_D)", "(ca * cb)",
     "(C[a] * C[b] - C2 * delta / (double)ORA_D)", "(C[a] * C[b])"),
    ("inner index a for b", "ca = (double)ORA_C[k][a], cb = (double)ORA_C[k][b]",
     "ca = (double)ORA_C[k][a], cb = (double)ORA_C[k][a]"),
    ("absolute instead of peculiar velocity", "C[a] = (double)ORA_C[i][a] - u[a]",
     "C[a] = (double)ORA_C[i][a]"),
    ("peculiar velocity takes u_x on both axes", "C[a] = (double)ORA_C[i][a] - u[a]",
     "C[a] = (double)ORA_C[i][a] - u[0]"),
    ("prefactor theta not squared", "(2.0 * rho * theta_eff * theta_eff)",
     "(2.0 * rho * theta_eff)"),
    ("prefactor rho dropped", "(2.0 * rho * theta_eff * theta_eff)",
     "(2.0 * theta_eff * theta_eff)"),
    ("OReg relaxation factor", "feq[i] + (1.0 - 1.0 / p->tau) * foreg[i]",
     "feq[i] + (1.0 - p->tau) * foreg[i]"),
    ("OReg term replaced by equilibrium", "feq[i] + (1.0 - 1.0 / p->tau) * foreg[i]",
     "feq[i] + (1.0 - 1.0 / p->tau) * feq[i]"),
    ("BGK relaxation", "f[i] - (1.0 / p->tau) * (f[i] - feq[i])",
     "f[i] - p->tau * (f[i] - feq[i])"),
    ("stream pulls instead of pushes (x)",
     "const int64_t xd = ora_wrap(x + ORA_C[i][0], nx);\n                dst[i * N + yd * nx + xd] = post[i];",
     "const int64_t xd = ora_wrap(x - ORA_C[i][0], nx);\n                dst[i * N + yd * nx + xd] = post[i];"),
    ("stream pulls instead of pushes (y)",
     "const int64_t yd = ora_wrap(y + ORA_C[i][1], ny);\n                const int64_t xd = ora_wrap(x + ORA_C[i][0], nx);\n                dst",
     "const int64_t yd = ora_wrap(y - ORA_C[i][1], ny);\n                const int64_t xd = ora_wrap(x + ORA_C[i][0], nx);\n                dst"),
    ("stream transposed", "dst[i * N + yd * nx + xd] = post[i];",
     "dst[i * N + (xd * ny + yd)] = post[i];"),
    ("first-order sign", "f1[i] = -tau * feq[i] * contraction", "f1[i] = tau * feq[i] * contraction"),
    ("first-order tau - 1/2 for tau", "f1[i] = -tau * feq[i] * contraction",
     "f1[i] = -(tau - 0.5) * feq[i] * contraction"),
    ("first-order absolute velocity", "Cp[a] = (double)ORA_C[i][a] - u[a]",
     "Cp[a] = (double)ORA_C[i][a]"),
    ("first-order theta squared", "grad[b * ORA_D + a]) / (2.0 * theta_eff)",
     "grad[b * ORA_D + a]) / (2.0 * theta_eff * theta_eff)"),
    ("first-order delta term dropped", "(Cp[a] * Cp[b] - Cp2 * delta / (double)ORA_D)",
     "(Cp[a] * Cp[b])"),
    ("first-order start without f1", "f[i * N + n] = feq[i] + f1[i];", "f[i * N + n] = feq[i];"),
    ("first-order gradient components swapped", "g[ab] = grad[ab * N + n]",
     "g[ab] = grad[(3 - ab) * N + n]"),
    ("bounce-back keeps the direction", "ORA_C[k][1] == -ORA_C[i][1]) post[i] = f[k];",
     "ORA_C[k][1] == -ORA_C[i][1]) post[i] = f[i];"),
    ("specular instead of bounce-back", "ORA_C[k][1] == -ORA_C[i][1]) post[i]",
     "ORA_C[k][1] == ORA_C[i][1]) post[i]"),
    ("wall column off by one", "if (p->walls && (x == 0 || x == nx - 1))",
     "if (p->walls && (x == 1 || x == nx - 1))"),
    ("walls ignored", "if (p->walls && (x == 0 || x == nx - 1))", "if (0)"),
    ("local theta keeps rho u^2", "return (c2f - rho * (ux * ux + uy * uy)) / ((double)ORA_D * rho);",
     "return c2f / ((double)ORA_D * rho);"),
    ("local theta not divided by D", "return (c2f - rho * (ux * ux + uy * uy)) / ((double)ORA_D * rho);",
     "return (c2f - rho * (ux * ux + uy * uy)) / rho;"),
    ("local theta missing in Eq. 6", "ora_foreg(f, feq, rho, ux, uy, ora_theta_eff(p->eq, theta), foreg);",
     "ora_foreg(f, feq, rho, ux, uy, ora_theta_eff(p->eq, p->theta), foreg);"),
    ("local theta ignored", "const double theta = p->theta_local ? ora_node_theta(f, rho, ux, uy) : p->theta;",
     "const double theta = p->theta;"),
    ("streaming-only path wraps the wrong axis", "ora_wrap(x + ORA_C[i][0], nx);\n                dst[i * N + yd * nx + xd] = post[i * N",
     "ora_wrap(x + ORA_C[i][1], nx);\n                dst[i * N + yd * nx + xd] = post[i * N"),
]


@pytest.mark.parametrize("mutation", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_mutation_is_caught(tmp_path, mutation):
    name, edits = mutation[0], mutation[1:]
    src = open(SRC).read()
    for old, new in zip(edits[::2], edits[1::2]):
        assert src.count(old) == 1, f"mutation anchor not unique/present: {old!r}"
        src = src.replace(old, new)
    mutated = tmp_path / "oreg_oracle_mutant.c"
    mutated.write_text(src)
    lib = O.build(force=True, src=str(mutated), out=str(tmp_path / "libmutant.so"))
    O.use(lib)
    caught = None
    try:
        for check in pins.FAST_CHECKS + pins.LATTICE_CHECKS:
            try:
                check()
            except AssertionError as e:
                caught = f"{check.__name__}: {str(e)[:120]}"
                break
    finally:
        O.reset()
    assert caught is not None, f"mutation '{name}' passed every pin"
