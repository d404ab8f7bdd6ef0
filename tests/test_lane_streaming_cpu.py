"""Lane-level streaming of the stream-collide kernels, restated on the CPU.

A warp pass covers 32 consecutive 16-byte vectors of V nodes of a population
plane in row-major order (rows of ceil(nx / V) vectors, back to back); lane
l of pass p holds vector 32 p + l.  The x-shift of streaming moves values one
node between lanes with warp shuffles, and a lane whose neighbour lane holds
another row (it starts a row, ends a row, or sits at the warp's edge) takes
the element from memory instead.  These tests replay the kernels' lane rules
(`fetch_row`/`shift_row` for the pull of the A-B and AA odd steps,
`store_row_shifted_raw` for the push of the AA odd step) on every lane of
every pass and check, for widths that put several rows, row ends and partial
vectors into one pass:

  * every memory access stays inside its row (0 <= x < pitch);
  * the pull gives every node x the value at x - c_x (periodic in x);
  * the push writes every node position x < nx exactly once, with the value
    of the node at x - c_x, and touches only row padding otherwise.
No GPU is used.
"""
import math

import numpy as np
import pytest

WARP = 32


def lane_nodes(v0, lane, nx, ny, v):
    """(y, xb) of a lane; idle lanes past the last vector get xb = nx."""
    vpr = math.ceil(nx / v)
    vec = v0 + lane
    row = vec // vpr
    if row >= ny:
        return ny - 1, nx
    return row, (vec - row * vpr) * v


def passes_of(nx, ny, v):
    return math.ceil(math.ceil(nx / v) * ny / WARP)


def shfl_up(vals, lane):
    return vals[lane - 1] if lane >= 1 else vals[lane]


def shfl_down(vals, lane):
    return vals[lane + 1] if lane + 1 < WARP else vals[lane]


class Row:
    """A row of `pitch` elements whose reads and writes are checked."""

    def __init__(self, data, pitch):
        self.data, self.pitch = data, pitch
        self.writes = np.zeros(pitch, dtype=int)

    def read(self, x, n=1):
        assert 0 <= x and x + n <= self.pitch, (x, n, self.pitch)
        return self.data[x:x + n].copy()

    def write(self, x, vals):
        vals = np.atleast_1d(vals)
        assert 0 <= x and x + len(vals) <= self.pitch, (x, len(vals), self.pitch)
        self.data[x:x + len(vals)] = vals
        self.writes[x:x + len(vals)] += 1


def pull_pass(rows, v0, nx, ny, v, cx, cy):
    """One warp pass of the pull: out[lane][j] is the value node xb + j
    receives from the source plane (rows[y - cy], shifted by cx)."""
    lanes = [lane_nodes(v0, l, nx, ny, v) for l in range(WARP)]
    vecs, halos, wraps = [], [], []
    for sub, (y, xb) in enumerate(lanes):
        row = rows[(y - cy) % ny]
        vec, halo, wrap = np.zeros(v), 0.0, 0.0
        if xb < nx:
            vec = row.read(xb, v)
            if cx == 1 and (sub == 0 or xb == 0):
                halo = row.read(nx - 1 if xb == 0 else xb - 1)[0]
            elif cx == -1:
                if sub == WARP - 1 and xb + v < nx:
                    halo = row.read(xb + v)[0]
                if xb + v >= nx:
                    wrap = row.read(0)[0]
        vecs.append(vec)
        halos.append(halo)
        wraps.append(wrap)
    out = []
    for sub, (y, xb) in enumerate(lanes):
        a = vecs[sub]
        if cx == 0:
            o = a.copy()
        elif cx == 1:
            left = shfl_up([x[v - 1] for x in vecs], sub)
            if xb < nx and (sub == 0 or xb == 0):
                left = halos[sub]
            o = np.concatenate([[left], a[:-1]])
        else:
            right = shfl_down([x[0] for x in vecs], sub)
            if xb < nx and sub == WARP - 1 and xb + v < nx:
                right = halos[sub]
            o = np.concatenate([a[1:], [right]])
            for j in range(v):
                if xb + j == nx - 1:
                    o[j] = wraps[sub]
        out.append((y, xb, o))
    return out


def push_pass(rows, v0, nx, ny, v, cx, cy, values):
    """One warp pass of the AA odd push: node (x, y) sends values[y, x] to
    (x + cx, y + cy), both periodic."""
    lanes = [lane_nodes(v0, l, nx, ny, v) for l in range(WARP)]
    es = []
    for y, xb in lanes:
        e = np.zeros(v)
        if xb < nx:
            for j in range(v):
                if xb + j < nx:
                    e[j] = values[y, xb + j]
        es.append(e)
    for sub, (y, xb) in enumerate(lanes):
        if xb >= nx:
            continue
        row = rows[(y + cy) % ny]
        e = es[sub]
        if cx == 0:
            row.write(xb, e)
        elif cx == 1:
            from_left = shfl_up([x[v - 1] for x in es], sub)
            vec = np.concatenate([[from_left], e[:-1]])
            if not (sub == 0 or xb == 0):
                row.write(xb, vec)
            else:                                   # elements 1 .. v-1 only
                row.write(xb + 1, vec[1:])
            if xb + v > nx - 1:                     # node nx - 1 wraps to x = 0
                row.write(0, e[nx - 1 - xb])
            if sub == WARP - 1 and xb + v < nx:
                row.write(xb + v, e[v - 1])
        else:
            from_right = shfl_down([x[0] for x in es], sub)
            vec = np.concatenate([e[1:], [from_right]])
            has_row_end = xb + v > nx - 1
            last_foreign = sub == WARP - 1 and xb + v < nx
            if not has_row_end and not last_foreign:
                row.write(xb, vec)
            else:                                   # the first L elements only
                n = nx - 1 - xb if has_row_end else v - 1
                if n:
                    row.write(xb, vec[:n])
            if xb == 0:
                row.write(nx - 1, e[0])
            elif sub == 0:
                row.write(xb - 1, e[0])


WIDTHS = (1, 2, 3, 7, 8, 9, 15, 16, 17, 31, 33, 63, 100, 257)


@pytest.mark.parametrize("v", [2, 4, 8])
@pytest.mark.parametrize("cx,cy", [(0, 0), (1, 0), (-1, 0), (1, 1), (-1, -1), (0, 1), (1, -1)])
def test_pull_reads_inside_rows_and_shifts_periodically(v, cx, cy):
    rng = np.random.default_rng(7)
    for nx in WIDTHS:
        for ny in (1, 2, 3, 5):
            pitch = math.ceil(nx / v) * v
            plane = rng.standard_normal((ny, pitch))
            rows = [Row(plane[y].copy(), pitch) for y in range(ny)]
            seen = np.zeros((ny, nx), dtype=int)
            for p in range(passes_of(nx, ny, v)):
                for y, xb, o in pull_pass(rows, WARP * p, nx, ny, v, cx, cy):
                    for j in range(v):
                        x = xb + j
                        if x < nx:
                            want = plane[(y - cy) % ny, (x - cx) % nx]
                            assert o[j] == want, (nx, ny, p, x, y)
                            seen[y, x] += 1
            assert (seen == 1).all(), (nx, ny)


@pytest.mark.parametrize("v", [2, 4, 8])
@pytest.mark.parametrize("cx,cy", [(0, 0), (1, 0), (-1, 0), (1, 1), (-1, -1), (0, -1), (-1, 1)])
def test_push_writes_each_node_position_exactly_once(v, cx, cy):
    rng = np.random.default_rng(11)
    for nx in WIDTHS:
        for ny in (1, 2, 3, 5):
            pitch = math.ceil(nx / v) * v
            values = rng.standard_normal((ny, nx))
            rows = [Row(np.full(pitch, np.nan), pitch) for _ in range(ny)]
            for p in range(passes_of(nx, ny, v)):
                push_pass(rows, WARP * p, nx, ny, v, cx, cy, values)
            for yd, row in enumerate(rows):
                assert (row.writes[:nx] == 1).all(), (nx, ny, yd, row.writes)
                want = values[(yd - cy) % ny, (np.arange(nx) - cx) % nx]
                assert np.array_equal(row.data[:nx], want), (nx, ny, yd)
