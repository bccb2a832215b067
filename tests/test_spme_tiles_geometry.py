"""The geometric fact the tiled SPME spreading and gather rely on (no GPU): with particles
binned into cells of the real-space grid (cell = min(floor(x nc / L), nc - 1) of the wrapped
position) and bricks of bc cells per side, every particle of the cells [c0, c1) of an axis
has its mesh base floor(x K / L) within [floor(c0 K / nc), floor(c1 K / nc)], up to the
rounding of positions on a cell boundary; a tile that starts at floor(c0 K / nc) - P and is
floor(c1 K / nc) - floor(c0 K / nc) + P + 2 points wide therefore holds the whole footprint
[base - P + 1, base] of every particle of its brick (the kernels' test: P - 1 <= base - start
<= width - 1), the spare point at each end absorbing that rounding, e.g. a wrapped position
of -5e-324 (x / L underflows to -0, so the wrap leaves it below 0 and its base is -1).
Checked on the benchmark workloads' grids, with positions at and next to cell boundaries."""
import math

import numpy as np
import pytest

from paper_1708_01135_gb300 import workloads as W


def _grid(L, rc, n):
    # the library's grid rule: the finest of w = 3, 2, 1 cells per cutoff that gives at
    # least 2w + 1 cells, w = 3 only when cells hold >= 16 particles
    rho = n / L ** 3
    for w in (3, 2, 1):
        nc = min(256, int(math.floor(L * w / rc * (1.0 - 1e-12))))
        if nc < 2 * w + 1:
            continue
        if w == 3 and rho * (L / nc) ** 3 < 16.0:
            continue
        return nc
    return 1


def _check(x, L, nc, K, P, bc, strict):
    w = x - L * np.floor(x / L)
    w[w >= L] = 0.0
    cell = np.minimum((w * (nc / L)).astype(np.int64), nc - 1)
    c0 = (cell // bc) * bc
    c1 = np.minimum(c0 + bc, nc)
    lo = (c0 * K) // nc
    hi = (c1 * K) // nc
    base = np.floor(w * (K / L)).astype(np.int64)
    if strict:
        assert np.all(base >= lo) and np.all(base <= hi)
    local = base - (lo - P)
    width = hi - lo + P + 2
    assert np.all(local >= P - 1) and np.all(local <= width - 1)


@pytest.fixture(scope="module")
def random_32768():
    return W.random_32768()


@pytest.mark.parametrize("K,P", [(100, 8), (96, 6), (80, 10), (70, 12), (45, 4)])
@pytest.mark.parametrize("bc", [1, 2, 3, 4])
def test_every_footprint_lies_inside_its_brick_tile(K, P, bc, random_32768):
    pos, q, L = random_32768
    nc = _grid(L, 4.0, len(q))
    x = pos.reshape(-1)
    # adversarial positions: on and next to every cell boundary and the box edges
    edges = np.arange(nc + 1) * (L / nc)
    extra = np.concatenate([edges, np.nextafter(edges, -np.inf), np.nextafter(edges, np.inf),
                            [L, np.nextafter(L, 0.0), -0.0, -1e-300, 2 * L - 1e-12]])
    _check(x, L, nc, K, P, bc, strict=True)
    _check(extra, L, nc, K, P, bc, strict=False)


def test_rocksalt_grid_and_mesh():
    pos, q, L = W.rocksalt_262144()
    nc = _grid(L, 4.0, len(q))
    for K, P in ((200, 8), (192, 8), (160, 10)):
        for bc in (2, 3):
            _check(pos.reshape(-1), L, nc, K, P, bc, strict=True)
