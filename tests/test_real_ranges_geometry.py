"""CPU check of the candidate ranges of the real-space cell kernel (k_real_rows): its cell
grid rule, for every target the per-row ranges of sorted particles it visits, and the
staged union of a warp's ranges in each row (parts A, B, C of the row in bin order, each
target's [off0, off1) inside it), restated here in NumPy with the kernel's FP32 arithmetic.
On the benchmark systems (and on boxes with particles placed at cell and box boundaries)
every pair closer than r_c must be among the candidates of both of its particles exactly
once, every index must lie in [0, n), and the union layout must give each target exactly
its own ranges.  (The pair arithmetic itself is checked against the oracle by the GPU
tests.)"""
import math

import numpy as np
import pytest

from paper_1708_01135_gb300 import workloads as W


def cell_grid(L, rc, n):
    """The grid rule of the library (cell_grid in capi.cu)."""
    rho = n / L ** 3
    s_t = max(1.33 * rho ** (-1.0 / 3.0), rc / 5.0)
    nc = min(int(math.floor(L / s_t)), 160)
    while nc >= 3:
        w = int(math.ceil(rc * nc / L * (1.0 - 1e-12)))
        if w >= 1 and 2 * w + 1 <= nc:
            return nc, w
        nc -= 1
    return 1, 0


def sort_cells(pos, L, nc):
    """Binning as the library does it in cell mode: stable sort by cell key, then every cell
    of at most 256 particles ordered by the fixed-point x fraction relative to the cell
    centre (k_rowsort).  Returns the sorted positions, cells, keys, x fractions and the
    cell starts."""
    x = pos - L * np.floor(pos / L)
    x[x >= L] = 0.0
    c = np.minimum((x * (nc / L)).astype(np.int64), nc - 1)
    key = (c[:, 2] * nc + c[:, 1]) * nc + c[:, 0]
    scale = 4294967296.0 / L
    ux = np.rint(x[:, 0] * scale).astype(np.int64) & 0xFFFFFFFF
    uc = np.rint((c[:, 0] + 0.5) * (L / nc) * scale).astype(np.int64) & 0xFFFFFFFF
    xkey = ((ux - uc) & 0xFFFFFFFF).astype(np.uint32).view(np.int32).astype(np.int64)
    counts = np.bincount(key, minlength=nc ** 3)
    xkey = np.where(counts[key] <= 256, xkey, 0)
    order = np.lexsort((np.arange(len(key)), xkey, key))
    start = np.zeros(nc ** 3 + 1, dtype=np.int64)
    np.cumsum(np.bincount(key, minlength=nc ** 3), out=start[1:])
    return x[order], c[order], key[order], ux[order], start


def xwin_allowed(L, rc, nc, w):
    """The host's condition for the x windows (use_xwin, FP32 records)."""
    return w >= 5 and rc * 1.00001 + L / nc < 0.5 * L * (1.0 - 1e-6)


def first_within(d, lo, hi, R):
    """First g in [lo, hi) with d[g] <= R (binary search, as the kernel)."""
    while lo < hi:
        mid = (lo + hi) >> 1
        if d[mid] <= R:
            hi = mid
        else:
            lo = mid + 1
    return lo


def window(idx, ux, u, R):
    """The kernel's x-window cut of a target's candidates idx (global indices in union
    order): two binary searches on the int32 x displacements u - ux[j]."""
    if R is None or idx.size == 0:
        return idx
    d = ((u - ux[idx]) & 0xFFFFFFFF).astype(np.uint32).view(np.int32).astype(np.int64)
    lo = first_within(d, 0, idx.size, R)
    hi = first_within(d, lo, idx.size, -R - 1)
    # the searches rely on the x order: they must keep exactly the candidates inside
    keep = (d >= -R) & (d <= R)
    assert np.array_equal(idx[lo:hi], idx[keep]), "candidates not in x order"
    return idx[lo:hi]


def target_row(xs, c, L, rc, nc, w, i, dy, dz, xwin):
    """Unwrapped bins [a0, a1] of target i in row (dy, dz) and its x-window half-width R in
    fixed-point units (None without windows), or None out of reach (the kernel's FP32
    arithmetic)."""
    f32 = np.float32
    side = L / nc
    sidef, inv_side = f32(side), f32(1.0 / side)
    rc2m = f32(f32(rc * rc) * (f32(1.0) + f32(1e-5)))
    cx, cy, cz = c[i]
    xl = f32(xs[i, 0] - cx * side)
    yl = f32(xs[i, 1] - cy * side)
    zl = f32(xs[i, 2] - cz * side)
    gy = f32(dy * sidef - yl) if dy > 0 else (f32(yl - (dy + 1) * sidef) if dy < 0 else f32(0))
    gz = f32(dz * sidef - zl) if dz > 0 else (f32(zl - (dz + 1) * sidef) if dz < 0 else f32(0))
    d2 = f32(gy * gy + gz * gz)
    if not d2 < rc2m:
        return None
    reach = f32(np.sqrt(f32(rc2m - d2)))
    b0 = int(np.floor(f32((xl - reach) * inv_side)))
    b1 = int(np.floor(f32((xl + reach) * inv_side)))
    a0, a1 = cx + max(b0, -w), cx + min(b1, w)
    R = int(math.ceil(f32(reach * f32(4294967296.0 / L)))) + 1 if xwin else None
    return a0, a1, R


def union_check(xs, c, ux, start, L, rc, nc, w, group, xwin):
    """The staged union of a warp's targets in every row, as the kernel lays it out; returns
    per target the global indices it reads through the union."""
    f32 = np.float32
    sidef = f32(L / nc)
    rc2m = f32(f32(rc * rc) * (f32(1.0) + f32(1e-5)))
    got = {int(i): [] for i in group}
    for dz in range(-w, w + 1):
        mz = f32((abs(dz) - 1) * sidef) if dz else f32(0)
        for dy in range(-w, w + 1):
            my = f32((abs(dy) - 1) * sidef) if dy else f32(0)
            if my * my + mz * mz >= rc2m:
                continue
            rows = {int(i): target_row(xs, c, L, rc, nc, w, i, dy, dz, xwin) for i in group}
            live = [b for b in rows.values() if b]
            if not live:
                continue
            A0, A1 = min(b[0] for b in live), max(b[1] for b in live)
            # all targets of a warp may sit in different rows: the union uses each target's
            # own row; the kernel's warp shares one row only because every lane computes
            # the same (dy, dz) relative to its own cell, so check per target row
            for i in group:
                i = int(i)
                if not rows[i]:
                    continue
                a0, a1, R = rows[i]
                ci = c[i]
                base = (((ci[2] + dz) % nc) * nc + (ci[1] + dy) % nc) * nc
                cs = start[base:base + nc + 1]
                sA = lenA = lenC = 0
                sC = cs[0]
                if A0 < 0:
                    sA = cs[A0 + nc]; lenA = cs[nc] - sA
                b0, b1 = max(A0, 0), min(A1, nc - 1)
                sB = cs[b0]; lenB = cs[b1 + 1] - sB
                if A1 >= nc:
                    lenC = cs[A1 - nc + 1] - sC
                def off(b):
                    if b < 0:
                        return cs[b + nc] - sA
                    if b < nc:
                        return lenA + cs[b] - sB
                    return lenA + lenB + cs[b - nc] - sC
                o0, o1 = off(a0), off(a1 + 1)
                assert 0 <= o0 <= o1 <= lenA + lenB + lenC
                idx = []
                for q in range(o0, o1):
                    if q < lenA:
                        idx.append(sA + q)
                    elif q < lenA + lenB:
                        idx.append(sB + q - lenA)
                    else:
                        idx.append(sC + q - lenA - lenB)
                got[i].extend(window(np.array(idx, dtype=np.int64), ux, int(ux[i]), R).tolist())
    return got


def candidate_ranges(xs, c, ux, start, L, rc, nc, w, targets, xwin):
    """For each target: the candidate indices of every row, as the kernel computes them
    (FP32 reach and bin arithmetic, wrapped rows, clamped bins, x windows)."""
    f32 = np.float32
    sidef = f32(L / nc)
    rc2m = f32(f32(rc * rc) * (f32(1.0) + f32(1e-5)))
    out = []
    for i in targets:
        cx, cy, cz = c[i]
        rr = []
        for dz in range(-w, w + 1):
            mz = f32((abs(dz) - 1) * sidef) if dz else f32(0)
            for dy in range(-w, w + 1):
                my = f32((abs(dy) - 1) * sidef) if dy else f32(0)
                if my * my + mz * mz >= rc2m:
                    continue
                t = target_row(xs, c, L, rc, nc, w, i, dy, dz, xwin)
                if t is None:
                    continue
                a0, a1, R = t
                base = (((cz + dz) % nc) * nc + (cy + dy) % nc) * nc
                if a0 < 0:
                    parts = [(start[base + a0 + nc], start[base + nc]), (start[base], start[base + a1 + 1])]
                elif a1 >= nc:
                    parts = [(start[base + a0], start[base + nc]), (start[base], start[base + a1 - nc + 1])]
                else:
                    parts = [(start[base + a0], start[base + a1 + 1])]
                idx = np.concatenate([np.arange(a, b) for a, b in parts])
                rr.append(window(idx, ux, int(ux[i]), R))
        out.append(rr)
    return out


def check(pos, L, rc, targets=None, xwin=None):
    n = len(pos)
    nc, w = cell_grid(L, rc, n)
    assert w >= 1
    if xwin is None:
        xwin = xwin_allowed(L, rc, nc, w)
    xs, c, key, ux, start = sort_cells(pos, L, nc)
    if targets is None:
        targets = np.arange(n)
    ranges = candidate_ranges(xs, c, ux, start, L, rc, nc, w, targets, xwin)
    ncand = 0
    for i, rr in zip(targets, ranges):
        idx = np.concatenate(rr) if rr else np.zeros(0, int)
        assert idx.size == 0 or (idx.min() >= 0 and idx.max() < n)
        assert np.unique(idx).size == idx.size, "a candidate visited twice"
        d = xs - xs[i]
        d -= L * np.round(d / L)
        r2 = (d * d).sum(axis=1)
        partners = np.nonzero((r2 < rc * rc) & (np.arange(n) != i))[0]
        missing = np.setdiff1d(partners, idx)
        assert missing.size == 0, f"target {i}: partners {missing[:5]} not among the candidates"
        ncand += idx.size
    # the staged union of a warp's tile (up to 8 consecutive sorted targets of one row of
    # cells, as k_row_tiles cuts them) gives each target exactly its ranges
    tg = 8
    row_of = key // nc
    for g0 in list(targets[:: max(1, len(targets) // 40)])[:40]:
        r = row_of[g0]
        first = start[r * nc] + tg * ((g0 - start[r * nc]) // tg)
        group = np.arange(first, min(first + tg, start[(r + 1) * nc]))
        assert np.all(row_of[group] == r)
        got = union_check(xs, c, ux, start, L, rc, nc, w, group, xwin)
        own = candidate_ranges(xs, c, ux, start, L, rc, nc, w, group, xwin)
        for i, rr in zip(group, own):
            idx = np.concatenate(rr) if rr else np.zeros(0, int)
            assert sorted(got[int(i)]) == sorted(idx.tolist()), f"union layout of target {i}"
    return nc, w, ncand / len(targets)


def test_grid_rule_matches_the_library():
    from paper_1708_01135_gb300 import Ewald, ewald as E
    try:
        E.lib()
    except RuntimeError as e:
        pytest.skip(str(e))
    for n, L, rc in ((32768, 32.0, 4.0), (262144, 64.0, 6.8), (2097152, 128.0, 9.6),
                     (512, 8.0, 2.6), (4002, 15.87, 4.0)):
        # the plan's grid is chosen when its workspace is sized for n particles; plan_info
        # reports the grid of the density-free set-up until then, so compare the rule only
        nc, w = cell_grid(L, rc, n)
        assert 2 * w + 1 <= nc and w * (L / nc) >= rc * (1 - 1e-12)


@pytest.mark.parametrize("name,rc", [("random_32768", 4.0), ("rocksalt_512", 2.6)])
def test_every_partner_is_a_candidate_once(name, rc):
    pos, q, L = getattr(W, name)()
    rng = np.random.default_rng(3)
    targets = None if len(q) <= 4096 else np.sort(rng.choice(len(q), 3000, replace=False))
    nc, w, per_target = check(pos, L, rc, targets)
    assert w >= 2
    # the x windows (valid wherever reach + side < L/2; the library takes them from w >= 5)
    # drop candidates: fewer per target than with whole cells
    sub = targets[:300] if targets is not None else None
    _, _, whole = check(pos, L, rc, sub, xwin=False)
    _, _, cut = check(pos, L, rc, sub, xwin=True)
    assert cut < whole


def test_boundary_positions():
    """Particles on cell faces, at 0 and just below L, and a cutoff that is an exact
    multiple of the cell side."""
    rng = np.random.default_rng(5)
    L, n = 12.0, 1500
    pos = rng.uniform(0, L, size=(n, 3))
    side = L / cell_grid(L, 2.4, n)[0]
    pos[:200] = np.round(pos[:200] / side) * side          # on cell faces
    pos[200:220, 0] = 0.0
    pos[220:240, 1] = np.nextafter(L, 0)
    pos[240:260] = -1e-300
    for rc in (2.4, 3.0, 3.9):
        check(pos, L, rc)
        check(pos, L, rc, xwin=True)


def test_large_system_sample():
    pos, q, L = W.rocksalt_262144()
    rng = np.random.default_rng(11)
    nc, w, _ = check(pos, L, 6.8, np.sort(rng.choice(len(q), 400, replace=False)))
    assert xwin_allowed(L, 6.8, nc, w)          # the library's windows are on here
