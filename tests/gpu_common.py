"""Helpers for the GPU tests (device tensors, error norms, oracle caching)."""
import functools
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def dev(a, dtype=None):
    return torch.tensor(np.ascontiguousarray(a), device="cuda", dtype=dtype or torch.float64)


def rel_rms(a, b):
    a = np.asarray(a); b = np.asarray(b)
    return math.sqrt(float(((a - b) ** 2).sum()) / float((b ** 2).sum()))


def rel(a, b):
    return abs(a - b) / abs(b)


def rel_total(e_total, ref):
    """Error of a total energy relative to the size of its parts, |E_real| + |E_recip| +
    |E_self| of the oracle: at large beta the total is a small difference of the reciprocal
    and self energies, and a path's error is set by the parts it sums."""
    return abs(e_total - ref["E_total"]) / (abs(ref["E_real"]) + abs(ref["E_recip"]) +
                                            abs(ref["E_self"]))


# Per-particle factor of assert_close: no single particle may be off by more than this many
# times the tolerance, measured in units of the RMS size of the reference values.
LOCAL_FACTOR = 20.0


def local_max(a, b):
    """Largest per-particle error relative to the RMS size of the reference: max_i |a_i - b_i|
    / sqrt(mean_i |b_i|^2), where a_i is a row (a force vector) for 2-D arrays and an element
    for 1-D ones."""
    a = np.asarray(a, dtype=np.float64); b = np.asarray(b, dtype=np.float64)
    if a.ndim == 1:
        a = a[:, None]; b = b[:, None]
    d = np.sqrt(((a - b) ** 2).sum(axis=1))
    scale = math.sqrt(float((b ** 2).sum(axis=1).mean()))
    return float(d.max()) / scale


def assert_close(a, b, tol):
    """Global and local parity: the relative RMS error over all particles is below tol, and
    no particle's error exceeds LOCAL_FACTOR * tol times the RMS size of the reference (a
    wrong result on a few particles of a large system, e.g. at a tile edge or in a ragged
    tail, barely moves the RMS but fails the local bound)."""
    g = rel_rms(a, b)
    loc = local_max(a, b)
    assert g < tol, f"relative RMS error {g:.3e} >= {tol:.1e}"
    assert loc <= LOCAL_FACTOR * tol, (
        f"largest per-particle error {loc:.3e} of the RMS size > {LOCAL_FACTOR:g} x {tol:.1e}")


@functools.lru_cache(maxsize=None)
def oracle_cached(name, beta, rc, kmax, sub=None):
    import oracle
    from paper_1708_01135_gb300 import workloads as W
    pos, q, L = getattr(W, name)()
    sub_idx = None if sub is None else np.array(sub, dtype=np.int64)
    return oracle.ewald(pos, q, L, beta, rc, kmax, sub=sub_idx)


def mode_scale(q, m, S):
    """Error scale of every structure factor: sqrt(sum q^2) (a random-phase sum) plus |S(k)|
    and |S(k')| of the mode k' = (-m_x, m_y, m_z) that shares its four real partial sums
    (S(+m_x) and S(-m_x) come from the same Re/Im products, which can both be large where
    the two modes differ greatly)."""
    idx = {tuple(v): i for i, v in enumerate(np.asarray(m).tolist())}
    partner = np.array([idx.get((-a, b, c), i) for i, (a, b, c) in enumerate(np.asarray(m).tolist())])
    return np.sqrt((np.asarray(q) ** 2).sum()) + np.abs(S) + np.abs(S[partner])
