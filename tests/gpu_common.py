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
