"""Seeded synthetic inputs: ionic lattices, random neutral ionic systems, request streams.

This module holds no Ewald arithmetic.  It only produces positions, charges and box
lengths, and it is the one module that both the oracle-side tests and the CUDA path
draw their inputs from.

The workloads follow the paper's benchmark system (Section 4.1): an NaCl-like ionic
system at a number density of one ion per (2.5 Angstrom)^3.  With 2.5 Angstrom as
the unit of length that density is 1.0, which is what every generator here uses by
default.  Units are Gaussian with the Coulomb constant equal to 1 (Section 2.1 and
the Poisson equation, Eq. 2).

All generators are deterministic functions of their arguments and ``seed``
(numpy PCG64).  Positions are float64 arrays of shape [n, 3]; charges are float64
of shape [n]; every system is exactly neutral.
"""
from __future__ import annotations

import ctypes
import hashlib
import math
import os
import subprocess
from dataclasses import dataclass

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def rocksalt(m: int, a: float = 1.0, jitter: float = 0.0, seed: int = 0):
    """Rock-salt lattice with m^3 ions on a simple cubic grid of spacing ``a``.

    Site (i, j, k) sits at a*(i, j, k) with charge (-1)^(i+j+k); the box is cubic with
    side L = m*a.  ``m`` must be even so that the periodic lattice is neutral and
    alternating across the boundary.  With ``jitter`` > 0 each coordinate gets an
    independent N(0, jitter^2) displacement (positions are not wrapped).

    Returns (pos [m^3, 3], q [m^3], L).
    """
    if m < 2 or m % 2:
        raise ValueError("rock-salt needs an even number of sites per side")
    idx = np.arange(m)
    i, j, k = np.meshgrid(idx, idx, idx, indexing="ij")
    sites = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1)
    pos = sites.astype(np.float64) * a
    q = np.where((sites.sum(axis=1) % 2) == 0, 1.0, -1.0)
    if jitter > 0:
        pos = pos + _rng(seed).normal(0.0, jitter, size=pos.shape)
    return np.ascontiguousarray(pos), q.astype(np.float64), float(m * a)


def cscl(m: int, c: float = 1.0, jitter: float = 0.0, seed: int = 0):
    """Caesium-chloride lattice: cations (+1) on a simple cubic lattice of edge ``c``
    and anions (-1) at the body centres; m^3 cells, N = 2 m^3 ions, L = m*c.

    Returns (pos [2 m^3, 3], q [2 m^3], L).  The nearest-neighbour distance is c*sqrt(3)/2.
    """
    idx = np.arange(m)
    i, j, k = np.meshgrid(idx, idx, idx, indexing="ij")
    cat = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1).astype(np.float64) * c
    ani = cat + 0.5 * c
    pos = np.concatenate([cat, ani], axis=0)
    q = np.concatenate([np.ones(len(cat)), -np.ones(len(ani))])
    if jitter > 0:
        pos = pos + _rng(seed).normal(0.0, jitter, size=pos.shape)
    return np.ascontiguousarray(pos), q, float(m * c)


def _neutral_charges(n: int, mix, rng: np.random.Generator) -> np.ndarray:
    """Exactly neutral charge vector: ``mix`` is a list of (charge, fraction) for the
    positive species; each gets an equal-count negative partner.  Counts are rounded
    down and the remainder goes to the first species, so that sum(q) == 0 exactly."""
    if n % 2:
        raise ValueError("a neutral system of +-q pairs needs an even particle count")
    half = n // 2
    counts = [int(math.floor(f * n)) for _, f in mix]
    # fractions are per sign: e.g. [(1, 0.4), (2, 0.1)] -> 40 % +1, 40 % -1, 10 % +2, 10 % -2
    counts[0] = half - sum(counts[1:])
    q = []
    for (val, _), c in zip(mix, counts):
        q.append(np.full(c, float(val)))
        q.append(np.full(c, -float(val)))
    q = np.concatenate(q)
    if q.size != n or q.sum() != 0.0:
        raise AssertionError("charge assignment is not neutral")
    return q[rng.permutation(n)]


_RSA_SRC = os.path.join(os.path.dirname(os.path.abspath(__file__)), "rsa.c")
_RSA_LIB = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "librsa.so")
_rsa = None


def build_rsa(force: bool = False) -> str:
    """Compile the sequential-insertion helper (rsa.c) with gcc into _build/librsa.so."""
    if force or not os.path.exists(_RSA_LIB) or os.path.getmtime(_RSA_LIB) < os.path.getmtime(_RSA_SRC):
        os.makedirs(os.path.dirname(_RSA_LIB), exist_ok=True)
        tmp = f"{_RSA_LIB}.tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11",
                               "-o", tmp, _RSA_SRC, "-lm"])
        os.replace(tmp, _RSA_LIB)
    return _RSA_LIB


def _rsa_lib():
    global _rsa
    if _rsa is None:
        lib = ctypes.CDLL(build_rsa())
        p = ctypes.c_void_p
        lib.rsa_insert.restype = ctypes.c_int64
        lib.rsa_insert.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int64,
                                   ctypes.c_int64, p, p, p, p, ctypes.c_int64, p]
        _rsa = lib
    return _rsa


def random_neutral(n: int, L: float | None = None, density: float = 1.0, hard_core: float = 0.8,
                   mix=((1.0, 0.5),), seed: int = 0):
    """Random neutral ionic system: n points uniform in a cubic box by random sequential
    insertion: candidates uniform in the box, in the order the seeded generator draws them,
    each accepted unless it lies closer than ``hard_core`` to an accepted point under
    periodic images.  Charges follow ``mix`` (see :func:`_neutral_charges`); the default is
    half +1 and half -1.  The box side defaults to (n / density)^(1/3).

    The charges are drawn first, then the candidate stream (uniform doubles of the same
    generator, x, y, z per candidate); the accept/reject pass over the stream is the C helper
    rsa.c (a cell grid of side >= hard_core, so a candidate meets only the points of 27
    cells).  Returns (pos [n, 3], q [n], L).
    """
    rng = _rng(seed)
    if L is None:
        L = (n / density) ** (1.0 / 3.0)
        if abs(L - round(L)) < 1e-9 * L:
            L = float(round(L))
    L = float(L)
    q = _neutral_charges(n, list(mix), rng)
    if hard_core <= 0:
        return rng.uniform(0.0, L, size=(n, 3)), q, L
    # cells at least a little wider than the hard core, so that rounding of the cell index
    # can never hide a point closer than the hard core two cells away
    g = int(math.floor(L / (hard_core * (1.0 + 1e-9))))
    lib = _rsa_lib()
    pts = np.zeros((n, 3), dtype=np.float64)
    head = np.full(max(1, g) ** 3 if g >= 3 else 1, -1, dtype=np.int64)
    nxt = np.full(max(1, n), -1, dtype=np.int64)
    count, drawn = 0, 0
    used = ctypes.c_int64(0)
    while count < n:
        chunk = max(1 << 16, 2 * (n - count))
        cand = np.ascontiguousarray(rng.uniform(0.0, L, size=(chunk, 3)))
        drawn += chunk
        count = lib.rsa_insert(L, float(hard_core), g, n, count, pts.ctypes.data,
                               head.ctypes.data, nxt.ctypes.data, cand.ctypes.data, chunk,
                               ctypes.byref(used))
        if count < n and drawn > 1000 * n + (1 << 20):
            raise RuntimeError("random sequential insertion stalled (hard core too large)")
    return np.ascontiguousarray(pts), q, L


# ---- the named workloads --------------------------------------------------------------

def rocksalt_512(seed: int = 1235):
    """Rock-salt 8x8x8 = 512 ions, a = 1, L = 8, jitter N(0, 0.05^2)."""
    return rocksalt(8, 1.0, 0.05, seed)


def random_32768(seed: int = 1236):
    """N = 32,768 (16,384 of each sign) uniform at density 1.0 (L = 32) with a 0.8 hard core."""
    return random_neutral(32768, density=1.0, hard_core=0.8, seed=seed)


def rocksalt_262144(seed: int = 1237):
    """Rock-salt 64x64x64 = 262,144 ions, a = 1, L = 64, jitter N(0, 0.05^2)."""
    return rocksalt(64, 1.0, 0.05, seed)


def random_2097152(seed: int = 1239):
    """N = 2,097,152 with charges +-1 (40 % each) and +-2 (10 % each), uniform at
    density 1.0 (L = 128) with a 0.8 hard core.  The result is also kept in the on-disk
    cache (see :func:`_cached`)."""
    return _cached(f"random_2097152_s{seed}",
                   lambda: random_neutral(2097152, density=1.0, hard_core=0.8,
                                          mix=((1.0, 0.4), (2.0, 0.1)), seed=seed))


def _cache_dir() -> str:
    d = os.environ.get("EWALD_WORKLOAD_CACHE")
    if d:
        return d
    return os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                        "_build", "workloads")


def _cached(key: str, make):
    """Return make() = (pos, q, L), stored once as .npz under the cache directory
    (EWALD_WORKLOAD_CACHE, default _build/workloads at the repository root).  The file
    name carries a digest of this module's source, so an edited generator never reads an
    older result."""
    with open(os.path.abspath(__file__), "rb") as f:
        tag = hashlib.sha256(f.read()).hexdigest()[:12]
    path = os.path.join(_cache_dir(), f"{key}-{tag}.npz")
    try:
        with np.load(path) as z:
            return np.ascontiguousarray(z["pos"]), np.ascontiguousarray(z["q"]), float(z["L"])
    except (OSError, KeyError, ValueError):
        pass
    pos, q, L = make()
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = f"{path}.tmp{os.getpid()}.npz"
        np.savez(tmp, pos=pos, q=q, L=np.float64(L))
        os.replace(tmp, path)
    except OSError:
        pass
    return pos, q, L


@dataclass
class Request:
    """One system of a request stream: arrival time (s), kind, positions, charges, box."""
    t_arrive: float
    kind: str
    pos: np.ndarray
    q: np.ndarray
    L: float


def request_sizes(count: int = 256, n_min: int = 256, n_max: int = 65536, seed: int = 1238):
    """Sizes and kinds of a serving stream: N log-uniform in [n_min, n_max], alternating
    rock-salt / random neutral, density U[0.8, 1.2].  Rock-salt sizes are rounded to the
    nearest m^3 with m even; random sizes to the nearest even N."""
    rng = _rng(seed)
    out = []
    for r in range(count):
        n = math.exp(rng.uniform(math.log(n_min), math.log(n_max)))
        rho = rng.uniform(0.8, 1.2)
        if r % 2 == 0:
            m = max(2, 2 * int(round(n ** (1.0 / 3.0) / 2.0)))
            out.append(("rocksalt", m ** 3, rho, m))
        else:
            nn = max(2, 2 * int(round(n / 2.0)))
            out.append(("random", nn, rho, None))
    return out


def request_stream(count: int = 256, rate_hz: float = 100.0, n_min: int = 256, n_max: int = 65536,
                   seed: int = 1238):
    """A serving stream of ``count`` independent systems with Poisson arrivals at
    ``rate_hz``.  Each system has its own box L = (N/rho)^(1/3)."""
    rng = _rng(seed + 7)
    t = 0.0
    reqs = []
    for r, (kind, n, rho, m) in enumerate(request_sizes(count, n_min, n_max, seed)):
        t += rng.exponential(1.0 / rate_hz)
        L = (n / rho) ** (1.0 / 3.0)
        if kind == "rocksalt":
            pos, q, L = rocksalt(m, a=L / m, jitter=0.05 * L / m, seed=seed * 1000 + r)
        else:
            pos, q, L = random_neutral(n, L=L, hard_core=0.8 * (1.0 / rho) ** (1.0 / 3.0),
                                       seed=seed * 1000 + r)
        reqs.append(Request(t, kind, pos, q, L))
    return reqs
