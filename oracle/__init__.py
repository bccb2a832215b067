"""Plain FP64 CPU Ewald oracle (Python side of ``oracle/ewald_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` use it.  The product library never imports it, and it imports nothing from
the product package.  It shares no code with the CUDA path.

The C source states the formulas and the paper passages they follow (Sections 3.1-3.2,
Eqs. 2-4, Listing 1, Algorithms 1-2).  This module only marshals numpy arrays, builds the
shared library with gcc on first use, and adds up the components.

Parity status: every function here is pinned by tests in ``tests/test_oracle.py``
(Madelung constants, beta invariance, sum of forces, finite differences, brute-force
image sums, the exact S(k) of an unjittered rock-salt lattice, lattice-point counts).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ewald_oracle.c")
_LIB = os.path.join(_HERE, "libewald_oracle.so")
_lock = threading.Lock()
_lib = None

_d = ctypes.c_double
_i64 = ctypes.c_int64
_p = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP, no fast-math) into oracle/libewald_oracle.so."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            L.ewo_kset_half.restype = _i64
            L.ewo_kset_half.argtypes = [ctypes.c_int, _p, _i64]
            L.ewo_real.restype = None
            L.ewo_real.argtypes = [_i64, _p, _p, _d, _d, _d, _i64, _p, _p, _p, _p, ctypes.c_int]
            L.ewo_real_cells.restype = ctypes.c_int
            L.ewo_real_cells.argtypes = [_i64, _p, _p, _d, _d, _d, _i64, _p, _p, _p, _p]
            L.ewo_structure_factor.restype = None
            L.ewo_structure_factor.argtypes = [_i64, _p, _p, _d, _i64, _p, _p]
            L.ewo_recip_energy.restype = _d
            L.ewo_recip_energy.argtypes = [_i64, _p, _p, _d, _d, _p]
            L.ewo_recip_forces.restype = None
            L.ewo_recip_forces.argtypes = [_i64, _p, _p, _d, _d, _i64, _p, _p, _i64, _p, _p, _p]
            L.ewo_virial_real.restype = None
            L.ewo_virial_real.argtypes = [_i64, _p, _p, _d, _d, _d, _p]
            L.ewo_virial_recip.restype = None
            L.ewo_virial_recip.argtypes = [_i64, _p, _p, _d, _d, _p]
            L.ewo_lj.restype = ctypes.c_int
            L.ewo_lj.argtypes = [_i64, _p, _p, ctypes.c_int, _p, _p, _d, _d, _p, _p, _p]
            L.ewo_self.restype = _d
            L.ewo_self.argtypes = [_i64, _p, _d]
            L.ewo_coulomb_cube.restype = None
            L.ewo_coulomb_cube.argtypes = [_i64, _p, _p, _d, ctypes.c_int, _p, _p]
            L.ewo_num_threads.restype = ctypes.c_int
            L.ewo_set_threads.argtypes = [ctypes.c_int]
            _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return int(lib().ewo_num_threads())


def set_threads(t: int) -> None:
    lib().ewo_set_threads(int(t))


def kset_half(kmax: int) -> np.ndarray:
    """Half-space k set (int32 [nk, 3]): m != 0, |m|^2 <= kmax^2, first nonzero of (mz, my, mx)
    positive; ordered by mz, then my, then mx."""
    n = lib().ewo_kset_half(int(kmax), None, 0)
    m = np.zeros((n, 3), dtype=np.int32)
    lib().ewo_kset_half(int(kmax), _ptr(m), n)
    return m


def _sub(sub):
    return None if sub is None else np.ascontiguousarray(sub, dtype=np.int64)


def real(pos, q, L, beta, rc, sub=None, images=False):
    """Real-space part: (E_real or None when sub is given, F [nt, 3], phi [nt]).  With
    images=True the sum runs over explicit image shifts even where r_c <= L/2 would take
    the minimum image directly (the same sum; used to check one branch against the other)."""
    pos, q, sub = _f64(pos), _f64(q), _sub(sub)
    nt = len(q) if sub is None else len(sub)
    F = np.zeros((nt, 3))
    phi = np.zeros(nt)
    e = _d(0.0)
    lib().ewo_real(len(q), _ptr(pos), _ptr(q), float(L), float(beta), float(rc),
                   0 if sub is None else len(sub), _ptr(sub), _ptr(F), _ptr(phi),
                   ctypes.byref(e) if sub is None else None, int(bool(images)))
    return (e.value if sub is None else None), F, phi


def real_cells(pos, q, L, beta, rc, sub=None):
    """Real-space part through a cell list (needs r_c <= L/2 and floor(L / r_c) >= 3):
    (E_real or None when sub is given, F [nt, 3], phi [nt]); the same sums as real()."""
    pos, q, sub = _f64(pos), _f64(q), _sub(sub)
    nt = len(q) if sub is None else len(sub)
    F = np.zeros((nt, 3))
    phi = np.zeros(nt)
    e = _d(0.0)
    rc_ = lib().ewo_real_cells(len(q), _ptr(pos), _ptr(q), float(L), float(beta), float(rc),
                               0 if sub is None else len(sub), _ptr(sub), _ptr(F), _ptr(phi),
                               ctypes.byref(e) if sub is None else None)
    if rc_ != 0:
        raise ValueError("real_cells needs r_c <= L/2 and at least 3 cells per side")
    return (e.value if sub is None else None), F, phi


def structure_factor(pos, q, L, m) -> np.ndarray:
    """S(k) = sum_j q_j exp(i k.r_j) for k = 2 pi m / L; complex128 [nk]."""
    pos, q = _f64(pos), _f64(q)
    m = np.ascontiguousarray(m, dtype=np.int32)
    S = np.zeros((len(m), 2))
    lib().ewo_structure_factor(len(q), _ptr(pos), _ptr(q), float(L), len(m), _ptr(m), _ptr(S))
    return S[:, 0] + 1j * S[:, 1]


def recip(pos, q, L, beta, kmax, sub=None, S=None):
    """Reciprocal part over K_half(kmax): (E_recip, F [nt, 3], phi [nt], S [nk], m [nk, 3])."""
    pos, q, sub = _f64(pos), _f64(q), _sub(sub)
    m = kset_half(kmax)
    if S is None:
        S = structure_factor(pos, q, L, m)
    S2 = np.ascontiguousarray(np.stack([S.real, S.imag], axis=1))
    e = lib().ewo_recip_energy(len(m), _ptr(m), _ptr(S2), float(L), float(beta), None)
    nt = len(q) if sub is None else len(sub)
    F = np.zeros((nt, 3))
    phi = np.zeros(nt)
    lib().ewo_recip_forces(len(q), _ptr(pos), _ptr(q), float(L), float(beta), len(m), _ptr(m),
                           _ptr(S2), 0 if sub is None else len(sub), _ptr(sub), _ptr(F), _ptr(phi))
    return e, F, phi, S, m


def virial_real(pos, q, L, beta, rc) -> np.ndarray:
    """Real-space virial tensor W_ab = -dE_real/d(eps_ab) at fixed beta ([3, 3])."""
    pos, q = _f64(pos), _f64(q)
    W = np.zeros(9)
    lib().ewo_virial_real(len(q), _ptr(pos), _ptr(q), float(L), float(beta), float(rc), _ptr(W))
    return W.reshape(3, 3)


def virial_recip(pos, q, L, beta, kmax, S=None) -> np.ndarray:
    """Reciprocal-space virial tensor W_ab = -dE_recip/d(eps_ab) at fixed beta over
    K_half(kmax) ([3, 3]); S (complex, K_half order) is computed when not given."""
    pos, q = _f64(pos), _f64(q)
    m = kset_half(kmax)
    if S is None:
        S = structure_factor(pos, q, L, m)
    S2 = np.ascontiguousarray(np.stack([S.real, S.imag], axis=1))
    W = np.zeros(9)
    lib().ewo_virial_recip(len(m), _ptr(m), _ptr(S2), float(L), float(beta), _ptr(W))
    return W.reshape(3, 3)


def lj(pos, types, eps, sigma, L, rc):
    """Truncated and shifted Lennard-Jones pairs inside r_c (minimum image): (E, F [n, 3],
    W [3, 3]).  types int [n] in [0, T); eps and sigma symmetric [T, T]."""
    pos = _f64(pos)
    types = np.ascontiguousarray(types, dtype=np.int32)
    eps, sigma = _f64(eps), _f64(sigma)
    T = eps.shape[0]
    F = np.zeros((len(types), 3))
    Wv = np.zeros(9)
    e = _d(0.0)
    r = lib().ewo_lj(len(types), _ptr(pos), _ptr(types), int(T), _ptr(eps), _ptr(sigma),
                     float(L), float(rc), _ptr(F), ctypes.byref(e), _ptr(Wv))
    if r != 0:
        raise ValueError("lj needs r_c <= L/2 and types in [0, T)")
    return e.value, F, Wv.reshape(3, 3)


def self_energy(q, beta) -> float:
    q = _f64(q)
    return float(lib().ewo_self(len(q), _ptr(q), float(beta)))


def ewald(pos, q, L, beta, rc, kmax, sub=None):
    """Full Ewald evaluation.  Returns a dict with E_real, E_recip, E_self, E_total (E_real and
    E_total are None when a subset is requested), F, F_real, F_recip, phi_real, phi_recip, S, m."""
    er, Fr, pr = real(pos, q, L, beta, rc, sub)
    ek, Fk, pk, S, m = recip(pos, q, L, beta, kmax, sub)
    es = self_energy(q, beta)
    return dict(E_real=er, E_recip=ek, E_self=es,
                E_total=None if er is None else er + ek + es,
                F=Fr + Fk, F_real=Fr, F_recip=Fk, phi_real=pr, phi_recip=pk, S=S, m=m)


def coulomb_cube(pos, q, L, shells: int, forces: bool = False):
    """Brute-force lattice sum over cubes of whole image cells: (E after each shell
    [shells + 1], F after the last shell or None).  Positions are used as given."""
    pos, q = _f64(pos), _f64(q)
    E = np.zeros(shells + 1)
    F = np.zeros((len(q), 3)) if forces else None
    lib().ewo_coulomb_cube(len(q), _ptr(pos), _ptr(q), float(L), int(shells), _ptr(E), _ptr(F))
    return E, F
