"""Plain FP64 smooth particle-mesh Ewald (SPME): the oracle for the SPME reciprocal part.

TEST INFRASTRUCTURE ONLY (as the rest of ``oracle/``): the product library never imports
it, and it imports nothing from the product package.

The paper names SPME as the faster successor of its classical Ewald sum at large N
(Sections 1 and 5) without stating it; the method is that of Essmann et al., J. Chem. Phys.
103, 8577 (1995), Sections II-III, restated here in the paper's Gaussian units (Coulomb
constant 1, splitting parameter beta, E_recip as in Eq. 3):

* scaled fractional coordinates u_a = K x_a / L in [0, K) on a K^3 mesh;
* cardinal B-splines of order p: M_2(u) = 1 - |u - 1| on [0, 2], and
  M_n(u) = u/(n-1) M_{n-1}(u) + (n-u)/(n-1) M_{n-1}(u-1), dM_n/du = M_{n-1}(u) - M_{n-1}(u-1);
* the charge mesh Q(k) = sum_i q_i prod_a M_p(u_ia - k_a - n_a K) (n_a: periodic images);
* with F(Q)(m) = sum_k Q(k) exp(2 pi i m.k / K), the structure factor S(m / L) is
  approximated by b_1 b_2 b_3 F(Q)(m), |b(m)|^2 = 1 / |sum_{k=0}^{p-2} M_p(k+1)
  exp(2 pi i m k / K)|^2 (the Euler exponential spline);
* E_recip = 1/2 sum_{m != 0} G(m) |F(Q)(m)|^2, G(m) = exp(-pi^2 |m~|^2 / beta^2) /
  (pi V |m~|^2) B(m), B = prod_a |b(m_a)|^2, m~ = m / L with every m_a taken in
  (-K/2, K/2] (the mesh aliases frequencies beyond);
* the mesh potential phi(k) = dE/dQ(k) = sum_m G(m) conj(F(Q)(m)) exp(2 pi i m.k / K),
  so that E = 1/2 sum_k Q(k) phi(k); forces F_i = -sum_k dQ(k)/dr_i phi(k) (the exact
  gradient of this E) and potentials phi_i = sum_k dQ(k)/dq_i phi(k), E = 1/2 sum q_i phi_i.
* virial W_ab = 1/2 sum_m G(m) |F(Q)(m)|^2 [delta_ab - 2 m~_a m~_b (1/|m~|^2 + pi^2/beta^2)]
  (the strain derivative at fixed beta, as for the classical sum: B(m) depends on the
  integers m only).

Only even orders p are accepted: for odd p the Euler spline's denominator vanishes at
m = K/2.  numpy's FFT is used as the library primitive for F and its inverse; nothing is
blocked, fused or reordered beyond the formulas above.

Parity pins (tests/test_oracle_spme.py): the B-spline partition of unity, symmetry and unit
integral; convergence to the classical Ewald reciprocal energy and forces of
``oracle.recip`` as K and p grow; central finite differences of the SPME energy against the
SPME forces; E = 1/2 sum q_i phi_i; invariance under a shift by one mesh spacing.
"""
from __future__ import annotations

import numpy as np


def bspline(p: int, u):
    """Cardinal B-spline M_p(u) (support [0, p]), by the order recursion."""
    u = np.asarray(u, dtype=np.float64)
    if p == 2:
        return np.where((u >= 0.0) & (u <= 2.0), 1.0 - np.abs(u - 1.0), 0.0)
    return u / (p - 1) * bspline(p - 1, u) + (p - u) / (p - 1) * bspline(p - 1, u - 1.0)


def bspline_deriv(p: int, u):
    """dM_p/du = M_{p-1}(u) - M_{p-1}(u - 1)."""
    u = np.asarray(u, dtype=np.float64)
    return bspline(p - 1, u) - bspline(p - 1, u - 1.0)


def _check(K: int, p: int):
    if p < 4 or p % 2:
        raise ValueError("SPME needs an even B-spline order p >= 4")
    if K < p:
        raise ValueError("SPME needs a mesh of at least p points per side")


def _signed(K: int):
    m = np.arange(K)
    return np.where(m <= K // 2, m, m - K).astype(np.float64)


def bspline_moduli(K: int, p: int) -> np.ndarray:
    """|b(m)|^2 for m = 0..K-1 (one axis)."""
    m = np.arange(K)[:, None]
    k = np.arange(p - 1)[None, :]
    den = (bspline(p, k + 1.0) * np.exp(2j * np.pi * m * k / K)).sum(axis=1)
    return 1.0 / np.abs(den) ** 2


def influence(K: int, p: int, L: float, beta: float) -> np.ndarray:
    """G(m) on the full K^3 mesh of frequencies (G(0) = 0)."""
    _check(K, p)
    s = _signed(K) / L
    b2 = bspline_moduli(K, p)
    m2 = s[:, None, None] ** 2 + s[None, :, None] ** 2 + s[None, None, :] ** 2
    B = b2[:, None, None] * b2[None, :, None] * b2[None, None, :]
    V = L ** 3
    with np.errstate(divide="ignore", invalid="ignore"):
        G = np.exp(-np.pi ** 2 * m2 / beta ** 2) / (np.pi * V * m2) * B
    G[0, 0, 0] = 0.0
    return G


def _weights(pos, L, K, p):
    """Per particle and axis: mesh indices k [n, 3, p] (mod K) and M_p, dM_p/du there."""
    x = np.asarray(pos, dtype=np.float64)
    x = x - L * np.floor(x / L)
    u = K * x / L
    base = np.floor(u).astype(np.int64)
    j = np.arange(p)
    k = base[:, :, None] - j[None, None, :]            # M_p(u - k) > 0 for k in (u - p, u]
    t = u[:, :, None] - k
    return np.mod(k, K), bspline(p, t), bspline_deriv(p, t)


def charge_mesh(pos, q, L, K, p, block: int = 4096) -> np.ndarray:
    """Q(k) on the K^3 mesh: every particle adds q_i M_p M_p M_p to its p^3 points (in
    blocks of particles, each an unbuffered np.add.at over their flattened point indices)."""
    idx, w, _ = _weights(pos, L, K, p)
    q = np.asarray(q, dtype=np.float64)
    Q = np.zeros(K * K * K)
    for s in range(0, len(q), block):
        e = min(len(q), s + block)
        wq = (q[s:e, None, None, None] * w[s:e, 0][:, :, None, None] *
              w[s:e, 1][:, None, :, None] * w[s:e, 2][:, None, None, :])
        flat = ((idx[s:e, 0][:, :, None, None] * K + idx[s:e, 1][:, None, :, None]) * K +
                idx[s:e, 2][:, None, None, :])
        np.add.at(Q, flat.ravel(), wq.ravel())
    return Q.reshape(K, K, K)


def recip(pos, q, L, beta, K, p, sub=None, Q=None):
    """SPME reciprocal part: dict with E, F [n, 3], phi [n], W [3, 3], Q, phi_mesh.  With
    `sub` (particle indices) F and phi hold only those particles, in that order; the mesh
    still takes every particle.  Q, if given, is charge_mesh(pos, q, L, K, p) computed
    before."""
    _check(K, p)
    q = np.asarray(q, dtype=np.float64)
    G = influence(K, p, L, beta)
    if Q is None:
        Q = charge_mesh(pos, q, L, K, p)
    FQ = np.fft.fftn(Q)                     # conj(F(Q)) for real Q; |.|^2 is the same
    A = G * np.abs(FQ) ** 2
    E = 0.5 * float(A.sum())
    phi_mesh = np.real(np.fft.ifftn(G * FQ)) * K ** 3
    sel = np.arange(len(q)) if sub is None else np.asarray(sub)
    idx, w, dw = _weights(np.asarray(pos)[sel], L, K, p)
    n = len(sel)
    F = np.zeros((n, 3))
    phi = np.zeros(n)
    qs = q[sel]
    for i in range(n):
        P = phi_mesh[np.ix_(idx[i, 0], idx[i, 1], idx[i, 2])]
        wx, wy, wz = w[i]
        dx, dy, dz = dw[i]
        phi[i] = np.einsum("a,b,c,abc->", wx, wy, wz, P)
        g = np.array([np.einsum("a,b,c,abc->", dx, wy, wz, P),
                      np.einsum("a,b,c,abc->", wx, dy, wz, P),
                      np.einsum("a,b,c,abc->", wx, wy, dz, P)])
        F[i] = -qs[i] * (K / L) * g
    s = _signed(K) / L
    M = [s[:, None, None] + 0 * s[None, :, None] + 0 * s[None, None, :],
         0 * s[:, None, None] + s[None, :, None] + 0 * s[None, None, :],
         0 * s[:, None, None] + 0 * s[None, :, None] + s[None, None, :]]
    m2 = M[0] ** 2 + M[1] ** 2 + M[2] ** 2
    m2[0, 0, 0] = 1.0
    c = 2.0 * (1.0 / m2 + np.pi ** 2 / beta ** 2)
    W = np.zeros((3, 3))
    for a in range(3):
        for b in range(3):
            W[a, b] = 0.5 * float((A * ((1.0 if a == b else 0.0) - c * M[a] * M[b])).sum())
    return dict(E=E, F=F, phi=phi, W=W, Q=Q, phi_mesh=phi_mesh)
