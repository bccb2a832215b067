"""Lennard-Jones pairs fused into the real-space kernel (ewald_set_lj) against the oracle's
ewo_lj on every path (FP64, mixed, FP32) through the cell-list and all-pairs kernels:
forces (Ewald + LJ), the LJ energy (energy[3] minus the three Ewald parts) and the LJ
virial (the sum tensor minus the real and reciprocal ones).  Then: a bad type is reported,
switching the pairs off restores the plain results bit for bit, the FP64 MD trajectory
follows an oracle-driven Verlet loop, and a rock-salt crystal held by the LJ repulsion
conserves its energy over 10,000 velocity-Verlet steps on the mixed path."""
import math

import numpy as np
import pytest

from gpu_common import dev, need_gpu, rel, rel_rms, assert_close, torch

import oracle
from paper_1708_01135_gb300 import MD_RECORD, Ewald, EwaldError
from paper_1708_01135_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "mixed": 2e-5, "fp32": 2e-5}
EPS = np.array([[0.30, 0.05], [0.05, 0.20]])
SIG = np.array([[0.90, 0.80], [0.80, 1.00]])


def _types(q):
    return (np.asarray(q) < 0).astype(np.int32)


def _eval(ew, pos, q):
    n = len(q)
    F = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    V = torch.empty((4, 3, 3), dtype=torch.float64, device="cuda")
    E = torch.empty(4, dtype=torch.float64, device="cuda")
    ew.compute_virial_async(dev(pos), dev(q), F, V, E)
    st = ew.status()
    return st, F.cpu().numpy(), V.cpu().numpy(), E.cpu().numpy()


CASES = {
    "cells": dict(n=20000, seed=51, rc_frac=0.2, beta_rc=3.3, kmax=16),
    "allpairs": dict(n=600, seed=52, rc_frac=0.45, beta_rc=3.3, kmax=10),
}


@pytest.mark.parametrize("precision", ["fp64", "mixed", "fp32"])
@pytest.mark.parametrize("case", ["cells", "allpairs"])
def test_lj_matches_oracle(precision, case):
    need_gpu()
    c = CASES[case]
    pos, q, L = W.random_neutral(c["n"], density=1.0, hard_core=0.8, seed=c["seed"])
    rc = c["rc_frac"] * L
    beta = c["beta_rc"] / rc
    types = _types(q)
    e_lj, F_lj, W_lj = oracle.lj(pos, types, EPS, SIG, L, rc)
    sub = np.sort(np.random.default_rng(c["seed"]).choice(len(q), min(len(q), 512), replace=False))
    ref = oracle.ewald(pos, q, L, beta, rc, c["kmax"], sub=sub)
    t_types = dev(types, torch.int32)
    with Ewald(L, beta, rc, c["kmax"], precision) as ew:
        ew.set_lj(EPS, SIG, t_types)
        st, F, V, E = _eval(ew, pos, q)
    assert st == 0
    tol = TOL[precision]
    F_ref = ref["F"] + F_lj[sub]
    assert_close(F[sub], F_ref, tol)
    # the LJ parts alone: energy and virial by difference of the reported parts
    assert rel(E[3] - E[0] - E[1] - E[2], e_lj) < tol
    W_gpu = V[3] - V[0] - V[1]
    assert np.abs(W_gpu - W_lj).max() < tol * np.abs(W_lj).max()


def test_bad_type_and_switching_off():
    need_gpu()
    pos, q, L = W.random_neutral(4000, density=1.0, hard_core=0.8, seed=53)
    rc = 0.25 * L
    beta = 3.3 / rc
    types = _types(q)
    with Ewald(L, beta, rc, 12, "mixed") as ew:
        st0, F0, V0, E0 = _eval(ew, pos, q)
        bad = types.copy()
        bad[17] = 2                       # outside [0, 2): reported, taken as type 0
        t_bad = dev(bad, torch.int32)
        ew.set_lj(EPS, SIG, t_bad)
        st1, _, _, _ = _eval(ew, pos, q)
        t_ok = dev(types, torch.int32)
        ew.set_lj(EPS, SIG, t_ok)
        st2, F2, _, E2 = _eval(ew, pos, q)
        ew.set_lj()
        st3, F3, V3, E3 = _eval(ew, pos, q)
        with pytest.raises(EwaldError):
            ew.set_lj(np.array([[0.1, 0.2], [0.3, 0.1]]), SIG, t_ok)     # not symmetric
        with pytest.raises(EwaldError):
            ew.set_lj(np.full((9, 9), 0.1), np.full((9, 9), 1.0), t_ok)  # too many types
    assert st0 == 0 and st2 == 0 and st3 == 0
    assert st1 != 0
    assert np.array_equal(F3, F0) and np.array_equal(E3, E0) and np.array_equal(V3, V0)
    assert np.allclose(E2[:3], E0[:3], rtol=1e-12, atol=0) and E2[3] != E0[3]
    assert np.abs(F2 - F0).max() > 0


def _verlet_oracle_lj(pos, vel, q, types, L, beta, rc, kmax, dt, steps):
    x, v = pos.copy(), vel.copy()

    def force(x):
        r = oracle.ewald(x, q, L, beta, rc, kmax)
        e, F, _ = oracle.lj(x, types, EPS, SIG, L, rc)
        return r["F"] + F, r["E_total"] + e

    F, ep = force(x)
    log = [[ep, 0.5 * float((v * v).sum())]]
    for _ in range(steps):
        v = v + 0.5 * dt * F
        x = x + dt * v
        F, ep = force(x)
        v = v + 0.5 * dt * F
        log.append([ep, 0.5 * float((v * v).sum())])
    return x, v, np.array(log)


def test_fp64_md_with_lj_matches_oracle_verlet():
    need_gpu()
    pos, q, L = W.random_neutral(800, density=1.0, hard_core=0.85, seed=54)
    vel = np.random.default_rng(54).normal(0.0, 0.2, size=pos.shape)
    types = _types(q)
    beta, rc, kmax, dt, steps = 0.9, 0.45 * L, 12, 2e-3, 6
    xr, vr, logr = _verlet_oracle_lj(pos, vel, q, types, L, beta, rc, kmax, dt, steps)
    t_types = dev(types, torch.int32)
    with Ewald(L, beta, rc, kmax, "fp64") as ew:
        ew.set_lj(EPS, SIG, t_types)
        tp, tv = dev(pos), dev(vel)
        F = torch.empty_like(tp)
        log = torch.empty((steps + 1, MD_RECORD), dtype=torch.float64, device="cuda")
        ew.md(tp, tv, dev(q), F, dt, steps, log=log)
        assert ew.status() == 0
    x, v, log = tp.cpu().numpy(), tv.cpu().numpy(), log.cpu().numpy()
    assert np.abs(x - xr).max() < 1e-10 * L
    assert np.abs(v - vr).max() < 1e-9 * np.abs(vr).max()
    assert np.abs(log[:, 3] - logr[:, 0]).max() < 1e-9 * np.abs(logr[:, 0]).max()
    assert np.abs(log[:, 4] - logr[:, 1]).max() < 1e-9 * np.abs(logr[:, 1]).max()


def _md_log(precision, pos, vel, q, L, eps, sig, dt, steps):
    n = len(q)
    t_types = torch.zeros(n, dtype=torch.int32, device="cuda")
    with Ewald(L, 0.66, 5.0, 11, precision) as ew:
        ew.set_lj(eps, sig, t_types)
        tp, tv = dev(pos), dev(vel)
        F = torch.empty_like(tp)
        log = torch.empty((steps + 1, MD_RECORD), dtype=torch.float64, device="cuda")
        ew.md(tp, tv, dev(q), F, dt, steps, log=log)
        assert ew.status() == 0
    return tp.cpu().numpy(), log.cpu().numpy()


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_rock_salt_with_lj_conserves_energy_over_10000_steps(precision):
    """NaCl-like crystal in reduced units: 16^3 ions of charge +-1 at spacing 1, every pair
    with sigma = 1 and eps = 0.0182 (about zero pressure at this spacing: the LJ virial
    balances the Madelung energy), unit masses, random velocities of kT = 0.01 (half of it
    ends as potential energy; rock-salt melts near kT = 0.018 in these units).  Over 10,000
    steps of dt = 2e-3 (about 10 vibration periods) the total energy stays within 1e-6 of
    |E_pot| with no systematic drift, and every ion stays near its site."""
    need_gpu()
    pos, q, L = W.rocksalt(16)
    rng = np.random.default_rng(55)
    vel = rng.normal(0.0, math.sqrt(0.01), size=pos.shape)
    vel -= vel.mean(axis=0)
    steps, dt = 10000, 2e-3
    x, log = _md_log(precision, pos, vel, q, L, np.full((1, 1), 0.0182), np.ones((1, 1)), dt, steps)
    et, ke, ep = log[:, 5], log[:, 4], log[:, 3]
    dev_max = np.abs(et - et[0]).max() / abs(ep[0])
    # linear trend of the total energy over the run, relative to |E_pot|
    slope = np.polyfit(np.arange(steps + 1), et, 1)[0] * steps / abs(ep[0])
    disp = np.abs(((x - pos + L / 2) % L) - L / 2).max()
    print(f"LJ rock-salt 10k steps ({precision}): max |dE|/|E_pot| {dev_max:.2e}, trend "
          f"{slope:.2e}, max |dE|/KE {np.abs(et - et[0]).max() / ke.mean():.2e}, "
          f"KE {ke[0]:.2f}->{ke[-1]:.2f}, max displacement {disp:.3f}")
    assert ke.min() > 0.2 * ke[0]           # neither frozen nor collapsed
    assert disp < 0.5                       # still a crystal
    assert dev_max < 1e-5 and abs(slope) < 1e-5
