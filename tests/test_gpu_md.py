"""ewald_md: velocity-Verlet time steps driven by the Ewald forces.

The trajectory of the FP64 plan is compared with a plain NumPy velocity-Verlet loop whose
forces come from the FP64 oracle (same masses, time step and initial state); the per-step
energy log with the oracle's energies and the kinetic energy of the reference trajectory.
The mixed plan is checked for energy conservation over a longer run and for staying close
to the FP64 trajectory; both for bit-identical repeats.
"""
import numpy as np
import pytest

from gpu_common import dev, need_gpu, rel, torch

import oracle
from paper_1708_01135_gb300 import MD_RECORD, Ewald
from paper_1708_01135_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _system(n=1000, seed=31):
    pos, q, L = W.random_neutral(n, density=1.0, hard_core=0.8, seed=seed,
                                 mix=((1.0, 0.4), (2.0, 0.1)))
    rng = np.random.default_rng(seed)
    vel = rng.normal(0.0, 0.3, size=pos.shape)
    mass = rng.uniform(1.0, 3.0, size=len(q))
    return pos, q, L, vel, mass


def _verlet_oracle(pos, vel, q, mass, L, beta, rc, kmax, dt, steps):
    """Reference trajectory: v += dt/2 F/m; x += dt v; F = F(x); v += dt/2 F/m."""
    x, v = pos.copy(), vel.copy()
    r = oracle.ewald(x, q, L, beta, rc, kmax)
    F = r["F"]
    log = []

    def rec(r, v):
        ke = 0.5 * float((mass[:, None] * v * v).sum())
        return [r["E_real"], r["E_recip"], r["E_self"], r["E_total"], ke, r["E_total"] + ke]

    log.append(rec(r, v))
    for _ in range(steps):
        v = v + 0.5 * dt * F / mass[:, None]
        x = x + dt * v
        r = oracle.ewald(x, q, L, beta, rc, kmax)
        F = r["F"]
        v = v + 0.5 * dt * F / mass[:, None]
        log.append(rec(r, v))
    return x, v, F, np.array(log)


def _run(ew, pos, vel, q, mass, dt, steps):
    n = len(q)
    tp, tv = dev(pos), dev(vel)
    F = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    log = torch.empty((steps + 1, MD_RECORD), dtype=torch.float64, device="cuda")
    ew.md(tp, tv, dev(q), F, dt, steps, mass=None if mass is None else dev(mass), log=log)
    assert ew.status() == 0
    return tp.cpu().numpy(), tv.cpu().numpy(), F.cpu().numpy(), log.cpu().numpy()


def test_fp64_trajectory_matches_oracle_verlet():
    need_gpu()
    pos, q, L, vel, mass = _system()
    beta, rc, kmax, dt, steps = 0.9, 0.45 * L, 12, 2e-3, 8
    xr, vr, Fr, logr = _verlet_oracle(pos, vel, q, mass, L, beta, rc, kmax, dt, steps)
    with Ewald(L, beta, rc, kmax, "fp64") as ew:
        x, v, F, log = _run(ew, pos, vel, q, mass, dt, steps)
    assert np.abs(x - xr).max() < 1e-10 * L
    assert np.abs(v - vr).max() < 1e-9 * np.abs(vr).max()
    assert np.abs(F - Fr).max() < 1e-9 * np.abs(Fr).max()
    scale = np.abs(logr).max(axis=0)
    assert np.all(np.abs(log - logr) <= 1e-9 * scale + 1e-12)


def test_zero_steps_is_one_evaluation():
    need_gpu()
    pos, q, L, vel, mass = _system(600, seed=5)
    with Ewald(L, 0.9, 0.45 * L, 10, "mixed") as ew:
        x, v, F, log = _run(ew, pos, vel, q, None, 1e-3, 0)
        F1, e1 = ew.compute(dev(pos), dev(q))
    assert np.array_equal(x, pos) and np.array_equal(v, vel)
    assert np.array_equal(F, F1.cpu().numpy())
    assert np.array_equal(log[0, :4], e1)
    assert rel(log[0, 4], 0.5 * float((vel * vel).sum())) < 1e-13


def test_mixed_energy_conservation_and_repeatability():
    """Jittered rock-salt 16^3 from rest: over 200 steps of dt = 1e-3 the total energy stays
    within 1e-7 of |E_pot| (the velocity-Verlet fluctuation is O(dt^2) and the mixed-path
    force error ~1e-6 enters the energy only through the work it does), and the trajectory
    stays within 1e-5 of the FP64 plan's."""
    need_gpu()
    pos, q, L = W.rocksalt(16, 1.0, 0.05, seed=77)
    vel = np.zeros_like(pos)
    beta, rc, kmax, dt, steps = 0.75, 5.0, 14, 1e-3, 200
    with Ewald(L, beta, rc, kmax, "mixed") as ew:
        x1, v1, F1, log1 = _run(ew, pos, vel, q, None, dt, steps)
        x2, v2, F2, log2 = _run(ew, pos, vel, q, None, dt, steps)
    with Ewald(L, beta, rc, kmax, "fp64") as ew:
        x3, v3, F3, log3 = _run(ew, pos, vel, q, None, dt, steps)
    assert np.array_equal(x1, x2) and np.array_equal(log1, log2)
    drift = np.abs(log1[:, 5] - log1[0, 5]).max() / abs(log1[0, 3])
    drift64 = np.abs(log3[:, 5] - log3[0, 5]).max() / abs(log3[0, 3])
    print(f"energy drift: mixed {drift:.2e}, fp64 {drift64:.2e}; KE(end) {log1[-1, 4]:.4e}")
    assert log1[-1, 4] > 0.0
    assert drift < 1e-7 and drift64 < 1e-7
    disp = np.abs(x3 - pos).max()
    assert np.abs(x1 - x3).max() < 1e-5 * max(disp, 1e-3)
