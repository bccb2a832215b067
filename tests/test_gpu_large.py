"""Full-size parity at the two large workloads (262,144-ion rock-salt, 2,097,152-ion random
+-1/+-2 system), in the configuration the benchmark times: parameters from the tuner at the benchmark's tuning
tolerance (bench.TUNE_TOL) and r_c where bench.WORKLOADS fixes it, and the crystal's near pairs
in double-float.

The oracle cannot evaluate these systems in seconds, so the checks are on samples and on
stored oracle sums:
  * S(k) on 2,048 seed-chosen modes (and their +-m_x partners) evaluated by the oracle from
    every particle;
  * forces of 4,096 seed-chosen particles: the oracle's real-space sum (cell list) plus its
    reciprocal force from the structure factor the GPU produced (checked above), so that the
    back-scatter is compared on its own;
  * E_recip against the oracle's energy formula applied to the GPU's structure factor, and,
    where stored, against the oracle's full reciprocal sum;
  * E_real and E_self against oracle sums stored by tests/golden/make_large_energies.py,
    with a digest of the generated inputs so that a changed generator is reported as such.
Bounds: relative RMS force error and relative structure-factor error 1e-5 on the mixed path,
1e-9 on the FP64 path; E_real within the bound times 1/2 sum_i |q_i phi_i|.
"""
import hashlib
import json
import os

import numpy as np
import pytest

from gpu_common import dev, need_gpu, rel, rel_rms, assert_close, local_max, torch

import bench
import oracle
from paper_1708_01135_gb300 import Ewald, tune
from paper_1708_01135_gb300 import workloads as W

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def _gold():
    with open(os.path.join(HERE, "golden", "large_energies.json")) as f:
        return json.load(f)


TOL = {"mixed": 1e-5, "fp64": 1e-9}


def _digest(a):
    return hashlib.sha256(np.ascontiguousarray(a, dtype=np.float64).tobytes()).hexdigest()


def _load(name):
    pos, q, L = getattr(W, name)()
    g = _gold()[name]
    assert _digest(pos) == g["pos_sha256"] and _digest(q) == g["q_sha256"], \
        "generated inputs differ from the ones the stored energies belong to"
    rc, beta, km = tune(len(q), L, bench.TUNE_TOL.get(name, bench.TOL), r_c=bench.WORKLOADS[name][1])
    assert rc == g["r_c"] and km == g["k_max"] and abs(beta - g["beta"]) <= 1e-12 * beta
    return pos, q, L, g


def _partner_index(m, sel):
    """For each selected mode m, the index of (-m_x, m_y, m_z) in the k set (itself when
    that mode is not in the half space)."""
    idx = {tuple(v): i for i, v in enumerate(m.tolist())}
    return np.array([idx.get((-int(m[i, 0]), int(m[i, 1]), int(m[i, 2])), i) for i in sel])


@pytest.mark.parametrize("name,precision", [("rocksalt_262144", "mixed"),
                                            ("rocksalt_262144", "fp64"),
                                            ("random_2097152", "mixed")])
def test_full_size_sampled(name, precision):
    need_gpu()
    pos, q, L, g = _load(name)
    n, rc, beta, km = len(q), g["r_c"], g["beta"], g["k_max"]
    tol = TOL[precision]
    with Ewald(L, beta, rc, km, precision) as ew:
        if name in bench.NEAR_DF:
            ew.set_near_pairs(True)
        F, e = ew.compute(dev(pos), dev(q))
        Sg = ew.structure_factor()
        m = ew.kset()
    F = F.cpu().numpy()
    assert np.array_equal(m, oracle.kset_half(km))
    rng = np.random.default_rng(4096)

    # structure factors on sampled modes
    sel = np.sort(rng.choice(len(m), 2048, replace=False))
    part = _partner_index(m, sel)
    S_or = oracle.structure_factor(pos, q, L, m[sel])
    S_par = oracle.structure_factor(pos, q, L, m[part])
    scale = np.sqrt((q ** 2).sum()) + np.abs(S_or) + np.abs(S_par)
    err_S = np.abs(Sg[sel] - S_or) / scale
    assert err_S.max() < tol, err_S.max()

    # forces on sampled particles
    sub = np.sort(rng.choice(n, 4096, replace=False))
    _, Fr, _ = oracle.real_cells(pos, q, L, beta, rc, sub=sub)
    ek_gpuS, Fk, _, _, _ = oracle.recip(pos, q, L, beta, km, sub=sub, S=Sg)
    err_F = rel_rms(F[sub], Fr + Fk)
    assert_close(F[sub], Fr + Fk, tol)

    # energies
    assert rel(e[1], ek_gpuS) < 1e-12
    if "E_recip" in g:
        assert rel(e[1], g["E_recip"]) < tol
    assert abs(e[0] - g["E_real"]) < tol * g["E_real_scale"]
    assert rel(e[2], g["E_self"]) < 1e-13
    assert abs(e[3] - (e[0] + e[1] + e[2])) <= 1e-12 * abs(e[3])
    print(f"{name} {precision}: S err {err_S.max():.2e}, F err {err_F:.2e} "
          f"(largest particle {local_max(F[sub], Fr + Fk):.2e}), "
          f"E_real err {abs(e[0] - g['E_real']) / g['E_real_scale']:.2e}")
