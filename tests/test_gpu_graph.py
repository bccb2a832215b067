"""Graph replay of repeated evaluations: an evaluation with the same sizes and buffers as the
one before it is captured into a CUDA graph and replayed.  Every result must equal a fresh
plan's, whatever path produced it: first call (launch by launch), second (capture + launch),
later calls (replay), new data in the same buffers, other buffers, other parts, and a
re-parameterised plan."""
import numpy as np
import pytest

from gpu_common import dev, need_gpu, torch

from paper_1708_01135_gb300 import PART_ALL, PART_RECIP, Ewald
from paper_1708_01135_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _fresh(pos, q, L, beta, rc, km, parts=PART_ALL):
    with Ewald(L, beta, rc, km, "mixed") as ew:
        n = len(q)
        F = torch.empty((n, 3), dtype=torch.float64, device="cuda")
        E = torch.empty(4, dtype=torch.float64, device="cuda")
        ew.compute_async(dev(pos), dev(q), F, E, parts=parts)
        assert ew.status() == 0
        return F.cpu().numpy(), E.cpu().numpy()


def test_replay_matches_fresh_plans():
    need_gpu()
    pos, q, L = W.random_neutral(3000, density=1.0, hard_core=0.8, seed=41)
    beta, rc, km = 0.9, 4.0, 14
    F0, E0 = _fresh(pos, q, L, beta, rc, km)
    n = len(q)
    with Ewald(L, beta, rc, km, "mixed") as ew:
        tp, tq = dev(pos), dev(q)
        F = torch.empty((n, 3), dtype=torch.float64, device="cuda")
        E = torch.empty(4, dtype=torch.float64, device="cuda")
        for _ in range(4):                        # direct, capture, replay, replay
            F.fill_(float("nan")); E.fill_(float("nan"))
            ew.compute_async(tp, tq, F, E)
            assert ew.status() == 0
            assert np.array_equal(F.cpu().numpy(), F0) and np.array_equal(E.cpu().numpy(), E0)
        # new positions written into the same buffer: the replayed graph reads them
        pos2 = pos + 0.01 * np.random.default_rng(2).standard_normal(pos.shape)
        tp.copy_(dev(pos2))
        F2, E2 = _fresh(pos2, q, L, beta, rc, km)
        for _ in range(2):
            ew.compute_async(tp, tq, F, E)
            assert ew.status() == 0
            assert np.array_equal(F.cpu().numpy(), F2) and np.array_equal(E.cpu().numpy(), E2)
        # other output buffers, then another part mask
        G = torch.empty_like(F)
        for _ in range(3):
            ew.compute_async(tp, tq, G, E)
            assert np.array_equal(G.cpu().numpy(), F2)
        Fr, Er = _fresh(pos2, q, L, beta, rc, km, PART_RECIP)
        for _ in range(3):
            ew.compute_async(tp, tq, G, E, parts=PART_RECIP)
            assert np.array_equal(G.cpu().numpy(), Fr) and np.array_equal(E.cpu().numpy(), Er)


def test_synchronous_and_host_entry_points_repeat():
    need_gpu()
    pos, q, L = W.rocksalt_512()
    F0, E0 = _fresh(pos, q, L, 1.0, 4.0, 10)
    with Ewald(L, 1.0, 4.0, 10, "mixed") as ew:
        tp, tq = dev(pos), dev(q)
        for _ in range(4):
            F, e = ew.compute(tp, tq)
            assert np.array_equal(F.cpu().numpy(), F0) and np.array_equal(e, E0)
        for _ in range(3):
            Fh, eh = ew.compute_host(pos, q)
            assert np.array_equal(Fh, F0) and np.array_equal(eh, E0)


def test_results_do_not_depend_on_the_plans_history():
    """The cell grid follows each evaluation's particle count, so a plan that evaluated a
    larger system first (buffers kept, grid switched) gives the smaller system the same bits
    as a fresh plan, and switching back gives the larger one its own bits again."""
    need_gpu()
    L, beta, rc, km = 16.0, 0.9, 4.0, 14
    big_pos, big_q, _ = W.random_neutral(4096, L=L, hard_core=0.8, seed=51)
    small_pos, small_q, _ = W.random_neutral(1500, L=L, hard_core=0.8, seed=52)
    Fb0, Eb0 = _fresh(big_pos, big_q, L, beta, rc, km)
    Fs0, Es0 = _fresh(small_pos, small_q, L, beta, rc, km)
    with Ewald(L, beta, rc, km, "mixed") as ew:
        for pos, q, F0, E0 in ((big_pos, big_q, Fb0, Eb0), (small_pos, small_q, Fs0, Es0),
                               (big_pos, big_q, Fb0, Eb0), (small_pos, small_q, Fs0, Es0)):
            n = len(q)
            F = torch.empty((n, 3), dtype=torch.float64, device="cuda")
            E = torch.empty(4, dtype=torch.float64, device="cuda")
            for _ in range(3):                    # direct, capture, replay
                ew.compute_async(dev(pos), dev(q), F, E)
                assert ew.status() == 0
                assert np.array_equal(F.cpu().numpy(), F0) and np.array_equal(E.cpu().numpy(), E0)
