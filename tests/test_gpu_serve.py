"""Continuous-batching server (ewald_server_*): every result equals the same system evaluated
alone through a plan, admission respects the HBM budget, requests overlap when the budget
allows, and errors come back as statuses."""
import time

import numpy as np
import pytest

from gpu_common import assert_close, dev, need_gpu, rel_total, torch

import oracle

from paper_1708_01135_gb300 import Ewald, EwaldError, Server, tune
from paper_1708_01135_gb300 import ewald as E
from paper_1708_01135_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _systems(count=10, seed=5):
    out = []
    for i, (kind, n, rho, m) in enumerate(W.request_sizes(count, 256, 6000, seed)):
        L = (n / rho) ** (1.0 / 3.0)
        if kind == "rocksalt":
            pos, q, L = W.rocksalt(m, a=L / m, jitter=0.05 * L / m, seed=100 + i)
        else:
            pos, q, L = W.random_neutral(n, L=L, hard_core=0.8 * (1.0 / rho) ** (1.0 / 3.0), seed=100 + i)
        rc, beta, km = tune(len(q), L, 1e-5, r_c=min(4.0, 0.5 * L))
        out.append((pos, q, L, beta, rc, km))
    return out


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_results_equal_isolated_evaluations(precision):
    need_gpu()
    systems = _systems(10 if precision == "mixed" else 5)
    srv = Server(max_slots=4)
    try:
        reqs = []
        for pos, q, L, beta, rc, km in systems:
            tp, tq = dev(pos), dev(q)
            F = torch.empty((len(q), 3), dtype=torch.float64, device="cuda")
            t = srv.submit(tp, tq, F, L, beta, rc, km, precision)
            reqs.append((t, F))
        results = [srv.wait(t, 120.0) for t, _ in reqs]
        stats = srv.stats()
    finally:
        srv.close()
    assert stats["submitted"] == len(systems) and stats["completed"] == len(systems)
    for (pos, q, L, beta, rc, km), (t, F), res in zip(systems, reqs, results):
        assert res["status"] == 0
        assert res["t_submit"] <= res["t_admit"] <= res["t_done"]
        with Ewald(L, beta, rc, km, precision) as ew:
            F1, e1 = ew.compute(dev(pos), dev(q))
        # the same kernels and the same fixed reduction orders: identical results
        assert torch.equal(F, F1)
        assert np.array_equal(res["energy"], e1)


@pytest.mark.parametrize("precision,tol", [("mixed", 1e-5), ("fp64", 1e-10)])
def test_server_results_match_the_oracle(precision, tol):
    """Four requests of different sizes and kinds evaluated together by the server, each
    checked against the FP64 oracle at its own (beta, r_c, k_max), per particle and in
    energy (the mixed-path and FP64-path bounds of the parity tests)."""
    need_gpu()
    systems = _systems(4, seed=21)
    srv = Server(max_slots=4)
    try:
        reqs = []
        for pos, q, L, beta, rc, km in systems:
            F = torch.empty((len(q), 3), dtype=torch.float64, device="cuda")
            reqs.append((srv.submit(dev(pos), dev(q), F, L, beta, rc, km, precision), F))
        results = [srv.wait(t, 120.0) for t, _ in reqs]
    finally:
        srv.close()
    for (pos, q, L, beta, rc, km), (t, F), res in zip(systems, reqs, results):
        assert res["status"] == 0
        ref = oracle.ewald(pos, q, L, beta, rc, km)
        assert_close(F.cpu().numpy(), ref["F"], tol)
        assert rel_total(res["energy"][3], ref) < tol


def test_budget_limits_admission_and_requests_overlap():
    need_gpu()
    systems = _systems(8, seed=9)
    fp = []
    srv_probe = Server(max_slots=8)
    try:
        for pos, q, L, beta, rc, km in systems[:1]:
            tp, tq = dev(pos), dev(q)
            F = torch.empty((len(q), 3), dtype=torch.float64, device="cuda")
            fp.append(srv_probe.wait(srv_probe.submit(tp, tq, F, L, beta, rc, km), 60.0)["footprint_bytes"])
    finally:
        srv_probe.close()
    # largest footprint of the stream, estimated by submitting all of them to a wide server
    wide = Server(max_slots=8)
    tickets, keep = [], []
    try:
        for pos, q, L, beta, rc, km in systems:
            tp, tq = dev(pos), dev(q)
            F = torch.empty((len(q), 3), dtype=torch.float64, device="cuda")
            keep.append((tp, tq, F))
            tickets.append(wide.submit(tp, tq, F, L, beta, rc, km))
        res = [wide.wait(t, 120.0) for t in tickets]
        wide_stats = wide.stats()
    finally:
        wide.close()
    biggest = max(r["footprint_bytes"] for r in res)
    assert all(r["status"] == 0 for r in res)
    assert wide_stats["peak_concurrent"] >= 2          # requests overlapped on the device
    # a budget of 1.5x the largest request: never more than the budget admitted at once
    budget = int(1.5 * biggest)
    tight = Server(max_slots=8, hbm_budget_bytes=budget)
    try:
        tickets = [tight.submit(tp, tq, F, L, beta, rc, km)
                   for (tp, tq, F), (pos, q, L, beta, rc, km) in zip(keep, systems)]
        res2 = [tight.wait(t, 120.0) for t in tickets]
        tight_stats = tight.stats()
    finally:
        tight.close()
    assert all(r["status"] == 0 for r in res2)
    assert tight_stats["peak_admitted_bytes"] <= budget
    for a, b in zip(res, res2):
        assert np.array_equal(a["energy"], b["energy"])


def test_request_larger_than_budget_is_rejected():
    need_gpu()
    pos, q, L = W.rocksalt(8, 1.0, 0.05, seed=3)
    srv = Server(max_slots=2, hbm_budget_bytes=1 << 16)
    try:
        F = torch.empty((len(q), 3), dtype=torch.float64, device="cuda")
        with pytest.raises(EwaldError) as ex:
            srv.submit(dev(pos), dev(q), F, L, 1.0, 4.0, 8)
        assert ex.value.status == E.E_INVAL
    finally:
        srv.close()


def test_nonneutral_request_reports_status_and_server_continues():
    need_gpu()
    pos, q, L = W.rocksalt(8, 1.0, 0.05, seed=4)
    bad = q.copy()
    bad[0] = 0.3
    srv = Server(max_slots=2)
    try:
        F1 = torch.empty((len(q), 3), dtype=torch.float64, device="cuda")
        F2 = torch.empty((len(q), 3), dtype=torch.float64, device="cuda")
        t1 = srv.submit(dev(pos), dev(bad), F1, L, 1.0, 4.0, 8)
        t2 = srv.submit(dev(pos), dev(q), F2, L, 1.0, 4.0, 8)
        r1 = srv.wait(t1, 60.0)
        r2 = srv.wait(t2, 60.0)
    finally:
        srv.close()
    assert r1["status"] == E.E_NONNEUTRAL
    assert r2["status"] == 0


def test_poll_unknown_ticket_and_wait_timeout():
    need_gpu()
    srv = Server(max_slots=1)
    try:
        with pytest.raises(EwaldError) as ex:
            srv.poll(987654321)
        assert ex.value.status == E.E_NOTFOUND
        pos, q, L = W.random_32768()
        F = torch.empty((len(q), 3), dtype=torch.float64, device="cuda")
        t = srv.submit(dev(pos), dev(q), F, L, 0.93, 4.0, 36, "fp64")   # ~0.1 s on the GPU
        with pytest.raises(EwaldError) as ex:
            srv.wait(t, 0.0)
        assert ex.value.status == E.E_TIMEOUT
        assert srv.wait(t, 120.0)["status"] == 0
    finally:
        srv.close()


def test_destroy_with_work_in_flight():
    need_gpu()
    systems = _systems(6, seed=13)
    srv = Server(max_slots=2)
    keep = []
    for pos, q, L, beta, rc, km in systems:
        tp, tq = dev(pos), dev(q)
        F = torch.empty((len(q), 3), dtype=torch.float64, device="cuda")
        keep.append((tp, tq, F))
        srv.submit(tp, tq, F, L, beta, rc, km)
    t0 = time.time()
    srv.close()          # waits for running requests, drops queued ones
    assert time.time() - t0 < 60.0
