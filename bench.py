"""Benchmark: Ewald force evaluations per second (particles/s) on the GPU.

A step is one full evaluation of the hot path (binning, real-space pairs, S(k), energy,
back-scatter, self term, unsort) of one synthetic system through the C ABI.  Rank 0 prints
one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload random_32768]
                  [--precision mixed|fp64|fp32|mixed_bf16] [--impl ours|reference]
                  [--md STEPS [--dt DT] [--lj] [--kT KT]] [--spme auto|K,p [--spme-rc RC]]
  (--spme applies to single evaluations and to --md runs)

Timing: inputs resident in HBM; before every step a 512 MiB buffer is written to flush
the L2 (129 MB); every step is bracketed by CUDA events on the launching stream and the
per-step device times are summed.  The end-to-end figure times the host-buffer entry point
(pinned host -> device copies of positions and charges, evaluation, device -> host copies of
forces and energies) per step.  Multi-GPU: the method shards into independent systems, so
N ranks evaluate N independent replicas (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1708_01135_gb300 import workloads as W  # noqa: E402

TOL = 1e-6

WORKLOADS = {
    # name: (generator, fixed r_c or None)
    "rocksalt_512": (W.rocksalt_512, 4.0),
    "random_32768": (W.random_32768, 4.0),
    "rocksalt_262144": (W.rocksalt_262144, None),
    "random_2097152": (W.random_2097152, None),
}


# Smooth particle-mesh Ewald: the mesh spacing h = L / K that keeps the mesh error of the
# forces below about 1e-6 of the RMS force, as beta * h for each B-spline order p.  Calibrated
# against the FP64 oracle (SPME reciprocal forces against the converged classical sum, random
# +-1 ionic systems at density 1, beta 0.93 and 1.2: the error depends on beta * h and p
# only), with a margin for +-2 charge mixtures, whose relative error is a few times larger.
SPME_BETA_H = {6: 0.20, 8: 0.30, 10: 0.36, 12: 0.40}


def fft_size(k):
    """Smallest even K >= k whose prime factors are 2, 3, 5 and 7 (sizes cuFFT handles with
    its fastest kernels)."""
    k = max(4, int(math.ceil(k)))
    while True:
        if k % 2 == 0:
            r = k
            for f in (2, 3, 5, 7):
                while r % f == 0:
                    r //= f
            if r == 1:
                return k
        k += 1


def spme_params(spec, beta, L):
    """(K, p) from --spme: 'K,p', or 'auto' / 'auto:p' (mesh from SPME_BETA_H)."""
    if spec.startswith("auto"):
        p = int(spec.split(":")[1]) if ":" in spec else 8
        return fft_size(beta * L / SPME_BETA_H[p]), p
    K, p = (int(x) for x in spec.split(","))
    return K, p


def run_params(args, n, L):
    """(r_c, beta, k_max, spme) of a run: the tuned classical parameters, or with --spme the
    SPME mesh (K, p) at the same beta, or at beta r_c = sqrt(-ln tol) for --spme-rc; the
    classical k_max at that beta (for the accuracy check) may exceed the library's limit, in
    which case the plan carries an unused k_max and the classical comparison is skipped."""
    rc, beta, kmax = params_for(args.workload, n, L)
    spme = None
    if args.spme:
        if args.spme_rc:
            rc = args.spme_rc
            beta = math.sqrt(-math.log(TOL)) / rc
            kmax = int(math.ceil(math.sqrt(-math.log(TOL)) * beta * L / math.pi))
        K, order = spme_params(args.spme, beta, L)
        spme = {"K": K, "order": order, "beta_h": beta * L / K, "classical_k_max": kmax}
        kmax = min(kmax, 127)
    return rc, beta, kmax, spme


def params_for(workload, n, L):
    from paper_1708_01135_gb300 import tune
    if workload == "rocksalt_512":
        return 4.0, 1.0, 10          # r_c = L/2, k_max raised to 10 to reach 1e-6
    rc_fixed = WORKLOADS[workload][1]
    rc, beta, km = tune(n, L, TOL, r_c=rc_fixed)
    return rc, beta, km


# ---- roofline bookkeeping ---------------------------------------------------------------

def row_nxmax(kmax):
    """n_x,max of every row (m_y, m_z) of the half plane, in increasing order (the order the
    library processes the rows of the back-scatter in)."""
    out = []
    for mz in range(kmax + 1):
        for my in range(-kmax, kmax + 1):
            if my * my + mz * mz <= kmax * kmax and (mz > 0 or my >= 0):
                out.append(math.isqrt(kmax * kmax - my * my - mz * mz))
    return sorted(out)


def len_kset_half(kmax):
    """|K_half|: integer m != 0 with |m|^2 <= k_max^2 in the half space (m_z > 0, or m_z = 0
    and m_y > 0, or m_z = m_y = 0 and m_x > 0)."""
    cnt = 0
    for mz in range(kmax + 1):
        for my in range(-kmax, kmax + 1):
            r = kmax * kmax - my * my - mz * mz
            if r < 0:
                continue
            nx = math.isqrt(r)
            if mz > 0 or my > 0:
                cnt += 2 * nx + 1
            elif my == 0 and mz == 0:
                cnt += nx
    return cnt


def rows_count(kmax):
    return len(row_nxmax(kmax))


def tensor_flops(n, kmax):
    """Issued tensor-core flops of one evaluation (three split-term products each), following
    the library's tiling.  Forward: per group of 128 rows (forward order: decreasing n_x,max)
    one or two column passes, each an M = 128 x N = 256 product over K = n padded to
    32-particle stages.  Back-scatter: M = n padded to 256-particle CTA tiles; columns in
    passes of 256 (the last narrower, padded to 16), pass q over K = 32-deep blocks from the
    block holding the first row with n_x,max >= the smallest |m_x| of its columns."""
    nx = row_nxmax(kmax)
    R = len(nx)
    nf = 16 * math.ceil((2 * kmax + 1) / 16)
    kpad = 32 * math.ceil(n / 32)
    fwd = 0.0
    for g in range(math.ceil(R / 128)):
        first = nx[R - 1 - 128 * g]                     # forward order = reverse row order
        ncols = min(nf, 16 * math.ceil((2 * first + 1) / 16))
        fwd += math.ceil(ncols / 128) * 2.0 * 128 * 256 * kpad * 3
    ncol = 3 * (2 * kmax + 1)
    npass = math.ceil(ncol / 256)
    nkb = math.ceil(2 * R / 32)
    back = 0.0
    for q in range(npass):
        width = 16 * math.ceil(min(256, ncol - 256 * q) / 16)
        gc = 256 * q
        mlo = 0 if gc < 3 else 1 + (gc - 3) // 6
        r = next((i for i, v in enumerate(nx) if v >= mlo), R - 1)
        kb0 = r // 16
        back += 2.0 * (256 * math.ceil(n / 256)) * (32 * (nkb - kb0)) * width * 3
    return fwd, back


# DRAM bytes per launch of the back-scatter kernel from an ncu capture of the benchmark
# workload, valid while the kernel source is unchanged (sha256 prefix of recip_tc.cu)
BS_TRAFFIC = {("random_32768", "mixed", "b35ef610511fc771"): 4227328}


def bs_traffic(workload, precision):
    import hashlib
    src = os.path.join(ROOT, "paper_1708_01135_gb300", "csrc", "recip_tc.cu")
    try:
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    except OSError:
        return None
    return BS_TRAFFIC.get((workload, precision, h))


def simt_flops(n, kmax):
    """Multiply-add flops of the CUDA-core products (forward and back-scatter)."""
    R = rows_count(kmax)
    fwd = 2.0 * 4 * R * (kmax + 1) * n
    back = 2.0 * n * (2 * R) * 3 * (2 * kmax + 1)
    return fwd, back


def fp32_peak(pk):
    """FP32 CUDA-core peak in TFLOP/s: 152 SMs x 128 FP32 lanes x 2 flop (FMA) x the maximum
    SM clock (MEASURED_PEAKS.json's sm_max_mhz, else 2070 MHz)."""
    return 152 * 128 * 2 * float(pk.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# ---- multi-rank aggregation --------------------------------------------------------------

def max_over_ranks(ms, world, device=None):
    """The job's step time is its slowest rank's: the max of a per-rank time over the ranks
    of the default process group (the value itself when there is one rank)."""
    if world <= 1:
        return float(ms)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, ms, world):
    """Units per second of the whole job: every rank processes units_per_rank in ms."""
    return world * units_per_rank / (ms * 1e-3)


# ---- clocks ------------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---- CPU oracle baseline ------------------------------------------------------------------

def oracle_sample(pos, q, L, beta, rc, kmax, n_targets, seed=0, S_given=None,
                  max_sk_terms=8e9):
    """Time the FP64 oracle on a bounded sample of one evaluation and scale it to the whole
    evaluation.  Sample: S(k) over all particles (over a random subset of the modes when
    |K_half| N exceeds max_sk_terms, scaled by the mode count), then real-space and
    reciprocal forces for `n_targets` random particles; both force parts cost the same per
    target, so the full time is t_S + (N / n_targets) t_targets.  When S(k) is sampled the
    reciprocal forces use S_given (the structure factor of the path under test), so the
    returned forces compare that path's back-scatter and real-space sums with the oracle's.
    Returns (full time, CPU seconds spent, targets, target indices, oracle forces, note)."""
    import oracle
    n = len(q)
    rng = np.random.default_rng(seed)
    sub = np.sort(rng.choice(n, size=min(n_targets, n), replace=False))
    m = oracle.kset_half(kmax)
    nk = len(m)
    t0 = time.perf_counter()
    if nk * n <= max_sk_terms or S_given is None:
        S = oracle.structure_factor(pos, q, L, m)
        t_s = time.perf_counter() - t0
        note = f"S(k) over all {n} particles and all {nk} modes"
    else:
        ms = np.sort(rng.choice(nk, size=max(1, int(max_sk_terms // n)), replace=False))
        oracle.structure_factor(pos, q, L, m[ms])
        t_s = (time.perf_counter() - t0) * nk / len(ms)
        S = S_given
        note = (f"S(k) over all {n} particles for {len(ms)} random modes, scaled to {nk} modes "
                f"(reciprocal forces from the GPU's S(k))")
    t1 = time.perf_counter()
    _, Fr, _ = oracle.real(pos, q, L, beta, rc, sub=sub)
    _, Fk, _, _, _ = oracle.recip(pos, q, L, beta, kmax, sub=sub, S=S)
    t2 = time.perf_counter()
    full = t_s + (t2 - t1) * n / len(sub)
    return full, (t2 - t0), len(sub), sub, Fr + Fk, note


def spme_oracle_sample(pos, q, L, beta, rc, K, order, n_targets, seed=0):
    """Time the FP64 oracle's SPME evaluation on a bounded sample and scale it: the charge
    mesh of all particles and its transforms once, then real-space and SPME reciprocal forces
    of `n_targets` random particles (the full time is t_mesh + (N / n_targets) t_targets).
    Returns (full time, CPU seconds spent, targets, target indices, oracle forces, note)."""
    import oracle
    from oracle import spme as ospme
    n = len(q)
    rng = np.random.default_rng(seed)
    sub = np.sort(rng.choice(n, size=min(n_targets, n), replace=False))
    t0 = time.perf_counter()
    Q = ospme.charge_mesh(pos, q, L, K, order)
    t1 = time.perf_counter()
    ospme.recip(pos, q, L, beta, K, order, sub=sub[:1], Q=Q)     # transforms + one target
    t2 = time.perf_counter()
    _, Fr, _ = oracle.real(pos, q, L, beta, rc, sub=sub)
    Fk = ospme.recip(pos, q, L, beta, K, order, sub=sub, Q=Q)["F"]
    t3 = time.perf_counter()
    t_once = (t1 - t0) + (t2 - t1)                  # mesh and transforms
    t_targets = max((t3 - t2) - (t2 - t1), 0.0)     # per-target work of all the targets
    full = t_once + t_targets * n / len(sub)
    note = (f"SPME oracle: charge mesh of all {n} particles and its transforms on a {K}^3 mesh "
            f"(p = {order})")
    return full, (t3 - t0), len(sub), sub, Fr + Fk, note


# ---- main ---------------------------------------------------------------------------------

def _gen_request(item):
    """One system of the serving stream (runs in a worker process)."""
    import numpy as np_
    from paper_1708_01135_gb300 import workloads as W_
    r, kind, n, rho, m, seed = item
    L = (n / rho) ** (1.0 / 3.0)
    if kind == "rocksalt":
        pos, q, L = W_.rocksalt(m, a=L / m, jitter=0.05 * L / m, seed=seed * 1000 + r)
    else:
        pos, q, L = W_.random_neutral(n, L=L, hard_core=0.8 * (1.0 / rho) ** (1.0 / 3.0),
                                      seed=seed * 1000 + r)
    return np_.ascontiguousarray(pos), np_.ascontiguousarray(q), float(L)


def run_serving(args, rank, world, local):
    """Serving stream: independent systems of uneven N (log-uniform in [256, 65536], half
    jittered rock-salt, half random neutral, density U[0.8, 1.2], each with its own box and
    tuned parameters), submitted to the continuous-batching server.  First a closed-loop run
    measures the saturation rate; then Poisson arrivals at several fractions of it give p50/p99
    latency (submit -> result) and the aggregate particles/s."""
    import multiprocessing as mp
    seed = 1238
    count = args.requests
    items = [(r, kind, n, rho, m, seed) for r, (kind, n, rho, m) in
             enumerate(W.request_sizes(count, 256, 65536, seed))]
    ctx = mp.get_context("spawn")          # before the first CUDA call of this process
    with ctx.Pool(min(16, os.cpu_count() or 4)) as pool:
        systems = pool.map(_gen_request, items)
    import torch
    torch.cuda.set_device(local)
    from paper_1708_01135_gb300 import Server, tune
    dev = torch.device("cuda", local)
    reqs = []
    for pos, q, L in systems:
        rc, beta, km = tune(len(q), L, 1e-5, r_c=min(0.5 * L, 4.0 * (len(q) / L ** 3) ** (-1.0 / 3.0)))
        reqs.append(dict(pos=torch.tensor(pos, device=dev), q=torch.tensor(q, device=dev),
                         F=torch.empty((len(q), 3), dtype=torch.float64, device=dev),
                         L=L, beta=beta, rc=rc, km=km, n=len(q)))
    total_n = sum(r["n"] for r in reqs)
    srv = Server(max_slots=args.slots)

    def run(times):
        t0 = time.perf_counter()
        tickets = []
        for r, ta in zip(reqs, times):
            while time.perf_counter() - t0 < ta:
                time.sleep(0.0002)
            tickets.append(srv.submit(r["pos"], r["q"], r["F"], r["L"], r["beta"], r["rc"], r["km"],
                                      args.precision))
        res = [srv.wait(t, 600.0) for t in tickets]
        if any(x["status"] != 0 for x in res):
            raise RuntimeError("a serving request failed")
        lat = np.array([x["t_done"] - x["t_submit"] for x in res]) * 1e3
        span = max(x["t_done"] for x in res) - min(x["t_submit"] for x in res)
        return lat, span

    run([0.0] * min(16, count))            # warm-up: plans, pools, module load
    lat, span = run([0.0] * count)         # closed loop: everything at once
    sat_rate = count / span
    out = {"saturation": {"requests_per_s": sat_rate, "particles_per_s": total_n / span,
                          "p50_ms": float(np.percentile(lat, 50)),
                          "p99_ms": float(np.percentile(lat, 99))}}
    rng = np.random.default_rng(seed + 7)
    for frac in (0.25, 0.5, 0.75, 0.9, 1.1):
        rate = frac * sat_rate
        times = np.cumsum(rng.exponential(1.0 / rate, size=count))
        lat, span = run(list(times - times[0]))
        out[f"load_{frac}"] = {"arrival_per_s": rate, "p50_ms": float(np.percentile(lat, 50)),
                               "p99_ms": float(np.percentile(lat, 99)),
                               "particles_per_s": total_n / span}
    stats = srv.stats()
    srv.close()
    if rank == 0:
        print(json.dumps({"metric": "ewald_serving", "unit": "ms / particles/s", "n_gpus": world,
                          "requests": count, "total_particles": total_n, "slots": args.slots,
                          "precision": args.precision, "tol": 1e-5, "data": "synthetic",
                          "results": out, "server": stats}), flush=True)


def run_md(args, rank, world, local):
    """Molecular dynamics: `--md K` velocity-Verlet steps (unit masses, dt = 1e-3, the system
    starting at rest) in one ewald_md call per replica; every step is one full evaluation plus
    the kick/drift kernels.  Reports particle-steps/s over the K steps (the call also evaluates
    the initial forces, which is counted inside the timed region) and the energy drift
    max_s |E_tot(s) - E_tot(0)| relative to |E_pot(0)|."""
    import torch
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1708_01135_gb300 import MD_RECORD, Ewald
    gen, _ = WORKLOADS[args.workload]
    pos, q, L = gen()
    n = len(q)
    rc, beta, kmax, spme = run_params(args, n, L)
    dev = torch.device("cuda", local)
    tq = torch.tensor(q, device=dev)
    F = torch.empty((n, 3), dtype=torch.float64, device=dev)
    steps, dt = args.md, args.dt
    log = torch.empty((steps + 1, MD_RECORD), dtype=torch.float64, device=dev)
    ew = Ewald(L, beta, rc, kmax, args.precision)
    if spme:
        ew.set_spme(spme["K"], spme["order"])
    lj_cfg = None
    if args.lj:
        # one Lennard-Jones type for every pair, sigma = the rock-salt spacing and eps that
        # about balances the Madelung pressure there (reduced NaCl-like units)
        lj_cfg = {"types": 1, "sigma": 1.0, "epsilon": 0.0182, "cutoff": rc, "shifted": True}
        t_types = torch.zeros(n, dtype=torch.int32, device=dev)
        ew.set_lj(np.full((1, 1), lj_cfg["epsilon"]), np.full((1, 1), lj_cfg["sigma"]), t_types)
    v0 = np.zeros((n, 3))
    if args.kT > 0:
        v0 = np.random.default_rng(2024).normal(0.0, np.sqrt(args.kT), size=(n, 3))
        v0 -= v0.mean(axis=0)
    clocks = ClockSampler(local)
    clocks.start()
    t_warm = time.perf_counter()
    w = 0
    while w < args.warmup or time.perf_counter() - t_warm < 0.5:
        tp = torch.tensor(pos, device=dev)
        tv = torch.tensor(v0, device=dev)
        ew.md(tp, tv, tq, F, dt, 1)
        w += 1
        torch.cuda.synchronize()
    if ew.status() != 0:
        raise RuntimeError("warm-up MD step reported an error")
    ew.profile(1)
    ew.compute_async(tp, tq, F, torch.empty(4, dtype=torch.float64, device=dev))
    _, per_eval = ew.profile(-1)
    ew.profile(0)
    tp = torch.tensor(pos, device=dev)
    tv = torch.tensor(v0, device=dev)
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ev0.record(stream)
    ew.md(tp, tv, tq, F, dt, steps, log=log)
    ev1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    if ew.status() != 0:
        raise RuntimeError("MD run reported an error")
    ms = max_over_ranks(ev0.elapsed_time(ev1), world, dev)
    lg = log.cpu().numpy()
    e_tot = lg[:, 5]
    drift = float(np.abs(e_tot - e_tot[0]).max() / abs(lg[0, 3]))
    if rank == 0:
        print(json.dumps({
            "metric": "ewald_md_particle_steps_per_s", "value": whole_job_rate(n * steps, ms, world),
            "unit": "particle-steps/s", "n_gpus": world, "steps": steps, "warmup": w,
            "ms_per_step": ms / steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
            "config": {"workload": args.workload, "n": n, "L": L, "r_c": rc, "beta": beta,
                       "k_max": kmax, "dt": dt, "mass": 1.0, "kT0": args.kT, "lj": lj_cfg,
                       "reciprocal": ({"method": "spme", **spme} if spme else
                                      {"method": "classical k-space sum"}),
                       "precision": args.precision,
                       "l2": "not flushed: the MD state stays resident from step to step",
                       "parallelism": f"replicas x{world}"},
            "energy": {"E_pot0": float(lg[0, 3]), "E_tot0": float(e_tot[0]),
                       "E_kin_end": float(lg[-1, 4]), "drift_rel_max": drift,
                       "drift_rel_end": float(abs(e_tot[-1] - e_tot[0]) / abs(lg[0, 3]))},
            "gpu_launches": (steps + 1) * (per_eval + 2) + steps,
            "clocks": clk}), flush=True)
    ew.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle
    gen, _ = WORKLOADS[args.workload]
    pos, q, L = gen()
    n = len(q)
    rc, beta, kmax = params_for(args.workload, n, L)
    nk = len(oracle.kset_half(kmax))
    S0 = np.zeros(nk, dtype=complex)
    # every step times a sample sized so that the whole run takes about two and a half
    # minutes (between 0.5 s and 10 s of oracle work a step): a small probe measures the
    # oracle's rates, then each step takes S(k) over the modes and the forces of the targets
    # that fill half of its budget each (see oracle_sample for the scaling to the full N)
    budget = min(10.0, max(0.5, 150.0 / (args.warmup + args.steps)))
    ms = oracle.kset_half(kmax)[: max(1, min(nk, int(2e7 // n)))]
    t0 = time.perf_counter()
    oracle.structure_factor(pos, q, L, ms)
    c_s = max(1e-13, (time.perf_counter() - t0) / (len(ms) * n))      # s per (mode, particle)
    probe = np.arange(min(16, n))
    t0 = time.perf_counter()
    oracle.real(pos, q, L, beta, rc, sub=probe)
    oracle.recip(pos, q, L, beta, kmax, sub=probe, S=S0)
    c_t = max(1e-9, (time.perf_counter() - t0) / len(probe))          # s per target
    targets = int(min(args.cpu_targets, max(16, 0.5 * budget / c_t)))
    max_terms = max(float(n), 0.5 * budget / c_s)
    times = []
    for s in range(args.warmup + args.steps):
        full, wall, nt, _, _, note = oracle_sample(pos, q, L, beta, rc, kmax, targets, seed=s,
                                                   S_given=S0, max_sk_terms=max_terms)
        if s >= args.warmup:
            times.append(full)
    t = float(np.mean(times))
    value = n / t
    note = note.replace("(reciprocal forces from the GPU's S(k))",
                        "(reciprocal forces of the targets timed against a stand-in S(k) of "
                        "the same size)")
    line = {
        "impl": "reference", "metric": "ewald_particles_per_s", "value": value,
        "unit": "particles/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "n": n, "L": L, "r_c": rc, "beta": beta,
                   "k_max": kmax, "tol": TOL},
        "cpu_baseline": {"value": value, "unit": "particles/s", "cores": oracle.num_threads(),
                         "kind": "oracle",
                         "sample": f"{note}; forces of {targets} random particles, scaled "
                                   f"to {n}"},
        "e2e": {"value": value, "unit": "particles/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default="random_32768", choices=sorted(WORKLOADS) + ["serving"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64", "fp32", "mixed_bf16"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-targets", type=int, default=2048)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--requests", type=int, default=256)
    ap.add_argument("--slots", type=int, default=8)
    ap.add_argument("--fp64-max-n", type=int, default=300000,
                    help="time the FP64 GPU path beside the line up to this N")
    ap.add_argument("--md", type=int, default=0, help="velocity-Verlet MD steps (0: single evaluations)")
    ap.add_argument("--dt", type=float, default=1e-3)
    ap.add_argument("--lj", action="store_true", help="MD with Lennard-Jones pairs (sigma 1, eps 0.0182)")
    ap.add_argument("--kT", type=float, default=0.0, help="MD initial Maxwell velocities (unit masses)")
    ap.add_argument("--spme", default="", help="reciprocal part by smooth particle-mesh Ewald: "
                    "'auto' (order 8), 'auto:P' or 'K,P'")
    ap.add_argument("--spme-rc", type=float, default=0.0,
                    help="real-space cutoff of the SPME line (beta from the tuner at this r_c)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    rank, world, local = dist_env()

    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload == "serving":
        return run_serving(args, rank, world, local)
    if args.md:
        return run_md(args, rank, world, local)

    import torch
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1708_01135_gb300 import Ewald

    gen, _ = WORKLOADS[args.workload]
    pos, q, L = gen()
    n = len(q)
    rc, beta, kmax, spme = run_params(args, n, L)
    dev = torch.device("cuda", local)
    tp = torch.tensor(pos, device=dev)
    tq = torch.tensor(q, device=dev)
    F = torch.empty((n, 3), dtype=torch.float64, device=dev)
    E = torch.empty(4, dtype=torch.float64, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    ew = Ewald(L, beta, rc, kmax, args.precision)
    if spme:
        ew.set_spme(spme["K"], spme["order"])

    # the clock sampler runs through the warm-up (at least ~0.5 s of back-to-back steps) and
    # the timed steps, so that its samples see the GPU under this workload's load
    clocks = ClockSampler(local)
    clocks.start()
    t_warm = time.perf_counter()
    w = 0
    while w < args.warmup or time.perf_counter() - t_warm < 0.5:
        ew.compute_async(tp, tq, F, E)
        w += 1
        if w % 8 == 0:
            torch.cuda.synchronize()
    torch.cuda.synchronize()
    if ew.status() != 0:
        raise RuntimeError("warm-up evaluation reported an error")

    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    stage = {k: [] for k in ("binning", "real", "recip_forward", "recip_coef", "recip_back",
                             "finalize", "total", "recip_branch")}
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    for s in range(args.steps):
        flush.fill_(float(s))
        ev0[s].record(stream)
        ew.compute_async(tp, tq, F, E)
        ev1[s].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    if ew.status() != 0:
        raise RuntimeError("timed evaluation reported an error")
    _, per_step = ew.profile(-1)        # kernels of one evaluation (one graph launch replays them)
    launches = per_step * args.steps
    # stage breakdown (not part of the timed steps): evaluations with stage events recorded,
    # which run the pipeline launch by launch
    ew.profile(1)
    for s in range(min(args.steps, 10)):
        flush.fill_(float(s))
        ew.compute_async(tp, tq, F, E)
        t, _ = ew.profile(-1)           # synchronises on the last stage event
        for k, v in t.items():
            stage[k].append(v)
    ew.profile(0)
    ms = max_over_ranks(float(np.mean([a.elapsed_time(b) for a, b in zip(ev0, ev1)])), world, dev)
    value = whole_job_rate(n, ms, world)

    # end to end through the host-buffer entry point (pinned host memory)
    hp = torch.tensor(pos).pin_memory().numpy()
    hq = torch.tensor(q).pin_memory().numpy()
    hf = torch.empty((n, 3), dtype=torch.float64).pin_memory().numpy()
    for _ in range(2):
        ew.compute_host(hp, hq, hf)
    torch.cuda.synchronize()
    e_times = []
    for _ in range(max(3, args.steps // 2)):
        t0 = time.perf_counter()
        _, eh = ew.compute_host(hp, hq, hf)
        e_times.append(time.perf_counter() - t0)
    e2e = whole_job_rate(n, max_over_ranks(1e3 * float(np.mean(e_times)), world, dev), world)

    pk, pk_kind = peaks()
    tc = args.precision in ("mixed", "mixed_bf16")
    back_ms = float(np.median(stage["recip_back"]))
    fwd_ms = float(np.median(stage["recip_forward"]))
    if spme:
        # the dominant kernel of an SPME step is the real-space pair kernel (FP32 on the mixed
        # path): 40 flop per pair evaluation within r_c, each pair evaluated from both sides
        # (no atomics), N (4 pi / 3) r_c^3 rho pairs per side for density rho
        real_ms = float(np.median(stage["real"]))
        pairs = n * (4.0 * math.pi / 3.0) * rc ** 3 * (n / L ** 3)
        achieved = 40.0 * pairs / (real_ms * 1e-3) / 1e12
        fp32 = args.precision != "fp64"
        peak = fp32_peak(pk) if fp32 else 1.25
        roof = {"bound": "alu", "kernel": "real-space pairs (a4)", "achieved": achieved,
                "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                "work": "40 flop per pair evaluation within r_c (both sides of every pair)",
                "peak_kind": ("FP32 CUDA-core rate from unit counts and the maximum SM clock "
                              "(152 SMs x 128 lanes x 2 flop x 2.07 GHz)" if fp32 else
                              "nominal FP64 rate")}
    elif tc:
        fwd_f, back_f = tensor_flops(n, kmax)
        achieved = back_f / (back_ms * 1e-3) / 1e12
        peak = pk.get("bf16_tflops_sustained", pk.get("bf16_tflops"))
        roof = {"bound": "tensor", "kernel": "back-scatter product (a8)", "achieved": achieved,
                "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": bs_traffic(args.workload, args.precision),
                "work": "issued MMA flop (three split-FP16 products, padded tiles)",
                "peak_kind": f"{pk_kind} bf16 dense sustained (fp16 dense rate is equal)"}
    else:
        fwd_f, back_f = simt_flops(n, kmax)
        achieved = back_f / (back_ms * 1e-3) / 1e12
        peak = 1.25 if args.precision == "fp64" else 76.0
        roof = {"bound": "alu", "kernel": "back-scatter product (a8)", "achieved": achieved,
                "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                "peak_kind": "nominal FP64/FP32 CUDA-core rate (unit counts x clock)"}
    stages_ms = {k: float(np.median(v)) for k, v in stage.items()}
    # the method's own work per evaluation, whatever the kernels issue: 40 flop per pair
    # evaluation within r_c (each pair from both sides, N (4 pi / 3) r_c^3 rho of them) and,
    # for the classical sum, 18 flop per (particle, mode) term (one complex multiply-add for
    # S(k), ~10 flop for the back-scatter), over the whole step time
    pairs = n * (4.0 * math.pi / 3.0) * rc ** 3 * (n / L ** 3)
    nk = 0 if spme else len_kset_half(kmax)
    algo = {"real_pair_evaluations": pairs, "recip_terms": float(n) * nk,
            "flop": 40.0 * pairs + 18.0 * n * nk,
            "tflops_over_step": (40.0 * pairs + 18.0 * n * nk) / (ms * 1e-3) / 1e12,
            "note": ("SPME mesh work not counted" if spme else
                     "classical k-space sum over the half-space modes")}

    # the plain FP64 GPU path on the same system and parameters
    fp64 = None
    if args.precision != "fp64" and n <= args.fp64_max_n:
        with Ewald(L, beta, rc, kmax, "fp64") as ew64:
            for _ in range(2):
                ew64.compute_async(tp, tq, F, E)
            torch.cuda.synchronize()
            t64 = []
            for s in range(3):
                flush.fill_(float(s))
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                ew64.compute_async(tp, tq, F, E)
                b.record(stream)
                torch.cuda.synchronize()
                t64.append(a.elapsed_time(b))
            if ew64.status() != 0:
                raise RuntimeError("FP64 evaluation reported an error")
        ms64 = float(np.mean(t64))
        fp64 = {"value": world * n / (ms64 * 1e-3), "unit": "particles/s", "ms_per_step": ms64,
                "steps": 3, "speedup_of_this_line": ms64 / ms}

    cpu = None
    accuracy = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        Fg = hf                 # forces of the last end-to-end evaluation (same input)
        if spme:
            full, wall, nt, sub, Fo, note = spme_oracle_sample(pos, q, L, beta, rc, spme["K"],
                                                               spme["order"], args.cpu_targets)
            ref_note = ("FP64 oracle at the same (beta, r_c, K, p): real-space pairs plus "
                        "the SPME reciprocal part; arithmetic error of this path (the mesh "
                        "error of (K, p) is the separate spme_vs_classical figure)")
        else:
            full, wall, nt, sub, Fo, note = oracle_sample(pos, q, L, beta, rc, kmax,
                                                          args.cpu_targets,
                                                          S_given=ew.structure_factor())
            ref_note = ("FP64 oracle at the same (beta, r_c, k_max): arithmetic error of this "
                        "path; the truncation error of the parameters is stated separately")
        cpu = {"value": n / full, "unit": "particles/s", "cores": oracle.num_threads(),
               "kind": "oracle", "sample": f"{note}; forces of {nt} random particles, scaled "
                                           f"to {n} ({wall:.1f} s of CPU work)"}
        accuracy = {"rel_force_rms_vs_oracle": float(np.sqrt(((Fg[sub] - Fo) ** 2).sum() /
                                                             (Fo ** 2).sum())),
                    "particles": int(nt), "reference": ref_note, "oracle_sample": note}
    if rank == 0 and spme and spme["classical_k_max"] <= 127:
        # the mesh error of SPME: its forces against the classical k-space sum at the same
        # beta and r_c (the tensor-core path, itself within ~1e-6 of the oracle)
        with Ewald(L, beta, rc, kmax, "mixed") as ewc:
            Fc = torch.empty_like(F)
            ewc.compute_async(tp, tq, Fc, torch.empty_like(E))
            Fc = Fc.cpu().numpy()
        Fs = hf
        spme["vs_classical_rel_force_rms"] = float(np.sqrt(((Fs - Fc) ** 2).sum() / (Fc ** 2).sum()))
    if rank == 0:
        line = {
            "metric": "ewald_particles_per_s", "value": value, "unit": "particles/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"mixed": "fp32 pairs + fp16x2 tensor products (fp32 accum) + f64 reductions",
                      "mixed_bf16": "fp32 pairs + bf16x2 tensor products (fp32 accum) + f64 reductions",
                      "fp64": "f64", "fp32": "f32 (f64 reductions)"}[args.precision],
            "data": "synthetic",
            "config": {"workload": args.workload, "n": n, "L": L, "r_c": rc, "beta": beta,
                       "k_max": kmax, "tol": TOL, "precision": args.precision,
                       "reciprocal": ({"method": "spme", **spme} if spme else
                                      {"method": "classical k-space sum"}),
                       "l2": "flushed before every step (512 MiB write)",
                       "parallelism": f"replicas x{world}"},
            "e2e": {"value": e2e, "unit": "particles/s", "h2d_bytes_per_step": 32 * n,
                    "d2h_bytes_per_step": 24 * n + 32},
            "gpu_launches": launches,
            "roofline": roof,
            "stages_ms": stages_ms,
            "algorithmic": algo,
            "clocks": clk,
            "cpu_baseline": cpu,
            "accuracy": accuracy,
            "fp64_gpu": fp64,
        }
        print(json.dumps(line), flush=True)
    ew.close()
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
