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
    "rocksalt_262144": (W.rocksalt_262144, 12.0),   # (reading 19 of the design notes)
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


# (r_c, beta, k_max) of every named workload at a 1e-6 relative force error: the library
# tuner's choices (ewald_tune at TUNE_TOL, r_c fixed where WORKLOADS fixes it), written out
# as plain numbers so that the oracle's reference arm needs nothing from the library;
# tests/test_bench_params.py checks that the tuner still returns them.
PARAMS = {
    "rocksalt_512": (4.0, 1.0, 10),          # r_c = L/2, k_max raised to 10 to reach 1e-6
    "random_32768": (4.0, 0.9292305472124596, 36),
    "rocksalt_262144": (12.0, 0.31985023936817364, 26),
    "random_2097152": (10.72, 0.34672781612405207, 53),
}
# The tuner's rule takes the truncation error relative to the force scale of disordered
# ionic systems; in the rock-salt crystal the net force is a small sum of large pair forces,
# and its relative errors are larger by that factor.  Measured total errors of the crystal
# (mixed path, double-float near pairs): 1.34e-6 at the tuner's r_c = 7.84 for 4e-7, 1.15e-6
# for 1e-7, 1.06e-6 at r_c = 11, 9.5e-7 at r_c = 12 (4e-7): the floor is the reciprocal
# part's arithmetic, whose share of the force falls as beta does.  So the crystal runs at
# r_c = 12, tuned for 4e-7.
TUNE_TOL = {"rocksalt_262144": 4e-7}
# Crystals: the near real-space pairs in double-float arithmetic (ewald_set_near_pairs); with
# FP32 near pairs their rounding gives 1e-6 of the crystal's RMS force.  (Not on the SPME
# lines, whose mesh error is larger.)
NEAR_DF = {"rocksalt_262144"}


def near_pairs_of(workload):
    return "double-float" if workload in NEAR_DF else "fp32"


def params_for(workload, n, L):
    return PARAMS[workload]


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


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of a kernel from an
# ncu capture of the same workload, valid while that kernel's source file is unchanged (its
# sha256 prefix is part of the key); the capture each figure comes from is named in
# profiles/.  Kernels without a current capture, and SPME runs (whose real-space kernel runs
# at another cutoff), report null.
TRAFFIC = {
    # profiles/k_real_rows_random_2097152.md: 117.569792 MB read + 38.573312 MB written
    ("real", "random_2097152", "mixed", "9f3e9833cb893640"): 156143104,
    # profiles/k_real_rows_rocksalt_262144_near_df.md (double-float near pairs, the crystal
    # line's kernel): 14.301696 MB read + 0.612864 MB written
    ("real", "rocksalt_262144", "mixed", "9f3e9833cb893640"): 14914560,
}


def kernel_traffic(kernel, workload, precision):
    import hashlib
    src = {"real": "realspace.cu", "forward": "recip_tc.cu", "back": "recip_tc.cu"}.get(kernel)
    if not src:
        return None
    try:
        path = os.path.join(ROOT, "paper_1708_01135_gb300", "csrc", src)
        h = hashlib.sha256(open(path, "rb").read()).hexdigest()[:16]
    except OSError:
        return None
    return TRAFFIC.get((kernel, workload, precision, h))


def unique_pairs(n, L, rc):
    """Unique pairs within r_c of a homogeneous system: N (2 pi / 3) r_c^3 rho."""
    return n * (2.0 * math.pi / 3.0) * rc ** 3 * (n / L ** 3)


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
    oracle_sample.parts = (Fr, Fk)      # the two parts of the returned forces
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


def serving_systems(count, seed=1238):
    """The serving stream's systems, generated in spawned worker processes (before any CUDA
    call of this process)."""
    import multiprocessing as mp
    items = [(r, kind, n, rho, m, seed) for r, (kind, n, rho, m) in
             enumerate(W.request_sizes(count, 256, 65536, seed))]
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(16, os.cpu_count() or 4)) as pool:
        return pool.map(_gen_request, items)


def serving_summary(systems, local, precision, slots, tol, loads=(0.25, 0.5, 0.75, 0.9, 1.1),
                    comparators=True, seed=1238):
    """Serving stream: independent systems of uneven N (log-uniform in [256, 65536], half
    jittered rock-salt, half random neutral, density U[0.8, 1.2], each with its own box and
    tuned parameters), submitted to the continuous-batching server.  A closed-loop run (all
    requests at once) gives the saturation rate; Poisson arrivals at fractions of it give
    p50/p99 latency (submit -> result) and the aggregate particles/s.  With comparators, the
    same requests are also evaluated one at a time through plans on one stream (mixed and
    FP64: the sequential baseline at the same accuracy), and the server's results are
    compared with the one-at-a-time ones."""
    import torch
    torch.cuda.set_device(local)
    from paper_1708_01135_gb300 import Ewald, Server, tune
    dev = torch.device("cuda", local)
    reqs = []
    for pos, q, L in systems:
        rc, beta, km = tune(len(q), L, tol, r_c=min(0.5 * L, 4.0 * (len(q) / L ** 3) ** (-1.0 / 3.0)))
        reqs.append(dict(pos=torch.tensor(pos, device=dev), q=torch.tensor(q, device=dev),
                         F=torch.empty((len(q), 3), dtype=torch.float64, device=dev),
                         L=L, beta=beta, rc=rc, km=km, n=len(q)))
    count = len(reqs)
    total_n = sum(r["n"] for r in reqs)

    def run(srv, times):
        t0 = time.perf_counter()
        tickets = []
        for r, ta in zip(reqs, times):
            while time.perf_counter() - t0 < ta:
                time.sleep(0.0002)
            tickets.append(srv.submit(r["pos"], r["q"], r["F"], r["L"], r["beta"], r["rc"], r["km"],
                                      precision))
        res = [srv.wait(t, 600.0) for t in tickets]
        bad = [(i, x["status"]) for i, x in enumerate(res) if x["status"] != 0]
        if bad:
            raise RuntimeError(f"serving requests failed (index, status): {bad[:8]}")
        lat = np.array([x["t_done"] - x["t_submit"] for x in res]) * 1e3
        span = max(x["t_done"] for x in res) - min(x["t_submit"] for x in res)
        return lat, span

    srv = Server(max_slots=slots)
    run(srv, [0.0] * min(16, count))            # warm-up: plans, pools, module load
    lat, span = run(srv, [0.0] * count)         # closed loop: everything at once
    sat_rate = count / span
    F_srv = [r["F"].clone() for r in reqs]
    out = {"requests": count, "total_particles": total_n, "slots": slots, "tol": tol,
           "precision": precision,
           "saturation": {"requests_per_s": sat_rate, "particles_per_s": total_n / span,
                          "p50_ms": float(np.percentile(lat, 50)),
                          "p99_ms": float(np.percentile(lat, 99))}}
    rng = np.random.default_rng(seed + 7)
    for frac in loads:
        rate = frac * sat_rate
        times = np.cumsum(rng.exponential(1.0 / rate, size=count))
        lat, span = run(srv, list(times - times[0]))
        out[f"load_{frac}"] = {"arrival_per_s": rate, "p50_ms": float(np.percentile(lat, 50)),
                               "p99_ms": float(np.percentile(lat, 99)),
                               "particles_per_s": total_n / span}
    out["server"] = srv.stats()
    srv.close()
    if comparators:
        # one request at a time through a plan per request on one stream (no overlap), with
        # the precision of the server and with the plain FP64 path, at the same parameters
        for prec, key in ((precision, "sequential_same_precision"), ("fp64", "sequential_fp64")):
            E = torch.empty(4, dtype=torch.float64, device=dev)
            plans = [Ewald(r["L"], r["beta"], r["rc"], r["km"], prec) for r in reqs]
            Fs = [torch.empty_like(r["F"]) for r in reqs]
            for ew, r, F in zip(plans, reqs, Fs):        # warm-up (workspaces, graphs)
                ew.compute_async(r["pos"], r["q"], F, E)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for ew, r, F in zip(plans, reqs, Fs):
                ew.compute_async(r["pos"], r["q"], F, E)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            for ew in plans:
                ew.close()
            diff = max(math.sqrt(float(((a - b) ** 2).sum()) / float((b ** 2).sum()))
                       for a, b in zip(F_srv, Fs))
            out[key] = {"particles_per_s": total_n / dt, "seconds": dt,
                        "server_speedup": (total_n / dt) and (out["saturation"]["particles_per_s"]
                                                              / (total_n / dt)),
                        "max_rel_force_rms_server_vs_this": diff}
    return out


def run_serving(args, rank, world, local):
    """--workload serving: the serving summary as its own JSON line."""
    systems = serving_systems(args.requests)
    out = serving_summary(systems, local, args.precision, args.slots, args.serving_tol)
    if rank == 0:
        print(json.dumps({"metric": "ewald_serving", "unit": "ms / particles/s", "n_gpus": world,
                          "data": "synthetic", "results": out}), flush=True)


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
    if args.workload in NEAR_DF and not spme:
        ew.set_near_pairs(True)
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


def cpu_model():
    """The host CPU's model name (from /proc/cpuinfo or lscpu), and its core count."""
    name = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                k, _, v = line.partition(":")
                if k.strip() in ("model name", "Model Name", "CPU part") and v.strip():
                    name = v.strip()
                    break
    except OSError:
        pass
    try:
        r = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10)
        for line in r.stdout.splitlines():
            k, _, v = line.partition(":")
            if k.strip() == "Model name" and v.strip():
                name = v.strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return {"model": name, "cores": os.cpu_count()}


def oracle_one_thread():
    """The oracle on one host thread: a full evaluation of the 512-ion lattice and a sampled
    evaluation of the 32,768-ion system (S(k) on a subset of modes, forces of 64 particles,
    scaled as oracle_sample does)."""
    import oracle
    out = {}
    prev = oracle.num_threads()
    oracle.set_threads(1)
    try:
        for name in ("rocksalt_512", "random_32768"):
            pos, q, L = WORKLOADS[name][0]()
            n = len(q)
            rc, beta, kmax = PARAMS[name]
            if n <= 4096:
                t0 = time.perf_counter()
                oracle.ewald(pos, q, L, beta, rc, kmax)
                t = time.perf_counter() - t0
                note = "full evaluation"
            else:
                t, _, nt, _, _, note = oracle_sample(pos, q, L, beta, rc, kmax, 64,
                                                     S_given=np.zeros(len(oracle.kset_half(kmax)),
                                                                      dtype=complex),
                                                     max_sk_terms=2e8)
                note = (note.replace("(reciprocal forces from the GPU's S(k))",
                                     "(reciprocal forces against a stand-in S(k))")
                        + f"; forces of {nt} particles, scaled to {n}")
            out[name] = {"particles_per_s": n / t, "seconds_per_evaluation": t, "sample": note}
    finally:
        oracle.set_threads(prev)
    return out


def run_reference(args, rank, world):
    """The oracle (plain FP64 CPU Ewald) as it stands, on the host cores, on the same workload,
    metric and parameters (plain numbers, PARAMS): every step a bounded sample of one
    evaluation scaled to the whole (see oracle_sample).  Nothing from the library is loaded."""
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
    nt = targets
    for st in range(args.warmup + args.steps):
        full, wall, nt, _, _, note = oracle_sample(pos, q, L, beta, rc, kmax, targets, seed=st,
                                                   S_given=S0, max_sk_terms=max_terms)
        if st >= args.warmup:
            times.append(full)
    t = float(np.mean(times))
    value = n / t
    note = note.replace("(reciprocal forces from the GPU's S(k))",
                        "(reciprocal forces of the targets timed against a stand-in S(k) of "
                        "the same size)")
    one = oracle_one_thread() if not args.no_one_thread else None
    line = {
        "impl": "reference", "metric": "ewald_particles_per_s", "value": value,
        "unit": "particles/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "n": n, "L": L, "r_c": rc, "beta": beta,
                   "k_max": kmax, "tol": TOL},
        "cpu_baseline": {"value": value, "unit": "particles/s", "cores": oracle.num_threads(),
                         "kind": "oracle", "cpu": cpu_model(),
                         "sample": f"{note}; forces of {nt} random particles, scaled "
                                   f"to {n}"},
        "one_thread": one,
        "e2e": {"value": value, "unit": "particles/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def converged_params(L, p=4.3):
    """Cutoffs at which both truncation errors are ~exp(-p^2) ~ 1e-8 of the force: r_c = L/2
    (the largest the minimum image allows), beta = p / r_c, k_max = ceil(p beta L / pi)."""
    rc = 0.5 * L
    beta = p / rc
    return rc, beta, int(math.ceil(p * beta * L / math.pi))


def accuracy_converged(pos, q, L, F_gpu, n_targets=1024, seed=11):
    """Total relative RMS force error of a result against the oracle at converged cutoffs
    (converged_params), on a random subset of particles: the truncation error of the
    benchmark's parameters and the arithmetic error of the path together."""
    import oracle
    n = len(q)
    rng = np.random.default_rng(seed)
    sub = np.sort(rng.choice(n, size=min(n_targets, n), replace=False))
    rc, beta, kmax = converged_params(L)
    t0 = time.perf_counter()
    _, Fr, _ = oracle.real(pos, q, L, beta, rc, sub=sub)
    _, Fk, _, _, _ = oracle.recip(pos, q, L, beta, kmax, sub=sub)
    Fo = Fr + Fk
    d = F_gpu[sub] - Fo
    scale = math.sqrt(float((Fo ** 2).sum(axis=1).mean()))
    return {"rel_force_rms": float(np.sqrt((d ** 2).sum() / (Fo ** 2).sum())),
            "largest_particle_rel": float(np.sqrt((d ** 2).sum(axis=1)).max() / scale),
            "particles": int(len(sub)),
            "reference": {"r_c": rc, "beta": beta, "k_max": kmax,
                          "note": "FP64 oracle, minimum-image pairs of the subset and the "
                                  "k-space sum of all particles"},
            "cpu_seconds": time.perf_counter() - t0}


def structure_factor_error(pos, q, L, m, S_gpu, modes=1024, seed=12):
    """Relative error of the path's S(k) on random modes: |S_gpu - S_oracle| over
    sqrt(sum q^2) + |S| (the size of a random-phase sum), the largest and the RMS."""
    import oracle
    rng = np.random.default_rng(seed)
    sel = np.sort(rng.choice(len(m), size=min(modes, len(m)), replace=False))
    So = oracle.structure_factor(pos, q, L, m[sel])
    e = np.abs(S_gpu[sel] - So) / (np.sqrt((q ** 2).sum()) + np.abs(So))
    return {"max": float(e.max()), "rms": float(np.sqrt((e ** 2).mean())), "modes": int(len(sel))}


def kernel_rooflines(n, L, rc, kmax, precision, spme, times, pk, pk_kind, alu_peaks,
                     workload, alone=None):
    """Roofline of the three kernels that carry the method's work, each from its own CUDA
    event bracket (ewald_profile): achieved = algorithmic flop per launch / kernel time, where
    the algorithmic work is 40 flop per unique pair within r_c (real space), 8 flop per
    (particle, mode) term for the S(k) product and 10 for the back-scatter; peak = the measured
    bf16 dense rate (sustained) for tensor-core products, the measured FP32/FP64 FMA rate for
    CUDA-core kernels.  The list is ordered by kernel time, the first entry dominating.  With
    `alone` (the kernel times of evaluations of one part only), every entry also gives the
    kernel's rate when it does not share the SMs with the other branch."""
    fp64 = precision == "fp64"
    tc = precision in ("mixed", "mixed_bf16")
    alu = alu_peaks["fp64" if fp64 else "fp32"]
    alu_kind = ("measured here (ewald_fma_peak, "
                + ("FP64" if fp64 else "FP32") + " FMA loop on every SM)")
    tensor_peak = pk.get("bf16_tflops_sustained", pk.get("bf16_tflops"))
    tensor_kind = f"{pk_kind} bf16 dense sustained (the fp16 dense rate is equal)"
    nk = len_kset_half(kmax)
    out = []
    pairs = unique_pairs(n, L, rc)
    rows = [("real", "real-space pairs (a4)", times.get("real_kernel"), 40.0 * pairs,
             "40 flop per unique pair within r_c", "alu", alu, alu_kind)]
    if not spme:
        fwd_f, back_f = tensor_flops(n, kmax) if tc else simt_flops(n, kmax)
        rows.append(("forward", "structure-factor product (a5-a6)", times.get("recip_forward"),
                     8.0 * n * nk, "8 flop per (particle, mode) term",
                     "tensor" if tc else "alu", tensor_peak if tc else alu,
                     tensor_kind if tc else alu_kind, fwd_f))
        rows.append(("back", "back-scatter product (a8)", times.get("backscatter_kernel"),
                     10.0 * n * nk, "10 flop per (particle, mode) term",
                     "tensor" if tc else "alu", tensor_peak if tc else alu,
                     tensor_kind if tc else alu_kind, back_f))
    for row in rows:
        key, name, ms, flop, work, bound, peak, kind = row[:8]
        if not ms or ms <= 0:
            continue
        achieved = flop / (ms * 1e-3) / 1e12
        r = {"kernel": name, "bound": bound, "achieved": achieved, "peak": peak,
             "unit": "TFLOP/s", "frac": achieved / peak, "ms": ms, "work": work,
             "flop_per_launch": flop, "peak_kind": kind,
             "traffic": None if spme else kernel_traffic(key, workload, precision)}
        akey = {"real": "real_kernel", "forward": "recip_forward", "back": "backscatter_kernel"}[key]
        ms_a = (alone or {}).get(akey)
        if ms_a and ms_a > 0:
            r["ms_alone"] = ms_a
            r["frac_alone"] = flop / (ms_a * 1e-3) / 1e12 / peak
        if len(row) > 8 and bound == "tensor":
            issued = row[8]
            r["issued_tensor_flop"] = issued
            r["issued_tensor_frac"] = issued / (ms * 1e-3) / 1e12 / peak
        out.append(r)
    out.sort(key=lambda r: -r["ms"])
    return out


def time_steps(ew, tp, tq, F, E, flush, stream, steps):
    """Device time (ms, mean) of `steps` evaluations, each bracketed by CUDA events on the
    launching stream after an L2 flush."""
    import torch
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    for st in range(steps):
        flush.fill_(float(st))
        ev0[st].record(stream)
        ew.compute_async(tp, tq, F, E)
        ev1[st].record(stream)
    torch.cuda.synchronize()
    return float(np.mean([a.elapsed_time(b) for a, b in zip(ev0, ev1)]))


def profiled_times(ew, tp, tq, F, E, flush, reps, parts=None):
    """Median kernel and stage times (ms) over `reps` evaluations with the plan's profiling
    events recorded (those evaluations run launch by launch instead of as a graph); parts
    selects the real-space or reciprocal part alone (default: the whole evaluation)."""
    from paper_1708_01135_gb300 import PART_ALL
    stage = {}
    ew.profile(1)
    for st in range(reps):
        flush.fill_(float(st))
        ew.compute_async(tp, tq, F, E, parts=PART_ALL if parts is None else parts)
        t, _ = ew.profile(-1)           # synchronises on the last stage event
        for k, v in t.items():
            stage.setdefault(k, []).append(v)
    ew.profile(0)
    return {k: float(np.median(v)) for k, v in stage.items()}


def measure_workload(args, workload, local, world, dev, flush, alu_peaks, steps, warmup,
                     e2e=True, spme_spec="", accuracy="full"):
    """One workload on this rank's GPU: device-timed evaluations, kernel times, the end-to-end
    figure through the host-buffer entry point, kernel rooflines and (rank 0) accuracy
    against the oracle.  Returns the fields of its JSON line and the inputs (for reuse)."""
    import torch
    from paper_1708_01135_gb300 import Ewald
    gen, _ = WORKLOADS[workload]
    pos, q, L = gen()
    n = len(q)

    class A:
        pass
    a = A()
    a.workload, a.spme, a.spme_rc = workload, spme_spec, args.spme_rc
    rc, beta, kmax, spme = run_params(a, n, L)
    tp = torch.tensor(pos, device=dev)
    tq = torch.tensor(q, device=dev)
    F = torch.empty((n, 3), dtype=torch.float64, device=dev)
    E = torch.empty(4, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    ew = Ewald(L, beta, rc, kmax, args.precision)
    if spme:
        ew.set_spme(spme["K"], spme["order"])
    if workload in NEAR_DF and not spme:
        ew.set_near_pairs(True)
    # the clock sampler runs through the warm-up (at least ~0.5 s of back-to-back steps) and
    # the timed steps, so that its samples see the GPU under this workload's load
    clocks = ClockSampler(local)
    clocks.start()
    t_warm = time.perf_counter()
    w = 0
    while w < warmup or time.perf_counter() - t_warm < 0.5:
        ew.compute_async(tp, tq, F, E)
        w += 1
        if w % 8 == 0:
            torch.cuda.synchronize()
    torch.cuda.synchronize()
    if ew.status() != 0:
        raise RuntimeError("warm-up evaluation reported an error")
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ms = time_steps(ew, tp, tq, F, E, flush, stream, steps)
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    if ew.status() != 0:
        raise RuntimeError("timed evaluation reported an error")
    _, per_step = ew.profile(-1)        # kernels of one evaluation (one graph launch replays them)
    times = profiled_times(ew, tp, tq, F, E, flush, min(steps, 10))
    # each branch alone (the other part not evaluated), for the kernels' own rates
    from paper_1708_01135_gb300 import PART_REAL, PART_RECIP
    alone = {"real_kernel": profiled_times(ew, tp, tq, F, E, flush, 3, PART_REAL).get("real_kernel")}
    rt = profiled_times(ew, tp, tq, F, E, flush, 3, PART_RECIP)
    alone["recip_forward"] = rt.get("recip_forward")
    alone["backscatter_kernel"] = rt.get("backscatter_kernel")
    ms = max_over_ranks(ms, world, dev)
    value = whole_job_rate(n, ms, world)
    out = {"n": n, "L": L, "r_c": rc, "beta": beta, "k_max": kmax, "spme": spme,
           "tune_tol": TUNE_TOL.get(workload, TOL),
           "near_pairs": "fp32" if spme else near_pairs_of(workload),
           "value": value, "ms_per_step": ms, "steps": steps, "warmup": w,
           "gpu_launches": per_step * steps, "clocks": clk}
    Fg = F.cpu().numpy()
    if e2e:
        # end to end through the host-buffer entry point (pinned host memory)
        hp = torch.tensor(pos).pin_memory().numpy()
        hq = torch.tensor(q).pin_memory().numpy()
        hf = torch.empty((n, 3), dtype=torch.float64).pin_memory().numpy()
        for _ in range(2):
            ew.compute_host(hp, hq, hf)
        torch.cuda.synchronize()
        e_times = []
        for _ in range(max(3, steps // 2)):
            t0 = time.perf_counter()
            ew.compute_host(hp, hq, hf)
            e_times.append(time.perf_counter() - t0)
        out["e2e"] = {"value": whole_job_rate(n, max_over_ranks(1e3 * float(np.mean(e_times)),
                                                                world, dev), world),
                      "unit": "particles/s", "h2d_bytes_per_step": 32 * n,
                      "d2h_bytes_per_step": 24 * n + 32}
        Fg = np.array(hf)
    pk, pk_kind = peaks()
    roofs = kernel_rooflines(n, L, rc, kmax, args.precision, spme, times, pk, pk_kind,
                             alu_peaks, workload, alone)
    out["roofline_kernels"] = roofs
    out["kernel_ms"] = {k: times.get(k) for k in ("real_kernel", "recip_forward",
                                                   "backscatter_kernel", "finalize_kernels",
                                                   "binning")}
    out["stage_spans_ms"] = {k: v for k, v in times.items() if k not in out["kernel_ms"]}
    nk = 0 if spme else len_kset_half(kmax)
    pairs = unique_pairs(n, L, rc)
    out["algorithmic"] = {"unique_pairs": pairs, "recip_terms": float(n) * nk,
                          "flop": 40.0 * pairs + 18.0 * n * nk,
                          "tflops_over_step": (40.0 * pairs + 18.0 * n * nk) / (ms * 1e-3) / 1e12,
                          "note": ("SPME mesh work not counted" if spme else
                                   "40 flop per unique pair, 18 per (particle, mode) term")}
    Sg = None if spme else ew.structure_factor()
    m = None if spme else ew.kset()
    # the real-space and reciprocal parts on their own (for the error of each part)
    from paper_1708_01135_gb300 import PART_REAL, PART_RECIP
    F_parts = {}
    if not spme and accuracy != "none":
        for nm, pt in (("real", PART_REAL), ("recip", PART_RECIP)):
            ew.compute_async(tp, tq, F, E, parts=pt)
            F_parts[nm] = F.cpu().numpy()
    ew.close()
    rank = int(os.environ.get("RANK", "0"))
    if rank == 0 and world == 1 and accuracy != "none":
        import oracle
        acc = {}
        if spme:
            full, wall, nt, sub, Fo, note = spme_oracle_sample(pos, q, L, beta, rc, spme["K"],
                                                               spme["order"], args.cpu_targets)
            acc["same_parameters"] = {
                "rel_force_rms": float(np.sqrt(((Fg[sub] - Fo) ** 2).sum() / (Fo ** 2).sum())),
                "particles": int(nt),
                "reference": "FP64 SPME oracle at the same (beta, r_c, K, p)"}
        else:
            full, wall, nt, sub, Fo, note = oracle_sample(pos, q, L, beta, rc, kmax,
                                                          args.cpu_targets, S_given=Sg)
            sk_all = note.startswith(f"S(k) over all {n} particles and all")
            acc["same_parameters"] = {
                "rel_force_rms": float(np.sqrt(((Fg[sub] - Fo) ** 2).sum() / (Fo ** 2).sum())),
                "particles": int(nt),
                "reference": ("FP64 oracle at the same (beta, r_c, k_max), S(k) of the oracle"
                              if sk_all else
                              "FP64 oracle at the same (beta, r_c, k_max); its reciprocal "
                              "forces use this path's S(k), whose own error is "
                              "structure_factor_error")}
            acc["structure_factor_error"] = structure_factor_error(pos, q, L, m, Sg)
            if F_parts:
                Fr_o, Fk_o = oracle_sample.parts
                scale = float(np.sqrt((Fo ** 2).sum()))
                acc["by_part"] = {
                    "real": float(np.sqrt(((F_parts["real"][sub] - Fr_o) ** 2).sum())) / scale,
                    "recip": float(np.sqrt(((F_parts["recip"][sub] - Fk_o) ** 2).sum())) / scale,
                    "note": "RMS error of each part over the RMS total force of the sample"}
        out["cpu_baseline"] = {"value": n / full, "unit": "particles/s",
                               "cores": oracle.num_threads(), "kind": "oracle",
                               "cpu": cpu_model(),
                               "sample": f"{note}; forces of {nt} random particles, scaled "
                                         f"to {n} ({wall:.1f} s of CPU work)"}
        if accuracy == "full" and not spme:
            acc["total_vs_converged"] = accuracy_converged(pos, q, L, Fg,
                                                           n_targets=args.converged_targets)
            acc["meets_tolerance"] = acc["total_vs_converged"]["rel_force_rms"] <= TOL
        out["accuracy"] = acc
    return out, (pos, q, L, tp, tq)


def run_capture(args, local):
    """--capture K: K evaluations of the workload, every kernel a separate launch (the plan's
    profiling mode), for kernel captures under a profiler; prints one status line."""
    import torch
    torch.cuda.set_device(local)
    from paper_1708_01135_gb300 import Ewald
    pos, q, L = WORKLOADS[args.workload][0]()
    n = len(q)
    rc, beta, kmax, spme = run_params(args, n, L)
    dev = torch.device("cuda", local)
    tp, tq = torch.tensor(pos, device=dev), torch.tensor(q, device=dev)
    F = torch.empty((n, 3), dtype=torch.float64, device=dev)
    E = torch.empty(4, dtype=torch.float64, device=dev)
    with Ewald(L, beta, rc, kmax, args.precision) as ew:
        if spme:
            ew.set_spme(spme["K"], spme["order"])
        if args.workload in NEAR_DF and not spme:
            ew.set_near_pairs(True)
        ew.profile(1)
        for _ in range(args.capture):
            ew.compute_async(tp, tq, F, E)
        torch.cuda.synchronize()
        st = ew.status()
    print(json.dumps({"capture": args.capture, "workload": args.workload, "status": st}))
    if st != 0:
        raise RuntimeError("evaluation reported an error")


def run_capture_serving(args, local):
    """--workload serving --capture K: the first K requests of the serving stream submitted at
    once to a server of --slots slots (tol --serving-tol), for launch lists under a profiler;
    prints one status line."""
    systems = serving_systems(args.capture)
    import torch
    torch.cuda.set_device(local)
    from paper_1708_01135_gb300 import Server, tune
    dev = torch.device("cuda", local)
    reqs = []
    for pos, q, L in systems:
        rc, beta, km = tune(len(q), L, args.serving_tol,
                            r_c=min(0.5 * L, 4.0 * (len(q) / L ** 3) ** (-1.0 / 3.0)))
        reqs.append((torch.tensor(pos, device=dev), torch.tensor(q, device=dev),
                     torch.empty((len(q), 3), dtype=torch.float64, device=dev), L, beta, rc, km))
    srv = Server(max_slots=args.slots)
    try:
        tickets = [srv.submit(p, q, F, L, b, rc, km, args.precision) for p, q, F, L, b, rc, km in reqs]
        res = [srv.wait(t, 600.0) for t in tickets]
    finally:
        srv.close()
    st = [r["status"] for r in res]
    print(json.dumps({"capture": args.capture, "workload": "serving", "n": [len(r[1]) for r in reqs],
                      "status": st}))
    if any(st):
        raise RuntimeError("a serving request failed")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default="random_2097152", choices=sorted(WORKLOADS) + ["serving"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64", "fp32", "mixed_bf16"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-targets", type=int, default=2048)
    ap.add_argument("--converged-targets", type=int, default=1024)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-one-thread", action="store_true")
    ap.add_argument("--extras", default="rocksalt_262144,serving",
                    help="comma list of extra keys beside the line: rocksalt_262144, serving ('' for none)")
    ap.add_argument("--requests", type=int, default=256)
    ap.add_argument("--extra-requests", type=int, default=128,
                    help="requests of the serving summary beside the line")
    ap.add_argument("--slots", type=int, default=8)
    ap.add_argument("--serving-tol", type=float, default=1e-6)
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
    ap.add_argument("--peaks", action="store_true",
                    help="print only the measured FP32/FP64 FMA rates of the GPU")
    ap.add_argument("--capture", type=int, default=0,
                    help="for profiler captures: run this many evaluations launch by launch "
                         "(no graph replay, no timing) and exit")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    rank, world, local = dist_env()

    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload == "serving" and args.capture:
        return run_capture_serving(args, local)
    if args.workload == "serving":
        return run_serving(args, rank, world, local)
    if args.md:
        return run_md(args, rank, world, local)

    if args.capture:
        return run_capture(args, local)
    extras = [x for x in args.extras.split(",") if x] if (rank == 0 and world == 1) else []
    systems = serving_systems(args.extra_requests) if "serving" in extras else None

    import torch
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1708_01135_gb300 import Ewald, fma_peak
    dev = torch.device("cuda", local)
    alu_peaks = {"fp32": fma_peak("fp32"), "fp64": fma_peak("fp64")}
    if args.peaks:
        if rank == 0:
            print(json.dumps({"metric": "fma_peak", "unit": "TFLOP/s", **alu_peaks}), flush=True)
        return
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    res, (pos, q, L, tp, tq) = measure_workload(args, args.workload, local, world, dev, flush,
                                                alu_peaks, args.steps, args.warmup,
                                                spme_spec=args.spme,
                                                accuracy="none" if args.no_cpu_baseline else "full")
    n = res["n"]
    ms = res["ms_per_step"]

    # the plain FP64 GPU path on the same system and parameters
    fp64 = None
    if args.precision != "fp64" and n <= args.fp64_max_n:
        F = torch.empty((n, 3), dtype=torch.float64, device=dev)
        E = torch.empty(4, dtype=torch.float64, device=dev)
        with Ewald(L, res["beta"], res["r_c"], res["k_max"], "fp64") as ew64:
            for _ in range(2):
                ew64.compute_async(tp, tq, F, E)
            torch.cuda.synchronize()
            ms64 = time_steps(ew64, tp, tq, F, E, flush, torch.cuda.current_stream(), 3)
            if ew64.status() != 0:
                raise RuntimeError("FP64 evaluation reported an error")
        fp64 = {"value": world * n / (ms64 * 1e-3), "unit": "particles/s", "ms_per_step": ms64,
                "steps": 3, "speedup_of_this_line": ms64 / ms}
    spme = res["spme"]
    if rank == 0 and spme and spme["classical_k_max"] <= 127:
        # the mesh error of SPME: its forces against the classical k-space sum at the same
        # beta and r_c (the tensor-core path)
        F = torch.empty((n, 3), dtype=torch.float64, device=dev)
        with Ewald(L, res["beta"], res["r_c"], res["k_max"], args.precision) as ew:
            ew.set_spme(spme["K"], spme["order"])
            ew.compute_async(tp, tq, F, torch.empty(4, dtype=torch.float64, device=dev))
            Fs = F.cpu().numpy()
        with Ewald(L, res["beta"], res["r_c"], res["k_max"], "mixed") as ewc:
            ewc.compute_async(tp, tq, F, torch.empty(4, dtype=torch.float64, device=dev))
            Fc = F.cpu().numpy()
        spme["vs_classical_rel_force_rms"] = float(np.sqrt(((Fs - Fc) ** 2).sum() / (Fc ** 2).sum()))
    del tp, tq

    extra = {}
    for x in extras:
        if x == "serving":
            extra["serving"] = serving_summary(systems, local, args.precision, args.slots,
                                               args.serving_tol, loads=(0.5, 0.9))
        elif x in WORKLOADS and x != args.workload:
            r, _ = measure_workload(args, x, local, world, dev, flush, alu_peaks,
                                    min(args.steps, 10), 3, e2e=False,
                                    accuracy="none" if args.no_cpu_baseline else "sample")
            r.pop("clocks", None)
            extra[x] = r
    if rank == 0:
        roofs = res["roofline_kernels"]
        line = {
            "metric": "ewald_particles_per_s", "value": res["value"], "unit": "particles/s",
            "n_gpus": world, "steps": args.steps, "warmup": res["warmup"], "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"mixed": "fp32 pairs + fp16x2 tensor products (fp32 accum) + f64 reductions",
                      "mixed_bf16": "fp32 pairs + bf16x2 tensor products (fp32 accum) + f64 reductions",
                      "fp64": "f64", "fp32": "f32 (f64 reductions)"}[args.precision],
            "data": "synthetic",
            "config": {"workload": args.workload, "n": n, "L": L, "r_c": res["r_c"],
                       "beta": res["beta"], "k_max": res["k_max"], "tol": TOL,
                       "tune_tol": TUNE_TOL.get(args.workload, TOL),
                       "near_pairs": "fp32" if spme else near_pairs_of(args.workload),
                       "precision": args.precision,
                       "reciprocal": ({"method": "spme", **spme} if spme else
                                      {"method": "classical k-space sum"}),
                       "l2": "flushed before every step (512 MiB write)",
                       "parallelism": f"replicas x{world}"},
            "e2e": res.get("e2e"),
            "gpu_launches": res["gpu_launches"],
            "roofline": roofs[0] if roofs else None,
            "roofline_kernels": roofs,
            "kernel_ms": res["kernel_ms"],
            "stage_spans_ms": res["stage_spans_ms"],
            "algorithmic": res["algorithmic"],
            "peaks_measured": {**alu_peaks, "unit": "TFLOP/s",
                               "how": "ewald_fma_peak: FMA loop on every SM, CUDA events"},
            "clocks": res["clocks"],
            "cpu_baseline": res.get("cpu_baseline"),
            "accuracy": res.get("accuracy"),
            "fp64_gpu": fp64,
            **extra,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
