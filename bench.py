#!/usr/bin/env python
"""Benchmark of the H-matrix BEM hot path on GB300.

Workload (default): Laplace single- and double-layer P0 on the icosphere of
level 6 (81,920 triangles), vertices jittered by 5% of the mean edge length
(uniform, seeded), cluster leaf 32, eta 1.2, ACA eps 1e-5, FP32 quadrature
with FP64 accumulation ("mixed"), all admissible blocks in one persistent
launch per operator.

One step = for both operators: hmat_assemble (near field: regular pairs +
Sauter-Schwab singular pairs; far field: persistent ACA) and one hmat_matvec
with a seeded N(0,1) vector.  The mesh geometry and the block tree are built
once per mesh before the timed region (they do not depend on the operator);
the end-to-end figure `e2e` rebuilds everything from host arrays every step.

Metric: Galerkin integrals/s = entries evaluated per step (all near-field
entries + every entry the ACA requested) / step time.  The FP64 path of the
same step is timed after the run for the mixed-vs-FP64 comparison.  On one
GPU the line also carries records of the level-9 sphere (`c4`: 5.24 M
triangles, assembly and 100 products), the Helmholtz ellipsoid (`c3`: 499,280
triangles, complex ACA) and a short request stream (`serving`: p50 / p99).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Galerkin integrals/s & H-assembly time; p50/p99 latency; mixed vs FP64 at tol"
UNIT = "integrals/s"
WORKLOAD = {"workload": "laplace_slp_dlp_p0_icosphere_l6_jitter5pct", "n_triangles": 81920,
            "leaf_size": 32, "eta": 1.2, "aca_eps": 1e-5, "operators": ["SLP", "DLP"],
            "quadrature": "6-pt degree-4 regular, Sauter-Schwab 4^4 GL singular",
            "precision": "BEM_MIXED: FP32 regular quadrature with float-float accumulation; FP64 singular pairs, ACA pivots, residual updates and norms",
            "l2": "flushed between timed steps (256 MiB write)"}
LEAF, ETA, EPS = 32, 1.2, 1e-5

# GB300 unit counts and the maximum SM clock (profiling recipe)
N_SM, MUFU_PER_SM_CLK, FP32_PER_SM_CLK, FP64_PER_SM_CLK, SM_MAX_MHZ = 152, 16, 128, 2, 2070.0
FP64_TFLOPS_NOMINAL = 1.25

# distance classes of the regular rule (bem_set_quadrature) that the autotuner
# chose for the default workload: python -m paper_1711_01897_gb300.autotune
# --level 6 --quadrature (eps 1e-5, products within 0.5 eps of the 6-point
# products); the C2 line reports them beside the paper's 6-point rule
AUTOTUNED_RHO_L6 = (4.0, 24.0)
# ACA work shapes (bem_set_tuning: warp_max_rows, lane_max_rows) the autotuner
# chose for the Helmholtz ellipsoid workload: python -m
# paper_1711_01897_gb300.autotune --ellipsoid-nu 158 --eps 1e-4 (confirmation
# round, three repetitions: 1325 ms against 1592 ms for the library default;
# single timings of this launch vary by up to 15 %)
AUTOTUNED_SHAPES_C3 = (1280, 48)

# DRAM bytes of the two k_aca launches of one level-6 step (SLP read, write;
# DLP read, write), dram__bytes_read.sum + dram__bytes_write.sum from one ncu
# capture of the current kernel (re-capture when k_aca changes)
ACA_TRAFFIC_BYTES_PER_STEP_L6 = (5.093048832 + 1.826512640 + 11.758856704 + 2.819681024) * 1e9


def rank_jitter_seed(rank: int) -> int:
    """Each rank solves its own problem: the workload's mesh with a
    rank-dependent jitter seed (rank 0 is the single-GPU workload)."""
    return 1001 + 7919 * rank


def reduce_over_ranks(total_ms: float, integrals: float, dist, device):
    """Whole-job figures of the weakly scaled run: the timed region lasts as
    long as the slowest rank (max), and the integrals of all ranks add up."""
    import torch
    t = torch.tensor([total_ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    e = torch.tensor([float(integrals)], device=device, dtype=torch.float64)
    dist.all_reduce(e, op=dist.ReduceOp.SUM)
    return float(t.item()), float(e.item())


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    """nvidia-smi sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        out_dir = os.environ.get("BEM_BENCH_OUT", os.path.join(ROOT, "bench_out"))
        self.path = os.path.join(out_dir, f"clocks_bench_gpu{gpu}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) < 9:
                    continue
                try:
                    sm.append(float(p[1]))
                    smax.append(float(p[2]))
                except ValueError:
                    continue
                for n, v in zip(names, p[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                "samples": len(sm), "reasons": sorted(reasons)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


# Algorithmic FP32 instructions and MUFU operations per Green's function
# evaluation of the regular quadrature (36 evaluations per entry):
# SLP 3 FADD (x - y) + 3 FMUL/FFMA (r^2) + 1 FFMA (w / r) and one rsqrt;
# DLP adds the normal product (3) and r^-3 (2).
QUAD_FP32_PER_EVAL = {0: 7, 1: 12}


def quadrature_roofline(bem, mesh, V, T, dev, stream, flush, reps: int = 3, peaks=None):
    """A3 alone: one bem_entries call over two opposite caps of the sphere
    (every pair regular and well separated), timed with CUDA events on the
    launching stream, against the FP32 and MUFU pipe peaks (measured on the
    box by bem_measure_peaks when given, else derived from unit counts)."""
    import torch
    cen = V[T].mean(axis=1)
    test = np.nonzero(cen[:, 2] > 0.5)[0].astype(np.int32)
    trial = np.nonzero(cen[:, 2] < -0.5)[0].astype(np.int32)
    ti = torch.from_numpy(test).to(dev)
    tj = torch.from_numpy(trial).to(dev)
    out = torch.empty(len(test) * len(trial), dtype=torch.float64, device=dev)
    ents = float(len(test)) * len(trial)
    f_fp32_d = N_SM * FP32_PER_SM_CLK * SM_MAX_MHZ * 1e6 / 1e9   # Gop/s
    f_mufu_d = N_SM * MUFU_PER_SM_CLK * SM_MAX_MHZ * 1e6 / 1e9
    f_fp32 = peaks["fp32_fma_per_s"] / 1e9 if peaks else f_fp32_d
    f_mufu = peaks["mufu_rsqrt_per_s"] / 1e9 if peaks else f_mufu_d
    res = {"kernel": "k_entries (bem_entries, mixed precision, regular far pairs)",
           "peak_source": ("measured on this box (bem_measure_peaks: FFMA and MUFU rsqrt "
                           "throughput kernels)" if peaks else "derived from unit counts"),
           "peaks_derived_gops": {"fp32": f_fp32_d, "mufu": f_mufu_d},
           "entries_per_launch": ents, "evals_per_entry": 36,
           "timing": "CUDA events around one bem_entries call (one k_entries launch, "
                     "3 empty singular launches); L2 flushed before each"}
    for op, name in ((bem.SLP, "SLP"), (bem.DLP, "DLP")):
        bem.bem_entries(mesh.handle, op, 0.0, bem.MIXED, ti, tj, out, stream.cuda_stream)  # warm-up
        ms = []
        for _ in range(reps):
            flush.fill_(3)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            bem.bem_entries(mesh.handle, op, 0.0, bem.MIXED, ti, tj, out, stream.cuda_stream)
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        t = float(np.median(ms)) * 1e-3
        fp32 = ents * 36 * QUAD_FP32_PER_EVAL[op] / t / 1e9
        mufu = ents * 36 / t / 1e9
        fr32, frmu = fp32 / f_fp32, mufu / f_mufu
        res[name] = {"ms": t * 1e3, "entries_per_s": ents / t,
                     "fp32": {"achieved": fp32, "peak": f_fp32, "unit": "Gop/s", "frac": fr32},
                     "mufu": {"achieved": mufu, "peak": f_mufu, "unit": "Gop/s", "frac": frmu},
                     "binding": "fp32" if fr32 >= frmu else "mufu", "frac": max(fr32, frmu)}
    del out
    torch.cuda.empty_cache()
    return res


# ---------------------------------------------------------------------------
# CPU oracle arm (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------

def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the ISA)."""
    import platform
    import subprocess
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.split(":")[0].strip().lower() == "model name":
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.machine()


def oracle_sample_rate(V, T, seconds_target: float = 15.0, seed: int = 7, nthreads: int = 0,
                       ops=None, k: float = 0.0, eps: float = EPS):
    """Times the oracle's H-matrix assembly (Algorithm "H-Matrix Assembly":
    dense near blocks + ACA blocks, SLP and DLP) on a seeded sample of the
    workload's leaf blocks; returns integrals/s, threads, description."""
    import oracle
    ct = oracle.cluster_tree(V, T, LEAF)
    bl = oracle.block_list(ct, oracle.block_tree(ct, ETA))
    rng = np.random.default_rng(seed)
    far = np.nonzero(bl[:, 4] == 1)[0]
    near = np.nonzero(bl[:, 4] == 0)[0]
    # stratified: the same fraction of near and far blocks, growing until the
    # sample takes about seconds_target
    frac, total_entries, total_t = 0.002, 0, 0.0
    used = 0
    while True:
        nf = max(1, int(frac * far.size))
        nn = max(1, int(frac * near.size))
        ids = np.concatenate([rng.choice(far, nf, replace=False), rng.choice(near, nn, replace=False)])
        t0 = time.perf_counter()
        ent = 0
        for op in (ops if ops is not None else (oracle.SLP, oracle.DLP)):
            hm = oracle.hmat_assemble(V, T, op, k, LEAF, ETA, eps, block_ids=ids, nthreads=nthreads)
            ent += hm.entries_evaluated
        dt = time.perf_counter() - t0
        total_entries += ent
        total_t += dt
        used += ids.size
        if total_t >= seconds_target or frac >= 0.5:
            break
        frac = min(0.5, frac * max(2.0, seconds_target / max(dt, 1e-3) * 0.7))
    names = "+".join({0: "SLP", 1: "DLP", 2: "ADLP"}[o] for o in (ops if ops is not None else (0, 1)))
    return (total_entries / total_t, nthreads if nthreads > 0 else oracle.num_threads(),
            f"{used} of {bl.shape[0]} leaf blocks (near and admissible, seeded stratified sample), "
            f"{names}{', k = %g' % k if k else ''}, FP64 oracle, {total_entries} integrals in "
            f"{total_t:.1f} s")


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    from paper_1711_01897_gb300 import meshes
    V, T = meshes.workload_mesh("sphere_l6_jitter")
    times, vals = [], []
    for s in range(args.warmup + args.steps):
        rate, cores, sample = oracle_sample_rate(V, T, seconds_target=args.ref_seconds, seed=100 + s)
        if s >= args.warmup:
            vals.append(rate)
    value = float(np.mean(vals))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": None,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": WORKLOAD,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "cpu": cpu_model(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def run_gpu(args):
    import torch
    from paper_1711_01897_gb300 import bem, meshes

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    torch.cuda.init()
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    sptr = stream.cuda_stream

    extras = {}
    if ws == 1 and not args.no_c4:
        # the largest single-GPU configuration (level 9, 100 products) first,
        # as its own job would run: its host tree build and upload touch
        # gigabytes of fresh host memory, and measured 0.75 s in a fresh
        # process against 1.06 s after the legs below (same library)
        extras["c4"] = large_record(args, LARGE["c4"], steps=1, warmup=1, cpu_baseline=False)
        torch.cuda.empty_cache()
    if ws == 1 and not args.no_c3:
        # the Helmholtz ellipsoid (complex ACA on the autotuned work shapes);
        # the library's work shapes are put back for the legs below
        from paper_1711_01897_gb300 import bem as _bem
        saved = _bem.bem_get_tuning()
        try:
            extras["c3"] = large_record(args, LARGE["c3"], steps=2, warmup=1, cpu_baseline=False)
        finally:
            _bem.bem_set_tuning(saved["warp_max_rows"], saved["lane_max_rows"], saved["use_graphs"])
        torch.cuda.empty_cache()

    # one problem (the workload's mesh); with N ranks each assembles and
    # applies the block rows of its part of a cost-balanced row partition
    # (hmat_build_tree_part), gathering x and the rows of y with all_gathers
    # (no reduction)
    V, T = meshes.icosphere_level(args.level)
    V = meshes.jitter(V, T, 0.05, rank_jitter_seed(0))
    n = T.shape[0]
    mesh = bem.Mesh(V, T)
    hs = {op: bem.HMatrix(mesh, LEAF, ETA, parts=ws, part=rank) for op in (bem.SLP, bem.DLP)}
    rng = np.random.default_rng(5)
    x_host = rng.normal(size=n)
    x = torch.from_numpy(x_host).to(dev)
    ys = {op: torch.zeros(n, dtype=torch.float64, device=dev) for op in hs}
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    if ws > 1:
        from paper_1711_01897_gb300 import sharding
        _, perm_np = hs[bem.SLP].blocks()
        perm_t = torch.from_numpy(perm_np.astype(np.int64)).to(dev)
        rb, re = hs[bem.SLP].part_rows()
        rows = torch.tensor([rb, re], dtype=torch.int64, device=dev)
        allr = [torch.empty_like(rows) for _ in range(ws)]
        dist.all_gather(allr, rows)
        bounds = [int(r[0]) for r in allr] + [int(allr[-1][1])]
        x_seg = x[perm_t][rb:re].contiguous()     # this rank's rows of x

    def product(op, h):
        if ws == 1:
            bem.hmat_matvec(h.handle, x, ys[op], 1, sptr)
            return
        xc = sharding.gather_segments(x_seg, bounds, dist)
        xf = torch.empty_like(xc)
        xf[perm_t] = xc
        bem.hmat_matvec(h.handle, xf, ys[op], 1, sptr)
        yc = sharding.gather_segments(ys[op][perm_t][rb:re].contiguous(), bounds, dist)
        ys[op][perm_t] = yc

    def step(prec):
        ent = 0
        for op, h in hs.items():
            bem.hmat_assemble(h.handle, op, 0.0, EPS, prec, sptr)
            product(op, h)
        for op, h in hs.items():
            st = h.stats()
            ent += st["near_entries"] + st["far_entries"]
        return ent

    for _ in range(args.warmup):
        step(bem.MIXED)
        flush.fill_(1)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    clocks = Clocks(local)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    phase = {"near_regular": 0.0, "singular": 0.0, "aca": 0.0}
    launches0 = bem.bem_kernel_launches()
    ents = 0
    torch.cuda.synchronize()
    for s in range(args.steps):
        flush.fill_(s & 0xff)
        ev[s][0].record(stream)
        ents += step(bem.MIXED)
        ev[s][1].record(stream)
        for h in hs.values():
            st = h.stats()
            phase["near_regular"] += st["time_near_regular_ms"]
            phase["singular"] += st["time_singular_ms"]
            phase["aca"] += st["time_far_ms"]
    torch.cuda.synchronize()
    launches = bem.bem_kernel_launches() - launches0
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = float(np.sum(step_ms))
    if ws > 1:
        total_ms, ents_all = reduce_over_ranks(total_ms, ents, dist, dev)
    else:
        ents_all = float(ents)
    value = ents_all / (total_ms * 1e-3)
    st_slp, st_dlp = hs[bem.SLP].stats(), hs[bem.DLP].stats()
    y_mixed = {op: ys[op].cpu().numpy().copy() for op in hs}

    # FP64 path of the same step (after the timed region)
    fp64_ms = []
    for r in range(2):
        flush.fill_(7)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step(bem.FP64)
        b.record(stream)
        torch.cuda.synchronize()
        fp64_ms.append(a.elapsed_time(b))
    y_fp64 = {op: ys[op].cpu().numpy().copy() for op in hs}
    mixed_vs_fp64 = {
        "fp64_ms_per_step": float(np.min(fp64_ms)),
        "mixed_ms_per_step": float(np.median(step_ms)),
        "speedup": float(np.min(fp64_ms) / np.median(step_ms)),
        "matvec_rel_diff": {("SLP" if op == 0 else "DLP"): float(
            np.linalg.norm(y_mixed[op] - y_fp64[op]) / np.linalg.norm(y_fp64[op])) for op in hs},
        "tolerance": 2 * EPS}

    # the same step in BEM_MIXED_SP (the norm's dot products and the Laplace
    # singular integrands in single precision as well), products against the
    # FP64 step above
    sp_ms, sp_ents, sp_phase = [], 0, {"singular": 0.0, "aca": 0.0}
    for _ in range(args.warmup):
        step(bem.MIXED_SP)
        flush.fill_(1)
    torch.cuda.synchronize()
    for s in range(args.steps):
        flush.fill_(s & 0xff)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sp_ents += step(bem.MIXED_SP)
        b.record(stream)
        torch.cuda.synchronize()
        sp_ms.append(a.elapsed_time(b))
        for h in hs.values():
            st = h.stats()
            sp_phase["singular"] += st["time_singular_ms"]
            sp_phase["aca"] += st["time_far_ms"]
    sp_total = float(np.sum(sp_ms))
    if ws > 1:
        sp_total, sp_ents_all = reduce_over_ranks(sp_total, sp_ents, dist, dev)
    else:
        sp_ents_all = float(sp_ents)
    y_sp = {op: ys[op].cpu().numpy().copy() for op in hs}
    mixed_sp = {
        "precision": "BEM_MIXED_SP: as BEM_MIXED, plus FP32 dot products in the ACA norm "
                     "and FP32 Sauter-Schwab integrands (float-float sums) for the singular pairs",
        "value": sp_ents_all / (sp_total * 1e-3), "unit": UNIT,
        "ms_per_step": sp_total / args.steps,
        "phase_ms_per_step": {k_: v / args.steps for k_, v in sp_phase.items()},
        "matvec_rel_diff_vs_fp64": {("SLP" if op == 0 else "DLP"): float(
            np.linalg.norm(y_sp[op] - y_fp64[op]) / np.linalg.norm(y_fp64[op])) for op in hs},
        "tolerance": 2 * EPS}

    # the same step on trees built with the autotuned distance classes of the
    # regular rule, products against the FP64 6-point step above
    auto_q = None
    if args.level == 6 and not (args.rho3 > 0 or args.rho1 > 0):
        saved_q = bem.bem_get_quadrature()
        bem.bem_set_quadrature(*AUTOTUNED_RHO_L6)
        try:
            hq = {op: bem.HMatrix(mesh, LEAF, ETA) for op in (bem.SLP, bem.DLP)}
        finally:
            bem.bem_set_quadrature(saved_q["rho3"], saved_q["rho1"])

        def step_q():
            ent = 0
            for op, h in hq.items():
                bem.hmat_assemble(h.handle, op, 0.0, EPS, bem.MIXED, sptr)
                bem.hmat_matvec(h.handle, x, ys[op], 1, sptr)
            for h in hq.values():
                st = h.stats()
                ent += st["near_entries"] + st["far_entries"]
            return ent

        for _ in range(args.warmup):
            step_q()
            flush.fill_(1)
        torch.cuda.synchronize()
        q_ms, q_ents, q_aca = [], 0, 0.0
        for s in range(args.steps):
            flush.fill_(s & 0xff)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            q_ents += step_q()
            b.record(stream)
            torch.cuda.synchronize()
            q_ms.append(a.elapsed_time(b))
            q_aca += sum(h.stats()["time_far_ms"] for h in hq.values())
        q_total = float(np.sum(q_ms))
        if ws > 1:
            q_total, q_ents_all = reduce_over_ranks(q_total, q_ents, dist, dev)
        else:
            q_ents_all = float(q_ents)
        y_q = {op: ys[op].cpu().numpy().copy() for op in hs}
        sq = hq[bem.SLP].stats()
        auto_q = {
            "rho3": AUTOTUNED_RHO_L6[0], "rho1": AUTOTUNED_RHO_L6[1],
            "value": q_ents_all / (q_total * 1e-3), "unit": UNIT,
            "ms_per_step": q_total / args.steps, "aca_ms_per_step": q_aca / args.steps,
            "blocks": {"rule3": sq["n_blocks_rule3"], "rule1": sq["n_blocks_rule1"],
                       "all_far": sq["n_blocks_far"]},
            "matvec_rel_diff_vs_fp64_6pt": {("SLP" if op == 0 else "DLP"): float(
                np.linalg.norm(y_q[op] - y_fp64[op]) / np.linalg.norm(y_fp64[op])) for op in hs},
            "tolerance": 2 * EPS,
            "source": "autotune --level 6 --quadrature (eps 1e-5)"}
        for h in hq.values():
            h.close()

    # end to end through the C ABI from host buffers: mesh, one tree for both
    # operators (as for `value`), each assembly and its product from host x to
    # host y (x and y in page-locked host memory, as a caller streaming
    # vectors would hold them)
    e2e_ms, parts = [], []
    h2d = V.nbytes + T.astype(np.int32).nbytes + 2 * x_host.nbytes
    d2h = 2 * x_host.nbytes
    x_pin_t = torch.from_numpy(x_host).pin_memory()
    y_pin_t = torch.zeros(n, dtype=torch.float64).pin_memory()
    x_pin, y_pin = x_pin_t.numpy(), y_pin_t.numpy()
    for r in range(max(1, min(args.steps, 3))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        m2 = bem.Mesh(V, T)
        t1 = time.perf_counter()
        h2 = bem.HMatrix(m2, LEAF, ETA, parts=ws, part=rank)
        t2 = time.perf_counter()
        ent2 = 0
        for op in (bem.SLP, bem.DLP):
            h2.assemble(op, 0.0, EPS, bem.MIXED, sptr)
            bem.hmat_matvec(h2.handle, x_pin, y_pin, 1, sptr)
            s2 = h2.stats()
            ent2 += s2["near_entries"] + s2["far_entries"]
        t3 = time.perf_counter()
        h2.close()
        m2.close()
        torch.cuda.synchronize()
        t4 = time.perf_counter()
        e2e_ms.append((t4 - t0) * 1e3)
        parts.append({"mesh_ms": (t1 - t0) * 1e3, "tree_ms": (t2 - t1) * 1e3,
                      "assemble_and_product_ms": (t3 - t2) * 1e3, "free_ms": (t4 - t3) * 1e3,
                      "tree_clusters_ms": s2["time_tree_clusters_ms"],
                      "tree_blocks_ms": s2["time_tree_blocks_ms"],
                      "tree_lists_ms": s2["time_tree_lists_ms"],
                      "tree_upload_ms": s2["time_tree_upload_ms"]})
    if ws > 1:
        e2e_t, e2e_ents = reduce_over_ranks(float(np.median(e2e_ms)), ent2, dist, dev)
        e2e_val = e2e_ents / (e2e_t * 1e-3)
    else:
        e2e_val = ent2 / (np.median(e2e_ms) * 1e-3)
    e2e_parts = parts[int(np.argsort(e2e_ms)[len(e2e_ms) // 2])]

    # roofline of the dominant kernel (device time share over the timed steps)
    steps = args.steps
    f_clk = (clk.get("sm_mhz") or SM_MAX_MHZ) * 1e6
    evals_far = 36.0 * (st_slp["far_entries"] + st_dlp["far_entries"])
    sing = [st_slp["singular_pairs"][c] + st_dlp["singular_pairs"][c] for c in range(3)]
    near_reg = st_slp["near_entries"] + st_dlp["near_entries"] - sum(sing)
    per_step = {k: v / steps for k, v in phase.items()}
    dom = max(per_step, key=per_step.get)
    fp64_peak_d = N_SM * FP64_PER_SM_CLK * SM_MAX_MHZ * 1e6 / 1e9        # Gop/s
    mufu_peak_d = N_SM * MUFU_PER_SM_CLK * SM_MAX_MHZ * 1e6 / 1e9        # Gop/s
    # measured on this machine by the library's calibration kernels
    peaks = bem.bem_measure_peaks(sptr)
    fp64_peak = peaks["fp64_fma_per_s"] / 1e9
    mufu_peak = peaks["mufu_rsqrt_per_s"] / 1e9
    if dom == "aca":
        # algorithmic work of the mixed ACA per step.  rank^2 (m+n) per block
        # (aca_fp64_fma) counts the residual updates (about half) and the
        # norm's dot products (the other half), both FP64 in BEM_MIXED.
        # FP64: those, one addition per entry (widening the float-float
        # quadrature sum) and one multiplication per column entry (1/pivot).
        # FP32: 7 (SLP) / 12 (DLP) operations per point pair (the per-unit
        # figures of the quadrature roofline), 36 pairs per entry.  MUFU: one
        # rsqrt per pair.
        k2 = st_slp["aca_fp64_fma"] + st_dlp["aca_fp64_fma"]
        far = st_slp["far_entries"] + st_dlp["far_entries"]
        t_s = per_step[dom] * 1e-3
        ops = k2 + 1.5 * far
        achieved = ops / t_s / 1e9
        fp32_ops = 36.0 * (QUAD_FP32_PER_EVAL[0] * st_slp["far_entries"]
                           + QUAD_FP32_PER_EVAL[1] * st_dlp["far_entries"])
        fp32_peak = peaks["fp32_fma_per_s"] / 1e9
        roof = {"kernel": "k_aca (persistent ACA + far-field quadrature)", "bound": "alu",
                "pipe": "FP64 (DFMA/DADD/DMUL): the largest single-pipe demand per step",
                "achieved": achieved, "peak": fp64_peak,
                "unit": "Gop/s", "frac": achieved / fp64_peak,
                "traffic": ACA_TRAFFIC_BYTES_PER_STEP_L6 if args.level == 6 else None,
                "traffic_unit": "DRAM bytes per step (both k_aca launches, ncu capture)",
                "algorithmic": {"fp64_ops": ops, "fp32_ops": fp32_ops, "mufu_ops": evals_far,
                                "how": "FP64 = rank^2(m+n)/2 residual multiply-adds + rank^2(m+n)/2 "
                                       "norm multiply-adds + 1.5 per entry; FP32 = 36 x (7 SLP | 12 DLP) "
                                       "per entry; MUFU = 36 rsqrt per entry"},
                "pipe_ms_at_peak": {"fp64": ops / (fp64_peak * 1e9) * 1e3,
                                    "fp32": fp32_ops / (fp32_peak * 1e9) * 1e3,
                                    "mufu": evals_far / (mufu_peak * 1e9) * 1e3},
                "secondary": [{"pipe": "MUFU (rsqrt per Green's function evaluation)",
                               "achieved": evals_far / t_s / 1e9, "peak": mufu_peak,
                               "frac": evals_far / t_s / 1e9 / mufu_peak},
                              {"pipe": "FP32 (quadrature + norm dot products)",
                               "achieved": fp32_ops / t_s / 1e9, "peak": fp32_peak,
                               "frac": fp32_ops / t_s / 1e9 / fp32_peak}]}
    elif dom == "near_regular":
        achieved = 36.0 * near_reg / (per_step[dom] * 1e-3) / 1e9
        roof = {"kernel": "k_near_regular", "bound": "alu", "pipe": "MUFU",
                "achieved": achieved, "peak": mufu_peak, "unit": "Gop/s",
                "frac": achieved / mufu_peak, "traffic": None}
    else:
        per_pair = [128 * 12, 80 * 18, 24 * 15]
        ops = sum(s_ * p_ for s_, p_ in zip(sing, per_pair))
        achieved = ops / (per_step[dom] * 1e-3) / 1e9
        roof = {"kernel": "k_singular (Sauter-Schwab, FP64)", "bound": "alu", "pipe": "FP64",
                "achieved": achieved, "peak": fp64_peak, "unit": "Gop/s",
                "frac": achieved / fp64_peak, "traffic": None}
    roof["peak_source"] = ("measured on this box (bem_measure_peaks: DFMA and MUFU rsqrt throughput "
                           "kernels, best of three launches); MEASURED_PEAKS.json holds no ALU peak")
    roof["peaks_derived_gops"] = {"fp64": fp64_peak_d, "mufu": mufu_peak_d,
                                  "how": "152 SMs x per-SM unit rate (FP64 2/clk, MUFU 16/clk) "
                                         "x 2070 MHz max SM clock"}
    roof["phase_ms_per_step"] = per_step

    quad = quadrature_roofline(bem, mesh, V, T, dev, stream, flush, peaks=peaks)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        rate, cores, sample = oracle_sample_rate(V, T, seconds_target=args.cpu_seconds)
        rate1, _, sample1 = oracle_sample_rate(V, T, seconds_target=args.cpu_seconds / 3, seed=8,
                                               nthreads=1)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "cpu": cpu_model(), "kind": "oracle", "sample": sample,
               "one_thread": {"value": rate1, "unit": UNIT, "cores": 1, "sample": sample1}}

    if ws == 1:
        # serving latency (a short stream) on this GPU, after the C2 step's
        # buffers are released
        for h in hs.values():
            h.close()
        mesh.close()
        del x, ys, flush
        torch.cuda.empty_cache()
        if args.serving_requests > 0:
            extras["serving"] = serving_record(args, args.serving_requests, 8)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
                "higher_is_better": True, "scaling": "strong" if ws > 1 else "weak",
                "vs_baseline": None, "dtype": "f32+f64",
                "data": "synthetic (seeded jittered icosphere)",
                "config": dict(WORKLOAD, parallelism=(f"block-row sharding over {ws} GPUs" if ws > 1
                                                      else "1 GPU")),
                "integrals_per_step": ents_all / args.steps,
                "entries": {"near": st_slp["near_entries"], "far_SLP": st_slp["far_entries"],
                            "far_DLP": st_dlp["far_entries"], "singular_pairs": st_slp["singular_pairs"],
                            "far_blocks": st_slp["n_blocks_far"], "near_blocks": st_slp["n_blocks_near"]},
                "h_assembly_ms": {"SLP": st_slp["time_near_ms"] + st_slp["time_far_ms"],
                                  "DLP": st_dlp["time_near_ms"] + st_dlp["time_far_ms"]},
                "integrals_per_s_by_phase": {
                    "far_field_aca": (st_slp["far_entries"] + st_dlp["far_entries"])
                                     / (per_step["aca"] * 1e-3),
                    "near_regular": near_reg / (per_step["near_regular"] * 1e-3),
                    "singular": sum(sing) / (per_step["singular"] * 1e-3)},
                "tree_ms": st_slp["time_tree_ms"],
                "ranks": {"SLP": [st_slp["rank_min"], st_slp["rank_mean"], st_slp["rank_max"]],
                          "DLP": [st_dlp["rank_min"], st_dlp["rank_mean"], st_dlp["rank_max"]]},
                "mixed_vs_fp64": mixed_vs_fp64,
                "roofline": roof, "quadrature_roofline": quad, "cpu_baseline": cpu, "clocks": clk,
                "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                        "d2h_bytes_per_step": int(d2h), "ms_per_step": float(np.median(e2e_ms)),
                        "parts_ms": e2e_parts},
                "gpu_launches": int(launches), "step_ms": step_ms}
        if auto_q is not None:
            line["autotuned_quadrature"] = auto_q
        line["mixed_sp"] = mixed_sp
        line["measured_peaks"] = peaks
        line.update(extras)
        if args.rho3 > 0 or args.rho1 > 0:
            line["quadrature_classes"] = {
                "rho3": args.rho3, "rho1": args.rho1,
                "blocks": {"rule3": st_slp["n_blocks_rule3"], "rule1": st_slp["n_blocks_rule1"],
                           "all_far": st_slp["n_blocks_far"]}}
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def serving_record(args, nreq: int, calib: int):
    """Serving workload: a Poisson stream of assembly-and-product requests
    (mesh size log-uniform in [1k, 200k] triangles, jittered spheres and
    ellipsoids, 50% Laplace / 50% Helmholtz SLP with k ~ U[1, 20], ACA eps in
    {1e-4, 1e-6}), admitted by HBM budget and served with continuous batching
    (each batch's assemblies share one persistent ACA launch per kind of
    matrix); every tenth request is followed by a product-only request
    against the matrix it left resident.  Latency p50/p99 and throughput."""
    import threading
    import torch
    from paper_1711_01897_gb300 import bem, meshes
    torch.cuda.set_device(0)
    torch.cuda.init()
    rng = np.random.default_rng(1004)
    cache = {}

    def mesh_for(i):
        nt = float(np.exp(rng.uniform(np.log(1000.0), np.log(200000.0))))
        nu = max(2, int(round(np.sqrt(nt / 20.0))))
        if nu not in cache:
            cache[nu] = meshes.icosphere(nu)
        V, T = cache[nu]
        if rng.uniform() < 0.5:
            V = meshes.jitter(V, T, 0.05, 2000 + i)
        else:
            V = V * rng.uniform(0.5, 2.0, size=3)
        return V, T

    reqs = []
    for i in range(nreq):
        V, T = mesh_for(i)
        helm = rng.uniform() < 0.5
        k = float(rng.uniform(1.0, 20.0)) if helm else 0.0
        eps = 1e-4 if rng.uniform() < 0.5 else 1e-6
        x = rng.normal(size=T.shape[0]) + (1j * rng.normal(size=T.shape[0]) if helm else 0)
        reqs.append(dict(V=V, T=T, x=x, k=k, eps=eps))
    budget = int(args.hbm_budget_gb * (1 << 30))
    srv = bem.Server(budget, max_slots=args.slots)
    # capacity: a closed-loop batch of the first requests
    t0 = time.perf_counter()
    cal = [srv.submit(r["V"], r["T"], r["x"], k=r["k"], aca_eps=r["eps"]) for r in reqs[:calib]]
    for rid in cal:
        srv.wait(rid)
    cap = calib / (time.perf_counter() - t0)
    rate = args.load * cap
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=nreq))
    ids = [None] * nreq
    st0 = srv.stats()
    clk = Clocks(0)
    clk.start()
    start = time.perf_counter()

    def submitter():
        for i, r in enumerate(reqs):
            dt = arrivals[i] - (time.perf_counter() - start)
            if dt > 0:
                time.sleep(dt)
            ids[i] = srv.submit(r["V"], r["T"], r["x"], k=r["k"], aca_eps=r["eps"])

    th = threading.Thread(target=submitter)
    th.start()
    lat, lat_prod, ints, fails, shared, mism, sizes, phases = [], [], 0, 0, [], 0, [], []
    prod_phases = []
    for i in range(nreq):
        while ids[i] is None:
            time.sleep(0.0005)
        rc, info, y = srv.wait(ids[i])
        if rc != 0:
            fails += 1
            continue
        lat.append(info.t_done_ms - info.t_submit_ms)
        phases.append((info.t_ready_ms - info.t_submit_ms, info.t_admit_ms - info.t_ready_ms,
                       info.t_launch_ms - info.t_admit_ms, info.t_done_ms - info.t_launch_ms))
        sizes.append(reqs[i]["T"].shape[0])
        ints += info.integrals
        shared.append(info.launch_requests)
        if i % 10 == 5:
            # a product-only request against the matrix this one left resident
            p = srv.submit_product(ids[i], reqs[i]["x"])
            rc2, info2, y2 = srv.wait(p)
            if rc2 == 0:
                lat_prod.append(info2.t_done_ms - info2.t_submit_ms)
                prod_phases.append((info2.t_ready_ms - info2.t_submit_ms,
                                    info2.t_admit_ms - info2.t_ready_ms,
                                    info2.t_launch_ms - info2.t_admit_ms,
                                    info2.t_done_ms - info2.t_launch_ms))
                mism += int(not np.array_equal(y, y2))
    th.join()
    span = time.perf_counter() - start
    st = srv.stats()
    srv.close()
    clocks = clk.stop()
    lat = np.array(lat)
    sizes = np.array(sizes)
    ph = np.array(phases) if phases else np.zeros((1, 4))
    worst = np.argsort(-lat)[:5]
    names = ("trees", "admission", "batch", "device")
    phase_ms = {"median": {n: float(np.median(ph[:, c])) for c, n in enumerate(names)},
                "p99": {n: float(np.percentile(ph[:, c], 99)) for c, n in enumerate(names)},
                "slowest_requests": [{"triangles": int(sizes[w]), **{n: float(ph[w, c])
                                                                    for c, n in enumerate(names)}}
                                     for w in worst],
                "slowest_products": [dict(zip(names, map(float, p_)))
                                     for p_ in sorted(prod_phases, key=lambda q: -sum(q))[:3]]}
    by_size = {}
    for name, sel in (("below_40k_triangles", sizes < 40000), ("from_40k_triangles", sizes >= 40000)):
        if sel.any():
            by_size[name] = {"count": int(sel.sum()), "p50": float(np.percentile(lat[sel], 50)),
                             "p99": float(np.percentile(lat[sel], 99))}
            if len(phases) == len(lat):
                by_size[name]["parts_p99_ms"] = {n: float(np.percentile(ph[sel, c], 99))
                                                 for c, n in enumerate(names)}
    return {
        "config": {"workload": "serving: Poisson stream, 1k-200k triangles, 50% Laplace / 50% "
                               "Helmholtz SLP k~U[1,20], eps in {1e-4,1e-6}, assemble + 1 matvec; "
                               "after every 10th completes, a product-only request on its resident "
                               "matrix",
                   "requests": nreq, "slots": args.slots, "hbm_budget_gb": args.hbm_budget_gb,
                   "offered_load": args.load, "capacity_req_per_s": cap},
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                       "mean": float(lat.mean()),
                       "p99_over_p50": float(np.percentile(lat, 99) / np.percentile(lat, 50))},
        "latency_ms_by_size": by_size,
        "latency_parts_ms": phase_ms,
        "product_only_latency_ms": ({"p50": float(np.percentile(lat_prod, 50)),
                                     "p99": float(np.percentile(lat_prod, 99)),
                                     "count": len(lat_prod), "differ_from_assembly": mism}
                                    if lat_prod else None),
        "throughput": {"requests_per_s": len(lat) / span, "integrals_per_s": ints / span},
        "batching": {"aca_launches": st["aca_launches"] - st0["aca_launches"],
                     "requests_in_aca_launches": st["aca_launch_requests"] - st0["aca_launch_requests"],
                     "max_requests_per_launch": st["max_launch_requests"],
                     "mean_requests_per_launch_seen": float(np.mean(shared)) if shared else 0.0},
        "residency": {"reuse_hits": st["reuse_hits"], "evictions": st["evictions"],
                      "resident_at_end": st["resident"]},
        "admission": {"peak_reserved_gb": st["peak_reserved_bytes"] / (1 << 30),
                      "budget_gb": args.hbm_budget_gb, "failed": fails},
        "clocks": clocks}


def run_serving(args):
    rec = serving_record(args, args.requests, args.calib)
    lat = rec["latency_ms"]
    line = {"metric": METRIC, "value": lat["p99"], "unit": "ms (p99 latency)",
            "n_gpus": 1, "steps": args.requests, "warmup": args.calib, "ms_per_step": None,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
            "data": "synthetic (seeded Poisson request stream)"}
    line.update(rec)
    print(json.dumps(line), flush=True)
    return 0


LARGE = {
    "c3": {"mesh": "ellipsoid_nu158", "op": 0, "helmholtz": True, "eps": 1e-4, "matvecs": 1,
           "workload": "helmholtz_slp_p0_ellipsoid_10x1x1_nu158 (499,280 triangles, "
                       "k = 2 pi / (10 h), h mean longest edge)"},
    "c4": {"mesh": "sphere_l9", "op": 0, "helmholtz": False, "eps": 1e-4, "matvecs": 100,
           "workload": "laplace_slp_p0_icosphere_l9 (5,242,880 triangles), then 100 matvecs"},
}


def large_record(args, spec, steps: int, warmup: int, cpu_baseline: bool = True):
    """Helmholtz ellipsoid (C3) and level-9 sphere (C4): one step = one mixed
    assembly (all blocks in one persistent launch) plus the products; sampled
    exact rows of the matrix (oracle) check the product."""
    import torch
    from paper_1711_01897_gb300 import bem, meshes
    torch.cuda.set_device(0)
    torch.cuda.init()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    V, T = meshes.workload_mesh(spec["mesh"])
    n = T.shape[0]
    k = meshes.helmholtz_k_10_per_wavelength(V, T) if spec["helmholtz"] else 0.0
    if spec["helmholtz"] and args.warp_max_rows <= 0 and args.lane_max_rows < 0:
        t = bem.bem_get_tuning()
        bem.bem_set_tuning(AUTOTUNED_SHAPES_C3[0], AUTOTUNED_SHAPES_C3[1], t["use_graphs"])
    t0 = time.perf_counter()
    mesh = bem.Mesh(V, T)
    h = bem.HMatrix(mesh, LEAF, ETA)
    setup_s = time.perf_counter() - t0
    rng = np.random.default_rng(7)
    xh = rng.normal(size=n) + (1j * rng.normal(size=n) if k else 0)
    x = torch.from_numpy(xh).to(dev)
    y = torch.zeros_like(x)
    clk = Clocks(0)
    asm_ms, mv_ms, ents = [], [], 0
    for s in range(warmup + steps):
        if s == warmup:
            clk.start()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        bem.hmat_assemble(h.handle, spec["op"], k, spec["eps"], bem.MIXED, stream.cuda_stream)
        b.record(stream)
        torch.cuda.synchronize()
        st = h.stats()
        mvs = []
        for _ in range(spec["matvecs"]):
            c, d = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            c.record(stream)
            bem.hmat_matvec(h.handle, x, y, 1, stream.cuda_stream)
            d.record(stream)
            d.synchronize()
            mvs.append(c.elapsed_time(d))
        if s >= warmup:
            asm_ms.append(a.elapsed_time(b))
            mv_ms.extend(mvs)
            ents += st["near_entries"] + st["far_entries"]
    clocks = clk.stop()
    # sampled exact rows of A (oracle, FP64) against the product
    import oracle
    rows = np.sort(rng.choice(n, 16, replace=False)).astype(np.int32)
    t1 = time.perf_counter()
    A = oracle.entries(V, T, 0, k, rows, np.arange(n, dtype=np.int32))
    ref = A @ xh
    t_or = time.perf_counter() - t1
    cpu = None
    if cpu_baseline and not args.no_cpu_baseline:
        # the oracle's H-matrix assembly on a stratified sample of this mesh's
        # leaf blocks, extrapolated to the whole assembly by its integrals
        rate, cores, sample = oracle_sample_rate(V, T, seconds_target=args.cpu_seconds,
                                                 ops=(spec["op"],), k=k, eps=spec["eps"])
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "cpu": cpu_model(), "kind": "oracle", "sample": sample,
               "extrapolated_assembly_s": (ents / steps) / rate}
    got = y.cpu().numpy()[rows]
    err = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    tot_ms = float(np.sum(asm_ms))
    line = {"metric": METRIC, "value": ents / (tot_ms * 1e-3), "unit": UNIT, "n_gpus": 1,
            "steps": steps, "warmup": warmup,
            "ms_per_step": tot_ms / steps + float(np.sum(mv_ms)) / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
            "data": "synthetic", "config": {"workload": spec["workload"], "n_triangles": n, "k": k,
                                           "aca_eps": spec["eps"], "leaf_size": LEAF, "eta": ETA},
            "h_assembly_ms": float(np.median(asm_ms)), "tree_and_upload_s": setup_s,
            "tree_parts_ms": {"clusters": st["time_tree_clusters_ms"], "blocks": st["time_tree_blocks_ms"],
                              "lists": st["time_tree_lists_ms"], "upload": st["time_tree_upload_ms"],
                              "tree_total": st["time_tree_ms"]},
            "integrals_per_assembly": ents / steps,
            "phase_ms": {"near": st["time_near_ms"], "singular": st["time_singular_ms"],
                         "aca": st["time_far_ms"]},
            "ranks": [st["rank_min"], st["rank_mean"], st["rank_max"]],
            "memory_gb": {"near": st["near_bytes"] / 2**30, "factors": st["factor_bytes"] / 2**30,
                          "factors_read_per_product": st["factor_read_bytes"] / 2**30},
            "matvec_ms": {"mean": float(np.mean(mv_ms)), "p50": float(np.percentile(mv_ms, 50)),
                          "p99": float(np.percentile(mv_ms, 99)), "count": len(mv_ms)},
            # algorithmic bytes of a product: the near blocks and rank (m + n)
            # factor entries per admissible block (the unused columns of a
            # block's last 4-column chunk are not read)
            "matvec_gbs": (st["near_bytes"] + st["factor_read_bytes"]) / (np.median(mv_ms) * 1e-3) / 1e9,
            "sampled_rows_rel_err": err, "tolerance": 2 * spec["eps"],
            "oracle_rows_s": t_or, "cpu_baseline": cpu, "clocks": clocks,
            "aca_work_shapes": bem.bem_get_tuning()}
    if args.rho3 > 0 or args.rho1 > 0:
        line["quadrature_classes"] = {"rho3": args.rho3, "rho1": args.rho1,
                                      "blocks": {"rule3": st["n_blocks_rule3"],
                                                 "rule1": st["n_blocks_rule1"],
                                                 "all_far": st["n_blocks_far"]}}
    h.close()
    mesh.close()
    del x, y
    torch.cuda.empty_cache()
    return line


def run_large(args, spec):
    print(json.dumps(large_record(args, spec, args.steps, args.warmup)), flush=True)
    return 0


def run_p1(args):
    """Continuous piecewise linear spaces (the paper's benchmark space, Sec.
    5.2): Laplace single layer, double layer and hypersingular operator (Eq.
    (9), through the DP1 single layer) on the jittered icosphere, as
    H-matrices of the DP1 element-pair matrices with the P1 transforms in the
    product.  One step = the three assemblies and one product each; the
    integrals are DP1 entries (near field + every entry ACA requested).
    Sampled exact rows of the P1 matrices (oracle, FP64) check the products."""
    import torch
    from paper_1711_01897_gb300 import bem, meshes
    torch.cuda.set_device(0)
    torch.cuda.init()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    sptr = stream.cuda_stream
    V, T = meshes.icosphere_level(args.level)
    V = meshes.jitter(V, T, 0.05, 1001)
    nv, nt = V.shape[0], T.shape[0]
    t0 = time.perf_counter()
    mesh = bem.Mesh(V, T)
    ops = {name: op for name, op in (("SLP", bem.SLP), ("DLP", bem.DLP), ("HYPS", bem.HYPS))
           if name in args.ops.split(",")}
    hs = {name: bem.HMatrix(mesh, LEAF, ETA, space=bem.P1) for name in ops}
    setup_s = time.perf_counter() - t0
    rng = np.random.default_rng(11)
    x_host = rng.normal(size=nv)
    x = torch.from_numpy(x_host).to(dev)
    ys = {name: torch.zeros(nv, dtype=torch.float64, device=dev) for name in ops}
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def step(prec):
        ent = 0
        for name, h in hs.items():
            bem.hmat_assemble(h.handle, ops[name], 0.0, EPS, prec, sptr)
            bem.hmat_matvec(h.handle, x, ys[name], 1, sptr)
        for h in hs.values():
            st = h.stats()
            ent += st["near_entries"] + st["far_entries"]
        return ent

    for _ in range(max(3, args.warmup)):
        step(bem.MIXED)
    torch.cuda.synchronize()
    clocks = Clocks(0)
    clocks.start()
    ms, ents = [], 0
    per_op = {name: {"assembly_ms": 0.0, "near_regular_ms": 0.0, "singular_ms": 0.0, "aca_ms": 0.0}
              for name in ops}
    for s_ in range(args.steps):
        flush.fill_(s_ & 0xff)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ents += step(bem.MIXED)
        b.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
        for name, h in hs.items():
            st = h.stats()
            per_op[name]["assembly_ms"] += (st["time_near_ms"] + st["time_far_ms"]) / args.steps
            per_op[name]["near_regular_ms"] += st["time_near_regular_ms"] / args.steps
            per_op[name]["singular_ms"] += st["time_singular_ms"] / args.steps
            per_op[name]["aca_ms"] += st["time_far_ms"] / args.steps
    clk = clocks.stop()
    stats = {name: h.stats() for name, h in hs.items()}
    y_mixed = {name: ys[name].cpu().numpy().copy() for name in ops}
    # FP64 comparison step
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    step(bem.FP64)
    b.record(stream)
    torch.cuda.synchronize()
    fp64_ms = a.elapsed_time(b)
    # sampled exact rows (oracle) against the mixed products
    import oracle
    rows = np.sort(rng.choice(nv, 6, replace=False))
    t1 = time.perf_counter()
    errs = {}
    for name, op in ops.items():
        if name == "HYPS":
            R = oracle.hypersingular_p1_rows(V, T, 0.0, rows).real
            # D 1 = 0: its rows cancel, so the error is taken against |R| |x|
            scale = np.linalg.norm(np.abs(R) @ np.abs(x_host))
        else:
            R = oracle.p1_rows(V, T, op, 0.0, rows).real
            scale = np.linalg.norm(R @ x_host)
        errs[name] = float(np.linalg.norm(y_mixed[name][rows] - R @ x_host) / scale)
    t_or = time.perf_counter() - t1
    tot = float(np.sum(ms))
    line = {"metric": METRIC, "value": ents / (tot * 1e-3), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
            "data": "synthetic (seeded jittered icosphere)",
            "config": {"workload": f"laplace_p1_{'_'.join(n_.lower() for n_ in ops)}_icosphere_l{args.level}_jitter5pct",
                       "n_vertices": nv, "n_triangles": nt, "dp1_dofs": 3 * nt, "leaf_size": LEAF,
                       "eta": ETA, "aca_eps": EPS,
                       "precision": "mixed (FP32 quadrature, float-float accumulation, FP64 ACA)",
                       "l2": "flushed between timed steps (256 MiB write)"},
            "integrals_per_step": ents / args.steps, "per_operator": per_op,
            "ranks": {n_: [st["rank_min"], st["rank_mean"], st["rank_max"]] for n_, st in stats.items()},
            "memory_gb": {n_: (st["near_bytes"] + st["factor_bytes"]) / 2**30 for n_, st in stats.items()},
            "mixed_vs_fp64": {"fp64_ms_per_step": fp64_ms, "mixed_ms_per_step": float(np.median(ms)),
                              "speedup": fp64_ms / float(np.median(ms))},
            "sampled_rows_rel_err": errs, "tolerance": 2 * EPS, "oracle_rows_s": t_or,
            "tree_and_upload_s": setup_s, "clocks": clk}
    print(json.dumps(line), flush=True)
    return 0


def run_dense(args):
    """Dense weak-form assembly (Sec. 3, Algorithm "Dense Assembly"): every
    entry of the P0 Galerkin matrix of the unit sphere with about 103k
    triangles (the size of the paper's largest dense Laplace case), regular
    pairs by the tiled quadrature kernel and touching pairs by Sauter-Schwab,
    single and double layer, mixed precision (FP64 for one comparison run).
    Checks: sampled rows against the oracle, and the double-layer row sums
    against -|T_i|/2 over all rows."""
    import torch
    from paper_1711_01897_gb300 import bem, meshes
    torch.cuda.set_device(0)
    torch.cuda.init()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    V, T = meshes.icosphere(args.nu)
    nt = T.shape[0]
    mesh = bem.Mesh(V, T)
    ids = torch.arange(nt, dtype=torch.int32, device=dev)
    out = torch.empty(nt * nt, dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    res = {}
    clocks = Clocks(0)
    for name, op in (("SLP", bem.SLP), ("DLP", bem.DLP)):
        bem.bem_entries(mesh.handle, op, 0.0, bem.MIXED, ids, ids, out, stream.cuda_stream)
        if name == "SLP":
            clocks.start()
        ms = []
        for _ in range(args.steps):
            flush.fill_(1)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            bem.bem_entries(mesh.handle, op, 0.0, bem.MIXED, ids, ids, out, stream.cuda_stream)
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        res[name] = {"ms": float(np.median(ms)), "entries_per_s": nt * nt / (np.median(ms) * 1e-3)}
        A = out.view(nt, nt)
        rng = np.random.default_rng(3 + op)
        rows = np.sort(rng.choice(nt, 4, replace=False)).astype(np.int32)
        import oracle
        ref = oracle.entries(V, T, op, 0.0, rows, np.arange(nt, dtype=np.int32)).real
        got = A[torch.from_numpy(rows).long().to(dev)].cpu().numpy()
        res[name]["sampled_rows_rel_err"] = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
        if name == "DLP":
            P = V[T]
            area = 0.5 * np.linalg.norm(np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0]), axis=1)
            rs = A.sum(dim=1).cpu().numpy()
            res[name]["row_sum_vs_minus_half_area_max_rel"] = float(np.max(np.abs(rs + area / 2) / (area / 2)))
    clk = clocks.stop()
    # FP64 comparison, single layer
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    bem.bem_entries(mesh.handle, bem.SLP, 0.0, bem.FP64, ids, ids, out, stream.cuda_stream)
    b.record(stream)
    torch.cuda.synchronize()
    fp64_ms = a.elapsed_time(b)
    del out
    tot_ms = res["SLP"]["ms"] + res["DLP"]["ms"]
    line = {"metric": METRIC, "value": 2 * nt * nt / (tot_ms * 1e-3), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": 1, "ms_per_step": tot_ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
            "data": "synthetic (unit icosphere)",
            "config": {"workload": f"laplace_slp_dlp_p0_dense_icosphere_nu{args.nu}",
                       "n_triangles": nt, "entries_per_operator": nt * nt,
                       "precision": "mixed (FP32 quadrature, float-float accumulation); touching pairs FP64",
                       "l2": "flushed between timed launches (256 MiB write); output 8 n^2 bytes"},
            "per_operator": res,
            "mixed_vs_fp64": {"fp64_slp_ms": fp64_ms, "mixed_slp_ms": res["SLP"]["ms"],
                              "speedup": fp64_ms / res["SLP"]["ms"]},
            "clocks": clk}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="c2", choices=["c2", "c3", "c4", "serving", "p1", "dense"])
    ap.add_argument("--ops", default="SLP,DLP,HYPS",
                    help="operators of the p1 workload (comma-separated SLP, DLP, HYPS)")
    ap.add_argument("--nu", type=int, default=72,
                    help="geodesic frequency of the dense workload's sphere (20 nu^2 triangles)")
    ap.add_argument("--requests", type=int, default=2000)
    ap.add_argument("--serving-requests", type=int, default=200,
                    help="requests of the short serving stream in the default line (0: none)")
    ap.add_argument("--no-c4", action="store_true",
                    help="leave the level-9 record out of the default line")
    ap.add_argument("--no-c3", action="store_true",
                    help="leave the Helmholtz ellipsoid record out of the default line")
    ap.add_argument("--slots", type=int, default=6)
    ap.add_argument("--hbm-budget-gb", type=float, default=96.0)
    ap.add_argument("--load", type=float, default=0.8)
    ap.add_argument("--calib", type=int, default=24)
    ap.add_argument("--level", type=int, default=6,
                    help="icosphere level of the mesh (6 = the workload; smaller for profiling)")
    ap.add_argument("--warp-max-rows", type=int, default=0,
                    help="ACA work shapes (bem_set_tuning): blocks up to this many rows on one warp, "
                         "larger ones on a CTA (0 = the library's setting)")
    ap.add_argument("--lane-max-rows", type=int, default=-1,
                    help="... and up to this many on one lane (-1 = the library's setting)")
    ap.add_argument("--rho3", type=float, default=0.0,
                    help="distance class of the 3-point regular rule (dist/h; 0 = the paper's "
                         "6-point rule for every block)")
    ap.add_argument("--rho1", type=float, default=0.0,
                    help="distance class of the centroid rule (dist/h; 0 = off)")
    args = ap.parse_args()
    if args.warp_max_rows > 0 or args.lane_max_rows >= 0:
        from paper_1711_01897_gb300 import bem
        t = bem.bem_get_tuning()
        bem.bem_set_tuning(args.warp_max_rows if args.warp_max_rows > 0 else t["warp_max_rows"],
                           args.lane_max_rows if args.lane_max_rows >= 0 else t["lane_max_rows"],
                           t["use_graphs"])
    if args.rho3 > 0 or args.rho1 > 0:
        from paper_1711_01897_gb300 import bem
        bem.bem_set_quadrature(args.rho3, args.rho1)
        WORKLOAD["quadrature_classes"] = {"rho3": args.rho3, "rho1": args.rho1}
    if args.warmup < 3 and args.workload == "c2":
        args.warmup = 3
    if args.level != 6:
        WORKLOAD["workload"] = f"laplace_slp_dlp_p0_icosphere_l{args.level}_jitter5pct (profiling size)"
        WORKLOAD["n_triangles"] = 20 * 4 ** args.level
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "serving":
        return run_serving(args)
    if args.workload in LARGE:
        return run_large(args, LARGE[args.workload])
    if args.workload == "p1":
        return run_p1(args)
    if args.workload == "dense":
        return run_dense(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
