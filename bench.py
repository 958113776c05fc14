#!/usr/bin/env python
"""Benchmark of the hybrid direct-iterative KKT solver on one B300.

Headline workload (the precision form): the 100 x 100 x 100 3-D grid system
(n = 1e6, m = 5e5; 7-point weighted Laplacian, barrier 10^U(-8,8) on 40 % of
the diagonal, J with one unit entry and 4-8 local N(0,1) entries per row
within +-500 columns, delta = 1e-8, gamma = 1e6) with ten successive value
refactorizations on the fixed pattern (barrier rescaled by 10^U(-1,1) per
entry, new right-hand sides). A step = one numeric factorization + one full
solve (CG on the Schur complement + FP64 refinement on K_delta) of the next
value set on the resident pattern: one interior iteration. The analysis is
done once before timing (the paper amortizes it over the sequence). Metric:
KKT solves/s at relative residual <= 1e-8, mixed precision (FP32 factor with
tensor-core updates, FP64 CG and refinement) against the plain FP64 method on
the same workload.

Secondary blocks: the 500 x 500 2-D grid (n = 250000) at gamma 1e4 and 1e6
in both precisions, and the batching forms on the 200 x 100 grid.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--fp64-steps F]
  python bench.py --impl reference     # the CPU oracle on bounded samples
Multi-GPU (torchrun): independent replicas, one per rank (weak scaling).
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "grid3d_n1m"
WORKLOAD_TEXT = ("grid3d 100x100x100, n=1000000, m=500000, 10 value refactorizations, gamma=1e6, delta=1e-8, "
                 "barrier 10^U(-8,8) on 40%")
SECONDARY = "grid2d_n250k"
N_VALUE_SETS = 10
RR_TARGET = 1e-8
# the oracle's bounded sample: the same generator recipe on a 16^3 grid
SAMPLE_DIMS, SAMPLE_M = (16, 16, 16), 2048


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0, "sm_max_mhz": 2032.0}, "fallback"


def make_value_sets(name, count, **over):
    import workloads as W
    base = W.make_config(name, **over)
    sets = [base]
    for t in range(1, count):
        sets.append(W.rescale_barrier(sets[-1], seed=(0, t)))
    return sets


# ------------------------------------------------------------------ replicas
# One KKT system does not shard (its factor is one elimination tree), so N
# GPUs run N independent replicas: rank r takes the value sets in the order
# r, r+1, ... (weak scaling; no collective on the data path). The only
# exchange is the max-over-ranks of the timed region.
def value_set(step, rank):
    return (step + rank) % N_VALUE_SETS


def max_over_ranks(value, device):
    """Max of a host float over all ranks (identity when not distributed)."""
    import torch
    import torch.distributed as D
    if not (D.is_available() and D.is_initialized()) or D.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    D.all_reduce(t, op=D.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) >= 9:
                try:
                    rows.append((float(p[1]), float(p[2]), p[5:9]))
                except ValueError:
                    pass
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[i] for _, _, r in rows for i in range(4) if r[i].lower().startswith("active")})
        return {"sm_mhz": float(np.median([r[0] for r in rows])), "sm_max_mhz": max(r[1] for r in rows),
                "samples": len(rows), "reasons": reasons}


# ------------------------------------------------------------------ roofline
def tf32x3_peak(peaks, sustained=True):
    """FP32-equivalent peak of the three-product split-TF32 tensor-core path:
    the measured cuBLAS bf16 rate x the nominal TF32/BF16 ratio (1.1 / 2.25
    PFLOP/s dense) / 3 products."""
    bf16 = peaks.get("bf16_tflops_sustained" if sustained else "bf16_tflops", 1400.0)
    return bf16 * (1.1 / 2.25) / 3.0


def ffma_peak(peaks):
    """FP32 FMA units: 148 SMs x 128 lanes x 2 flops x the maximum SM clock (TFLOP/s)."""
    return 148 * 128 * 2 * peaks.get("sm_max_mhz", 2032.0) * 1e-6


def solve_bytes(prec, nnz_l, iters_per_pass, nnz_j, n, m):
    """Algorithmic bytes of one launch of the persistent solve kernel (one
    refinement pass): (iterations + 1) H^-1 applications for the mixed form
    (dx accumulated along the recurrence), + 2 for FP64 (w and the
    back-substitution); each application reads L twice (nnz(L) entries of s
    bytes), plus the J and J^T products of every iteration."""
    s = 8 if prec == "fp64" else 4
    hs = iters_per_pass + (1 if prec == "mixed" else 2)
    return hs * 2 * s * nnz_l + iters_per_pass * 2 * (12 * nnz_j + 8 * (n + m))


# ------------------------------------------------------------------ timed steps
def time_steps(s, dsets, steps, warmup, rank, dev, barrier, clocks=True):
    """warmup + steps factor/solve pairs on the resident pattern; the steps
    are bracketed by a barrier and a synchronize on both sides and timed
    with CUDA events on the current stream (the library's calls run there)."""
    import torch
    stream = torch.cuda.current_stream()
    n, m = s.n, s.m
    dx = torch.empty(n, dtype=torch.float64, device=dev)
    dy = torch.empty(m, dtype=torch.float64, device=dev)

    def step(t):
        Hv, Jv, rx, ry, delta, gamma = dsets[value_set(t, rank)]
        s.factor(Hv, Jv, delta, gamma)
        s.solve(rx, ry, dx, dy)
        return s.info

    for t in range(warmup):
        step(t)
    s.profile(reset=True)            # the solve kernel's own event timing, timed region only
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    infos = []
    clk = ClockSampler(dev.index) if clocks else None
    if clk:
        clk.start()
    barrier()
    ev[0].record(stream)
    for t in range(steps):
        infos.append(step(warmup + t))
        ev[t + 1].record(stream)
    barrier()
    cl = clk.stop() if clk else None
    lat = [ev[i].elapsed_time(ev[i + 1]) for i in range(steps)]
    total_ms = max_over_ranks(ev[0].elapsed_time(ev[-1]), dev)
    cg_ms, cg_n = s.profile(reset=True)["cg_persistent"]
    rr = [i.rr for i in infos]
    return dict(total_ms=total_ms, lat=lat, rr_max=max(rr), iters=[i.cg_iters for i in infos],
                ir=[i.ir_steps for i in infos], clocks=cl, cg_live=(cg_ms, cg_n), ok=max(rr) <= RR_TARGET,
                steps=steps, warmup=warmup)


def summary(R, world):
    solves = R["steps"] * world
    return {"value": round(solves / (R["total_ms"] / 1e3), 4), "unit": "solves/s",
            "ms_per_step": round(R["total_ms"] / R["steps"], 3), "steps": R["steps"], "warmup": R["warmup"],
            "rr_max": R["rr_max"], "cg_iters_mean": float(np.mean(R["iters"])),
            "ir_steps_mean": float(np.mean(R["ir"])),
            "latency_ms": {"p50": round(float(np.percentile(R["lat"], 50)), 3),
                           "p99": round(float(np.percentile(R["lat"], 99)), 3)}}


# ------------------------------------------------------------------ our arm
def run_ours(args, rank, world):
    import torch
    import paper_2110_03636_b300 as K

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    dist = world > 1
    if dist:
        import torch.distributed as D

    def barrier():
        if dist:
            D.barrier()
        torch.cuda.synchronize()

    cu = lambda a: torch.as_tensor(np.ascontiguousarray(a), device=dev)
    peaks, peak_src = load_peaks()

    # ---------------- headline: the precision form, mixed, on the resident 100^3 pattern
    sets = make_value_sets(args.workload, N_VALUE_SETS)
    base = sets[0]
    n, m = base.n, base.m
    dsets = [(cu(x.H_vals), cu(x.J_vals), cu(x.r_x), cu(x.r_y), x.delta, x.gamma) for x in sets]
    t0 = time.time()
    hs = K.KKTSolver.host_only(n, m, base.H_colptr, base.H_rowidx, base.J_rowptr, base.J_colidx,
                               ordering=args.ordering)
    t_analyse = time.time() - t0
    s = K.KKTSolver.like(hs, precision="mixed", ordering=args.ordering)
    si = s.symbolic_info
    R = time_steps(s, dsets, args.steps, args.warmup, rank, dev, barrier)
    head = summary(R, world)

    # per-kernel split and rooflines: the same steps kernel by kernel, each
    # launch bracketed by CUDA events on the library's stream (profile mode;
    # outside the timed region, since the events serialise the launches)
    prof_steps = 2
    s.set_profile(True)
    s.profile(reset=True)
    dx = torch.empty(n, dtype=torch.float64, device=dev)
    dy = torch.empty(m, dtype=torch.float64, device=dev)
    for t in range(prof_steps):
        Hv, Jv, rx, ry, delta, gamma = dsets[value_set(t, rank)]
        s.factor(Hv, Jv, delta, gamma)
        s.solve(rx, ry, dx, dy)
    prof = s.profile(reset=True)
    s.set_profile(False)
    per_step = {k: v[0] / prof_steps for k, v in prof.items() if v[1]}
    launches_per_step = sum(v[1] for v in prof.values()) / prof_steps
    fac_kinds = ("assemble", "potrf", "trsm", "panel_update", "syrk", "extend_add", "tc_split", "tri_inv", "syrk_tc",
                 "block")
    fac_ms = sum(per_step.get(k, 0.0) for k in fac_kinds)
    tc_ms = per_step.get("syrk_tc", 0.0)
    tc_peak = tf32x3_peak(peaks, sustained=True)
    roof = None
    if tc_ms > 0:
        ach = si.tc_flops / (tc_ms / 1e3) / 1e12
        roof = {"kernel": "k_tc_update (tcgen05 update-matrix SYRK and in-panel updates)", "bound": "tensor",
                "achieved": round(ach, 2), "peak": round(tc_peak, 1), "unit": "TFLOP/s",
                "frac": round(ach / tc_peak, 4), "traffic": None,
                "traffic_note": ("no DRAM capture of this kernel at this size (a 100 GB workload exceeds the "
                                 "capture size rule); the 4000-column front capture is summarised under profiles/"),
                "peak_source": (f"{peak_src}: bf16_tflops_sustained {peaks.get('bf16_tflops_sustained')} x TF32/BF16 "
                                "nominal 1.1/2.25 / 3 split products (FP32-equivalent flops)"),
                "work_per_unit": f"{si.tc_flops:.4g} flop per factorization (all launches of the kernel)",
                "ms_per_factorization": round(tc_ms, 2), "share_of_step": round(tc_ms / sum(per_step.values()), 3),
                "timing": "profiled steps (per-launch CUDA events on the library's stream)"}
    fac_roof = {"flops": si.flops, "ms": round(fac_ms, 2),
                "achieved_tflops": round(si.flops / (fac_ms / 1e3) / 1e12, 2),
                "peak_ffma_tflops": round(ffma_peak(peaks), 1),
                "frac_of_ffma": round(si.flops / (fac_ms / 1e3) / 1e12 / ffma_peak(peaks), 4),
                "peak_tf32x3_tflops": round(tc_peak, 1),
                "frac_of_tf32x3": round(si.flops / (fac_ms / 1e3) / 1e12 / tc_peak, 4),
                "note": "sum_j c_j^2 over all factor kernels' time (explicit zeros of relaxed supernodes not counted)"}
    cg_ms, cg_n = R["cg_live"]
    solve_roof = None
    if cg_n:
        passes = np.mean(R["ir"]) + 1
        ipp = float(np.mean(R["iters"]) / passes)
        byts = solve_bytes("mixed", si.nnz_l, ipp, base.J_colidx.size, n, m)
        ach = byts / (cg_ms / cg_n / 1e3) / 1e9
        solve_roof = {"kernel": "k_cg (persistent CG + triangular sweeps)", "bound": "hbm",
                      "achieved": round(ach, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
                      "frac": round(ach / peaks["hbm_gbs"], 4), "ms_per_launch": round(cg_ms / cg_n, 2),
                      "work_per_unit": f"{byts:.4g} byte per launch ({ipp:.2f} CG products per pass)",
                      "timing": f"timed region (CUDA events around each of {cg_n} launches)"}

    # end to end through the host-buffer entry point on the same handle
    e2e = None
    if not args.no_e2e:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
        hsets = [(pin(x.H_vals), pin(x.J_vals), pin(x.r_x), pin(x.r_y), x.delta, x.gamma) for x in sets]
        hx, hy = pin(np.zeros(n)), pin(np.zeros(m))
        Hv, Jv, rx, ry, delta, gamma = hsets[value_set(0, rank)]
        s.factor_solve_host(Hv, Jv, delta, gamma, rx, ry, hx, hy)
        barrier()
        t0 = time.perf_counter()
        for t in range(args.steps):
            Hv, Jv, rx, ry, delta, gamma = hsets[value_set(args.warmup + t, rank)]
            s.factor_solve_host(Hv, Jv, delta, gamma, rx, ry, hx, hy)
        barrier()
        el = max_over_ranks(time.perf_counter() - t0, dev)
        e2e = {"value": round(args.steps * world / el, 4), "unit": "solves/s",
               "h2d_bytes_per_step": 8 * (base.H_vals.size + base.J_vals.size + n + m),
               "d2h_bytes_per_step": 8 * (n + m) + 2 * 64}
    s.close()
    del s, dsets
    torch.cuda.empty_cache()

    # ---------------- the plain FP64 method on the same workload
    fp64 = None
    if args.fp64_steps > 0:
        dsets = [(cu(x.H_vals), cu(x.J_vals), cu(x.r_x), cu(x.r_y), x.delta, x.gamma) for x in sets[:2]]
        sf = K.KKTSolver.like(hs, precision="fp64", ordering=args.ordering)
        F = time_steps(sf, dsets, args.fp64_steps, 0, rank, dev, barrier, clocks=False)
        fp64 = summary(F, world)
        fp64["note"] = (f"{args.fp64_steps} timed step(s) without warm-up: one FP64 factorization of this "
                        "workload takes minutes (B300's FP64 rate is ~1/64 of FP32)")
        fp64["device_gb"] = round(sf.symbolic_info.device_bytes / 1e9, 1)
        sf.close()
        del sf, dsets
        torch.cuda.empty_cache()
    hs.close()
    return dict(head=head, R=R, t_analyse=t_analyse, si=si, roof=roof, fac_roof=fac_roof, solve_roof=solve_roof,
                e2e=e2e, fp64=fp64, per_step=per_step, launches_per_step=launches_per_step)


# ------------------------------------------------------------------ secondary workload
def run_secondary(args, rank, world, dev, barrier):
    """The plain-method scale workload (500 x 500 grid, n = 250000) at
    gamma 1e4 and 1e6, both precisions, on one analysis of its pattern."""
    import torch
    import paper_2110_03636_b300 as K
    cu = lambda a: torch.as_tensor(np.ascontiguousarray(a), device=dev)
    sets = make_value_sets(SECONDARY, N_VALUE_SETS)
    base = sets[0]
    hs = K.KKTSolver.host_only(base.n, base.m, base.H_colptr, base.H_rowidx, base.J_rowptr, base.J_colidx,
                               ordering=args.ordering)
    out = {"workload": "grid2d 500x500, n=250000, m=125000, 10 value refactorizations, delta=1e-8"}
    steps = min(args.steps, 10)
    for gamma in (1e4, 1e6):
        dsets = [(cu(x.H_vals), cu(x.J_vals), cu(x.r_x), cu(x.r_y), x.delta, gamma) for x in sets]
        blk = {}
        for prec in ("mixed", "fp64"):
            s = K.KKTSolver.like(hs, precision=prec, ordering=args.ordering)
            blk[prec] = summary(time_steps(s, dsets, steps, args.warmup, rank, dev, barrier, clocks=False), world)
            s.close()
        out[f"gamma_{gamma:.0e}"] = blk
        del dsets
    hs.close()
    torch.cuda.empty_cache()
    return out


# ------------------------------------------------------------------ batching forms
def run_batching(args, dev, rank=0, world=1, group=None):
    """The batching workload (200 x 100 grid, n = 20000, m = 10000): nsys
    systems sharing one analysed pattern with per-system edge weights and
    barriers (independent seeds), factored and solved through the batched
    entry points; and one of them with 64 right-hand sides solved together
    (the triangular sweeps shared) against 64 separate solves. Mixed
    precision (FP32 factor, FP64 CG and refinement). With several ranks the
    systems are sharded by contiguous index (each rank its own block on its
    own GPU) and the per-system statistics gathered on rank 0 over a CPU
    group; the rate is all systems over the slowest rank's time."""
    import torch
    import paper_2110_03636_b300 as K
    from paper_2110_03636_b300 import shard
    import workloads as W
    base = W.make_config("grid2d_n20k")
    lo, hi = shard.partition(args.batch_systems, world)[rank]
    systems = [W.reweight(base, seed=(1, b)) for b in range(lo, hi)]
    cu = lambda a: torch.as_tensor(np.ascontiguousarray(a), device=dev)
    Hs = cu(np.stack([x.H_vals for x in systems]))
    Js = cu(np.stack([x.J_vals for x in systems]))
    rng = np.random.default_rng(11)
    RX = cu(rng.standard_normal((args.batch_systems, base.n))[lo:hi])
    RY = cu(rng.standard_normal((args.batch_systems, base.m))[lo:hi])
    out = {"workload": "grid2d 200x100, n=20000, m=10000, per-system weights and barriers (seeds (1, b))",
           "precision": "mixed"}
    # plan parameters picked by the autotuner (measured coordinate search on
    # two of this rank's systems; the analysis is exact for every set)
    opts = {}
    if not args.no_autotune and hi > lo:
        from paper_2110_03636_b300 import autotune as AT
        pattern = (base.n, base.m, base.H_colptr, base.H_rowidx, base.J_rowptr, base.J_colidx)
        vs = [(Hs[i], Js[i], RX[i], RY[i], base.delta, base.gamma) for i in range(min(2, hi - lo))]
        opts, t_best, t_def, evals = AT.tune(pattern, vs, ordering=args.ordering, sweeps=1)
        out["autotune"] = {"options": opts, "ms_factor_solve": round(1e3 * t_best, 3),
                           "ms_factor_solve_defaults": round(1e3 * t_def, 3), "evaluations": len(evals),
                           "search": "coordinate descent over relaxation, solve tile shape, tensor cores"}
    s = K.KKTSolver(base.n, base.m, base.H_colptr, base.H_rowidx, base.J_rowptr, base.J_colidx,
                    precision="mixed", ordering=args.ordering, **opts)

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            r = fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / reps, r

    def batch_step():
        code, st = s.factor_batch(Hs, Js, base.delta, base.gamma)
        dx, dy, infos, sst, code2 = s.solve_batch(RX, RY)
        return st, sst, infos
    sec, (st, sst, infos) = timed(batch_step, 2)
    sec = max_over_ranks(sec, dev)
    stats = shard.gather_blocks({"status": np.asarray(st) + np.asarray(sst), "rr": np.array([i.rr for i in infos])},
                                rank, world, group=group)
    if rank == 0:
        out["batch"] = {"systems": args.batch_systems, "solves_per_s": round(args.batch_systems / sec, 2),
                        "ms_per_system": round(1e3 * sec * world / args.batch_systems, 3),
                        "failed": int((stats["status"] != 0).sum()), "rr_max": float(stats["rr"].max()),
                        "ranks": world, "form": ("factor_batch: one graph replay factors every system (system = "
                                                 "blockIdx.y of each launch); solve_batch: 4 concurrent solves "
                                                 "reading the systems' factors in place")
                        + (", systems sharded by contiguous index over the ranks" if world > 1 else "")}
    s.factor(Hs[0], Js[0], base.delta, base.gamma)
    R64 = cu(rng.standard_normal((64, base.n)))
    Y64 = cu(rng.standard_normal((64, base.m)))
    sec_m, (dx, dy, infos) = timed(lambda: s.solve_multi(R64, Y64), 2)
    sec_1, _ = timed(lambda: [s.solve(R64[j], Y64[j]) for j in range(64)], 1)
    out["multi_rhs"] = {"nrhs": 64, "rhs_per_s": round(64 / sec_m, 2), "separate_rhs_per_s": round(64 / sec_1, 2),
                        "rr_max": max(i.rr for i in infos),
                        "form": "solve_multi: 8 right-hand sides per persistent launch sharing each sweep"}
    s.close()
    return out


# ------------------------------------------------------------------ serving form
def run_serving(args, dev):
    """The serving workload: 4 resident patterns (2-D grids 100^2 .. 800^2,
    n = 1e4 .. 6.4e5, m = n/2, gamma = 1e6), requests = value updates of a
    random pattern (barrier rescaled by 10^U(-1,1), new right-hand sides),
    through the continuous-batching request server (HBM-budget admission,
    4 requests in flight on their own streams). First the saturated rate (all
    requests queued at once), then Poisson arrivals at 0.5 / 0.8 / 0.95 of it:
    latency p50 / p99 (submission to completion) and served solves/s."""
    import torch
    import paper_2110_03636_b300 as K
    import workloads as W
    cu = lambda a: torch.as_tensor(np.ascontiguousarray(a), device=dev)
    sides = (100, 200, 400, 800)
    nval = 3
    srv = K.KKTServer(0, max_inflight=4, precision="mixed", ordering=args.ordering, solve_sms=37)
    t0 = time.time()
    vals, pids = [], []
    for side in sides:
        x = W.serving_pattern(side)
        pids.append(srv.add_pattern(x.n, x.m, x.H_colptr, x.H_rowidx, x.J_rowptr, x.J_colidx))
        vs = []
        for t in range(nval):
            x = W.rescale_barrier(x, seed=(side, t))
            vs.append((cu(x.H_vals), cu(x.J_vals), x.delta, x.gamma, cu(x.r_x), cu(x.r_y),
                       torch.empty(x.n, dtype=torch.float64, device=dev),
                       torch.empty(x.m, dtype=torch.float64, device=dev)))
        vals.append(vs)
    t_setup = time.time() - t0
    rng = np.random.default_rng(5)

    def submit(k, p):
        H, J, d, g, rx, ry, dx, dy = vals[p][k % nval]
        # each in-flight request writes its own outputs: a fresh pair per request
        return srv.submit(pids[p], H, J, d, g, rx, ry, torch.empty_like(dx), torch.empty_like(dy))

    for p in range(len(sides)):                 # warm every pattern's first slot
        srv.wait(submit(0, p))

    def run(count, rate):
        pats = rng.integers(0, len(sides), count)
        gaps = rng.exponential(1.0 / rate, count) if rate else np.zeros(count)
        ids = []
        start = time.perf_counter()
        due = start
        for k in range(count):
            due += gaps[k]
            wait = due - time.perf_counter()
            if wait > 0:
                time.sleep(wait)
            ids.append(submit(k, int(pats[k])))
        infos = [srv.wait(r) for r in ids]
        t_first = min(i.t_submit for i in infos)
        t_last = max(i.t_end for i in infos)
        lat = np.array([1e3 * (i.t_end - i.t_submit) for i in infos])
        return {"requests": count, "solves_per_s": round(count / (t_last - t_first), 2),
                "latency_ms": {"p50": round(float(np.percentile(lat, 50)), 2),
                               "p99": round(float(np.percentile(lat, 99)), 2)},
                "rr_max": max(i.rr for i in infos), "failed": int(sum(i.status != 0 for i in infos))}

    sat = run(args.serve_requests, None)
    out = {"workload": "4 patterns: 2-D grids 100^2, 200^2, 400^2, 800^2 (n = 1e4 .. 6.4e5), m = n/2, gamma = 1e6; "
                       "each request one value refactorization + solve (mixed)",
           "server": "continuous batching, 4 in flight, HBM-budget admission (90 % of free memory)",
           "setup_s": round(t_setup, 1), "saturated": sat}
    lam = sat["solves_per_s"]
    for f in (0.5, 0.8, 0.95):
        out[f"poisson_{f}"] = dict(run(args.serve_requests, f * lam), arrival_rate=round(f * lam, 2))
    st = srv.stats()
    out["slots"], out["peak_inflight"] = st.slots, st.peak_inflight
    out["device_gb_peak"] = round(st.bytes_peak / 1e9, 2)
    srv.close()
    return out


# ------------------------------------------------------------------ oracle (CPU) samples
def oracle_sample_setup(workload_flops):
    """The oracle's bounded sample: the headline workload's generator recipe
    (same distributions, J window and gamma) on a 16^3 grid, analysed once.
    Returns (symbolic, value sets, scale) where scale = the sample's factor
    flops / the headline system's (sum_j c_j^2 of each)."""
    import oracle as O
    sets = make_value_sets(WORKLOAD, 3, dims=SAMPLE_DIMS, m=SAMPLE_M)
    b = sets[0]
    sym = O.Symbolic(b.n, b.m, b.H_colptr, b.H_rowidx, b.J_rowptr, b.J_colidx, ordering="nd")
    return sym, sets, sym.flops / workload_flops


def oracle_solve(sym, x):
    """One oracle solve of the sample (assembly + Cholesky + CG on the Schur
    complement + 3 refinement passes), wall seconds."""
    import oracle as O
    t0 = time.perf_counter()
    f = O.Factor(sym, x.H_vals, x.J_vals, x.delta, x.gamma)
    f.solve(x.r_x, x.r_y, ir_maxit=3)
    return time.perf_counter() - t0


def sample_text(sym, scale):
    d = "x".join(map(str, SAMPLE_DIMS))
    return (f"oracle (1 thread, FP64) full factor + solve of the same recipe on a {d} grid (n={sym.n}, m={sym.m}, "
            f"sum c^2 = {sym.flops:.3g}); per-solve time scaled to the 100^3 system by the factor-flop ratio "
            f"{scale:.3g} (the oracle cannot hold the 100^3 factor: ~95 GB of values)")


def cpu_baseline(workload_flops, seconds):
    sym, sets, scale = oracle_sample_setup(workload_flops)
    ts = []
    t_start = time.perf_counter()
    while True:
        ts.append(oracle_solve(sym, sets[len(ts) % len(sets)]))
        if time.perf_counter() - t_start >= seconds or len(ts) >= 20:
            break
    per = float(np.median(ts))
    return {"value": round(scale / per, 8), "unit": "solves/s", "cores": 1, "kind": "oracle",
            "sample": sample_text(sym, scale) + f"; median of {len(ts)} timed solves ({per:.2f} s each)"}


# sum_j c_j^2 of the headline system's factor (nested dissection): the
# library's and the oracle's symbolic analyses agree on it bit for bit; the
# oracle cannot analyse the 100^3 pattern in a bounded time and memory, so
# the reference arm scales its samples by this recorded value
HEADLINE_FLOPS = 208656661746431.0


def run_reference(args, rank, world):
    if rank != 0:
        return None
    sym, sets, scale = oracle_sample_setup(HEADLINE_FLOPS)
    ts = []
    for t in range(args.warmup + args.steps):
        dt = oracle_solve(sym, sets[t % len(sets)])
        if t >= args.warmup:
            ts.append(dt)
    per = float(np.mean(ts))
    v = scale / per
    return {"metric": "KKT solves/s at relative residual <= 1e-8 (factor + solve per interior iteration)",
            "value": round(v, 8), "unit": "solves/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(per * 1e3, 1), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD_TEXT, "precision": "fp64 (CPU oracle)"},
            "cpu_baseline": {"value": round(v, 8), "unit": "solves/s", "cores": 1, "kind": "oracle",
                             "sample": sample_text(sym, scale) + "; each step one timed sample solve"},
            "e2e": {"value": round(v, 8), "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--fp64-steps", type=int, default=1, help="timed FP64 steps on the headline workload (0: skip)")
    ap.add_argument("--no-secondary", action="store_true", help="skip the 500x500 grid blocks")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-sample-seconds", type=float, default=15.0)
    ap.add_argument("--ordering", default="nd", choices=["nd", "amd"])
    ap.add_argument("--no-batch", action="store_true", help="skip the batched / multi-RHS measurements")
    ap.add_argument("--batch-systems", type=int, default=256)
    ap.add_argument("--no-autotune", action="store_true", help="batching block with the default plan parameters")
    ap.add_argument("--no-serving", action="store_true", help="skip the request-server block")
    ap.add_argument("--serve-requests", type=int, default=300, help="requests per serving rate point")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        line = run_reference(args, rank, world)
        if line is not None:
            print(json.dumps(line), flush=True)
        return
    import torch
    if world > 1:
        import torch.distributed as D
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        D.init_process_group("nccl")
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))

    def barrier():
        if world > 1:
            D.barrier()
        torch.cuda.synchronize()

    res = run_ours(args, rank, world)
    H, si, R = res["head"], res["si"], res["R"]
    line = {
        "metric": "KKT solves/s at relative residual <= 1e-8 (factor + solve per interior iteration)",
        "value": H["value"], "unit": "solves/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": H["ms_per_step"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 factor (3xTF32 tensor-core updates) + f32 trisolve, f64 CG/residual/refinement",
        "data": "synthetic (seeded grid-Laplacian + barrier + local J; paper's power-grid matrices unavailable)",
        "config": {"workload": WORKLOAD_TEXT, "precision": "mixed", "ordering": args.ordering,
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": "per-step working set > L2 (FP32 panels %.1f GB)" % (si.panel_entries * 4 / 1e9),
                   "nnz_L": si.nnz_l, "factor_flops": si.flops, "tensor_core_flops": si.tc_flops,
                   "nsuper": si.nsuper},
        "latency_ms": H["latency_ms"], "rr_max": H["rr_max"], "cg_iters_mean": H["cg_iters_mean"],
        "ir_steps_mean": H["ir_steps_mean"], "analyse_s": round(res["t_analyse"], 2),
        "clocks": R["clocks"], "gpu_launches": int(round(res["launches_per_step"] * args.steps)),
        "roofline": res["roof"], "factor_roofline": res["fac_roof"], "solve_roofline": res["solve_roof"],
        "e2e": res["e2e"],
        "kernel_ms_per_step": {k: round(v, 3) for k, v in res["per_step"].items()},
    }
    if res["fp64"] is not None:
        line["fp64"] = res["fp64"]
        line["mixed_over_fp64"] = round(H["value"] / res["fp64"]["value"], 2)
    if si.flops != HEADLINE_FLOPS and args.workload == WORKLOAD:
        line["warning"] = "factor flops differ from the recorded value the reference arm scales by"
    if not args.no_secondary:
        line["secondary"] = run_secondary(args, rank, world, dev, barrier)
    if not args.no_batch:
        group = D.new_group(backend="gloo") if world > 1 else None
        line["batching"] = run_batching(args, dev, rank, world, group)
    if not args.no_serving:
        line["serving"] = run_serving(args, dev)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(si.flops, args.cpu_sample_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        D.destroy_process_group()


if __name__ == "__main__":
    main()
