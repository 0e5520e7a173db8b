#!/usr/bin/env python
"""Benchmark of the LTMP2 hot path on one GB300 (and N replicas under torchrun).

Metric: seconds per E_MP2 and pair-tau contractions per second (unordered
occupied pairs i <= j times Laplace points, per second of ltmp2_energy), on the
seeded Gaussian-well model solid with 16 wells, a 24^3 grid, 3071 plane waves,
32 occupied orbitals and 8 Laplace points, in the plain FP64 path.  The
precision form (complex64 FFTs, split-precision GEMMs, FP64 sums) is timed on
the same inputs and its error against the FP64 path is reported in meV/atom.

  python bench.py [--steps K] [--warmup W] [--form fp64|fp32] [--impl ours|reference]

One JSON line on stdout (rank 0).  Everything else goes to stderr.
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "s per E_MP2 and pair-tau contractions/s at <=0.1 meV/atom vs FP64 plain path"
UNIT = "pair-tau contractions/s"
HARTREE_TO_MEV = 27211.386245988
# Peaks: HBM and bf16 tensor from MEASURED_PEAKS.json; FP64 / FP32 ALU derived from unit
# counts at the maximum SM clock (2 FP64 FMA and 128 FP32 FMA per SM per clock).
SM_COUNT = 152
SM_MAX_MHZ = 2070.0
FP64_ALU_TFLOPS = 2 * 2 * SM_COUNT * SM_MAX_MHZ * 1e6 / 1e12     # 1.259
FP32_ALU_TFLOPS = 128 * 2 * SM_COUNT * SM_MAX_MHZ * 1e6 / 1e12   # 80.5
TF32_OVER_BF16 = 1.1 / 2.25   # nominal dense tensor-rate ratio (tf32 / bf16)

WORKLOAD = "cfg2"
CPU_SAMPLE_ORBITALS = (0, 1)   # oracle sample: ordered pairs (0,0), (0,1), (1,0), (1,1)
E2E_REPS = 3                   # end-to-end repetitions (each a full setup + energy + destroy)


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# Source files that define each stage's kernel, its launch configuration and the data it
# reads: a stored DRAM measurement holds only while these are unchanged.
STAGE_SOURCES = {
    "plane_fft": ["kernels.cuh", "fft.cuh", "plan.h", "path_impl.cuh"],
    "column_fft_contract": ["kernels.cuh", "fft.cuh", "plan.h", "path_impl.cuh"],
    "w_gemm": ["kernels.cuh", "plan.h", "path_impl.cuh", "tcgen05.cuh", "gemm_tc.cuh", "gemm_tc.cu",
               "gemm_f64tc.cuh", "gemm_f64tc.cu"],
}


def source_sha(stage: str) -> str:
    h = hashlib.sha256()
    for name in sorted(STAGE_SOURCES[stage]):
        with open(os.path.join(ROOT, "paper_1611_06797_gb300", "csrc", name), "rb") as fh:
            h.update(name.encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_for(stage: str, precision: int):
    """DRAM bytes per launch of the stage's kernel from the committed ncu summary, if it was
    taken from the current sources of that kernel; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path) or stage not in STAGE_SOURCES:
        return None
    with open(path) as f:
        d = json.load(f)
    e = d.get("fp64" if precision == 0 else "fp32", {}).get(stage)
    if not e or e.get("source_sha") != source_sha(stage):
        return None
    return e.get("dram_bytes_per_launch")


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [l for l in out.splitlines() if l.strip()]
        return False

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            parts = [p.strip() for p in l.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if parts[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ CPU baseline (oracle)
def cpu_worker(workload: str, orbitals, quad_json: str, reps: int = 1):
    """Runs in a fresh process: time the FP64 oracle on a bounded sample of the workload
    (every ordered pair (i, j) of the sampled occupied orbitals), `reps` times (nothing is
    cached between repetitions), with the quadrature (tau, w) the GPU arm uses."""
    import numpy as np
    from oracle import OracleSystem, laplace_denominator, mp2_energy
    from synth import SPECS, build_model_solid
    q = json.loads(quad_json)
    tau, w = np.array(q["tau"]), np.array(q["w"])
    s = build_model_solid(SPECS[workload])
    o = OracleSystem.from_solid(s)
    pairs = [(i, j) for i in orbitals for j in orbitals]
    secs = []
    for _ in range(reps):
        t0 = time.perf_counter()
        r = mp2_energy(o, laplace_denominator(tau, w), pairs=pairs, method="fft")
        secs.append(time.perf_counter() - t0)
    e = {f"{i},{j}": float(r["e_d"][i, j] + r["e_x"][i, j]) for i, j in pairs}
    print(json.dumps({"seconds": secs, "ordered_pairs": len(pairs), "n_tau": len(tau), "e_pair": e}))


def run_cpu_baseline(workload: str, tau, w, reps: int = 1, skip: int = 0):
    """The oracle in a fresh process on all host cores; the first `skip` repetitions are warm-up.

    The sample evaluates o ordered pairs; the whole workload has n_occ^2 ordered pairs
    (each costs the oracle the same N_v^2 N_G multiply-adds), so one E_MP2 takes
    t_sample * n_occ^2 / o, and the throughput in the metric's unit is
    (n_occ (n_occ + 1) / 2) * n_tau / that time."""
    from synth import SPECS
    spec = SPECS[workload]
    cores = os.cpu_count() or 1
    env = dict(os.environ, OPENBLAS_NUM_THREADS=str(cores), OMP_NUM_THREADS=str(cores),
               MKL_NUM_THREADS=str(cores), CUDA_VISIBLE_DEVICES="")
    quad = json.dumps({"tau": [float(x) for x in tau], "w": [float(x) for x in w]})
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-worker", workload, "--quad", quad,
           "--reps", str(reps)]
    r = subprocess.run(cmd, capture_output=True, text=True, env=env, timeout=1800)
    if r.returncode != 0:
        raise RuntimeError("cpu baseline failed: " + r.stderr[-2000:])
    d = json.loads(r.stdout.strip().splitlines()[-1])
    secs = d["seconds"][skip:]
    t_sample = sum(secs) / len(secs)
    ordered_full = spec.n_occ * spec.n_occ
    t_full = t_sample * ordered_full / d["ordered_pairs"]
    value = spec.n_occ * (spec.n_occ + 1) // 2 * d["n_tau"] / t_full
    sample = (f"oracle (canonical MP2 with the Laplace denominator of the GPU arm's own (tau, w), explicit "
              f"sums over i,j,a,b; numpy FFT overlap densities + BLAS pair integrals): the "
              f"{d['ordered_pairs']} ordered pairs of occupied orbitals {list(CPU_SAMPLE_ORBITALS)} x "
              f"{d['n_tau']} tau of the {workload} workload, {t_sample:.2f} s per sample, scaled by "
              f"{ordered_full}/{d['ordered_pairs']} ordered pairs to one E_MP2 ({t_full:.0f} s)")
    return {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
            "seconds": secs, "ordered_pairs": d["ordered_pairs"], "s_per_E_MP2_extrapolated": t_full,
            "e_pair": d["e_pair"]}


def oracle_check(cb, e_pair):
    """Sampled pair energies of the timed GPU run against the oracle's (same inputs, same
    quadrature): the 1e-8 Ha parity bound, checked inside the benchmark."""
    diffs = {}
    for key, ref in cb["e_pair"].items():
        i, j = (int(x) for x in key.split(","))
        diffs[key] = abs(float(e_pair[i][j]) - ref)
    worst = max(diffs.values())
    return {"pairs": sorted(diffs), "max_abs_diff_Ha": worst, "within_1e-8_Ha": worst <= 1e-8}


# ------------------------------------------------------------------ cost model
def stage_costs(sizes, n_prim, real, reps, nxa, nv_tau, w_virtual, n_v, green_full=False):
    """Algorithmic work of `reps` ltmp2_energy calls, by stage (flops).

    Real orbitals use the real cos/sin basis: the Green's function is a real product
    (2 flops per term) and the transformed states a complex x real one (4 flops per term);
    general orbitals take complex products (8 flops per term).  Per Laplace point the
    library keeps nv_tau[k] virtuals (ltmp2_tau_virtuals); where w_virtual[k] is set the
    transformed states take two products over them (S^T R_v'^T, then times R_v') and no
    Green's function is built, else the Green's function sums over nv_tau[k] virtuals (all
    n_v on the tensor cores: green_full) and one product with it follows.  The plane FFT
    pass counts 5 n log2 n flops per line of n points: per (column, occupied i) it
    transforms n rows and nxa columns (the aux m1 range) on each of the n planes."""
    n_pw, n_occ, n = sizes["n_pw"], sizes["n_occ"], sizes["grid"]
    spp = 1 if real else 2
    ncols = n_prim * spp * n_occ
    fg, fw = (2.0, 4.0) if real else (8.0, 8.0)
    line = 5.0 * n * math.log2(n)
    green = sum(0.0 if wv else fg * n_pw * n_pw * (n_v if green_full else nv) for nv, wv in zip(nv_tau, w_virtual))
    wgemm = sum(fw * ncols * n_pw * (2.0 * nv if wv else n_pw) for nv, wv in zip(nv_tau, w_virtual))
    return {
        "green_gemm": {"flops": reps * green},
        "w_gemm": {"flops": reps * wgemm},
        "plane_fft": {"flops": reps * len(nv_tau) * ncols * n_occ * n * (n + nxa) * line},
    }


def aux_nxa(spec):
    """Width of the aux sphere's m1 range (cubic cell, E_aux = 2/3 E_cut)."""
    return 2 * int(math.floor(math.sqrt(2.0 * spec.r2 / 3.0) + 1e-12)) + 1


def measured_alu(L):
    """FP64 / FP32 FMA rates of this GPU, measured now (ltmp2_alu_peak, CUDA events)."""
    return {"fp64": L.ltmp2_alu_peak(L.FP64), "fp32": L.ltmp2_alu_peak(L.FP32),
            "kind": "measured in this run: independent FMA chains over a full grid, CUDA events, best of 5"}


def _stage_bound(stage, st, costs, precision, simt, peaks, peak_kind, alu):
    """achieved = algorithmic work per launch / mean launch time (CUDA events around each
    launch on the library's stream), against the rate that bounds the stage."""
    per_launch_ms = st[stage]["ms"] / st[stage]["launches"]
    out = {"avg_launch_ms": per_launch_ms}
    if stage in costs:
        work = costs[stage]["flops"] / st[stage]["launches"]
        if not simt and (stage == "w_gemm" or (stage == "green_gemm" and precision == 0)):
            # tensor products per real product: 3xTF32 in the precision form; in the FP64 path
            # the 36 slice products (orders s + t < 8 of 8 x 7-bit slices per operand)
            work *= 3.0 if precision != 0 else 36.0
            peak = peaks["bf16_tflops"] * TF32_OVER_BF16
            bound, pk = "tensor", f"tf32 = {peak_kind} bf16 {peaks['bf16_tflops']} x nominal 1.1/2.25"
        elif precision == 0:
            peak, bound, pk = alu["fp64"], "alu", "FP64 FMA rate " + alu["kind"]
        else:
            peak, bound, pk = alu["fp32"], "alu", "FP32 FMA rate " + alu["kind"]
        achieved = work / (per_launch_ms / 1e3) / 1e12
        out.update({"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                    "peak_kind": pk, "work_per_launch": work})
    traffic = traffic_for(stage, precision)
    if traffic:
        # DRAM bytes of a full launch (the stored capture) over the mean launch time: the
        # last slab of each tau is smaller, so this slightly overstates the rate
        gbs = traffic / (per_launch_ms / 1e3) / 1e9
        out.update({"dram_bytes_per_launch": traffic, "dram_gbs": gbs, "dram_frac": gbs / peaks["hbm_gbs"]})
    return out


def roofline_of(st, costs, precision, simt, peaks, peak_kind, alu):
    """Dominant stage against its bound."""
    dom = max(st, key=lambda k: st[k]["ms"])
    if dom not in costs or st[dom]["launches"] == 0:
        return {"kernel": dom, "bound": None, "achieved": None, "peak": None, "unit": None, "frac": None,
                "traffic": traffic_for(dom, precision)}
    r = _stage_bound(dom, st, costs, precision, simt, peaks, peak_kind, alu)
    return {"kernel": dom, "bound": r["bound"], "achieved": r["achieved"], "peak": r["peak"], "unit": "TFLOP/s",
            "frac": r["frac"], "peak_kind": r["peak_kind"], "traffic": traffic_for(dom, precision),
            "work_per_launch": r["work_per_launch"], "avg_launch_ms": r["avg_launch_ms"]}


def stage_rooflines(st, costs, precision, simt, peaks, peak_kind, alu):
    """Every timed stage against its bound, and the DRAM rate where its bytes are stored."""
    return {k: _stage_bound(k, st, costs, precision, simt, peaks, peak_kind, alu)
            for k in st if st[k]["launches"] > 0 and st[k]["ms"] > 0}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--form", default="fp64", choices=["fp64", "fp32"])
    ap.add_argument("--no-forms", action="store_true", help="skip the FP32 forms on the 24^3 workload")
    ap.add_argument("--no-workloads", action="store_true",
                    help="skip the forms on their own workloads (36^3 precision form, 8-system batch)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-worker", default=None)
    ap.add_argument("--quad", default=None)
    ap.add_argument("--reps", type=int, default=1)
    ap.add_argument("--slab", type=int, default=0, help="primary G' per slab (0 = library default)")
    ap.add_argument("--target", default="cfg5", help="learned workload: the system that is screened")
    ap.add_argument("--train", default="cfg1,cfg2,batch0,batch1,batch2,batch3,batch4,batch5,batch6,batch7,cfg3",
                    help="learned workload: systems whose exact pair energies train the model")
    ap.add_argument("--route", default="green", choices=["green", "overlap"],
                    help="transformed states from the per-tau Green's function (default) or from stored "
                         "overlap densities (the paper's steps (i)-(iii))")
    ap.add_argument("--workload", default="cfg2",
                    choices=["cfg2", "batch", "learned", "cfg3", "uhf", "fftcmp", "kpoints"],
                    help="cfg2: the 16-well 24^3 system; batch: 8 uneven systems in one graph launch; "
                         "learned: surrogate-screened pairs; cfg3: precision form on the 64-well 36^3 system")
    args = ap.parse_args()

    if args.cpu_worker:
        cpu_worker(args.cpu_worker, CPU_SAMPLE_ORBITALS, args.quad, args.reps)
        return

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "ours" and args.workload in ("batch", "learned", "cfg3", "uhf", "fftcmp", "kpoints"):
        import torch
        import paper_1611_06797_gb300 as L
        torch.cuda.set_device(local)
        if args.workload == "batch":
            out = form_batch(L, torch, local, args.steps, args.warmup)
        elif args.workload == "cfg3":
            out = form_cfg3(L, torch, local, args.steps, args.warmup)
        elif args.workload == "kpoints":
            out = form_kpoints(L, torch, local, args.steps, args.warmup)
        elif args.workload == "learned":
            out = run_learned(args, local)
        elif args.workload == "uhf":
            out = run_uhf(args, local)
        else:
            out = run_fftcmp(args, local)
        print(json.dumps(out), flush=True)
        return
    from synth import SPECS, build_model_solid
    import paper_1611_06797_gb300 as L
    spec = SPECS[WORKLOAD]
    n_tau = spec.n_tau
    pairs = spec.n_occ * (spec.n_occ + 1) // 2

    if args.impl == "reference":
        # The reference arm: the FP64 oracle on the host cores, rank 0 only, on the GPU
        # arm's workload and quadrature (ltmp2_laplace_grid is host code: no device).
        if rank != 0:
            return
        s = build_model_solid(spec)
        tau, w, _ = L.ltmp2_laplace_grid(s.gap, s.width, n_tau)
        cb = run_cpu_baseline(WORKLOAD, tau, w, reps=args.warmup + args.steps, skip=args.warmup)
        value = cb["value"]
        out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * cb["s_per_E_MP2_extrapolated"],
               "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f64",
               "data": "synthetic", "config": {"workload": _workload_desc(spec)},
               "cpu_baseline": {"value": value, "unit": UNIT, "cores": cb["cores"], "kind": "oracle",
                                "sample": cb["sample"]},
               "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(out), flush=True)
        return

    import numpy as np
    import torch
    from paper_1611_06797_gb300.shard import sharded_energy

    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)

    t0 = time.time()
    s = build_model_solid(spec)
    log(f"fixture {time.time() - t0:.1f} s; gap {s.gap:.5f} Ha, width {s.width:.3f} Ha")
    tau, w, qerr = L.ltmp2_laplace_grid(s.gap, s.width, n_tau)
    peaks, peak_kind = measured_peaks()
    alu = measured_alu(L)
    log(f"measured FMA rates: FP64 {alu['fp64']:.3f} TFLOP/s, FP32 {alu['fp32']:.2f} TFLOP/s")
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MiB > L2

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    route = L.ROUTE_OVERLAP if args.route == "overlap" else L.ROUTE_GREEN
    route_info = {}

    def evaluate(ctx):
        """One E_MP2: the whole loop on one GPU, or this rank's contiguous share of the outer
        G' loop (Sec. III B) and one FP64 sum all-reduce of (E_d, E_x, e_ij) over NCCL."""
        if dist is None:
            return L.ltmp2_energy(ctx, tau, w)

        def all_reduce_sum(v):
            t = torch.from_numpy(v).to(dev)
            dist.all_reduce(t, op=dist.ReduceOp.SUM)
            return t.cpu().numpy()
        return sharded_energy(ctx, tau, w, rank, world, all_reduce_sum)

    def time_form(precision, simt=False):
        ctx = L.setup_from_solid(s, precision=precision, real=True, simt_gemm=simt)
        L.ltmp2_set_stream(ctx, stream)
        if args.slab > 0:
            L.ltmp2_set_slab_size(ctx, args.slab)
        if route == L.ROUTE_OVERLAP:
            t_r = time.perf_counter()
            L.ltmp2_set_route(ctx, route)
            sz = L.ltmp2_sizes(ctx)
            route_info[precision] = {
                "overlap_setup_s": time.perf_counter() - t_r,
                "overlap_bytes": L.ltmp2_num_primary_gprime(ctx) * sz["n_occ"] * (s.n_orb - s.n_occ)
                * (16 if precision == L.FP64 else 8)}
        for _ in range(args.warmup):
            with torch.cuda.stream(stream):
                flush.fill_(1.0)
            evaluate(ctx)
        barrier()
        L.ltmp2_reset_stage_times(ctx)
        L.ltmp2_set_profiling(ctx, True)
        n0 = L.ltmp2_kernel_launches(ctx)
        evs = []
        with ClockSampler(local) as clk:
            barrier()
            for _ in range(args.steps):
                with torch.cuda.stream(stream):
                    flush.fill_(1.0)
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                res = evaluate(ctx)
                b.record(stream)
                evs.append((a, b))
            barrier()
        L.ltmp2_set_profiling(ctx, False)
        ms = sum(a.elapsed_time(b) for a, b in evs)
        launches = L.ltmp2_kernel_launches(ctx) - n0
        stages = L.ltmp2_stage_times(ctx)
        sizes = L.ltmp2_sizes(ctx)
        n_prim = L.ltmp2_num_primary_gprime(ctx)
        nv_tau, w_virtual = L.ltmp2_tau_virtuals(ctx, tau)
        green_full = L.ltmp2_get_tuning(ctx)["green_tc"] == 1
        L.ltmp2_destroy(ctx)
        return {"ms_total": ms, "result": res, "launches": launches, "stages": stages, "sizes": sizes,
                "n_prim": n_prim, "clocks": clk.summary(), "nv_tau": [int(x) for x in nv_tau],
                "w_virtual": [int(x) for x in w_virtual], "green_full": green_full}

    def roofline(r, precision, simt):
        n_prim = r["n_prim"]
        if dist is not None:   # this rank's share of the G' loop
            from paper_1611_06797_gb300.shard import gprime_share
            b0, e0 = gprime_share(n_prim, rank, world)
            n_prim = e0 - b0
        costs = stage_costs(r["sizes"], n_prim, True, args.steps, aux_nxa(spec), r["nv_tau"], r["w_virtual"],
                            s.n_orb - s.n_occ, r["green_full"])
        return (roofline_of(r["stages"], costs, precision, simt, peaks, peak_kind, alu),
                stage_rooflines(r["stages"], costs, precision, simt, peaks, peak_kind, alu))

    primary = L.FP64 if args.form == "fp64" else L.FP32
    r = time_form(primary)
    ms_step = r["ms_total"] / args.steps
    if dist is not None:
        t = torch.tensor([ms_step], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_step = float(t.item())
    value = pairs * n_tau / (ms_step / 1e3)   # one E_MP2 per step, on all ranks together
    ed, ex, ep = r["result"]
    sizes = r["sizes"]

    st = r["stages"]
    roof, stage_roofs = roofline(r, primary, False)

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "s_per_E_MP2": ms_step / 1e3,
        "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
        "dtype": "f64" if primary == L.FP64 else "c64/tf32x3/f64-sum",
        "data": "synthetic: seeded Gaussian-well model solid, orbitals from dense diagonalisation",
        "config": {"workload": _workload_desc(spec), "n_pw": sizes["n_pw"], "n_aux": sizes["n_aux"],
                   "n_occ": sizes["n_occ"], "grid": sizes["grid"], "n_tau": n_tau, "pairs": pairs,
                   "form": "plain FP64" if primary == L.FP64 else "precision (FP32 FFT, split GEMM)",
                   "gemm": ("FP64-accurate products on tcgen05: rows scaled by powers of two, 8 exact 7-bit "
                            "slices per operand, 36 slice products accumulated exactly in FP32 tensor memory, "
                            "FP64 sums" if primary == L.FP64 else "tcgen05 3xTF32, FP32 sums per k block"),
                   "time_reversal": True, "l2": "flushed (256 MiB write) before every timed step",
                   "laplace_max_rel_err": qerr,
                   "parallelism": (f"outer G' loop split over {world} GPUs (contiguous balanced shares), one "
                                   "FP64 sum all-reduce per E_MP2" if world > 1 else "one GPU")},
        "energy": {"E_d": ed, "E_x": ex, "E": ed + ex, "meV_per_atom": (ed + ex) * HARTREE_TO_MEV / s.n_atoms},
        "roofline": roof,
        "stage_rooflines": stage_roofs,
        "stages": {k: {"ms_per_step": v["ms"] / args.steps, "launches_per_step": v["launches"] // args.steps}
                   for k, v in st.items()},
        "clocks": r["clocks"],
        "gpu_launches": r["launches"],
        "peaks_source": peak_kind,
        "alu_peaks_tflops": alu,
    }
    out["config"]["route"] = ("overlap densities stored (paper's steps (i)-(iii))" if route == L.ROUTE_OVERLAP
                              else "per-tau Green's function")
    # virtuals kept per Laplace point (weight >= 2^-64 of the LUMO's) and the points where W
    # goes through the virtual space instead of the Green's function
    out["config"]["virtuals_per_tau"] = r["nv_tau"]
    out["config"]["w_through_virtual_space"] = r["w_virtual"]
    if route_info:
        out["route"] = {("fp64" if k == L.FP64 else "fp32"): v for k, v in route_info.items()}

    if rank == 0 and world == 1 and not args.no_forms:
        other = L.FP32 if primary == L.FP64 else L.FP64
        ro = time_form(other)
        ms_o = ro["ms_total"] / args.steps
        edo, exo, _ = ro["result"]
        d64 = (ed, ex) if primary == L.FP64 else (edo, exo)
        d32 = (edo, exo) if primary == L.FP64 else (ed, ex)
        err = {"E_d": abs(d32[0] - d64[0]) * HARTREE_TO_MEV / s.n_atoms,
               "E_x": abs(d32[1] - d64[1]) * HARTREE_TO_MEV / s.n_atoms,
               "E": abs(sum(d32) - sum(d64)) * HARTREE_TO_MEV / s.n_atoms}
        so = ro["stages"]
        ro_roof, ro_stages = roofline(ro, other, False)
        out["forms"] = {("fp32" if other == L.FP32 else "fp64"): {
            "value": pairs * n_tau / (ms_o / 1e3), "s_per_E_MP2": ms_o / 1e3,
            "speedup_vs_fp64": (ms_step / ms_o) if other == L.FP32 else (ms_o / ms_step),
            "err_vs_fp64_meV_per_atom": err, "within_0.1_meV_per_atom": max(err.values()) <= 0.1,
            "gemm": "tcgen05 3xTF32" if other == L.FP32 else "tcgen05, FP64-accurate exact slices",
            "roofline": ro_roof,
            "stage_rooflines": ro_stages,
            "stages": {k: {"ms_per_step": v["ms"] / args.steps} for k, v in so.items()},
            "gpu_launches": ro["launches"]}}
        if other == L.FP32:
            rs = time_form(L.FP32, simt=True)
            ms_s = rs["ms_total"] / args.steps
            out["forms"]["fp32_simt_gemm"] = {
                "value": pairs * n_tau / (ms_s / 1e3), "s_per_E_MP2": ms_s / 1e3,
                "speedup_vs_fp64": ms_step / ms_s,
                "err_vs_fp64_meV_per_atom": {
                    "E_d": abs(rs["result"][0] - d64[0]) * HARTREE_TO_MEV / s.n_atoms,
                    "E_x": abs(rs["result"][1] - d64[1]) * HARTREE_TO_MEV / s.n_atoms,
                    "E": abs(rs["result"][0] + rs["result"][1] - sum(d64)) * HARTREE_TO_MEV / s.n_atoms},
                "gemm": "SIMT FP32 two-level sum",
                "stages": {k: {"ms_per_step": v["ms"] / args.steps} for k, v in rs["stages"].items()}}

    if rank == 0 and world == 1 and not args.no_e2e:
        # end to end through the public API: host arrays in, host results out, every step
        times = []
        h2d = s.coeff.nbytes + s.eps.nbytes + s.miller.nbytes
        d2h = 8 * (2 + s.n_occ * s.n_occ)
        reps = min(args.steps, E2E_REPS)
        for k in range(reps):
            barrier()
            t1 = time.perf_counter()
            ctx = L.setup_from_solid(s, precision=primary, real=True)
            L.ltmp2_set_stream(ctx, stream)
            if route == L.ROUTE_OVERLAP:
                L.ltmp2_set_route(ctx, route)
            L.ltmp2_energy(ctx, tau, w)
            L.ltmp2_destroy(ctx)
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t1)
        out["e2e"] = {"value": pairs * n_tau / statistics.mean(times), "unit": UNIT,
                      "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                      "s_per_step": statistics.mean(times), "steps": reps}

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            cb = run_cpu_baseline(WORKLOAD, tau, w)
            if primary == L.FP64 and ep is not None:
                out["oracle_check"] = oracle_check(cb, ep)
            cb.pop("e_pair", None)
            out["cpu_baseline"] = cb
        except Exception as e:  # reported, never fatal
            out["cpu_baseline"] = {"value": None, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                                   "sample": f"failed: {e}"[:300]}

    if rank == 0 and world == 1 and not args.no_workloads:
        # the metric's forms on their own workloads, fixed repeat counts (steps / warm-up
        # below), so that the default run stays within minutes at any --steps
        out.setdefault("forms", {})
        for key, fn in (("cfg3_precision", form_cfg3), ("cfg4_batch", form_batch), ("kpoints_2x2x2", form_kpoints)):
            try:
                out["forms"][key] = fn(L, torch, local, 1, 1, alu=alu)
            except Exception as e:  # reported, never fatal
                out["forms"][key] = {"error": f"{type(e).__name__}: {e}"[:300]}

    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)


def form_batch(L, torch, local, steps, warmup, alu=None):
    """Batching form: the 8 uneven model solids (4..48 wells, 16^3..32^3 grids, 8..96
    occupied, 6..10 tau), precision form, every system's evaluation in one CUDA graph per
    step; compared with the same systems evaluated one after another."""
    from synth import SPECS, BATCH_NAMES, build_model_solid
    dev = torch.device("cuda", local)
    t0 = time.time()
    solids = [build_model_solid(SPECS[n], device="cuda") for n in BATCH_NAMES]
    t_fix = time.time() - t0
    log(f"batch fixtures {t_fix:.1f} s")
    quads = [L.ltmp2_laplace_grid(s.gap, s.width, s.spec.n_tau)[:2] for s in solids]
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    ctxs = [L.setup_from_solid(s, precision=L.FP32, real=True) for s in solids]
    for c in ctxs:
        L.ltmp2_set_stream(c, stream)
    t1 = time.time()
    tune = [L.ltmp2_autotune(c) for c in ctxs]
    t_tune = time.time() - t1
    units = sum(s.n_occ * (s.n_occ + 1) // 2 * s.spec.n_tau for s in solids)
    # one after another (same kernels, same tuning)
    seq = []
    for c, (t, w) in zip(ctxs, quads):
        L.ltmp2_energy(c, t, w, pairs=False)
    torch.cuda.synchronize()
    for _ in range(steps):
        with torch.cuda.stream(stream):
            flush.fill_(1.0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for c, (t, w) in zip(ctxs, quads):
            L.ltmp2_energy(c, t, w, pairs=False)
        b.record(stream)
        torch.cuda.synchronize()
        seq.append(a.elapsed_time(b))
    ref = [L.ltmp2_energy(c, t, w, pairs=False)[:2] for c, (t, w) in zip(ctxs, quads)]
    batch = L.ltmp2_batch_create(ctxs, [q[0] for q in quads], [q[1] for q in quads])
    for _ in range(warmup):
        batch.run()
    torch.cuda.synchronize()
    times = []
    with ClockSampler(local) as clk:
        for _ in range(steps):
            with torch.cuda.stream(stream):
                flush.fill_(1.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ed, ex = batch.run()
            b.record(stream)
            torch.cuda.synchronize()
            times.append(a.elapsed_time(b))
    ms = sum(times) / len(times)
    maxdiff = max(max(abs(ed[k] - ref[k][0]), abs(ex[k] - ref[k][1])) for k in range(len(solids)))
    nodes = batch.kernel_nodes()
    persistent = batch.persistent()
    batch.destroy()
    # end to end: setup from host arrays + autotune (cached) + one batch evaluation + destroy
    t1 = time.perf_counter()
    c2 = [L.setup_from_solid(s, precision=L.FP32, real=True) for s in solids]
    for c in c2:
        L.ltmp2_set_stream(c, stream)
    L.ltmp2_energy_batch(c2, [q[0] for q in quads], [q[1] for q in quads])
    for c in c2:
        L.ltmp2_destroy(c)
    for c in ctxs:
        L.ltmp2_destroy(c)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t1
    return {
        "metric": METRIC, "value": units / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": steps,
        "warmup": warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c64/tf32x3/f64-sum",
        "data": "synthetic: 8 seeded Gaussian-well model solids, orbitals from dense diagonalisation",
        "config": {"workload": "batching form: " + ", ".join(
            f"{s.spec.wells} wells {s.spec.grid}^3 {s.n_pw} PW {s.n_occ} occ {s.spec.n_tau} tau" for s in solids),
                   "systems": len(solids), "pair_tau_units": units, "form": "precision, one CUDA graph per step",
                   "graph_mode": ("rounds with shared persistent FFT stages" if persistent
                                  else "one graph branch per system (round counts too uneven for lockstep)"),
                   "l2": "flushed (256 MiB write) before every timed step",
                   "autotune": [{"slab": t[0], "gemm_variant": t[1]} for t in tune]},
        "sequential_ms_per_step": sum(seq) / len(seq), "speedup_vs_sequential": (sum(seq) / len(seq)) / ms,
        "max_abs_diff_vs_sequential_Ha": maxdiff, "graph_kernel_nodes": nodes,
        "gpu_launches": nodes * steps, "graph_launches": steps, "clocks": clk.summary(),
        "setup_s": {"fixtures": t_fix, "autotune": t_tune},
        "e2e": {"value": units / e2e_s, "unit": UNIT, "s_per_step": e2e_s,
                "h2d_bytes_per_step": int(sum(s.coeff.nbytes + s.eps.nbytes + s.miller.nbytes for s in solids)),
                "d2h_bytes_per_step": 16 * len(solids)},
    }


def run_learned(args, local):
    """Learned form on its own workload: 128 wells, 40^3 grid, 20,005 plane waves, 256 occupied
    orbitals (32,896 pairs), 10 Laplace points, precision form.  The pair model is trained on
    the exact exchange pair energies (ln|e^x_ij| labels from ltmp2_learned_training_data) of
    the 12^3 and 24^3 systems, the 8 batching systems and the 36^3 system; ltmp2_energy_screened
    then screens the cfg5 pairs for a budget of 0.1 meV/atom.  The all-pairs contraction of
    the same inputs is timed beside it and measures the realised error."""
    import numpy as np
    import torch
    import paper_1611_06797_gb300 as L
    from paper_1611_06797_gb300 import learned as LF
    from synth import SPECS, BATCH_NAMES, build_model_solid
    dev = torch.device("cuda", local)
    train_names = [n for n in args.train.split(",") if n and n != args.target]
    t0 = time.time()
    sets = []
    for nm in train_names:
        sp = build_model_solid(SPECS[nm], device="cuda")
        t, w, _ = L.ltmp2_laplace_grid(sp.gap, sp.width, sp.spec.n_tau)
        c = L.setup_from_solid(sp, precision=L.FP32, real=True)
        sets.append(L.ltmp2_learned_training_data(c, t, w))
        L.ltmp2_destroy(c)
    y = np.concatenate([v for _, v in sets])
    t_label = time.time() - t0
    t1 = time.time()
    margin = LF.calibrate_margin(sets, epochs=4000, seed=5)
    net = LF.train(sets, epochs=4000, seed=5)
    t_train = time.time() - t1
    spec = SPECS[args.target]
    t2 = time.time()
    s = build_model_solid(spec, device="cuda")
    t_fix = time.time() - t2
    log(f"learned: labels {t_label:.0f} s, train {t_train:.0f} s, cfg5 fixture {t_fix:.0f} s")
    tau, w, qerr = L.ltmp2_laplace_grid(s.gap, s.width, spec.n_tau)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    c = L.setup_from_solid(s, precision=L.FP32, real=True)
    L.ltmp2_set_stream(c, stream)
    budget = 0.1 / HARTREE_TO_MEV * s.n_atoms
    L.ltmp2_energy(c, tau[:1], w[:1], pairs=False)     # warm-up: one Laplace point

    def timed(fn):
        with torch.cuda.stream(stream):
            flush.fill_(1.0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        r = fn()
        b.record(stream)
        torch.cuda.synchronize()
        return r, a.elapsed_time(b)
    n_prim = L.ltmp2_num_primary_gprime(c)
    # the screening decision first (descriptors, model, rule: the library's own calls)
    X = L.ltmp2_pair_descriptors(c).astype(np.float32)
    keep, n_sel, _ = L.ltmp2_screen_select(s.n_occ, margin * np.exp(net.predict(X).astype(np.float64)), budget)
    with ClockSampler(local) as clk:
        # all pairs, with the exact exchange of every pair (the reference for the realised error, and the ceiling below)
        (ed, ex, pd, px), ms_all = timed(lambda: L.ltmp2_energy_partial(c, tau, w, 0, n_prim))
        if n_sel > 0:
            r, ms_scr = timed(lambda: L.ltmp2_energy_screened(c, net, tau, w, budget, margin))
        else:   # no pair qualifies: the screened evaluation is the all-pairs one
            r = {"E_d": ed, "E_x": ex, "E_x_contracted": ex, "E_x_estimated": 0.0, "screened_pairs": 0,
                 "pairs": s.n_occ * (s.n_occ + 1) // 2}
            ms_scr = ms_all
    L.ltmp2_destroy(c)
    pairs = s.n_occ * (s.n_occ + 1) // 2
    per_atom = HARTREE_TO_MEV / s.n_atoms
    # ceiling of any screening at this budget: with every |e^x_ij| known exactly, the
    # largest set of off-diagonal pairs whose dropped exchange stays within the budget
    iu = np.triu_indices(s.n_occ, 1)
    exact = np.sort(np.abs(px[iu] + px.T[iu]))
    ceiling = int(np.searchsorted(np.cumsum(exact), budget, side="right"))
    return {
        "metric": METRIC, "value": pairs * spec.n_tau / (ms_scr / 1e3), "unit": UNIT, "n_gpus": 1,
        "steps": 1, "warmup": 1, "ms_per_step": ms_scr, "s_per_E_MP2": ms_scr / 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "c64/tf32x3/f64-sum",
        "data": "synthetic: seeded Gaussian-well model solids, orbitals from dense diagonalisation",
        "config": {"workload": _workload_desc(spec) + "; learned form: pair model trained on " +
                   ",".join(train_names) + f" ({len(y)} exact pair labels)", "budget_meV_per_atom": 0.1,
                   "laplace_max_rel_err": qerr},
        "all_pairs": {"s_per_E_MP2": ms_all / 1e3, "value": pairs * spec.n_tau / (ms_all / 1e3),
                      "E_d": ed, "E_x": ex},
        "speedup_vs_all_pairs": ms_all / ms_scr,
        "screened_pairs": r["screened_pairs"], "pairs": r["pairs"],
        "screened_fraction": r["screened_pairs"] / max(1, r["pairs"] - s.n_occ),
        "ceiling_with_exact_pair_energies": {"pairs": ceiling, "fraction": ceiling / max(1, len(exact)),
                                             "smallest_pair_exchange_Ha": float(exact[0]),
                                             "median_pair_exchange_Ha": float(np.median(exact))},
        "estimated_screened_exchange_Ha": r["E_x_estimated"],
        "err_vs_all_pairs_meV_per_atom": {
            "E_d": abs(r["E_d"] - ed) * per_atom, "E_x": abs(r["E_x"] - ex) * per_atom,
            "E": abs(r["E_d"] + r["E_x"] - ed - ex) * per_atom,
            "E_dropping_screened": abs(r["E_x_contracted"] - ex) * per_atom},
        "within_0.1_meV_per_atom": abs(r["E_d"] + r["E_x"] - ed - ex) * per_atom <= 0.1,
        "mlp": {"train_loss_std_units": net.loss, "train_s": t_train, "label_s": t_label, "samples": int(len(y)),
                "residual_ln": net.residual(), "screening_margin": margin,
                "margin_from": "leave-one-system-out over the training systems, lowest 2 % of predictions, x2"},
        "clocks": clk.summary(), "setup_s": {"fixture": t_fix},
    }


def form_cfg3(L, torch, local, steps, warmup, alu=None):
    """Precision form on its own workload: 64 wells, 36^3 grid, 10059 plane waves, 128
    occupied orbitals, 10 Laplace points (FP32 FFTs, 3xTF32 tcgen05 GEMM, FP64 sums).
    A full FP64 evaluation of this system takes about 45 minutes on one GB300, so the
    error against the FP64 path is measured on the same inputs over four spread ranges
    of the outer G' loop (ltmp2_energy_partial, 24 of 2724 primary G'), where both paths
    run; it is reported in meV/atom on the sample and scaled to the full G' loop as if
    every sampled error had the same sign (a conservative estimate)."""
    from synth import SPECS, build_model_solid
    spec = SPECS["cfg3"]
    dev = torch.device("cuda", local)
    if alu is None:
        alu = measured_alu(L)
    t0 = time.time()
    s = build_model_solid(spec, device="cuda")
    t_fix = time.time() - t0
    log(f"cfg3 fixture {t_fix:.1f} s; gap {s.gap:.6f} Ha, width {s.width:.3f} Ha")
    n_tau = spec.n_tau
    tau, w, qerr = L.ltmp2_laplace_grid(s.gap, s.width, n_tau)
    peaks, peak_kind = measured_peaks()
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    pairs = s.n_occ * (s.n_occ + 1) // 2
    ctx = L.setup_from_solid(s, precision=L.FP32, real=True)
    L.ltmp2_set_stream(ctx, stream)
    for _ in range(warmup):   # one Laplace point per warm-up step
        L.ltmp2_energy(ctx, tau[:1], w[:1], pairs=False)
    torch.cuda.synchronize()
    L.ltmp2_reset_stage_times(ctx)
    L.ltmp2_set_profiling(ctx, True)
    n0 = L.ltmp2_kernel_launches(ctx)
    evs = []
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        for _ in range(steps):
            with torch.cuda.stream(stream):
                flush.fill_(1.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ed, ex, _ = L.ltmp2_energy(ctx, tau, w, pairs=False)
            b.record(stream)
            evs.append((a, b))
        torch.cuda.synchronize()
    L.ltmp2_set_profiling(ctx, False)
    ms = sum(a.elapsed_time(b) for a, b in evs) / steps
    launches = (L.ltmp2_kernel_launches(ctx) - n0) // steps
    st = L.ltmp2_stage_times(ctx)
    sizes = L.ltmp2_sizes(ctx)
    n_prim = L.ltmp2_num_primary_gprime(ctx)
    tuning = L.ltmp2_get_tuning(ctx)
    nv_tau, w_virtual = L.ltmp2_tau_virtuals(ctx, tau)
    costs = stage_costs(sizes, n_prim, True, steps, aux_nxa(spec), nv_tau, w_virtual, s.n_orb - s.n_occ,
                        tuning["green_tc"] == 1)
    roof = roofline_of(st, costs, L.FP32, False, peaks, peak_kind, alu)
    stage_roofs = stage_rooflines(st, costs, L.FP32, False, peaks, peak_kind, alu)
    # FP32 vs FP64 on the same inputs, over sampled G' ranges
    width = 6
    starts = [0, n_prim // 3, (2 * n_prim) // 3, n_prim - width]
    t1 = time.time()
    c64 = L.setup_from_solid(s, precision=L.FP64, real=True)
    samp = {"fp64": [0.0, 0.0], "fp32": [0.0, 0.0]}
    for g0 in starts:
        d, x, _, _ = L.ltmp2_energy_partial(c64, tau, w, g0, g0 + width)
        samp["fp64"][0] += d
        samp["fp64"][1] += x
        d, x, _, _ = L.ltmp2_energy_partial(ctx, tau, w, g0, g0 + width)
        samp["fp32"][0] += d
        samp["fp32"][1] += x
    L.ltmp2_destroy(c64)
    L.ltmp2_destroy(ctx)
    t_cmp = time.time() - t1
    scale = n_prim / (width * len(starts))
    per_atom = HARTREE_TO_MEV / s.n_atoms
    err = {"E_d": abs(samp["fp32"][0] - samp["fp64"][0]) * per_atom,
           "E_x": abs(samp["fp32"][1] - samp["fp64"][1]) * per_atom,
           "E": abs(sum(samp["fp32"]) - sum(samp["fp64"])) * per_atom}
    return {
        "metric": METRIC, "value": pairs * n_tau / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": steps,
        "warmup": warmup, "ms_per_step": ms, "s_per_E_MP2": ms / 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "c64/tf32x3/f64-sum",
        "data": "synthetic: seeded Gaussian-well model solid, orbitals from dense diagonalisation",
        "config": {"workload": _workload_desc(spec), "n_pw": sizes["n_pw"], "n_aux": sizes["n_aux"],
                   "n_occ": sizes["n_occ"], "grid": sizes["grid"], "n_tau": n_tau, "pairs": pairs,
                   "form": "precision (FP32 FFT, 3xTF32 tcgen05 GEMM, FP64 sums)", "time_reversal": True,
                   "l2": "flushed (256 MiB write) before every timed step; inputs exceed L2",
                   "laplace_max_rel_err": qerr, "tuning": tuning},
        "energy": {"E_d": ed, "E_x": ex, "E": ed + ex, "meV_per_atom": (ed + ex) * per_atom},
        "roofline": roof,
        "stage_rooflines": stage_roofs,
        "stages": {k: {"ms_per_step": v["ms"] / steps, "launches_per_step": v["launches"] // steps}
                   for k, v in st.items()},
        "clocks": clk.summary(), "gpu_launches": launches, "peaks_source": peak_kind,
        "setup_s": {"fixture": t_fix},
        "err_vs_fp64_sampled": {
            "sample": f"primary G' [{', '.join(f'{g}..{g + width - 1}' for g in starts)}] of {n_prim}, all "
                      f"{n_tau} tau, all pairs; FP32 and FP64 paths on the same inputs",
            "meV_per_atom_on_sample": err,
            "meV_per_atom_scaled_to_full_loop": {k: v * scale for k, v in err.items()},
            "within_0.1_meV_per_atom_scaled": max(err.values()) * scale <= 0.1,
            "sample_energy_fp64": samp["fp64"], "seconds": t_cmp},
        "cpu_baseline": {"value": None, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                         "sample": "not run: one occupied pair of this system costs the oracle ~5e11 complex "
                                   "multiply-adds (N_v^2 N_G), beyond a bounded sample"},
    }


def form_kpoints(L, torch, local, steps, warmup, alu=None, mesh=(2, 2, 2)):
    """k-point sampling (Sec. II C-D): the 2-well 6 bohr cell of the 12^3 workload (515 plane
    waves, 2 occupied bands per k) on a 2 x 2 x 2 mesh, 6 Laplace points, in both precisions;
    against the Gamma-point path on the same physics, the 12 bohr supercell with 16 wells
    (4120 plane waves {k + G}, 24^3 grid, 16 occupied), which the k-point path replaces."""
    from synth import SPECS, build_kpoint_pair
    from synth.model_solid import well_positions
    spec = SPECS["cfg1"]
    dev = torch.device("cuda", local)
    t0 = time.time()
    ks, sc = build_kpoint_pair(spec.a, spec.grid, spec.r2, mesh, well_positions(spec), 2, seed=spec.seed,
                               device="cuda")
    t_fix = time.time() - t0
    n_tau = 6
    tau, w, qerr = L.ltmp2_laplace_grid(ks.gap, ks.width, n_tau)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    NO = ks.n_k * ks.n_occ
    units = NO * (NO + 1) // 2 * n_tau
    per_atom = HARTREE_TO_MEV / ks.n_atoms
    res = {}

    def timed(ctx, reps):
        L.ltmp2_set_stream(ctx, stream)
        for _ in range(warmup):
            L.ltmp2_energy(ctx, tau, w, pairs=False)
        torch.cuda.synchronize()
        L.ltmp2_reset_stage_times(ctx)
        L.ltmp2_set_profiling(ctx, True)
        n0 = L.ltmp2_kernel_launches(ctx)
        evs = []
        with ClockSampler(local) as clk:
            for _ in range(reps):
                with torch.cuda.stream(stream):
                    flush.fill_(1.0)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                r = L.ltmp2_energy(ctx, tau, w, pairs=False)
                b.record(stream)
                evs.append((a, b))
            torch.cuda.synchronize()
        L.ltmp2_set_profiling(ctx, False)
        st = L.ltmp2_stage_times(ctx)
        out = {"ms": sum(x.elapsed_time(y) for x, y in evs) / reps, "E_d": r[0], "E_x": r[1],
               "launches": (L.ltmp2_kernel_launches(ctx) - n0) // reps, "clocks": clk.summary(),
               "stages": {k: {"ms_per_step": v["ms"] / reps} for k, v in st.items()}}
        L.ltmp2_destroy(ctx)
        return out
    for prec, key in ((L.FP64, "fp64"), (L.FP32, "fp32")):
        res[key] = timed(L.setup_from_kpoint_solid(ks, precision=prec), steps)
    ctx = L.ltmp2_setup(sc.lattice, sc.grid, sc.miller, sc.coeff, sc.eps, sc.n_occ, 2 * ks.ecut / 3, L.FP64, 0)
    res["gamma_supercell_fp64"] = timed(ctx, 1)
    k64, k32, g64 = res["fp64"], res["fp32"], res["gamma_supercell_fp64"]
    return {
        "metric": METRIC, "value": units / (k64["ms"] / 1e3), "unit": UNIT, "n_gpus": 1, "steps": steps,
        "warmup": warmup, "ms_per_step": k64["ms"], "s_per_E_MP2": k64["ms"] / 1e3, "higher_is_better": True,
        "dtype": "f64", "data": "synthetic: seeded Gaussian-well model solid on a k-mesh, dense diagonalisation per k",
        "config": {"workload": f"k-point form: cfg1 cell (a={spec.a} bohr, 2 wells, {spec.grid}^3 grid, "
                               f"{ks.n_pw} plane waves shared by every k), {mesh[0]}x{mesh[1]}x{mesh[2]} mesh, "
                               f"2 occupied bands per k ({NO} composite occupied), {n_tau} tau; pair units over "
                               f"the composite occupied orbitals", "n_k": ks.n_k, "indirect_gap_Ha": ks.gap,
                   "laplace_max_rel_err": qerr,
                   "supercell": f"{sc.n_pw} plane waves, {int(sc.grid[0])}^3 grid, {sc.n_occ} occupied, "
                                f"{ks.n_atoms * ks.n_k} wells"},
        "energy_per_cell": {"E_d": k64["E_d"], "E_x": k64["E_x"]},
        "forms": {"fp32": {"s_per_E_MP2": k32["ms"] / 1e3, "speedup_vs_fp64": k64["ms"] / k32["ms"],
                           "err_vs_fp64_meV_per_atom": {"E_d": abs(k32["E_d"] - k64["E_d"]) * per_atom,
                                                        "E_x": abs(k32["E_x"] - k64["E_x"]) * per_atom}}},
        "gamma_supercell": {"s_per_E_MP2": g64["ms"] / 1e3, "kpoint_speedup": g64["ms"] / k64["ms"],
                            "abs_diff_per_cell_Ha": {"E_d": abs(g64["E_d"] / ks.n_k - k64["E_d"]),
                                                     "E_x": abs(g64["E_x"] / ks.n_k - k64["E_x"])},
                            "stages": g64["stages"]},
        "stages": k64["stages"], "gpu_launches": k64["launches"], "clocks": k64["clocks"],
        "setup_s": {"fixtures": t_fix},
    }


def run_uhf(args, local):
    """Spin-unrestricted form on the 24^3 cell: alpha with 33 and beta with 31 singly
    occupied orbitals, the beta electrons in wells of 0.9 x the depth (synthetic spin
    polarisation); plain FP64, and the precision form's error against it."""
    import torch
    import paper_1611_06797_gb300 as L
    from synth import SPECS, spin_polarized_pair
    spec = SPECS["cfg2"]
    dev = torch.device("cuda", local)
    a, b = spin_polarized_pair(spec, 33, 31)
    n_tau = spec.n_tau
    lo, hi = min(a.gap, b.gap), max(a.width, b.width)
    tau, w, qerr = L.ltmp2_laplace_grid(lo, hi, n_tau)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    res = {}
    for prec in (L.FP64, L.FP32):
        ca = L.setup_from_solid(a, precision=prec, real=True)
        cb = L.setup_from_solid(b, precision=prec, real=True)
        L.ltmp2_set_stream(ca, stream)
        L.ltmp2_set_stream(cb, stream)
        for _ in range(args.warmup):
            L.ltmp2_energy_uhf(ca, cb, tau[:1], w[:1])
        n0 = L.ltmp2_kernel_launches(ca)
        evs = []
        with ClockSampler(local) as clk:
            torch.cuda.synchronize()
            for _ in range(args.steps):
                with torch.cuda.stream(stream):
                    flush.fill_(1.0)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                r = L.ltmp2_energy_uhf(ca, cb, tau, w)
                e1.record(stream)
                evs.append((e0, e1))
            torch.cuda.synchronize()
        res[prec] = {"ms": sum(x.elapsed_time(y) for x, y in evs) / args.steps, "result": r,
                     "launches": (L.ltmp2_kernel_launches(ca) - n0) // args.steps, "clocks": clk.summary()}
        L.ltmp2_destroy(ca)
        L.ltmp2_destroy(cb)
    r64, r32 = res[L.FP64], res[L.FP32]
    units = (a.n_occ * (a.n_occ + 1) // 2 + b.n_occ * (b.n_occ + 1) // 2 + a.n_occ * b.n_occ) * n_tau
    per_atom = HARTREE_TO_MEV / a.n_atoms
    ed, ex, es = r64["result"]
    out = {
        "metric": METRIC, "value": units / (r64["ms"] / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r64["ms"], "s_per_E_MP2": r64["ms"] / 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic: seeded Gaussian-well model solid, two spin channels from dense diagonalisation",
        "config": {"workload": _workload_desc(spec) + "; spin-unrestricted: alpha 33, beta 31 singly occupied, "
                   "beta wells of depth 1.8 Ha (alpha 2.0 Ha)", "pair_units": "same-spin i<=j pairs of each "
                   "channel plus all opposite-spin pairs, times tau", "laplace_max_rel_err": qerr},
        "energy": {"E_d": ed, "E_x": ex, "E": ed + ex, "E_same_alpha": es[0], "E_same_beta": es[1],
                   "E_opposite": es[2]},
        "gpu_launches": r64["launches"], "clocks": r64["clocks"],
        "forms": {"fp32": {"s_per_E_MP2": r32["ms"] / 1e3, "speedup_vs_fp64": r64["ms"] / r32["ms"],
                           "err_vs_fp64_meV_per_atom": {
                               "E_d": abs(r32["result"][0] - ed) * per_atom,
                               "E_x": abs(r32["result"][1] - ex) * per_atom,
                               "E": abs(r32["result"][0] + r32["result"][1] - ed - ex) * per_atom}}},
    }
    return out


def run_fftcmp(args, local):
    """cuFFT, timed only as a comparison: batched complex 3D FFTs of the co-density size
    (torch.fft.fftn, inputs larger than L2), scaled to the number of co-density transforms
    one Laplace point needs on the 24^3 workload (one per (G', j, i) item), against the
    library's plane + column stages, which also form the products conj(phi_i) w_j, prune to
    the auxiliary sphere and contract.  Both precisions."""
    import torch
    import paper_1611_06797_gb300 as L
    from synth import SPECS, build_model_solid
    spec = SPECS["cfg2"]
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    s = build_model_solid(spec)
    tau, w, _ = L.ltmp2_laplace_grid(s.gap, s.width, spec.n_tau)
    n = spec.grid
    out = {"metric": "cuFFT comparison", "config": {"workload": _workload_desc(spec)}, "results": {}}
    for prec, dt in ((L.FP32, torch.complex64), (L.FP64, torch.complex128)):
        ctx = L.setup_from_solid(s, precision=prec, real=True)
        L.ltmp2_set_profiling(ctx, True)
        L.ltmp2_energy(ctx, tau[:1], w[:1], pairs=False)
        L.ltmp2_reset_stage_times(ctx)
        L.ltmp2_energy(ctx, tau[:2], w[:2], pairs=False)
        st = L.ltmp2_stage_times(ctx)
        items = L.ltmp2_num_primary_gprime(ctx) * s.n_occ * s.n_occ
        L.ltmp2_destroy(ctx)
        ours = (st["plane_fft"]["ms"] + st["column_fft_contract"]["ms"]) / 2
        batch = 1024 if prec == L.FP32 else 512   # 113 MB in, 113 MB out: above the L2
        x = torch.randn(batch, n, n, n, dtype=dt, device=dev)
        for _ in range(3):
            y = torch.fft.fftn(x, dim=(1, 2, 3))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        reps = 5
        for _ in range(reps):
            y = torch.fft.fftn(x, dim=(1, 2, 3))
        b.record()
        torch.cuda.synchronize()
        per_fft_ms = a.elapsed_time(b) / reps / batch
        del x, y
        out["results"]["fp32" if prec == L.FP32 else "fp64"] = {
            "cufft_ms_per_fft": per_fft_ms, "ffts_per_tau": items,
            "cufft_transforms_only_ms_per_tau": per_fft_ms * items,
            "ours_plane_plus_column_ms_per_tau": ours,
            "ratio_cufft_over_ours": per_fft_ms * items / ours}
    # cuBLAS on the transformed-state product of one full slab (4096 complex columns =
    # 8192 stacked real rows times the real n_pw x n_pw Green's function), against the
    # library's kernel for the same launch (bench stage time per launch)
    npw = s.n_pw
    rows = 2 * 128 * s.n_occ
    torch.backends.cuda.matmul.allow_tf32 = False
    for prec, dt in ((L.FP64, torch.float64), (L.FP32, torch.float32)):
        A = torch.randn(rows, npw, dtype=dt, device=dev)
        B = torch.randn(npw, npw, dtype=dt, device=dev)
        for _ in range(3):
            C = A @ B
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        for _ in range(5):
            C = A @ B
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / 5
        ctx = L.setup_from_solid(s, precision=prec, real=True)
        L.ltmp2_set_profiling(ctx, True)
        L.ltmp2_energy(ctx, tau[:1], w[:1], pairs=False)
        L.ltmp2_reset_stage_times(ctx)
        L.ltmp2_energy(ctx, tau[:1], w[:1], pairs=False)
        st = L.ltmp2_stage_times(ctx)["w_gemm"]
        L.ltmp2_destroy(ctx)
        key = "gemm_fp64" if prec == L.FP64 else "gemm_fp32"
        out["results"][key] = {
            "shape": [rows, npw, npw], "cublas": "DGEMM" if prec == L.FP64 else "SGEMM (TF32 off)",
            "cublas_ms": ms, "cublas_tflops": 2.0 * rows * npw * npw / ms / 1e9,
            "ours_ms_per_launch": st["ms"] / max(1, st["launches"]),
            "ours": "k_rgemm FP64 (SIMT)" if prec == L.FP64 else "tcgen05 3xTF32 (k_tc_cgemm_stacked + packing)"}
        del A, B, C
    return out


def _workload_desc(spec):
    return (f"{spec.name}: cubic cell a={spec.a} bohr, {spec.wells} Gaussian wells (A=2 Ha, s=0.8 bohr) on a "
            f"jittered {spec.lattice_sites} site lattice, {spec.grid}^3 grid, plane-wave sphere r^2<={spec.r2} "
            f"(index units), {spec.n_occ} occupied, all other states virtual, {spec.n_tau} Laplace points, "
            f"E_aux = 2/3 E_cut, Gamma point, closed shell")


if __name__ == "__main__":
    main()
