"""Benchmark of the CVS-ADC(2) hot path on GB300.

Metric: CVS-ADC(2) sigma builds/s and time-to-roots, mixed vs FP64.

Timed step: one sigma build M x over a block of 4 trial vectors of the
large workload (two metal L-edges: ncore 12, nval 120, nvirt 600, naux
3000, 16 roots; N = 258 775 200 CVS-packed amplitudes, 4.14 GB per
complex128 vector) through the full sigma path -- doubles unpack, the
B^P coupling GEMMs, the <Kb||Ij> terms through the stored 1-external
block, M22 applied on the fly, CVS packing, the dense M11 x1 -- in the
mixed precision (tensor-core exact-slice GEMMs, SLICE4), with the problem
prepared on the device (t2 bands, M11) and the inputs (B^P, 25.7 GB,
larger than L2) resident in HBM.  value = sigma builds per second over all
ranks.

Also reported on the same line: sigma builds/s of the other precisions,
time-to-roots of full solves (mixed vs FP64-class, and their root
difference) on the small, medium and large workloads, the e2e sigma rate
through the C ABI with host buffers, the roofline of the tcgen05 slice GEMM
from CUDA-event timing of its launches inside the timed region, SM clocks
sampled during the timed region, and a CPU baseline (the oracle's
matrix-free sigma on a bounded sample of the same workload).

--impl reference times that CPU oracle alone (the reference arm).
Multi-GPU (torchrun): independent replicas, one per GPU (weak scaling).
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from synth import WORKLOADS, make_instance, physical_scale  # noqa: E402

METRIC = "CVS-ADC(2) sigma builds/s and time-to-roots, mixed vs FP64 (≤1e-5 Eh), 1 GB300"
UNIT = "sigma builds/s"
WORKLOAD = "large"
NVEC = 4
PRODUCTS = {"slice4": 10, "fp64_slice7": 28, "bf16x3": 3}


def n_amplitudes(w):
    return w["ncore"] * w["nvirt"] + w["ncore"] * w["nval"] * w["nvirt"] * (w["nvirt"] - 1) // 2


def workload_config(prec):
    w = WORKLOADS[WORKLOAD]
    n = w["ncore"] + w["nval"] + w["nvirt"]
    return {
        "workload": "%s CVS-ADC(2): ncore %d, nval %d, nvirt %d, naux %d, %d roots; "
                    "sigma on %d-vector Davidson blocks" % (
                        WORKLOAD, w["ncore"], w["nval"], w["nvirt"], w["naux"], w["nroots"],
                        NVEC),
        "precision": prec,
        "n_amplitudes": n_amplitudes(w),
        "l2": "inputs larger than L2 (B^P %.1f GB, trial block %.1f GB)" % (
            w["naux"] * n * n * 16 / 1e9, NVEC * n_amplitudes(w) * 16 / 1e9),
        "inputs": "seeded synthetic (synth.make_instance, seed 0)",
    }


# --------------------------------------------------------------- helpers

def max_over_ranks(ms, ws, device):
    """The slowest rank's time (ms): every rank contributes its own timed
    region, the job takes as long as the slowest replica."""
    if ws <= 1:
        return ms
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(ws, units_per_step, steps, t_max_ms):
    """Units per second over all ranks (weak scaling: each rank does
    units_per_step per step on its own replica)."""
    return ws * units_per_step * steps / (t_max_ms / 1e3)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clock and throttle samples while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.lines = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "fallback": True}


def traffic_from_profile(kernel):
    """Per-launch DRAM bytes of one kernel at the bench's launch shape, from
    its committed ncu summary profiles/<kernel>_large_sigma.md (None when
    absent or recorded as null)."""
    p = os.path.join(ROOT, "profiles", "%s_large_sigma.md" % kernel)
    try:
        for line in open(p):
            if line.startswith("traffic_bytes_per_launch:"):
                v = line.split(":", 1)[1].strip()
                return None if v in ("", "null") else float(v)
    except OSError:
        pass
    return None


# --------------------------------------------------------- CPU baseline

class OracleSigmaSample:
    """The oracle's matrix-free sigma of one vector in bounded units: a unit
    is the coupling block of one valence spinor j (explicit <ab||cj>)
    restricted to `rows` values of the first virtual index; nval x
    ceil(nvirt / rows) units plus one whole-vector doubles unpack and pack
    make one sigma build."""

    def __init__(self, inst, rows):
        from oracle import adc2

        self.adc2 = adc2
        nc, nw, nv = inst.ncore, inst.nval, inst.nvirt
        self.nw, self.nv, self.rows = nw, nv, min(rows, nv)
        N1, _, N2 = adc2.sizes(nc, nw, nv)
        # the dense M11 x1 product is N1^2 multiply-adds, negligible next to
        # the couplings; a zero M11 keeps the oracle from building it
        self.sig = adc2.Sigma(inst.eps, inst.B, nc, nw, nv,
                              M11=np.zeros((N1, N1), complex), cache_blocks=False)
        rng = np.random.default_rng(1)
        x = rng.standard_normal(N1 + N2) + 1j * rng.standard_normal(N1 + N2)
        self.X = x[:N1].reshape(nc, nv)
        t0 = time.perf_counter()
        self.Y = adc2.unpack(x[N1:], nc, nw, nv)
        s2 = np.zeros((nc, nw, nv, nv), dtype=np.complex128)
        adc2.pack(s2, nv)
        self.t_vector = time.perf_counter() - t0
        self.nslice = (nv + self.rows - 1) // self.rows
        self.units = nw * self.nslice
        self.i = 0

    def unit(self):
        j, q = divmod(self.i % self.units, self.nslice)
        r = slice(q * self.rows, min(self.nv, (q + 1) * self.rows))
        self.sig.coupling_block(self.X, self.Y, j, r)
        self.i += 1

    def rate(self, t_unit):
        """sigma builds/s from the mean time of one unit."""
        return 1.0 / (self.t_vector + self.units * t_unit)


def cpu_baseline(inst, seconds_hint=20.0, rows=None):
    """The oracle's matrix-free sigma, timed on a bounded sample of units
    (see OracleSigmaSample), scaled to one sigma build."""
    smp = OracleSigmaSample(inst, rows or inst.nvirt)
    t0 = time.perf_counter()
    n = 0
    while True:
        smp.unit()
        n += 1
        if time.perf_counter() - t0 > seconds_hint or n >= smp.units:
            break
    dt = time.perf_counter() - t0
    try:
        import threadpoolctl

        cores = max(i.get("num_threads", 1) for i in threadpoolctl.threadpool_info()) or os.cpu_count()
    except Exception:
        cores = os.cpu_count()
    return {"value": smp.rate(dt / n), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "oracle matrix-free sigma (explicit <ab||cj> per valence spinor) of the "
                      "%s workload, one vector: %d of %d units (valence spinor x %d rows "
                      "of the first virtual index) in %.1f s, scaled to all units, plus one "
                      "whole-vector doubles unpack and pack (%.1f s)" % (
                          WORKLOAD, n, smp.units, smp.rows, dt, smp.t_vector)}


# ------------------------------------------------------------- our arm

def run_ours(args):
    import torch

    import paper_2604_27451_gb300 as pkg
    from paper_2604_27451_gb300 import _lib

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    lib = _lib.load()
    prec = args.precision
    w = WORKLOADS[WORKLOAD]
    inst = make_instance(w["ncore"], w["nval"], w["nvirt"], w["naux"], seed=0)
    nc, nw, nv = inst.ncore, inst.nval, inst.nvirt
    stream = torch.cuda.current_stream(dev)
    ctx = pkg.Context(local, stream=stream.cuda_stream)
    eps = torch.from_numpy(inst.eps).to(dev)
    B = torch.from_numpy(inst.B).to(dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    # sigma needs no transition moments: prepared without dipoles
    ctx.prepare(eps, B, None, nc, nw, nv, precision=prec)
    torch.cuda.synchronize()
    prepare_s = time.perf_counter() - t0
    del B  # the library holds its own copy of B^P
    torch.cuda.empty_cache()
    N = ctx.shape["N"]
    g = torch.Generator(device=dev).manual_seed(11)
    X = torch.randn(NVEC, N, dtype=torch.complex128, device=dev, generator=g)
    X /= torch.linalg.vector_norm(X, dim=1, keepdim=True)
    S = torch.empty_like(X)

    def barrier():
        if ws > 1:
            import torch.distributed as dist

            dist.barrier()

    for _ in range(args.warmup):
        ctx.sigma(X, prec, out=S)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    lib.cvsadc_kernel_stats_reset()
    lib.cvsadc_kernel_timing(1)
    launches0 = lib.cvsadc_launch_count()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            ctx.sigma(X, prec, out=S)
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    launches = lib.cvsadc_launch_count() - launches0
    lib.cvsadc_kernel_timing(0)
    ms_total = ev0.elapsed_time(ev1)
    import ctypes

    kid = {"slice4": 1, "fp64_slice7": 1, "bf16x3": 0, "fp64": 2}[prec]
    cnt, kms, kfl = ctypes.c_int64(), ctypes.c_double(), ctypes.c_double()
    lib.cvsadc_kernel_stats(kid, ctypes.byref(cnt), ctypes.byref(kms), ctypes.byref(kfl))
    # max time over ranks
    t_max = max_over_ranks(ms_total, ws, dev)
    ms_per_step = t_max / args.steps
    value = whole_job_rate(ws, NVEC, args.steps, t_max)

    # roofline of the dominant kernel (CUDA-event timed inside the region)
    peaks = measured_peaks()
    roofline = None
    if cnt.value > 0 and prec in PRODUCTS:
        achieved = kfl.value / (kms.value / 1e3) / 1e12
        peak = peaks["bf16_tflops"] / PRODUCTS[prec]
        kname = {"slice4": "tc_slice4r_kernel", "fp64_slice7": "tc_slice_kernel",
                 "bf16x3": "tc_gemm_kernel"}[prec]
        roofline = {"bound": "tensor", "achieved": round(achieved, 2), "peak": round(peak, 2),
                    "unit": "TFLOP/s", "frac": round(achieved / peak, 4),
                    "traffic": traffic_from_profile(kname),
                    "kernel": kname,
                    "launches": int(cnt.value), "avg_launch_ms": round(kms.value / cnt.value, 4),
                    "share_of_step_time": round(kms.value / ms_total, 4),
                    "peak_basis": "measured bf16 burst %.1f TFLOP/s / %d bf16 products per "
                                  "algorithmic product (of measured)" % (
                                      peaks["bf16_tflops"], PRODUCTS[prec]),
                    "tensor_pipe_frac": round(achieved * PRODUCTS[prec] / peaks["bf16_tflops"], 4)}
    elif cnt.value > 0:
        achieved = kfl.value / (kms.value / 1e3) / 1e12
        roofline = {"bound": "alu", "achieved": round(achieved, 3), "peak": 1.1, "unit": "TFLOP/s",
                    "frac": round(achieved / 1.1, 4), "traffic": None, "kernel": "zgemm_f64_kernel",
                    "peak_basis": "cuBLAS DGEMM measured on this pool, 1.10 TFLOP/s"}

    out = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "c128 via %s tensor-core GEMMs" % prec if prec != "fp64" else "c128 (FP64 FMA)",
        "data": "synthetic", "config": workload_config(prec),
        "prepare_s": round(prepare_s, 3), "gpu_launches": int(launches),
        "clocks": clk.summary(), "roofline": roofline,
    }
    if rank == 0 and not args.core_only:
        state = {"ctx": ctx, "X": X, "S": S}
        del X, S
        out.update(extras(args, state, inst, stream, torch, pkg))
    elif rank == 0:
        out["e2e"] = None
    if rank == 0:
        print(json.dumps(out), flush=True)
    ctx.close()
    if ws > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


def extras(args, state, inst, stream, torch, pkg):
    """Everything on the JSON line besides the timed step.  state holds the
    prepared context and the trial block; both are released before the full
    solves so that those start from an empty device."""
    res = {}
    ctx, X = state["ctx"], state["X"]
    dev = X.device
    only_large = args.ttr_large_only
    if only_large:
        state.clear()
        del X
        ctx.close()
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
    # sigma builds/s of the other precisions on (part of) the same block;
    # FP64 FMA runs at ~1.1 TFLOP/s on this GPU: one vector is minutes at the
    # large workload, so it is timed on the medium solve below instead
    rates = {}
    for p, nvec in () if only_large else (("bf16x3", NVEC), ("slice4", NVEC), ("fp64_slice7", 2)):
        xs = X[:nvec].contiguous()
        ss = torch.empty_like(xs)
        ctx.sigma(xs, p, out=ss)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.sigma(xs, p, out=ss)
        e1.record(stream)
        torch.cuda.synchronize()
        rates[p] = round(nvec / (e0.elapsed_time(e1) / 1e3), 3)
        del xs, ss
    if not only_large:
        res["sigma_builds_per_s"] = rates
        res.update(_e2e_and_release(args, state, X, ctx, torch))
        del X

    # time-to-roots: full solves (prepare + Davidson + refinement) with
    # inputs resident, mixed vs FP64; the Schur-complement preconditioner
    # is on unless the entry says "diag"
    def solve_entry(e_, B_, d_, w, p, precond="schur", conv=1e-7, refine=True):
        c2 = pkg.Context(dev.index, stream=stream.cuda_stream)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        o = c2.solve(e_, B_, d_, w["ncore"], w["nval"], w["nvirt"], w["nroots"],
                     precision=p, conv=conv, precond=precond, refine=refine)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        c2.close()
        i = o["info"]
        return o["omega"].cpu().numpy(), {
            "s": round(dt, 3), "status": int(o["status"]), "iterations": i["iterations"],
            "sigma_vectors": i["sigma_vectors"], "coupling_vectors": i["coupling_vectors"],
            "schur_builds": i["schur_builds"], "t_schur_s": round(i["t_schur_ms"] / 1e3, 3),
            "t_prepare_s": round(i["t_prepare_ms"] / 1e3, 3)}

    if not only_large:
        res.update(_small_medium_ttr(args, dev, torch, solve_entry))
    if args.ttr_large:
        res.update(_large_ttr(args, inst, dev, torch, solve_entry))
    if not args.no_cpu_baseline and not only_large:
        res["cpu_baseline"] = cpu_baseline(inst, args.cpu_seconds, rows=max(1, inst.nvirt // 8))
    return res


def _e2e_and_release(args, state, X, ctx, torch):
    """e2e: the public API with host buffers (pinned), copies inside; then
    the prepared context and the trial block are released."""
    res = {}
    N = X.shape[1]
    xh = torch.empty((NVEC, N), dtype=torch.complex128, pin_memory=True)
    xh.copy_(X)
    sh = torch.empty_like(xh).pin_memory()
    xn, sn = xh.numpy(), sh.numpy()
    ctx.sigma(xn, args.precision, out=sn)
    reps = 2
    t0 = time.perf_counter()
    for _ in range(reps):
        ctx.sigma(xn, args.precision, out=sn)
    dt = (time.perf_counter() - t0) / reps
    nb = NVEC * N * 16
    res["e2e"] = {"value": round(NVEC / dt, 3), "unit": UNIT, "h2d_bytes_per_step": nb,
                  "d2h_bytes_per_step": nb,
                  "path": "cvsadc_sigma through the C ABI with pinned host buffers"}
    del xh, sh, xn, sn
    state.clear()
    ctx.close()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return res


def _small_medium_ttr(args, dev, torch, solve_entry):
    """Time-to-roots on the small and medium workloads, mixed vs FP64."""
    res = {}
    w = WORKLOADS["small"]
    sm = make_instance(w["ncore"], w["nval"], w["nvirt"], w["naux"], seed=0)
    e_, B_, d_ = (torch.from_numpy(a).to(dev) for a in (sm.eps, sm.B, sm.dip))
    ttr = {"workload": "small CVS-ADC(2): ncore 6, nval 14, nvirt 40, naux 240, 4 roots, "
                       "residual 1e-7, inputs resident"}
    roots = {}
    for p, pc in (("slice4", "schur"), ("fp64_slice7", "schur"), ("fp64", "schur"),
                  ("fp64", "diag")):
        key = p if pc == "schur" else p + "_diag_precond"
        roots[key], ttr[key] = solve_entry(e_, B_, d_, w, p, pc)
    ttr["max_abs_root_diff_mixed_vs_fp64_Eh"] = float(np.abs(roots["slice4"] - roots["fp64"]).max())
    ttr["max_abs_root_diff_fp64_slice7_vs_fp64_Eh"] = float(np.abs(roots["fp64_slice7"] - roots["fp64"]).max())
    ttr["speedup_mixed_vs_fp64"] = round(ttr["fp64"]["s"] / ttr["slice4"]["s"], 2)
    res["time_to_roots"] = ttr
    del e_, B_, d_
    # the medium workload: mixed vs FP64-class (7-slice) time-to-roots
    wm = WORKLOADS["medium"]
    me = make_instance(wm["ncore"], wm["nval"], wm["nvirt"], wm["naux"], seed=0)
    e_, B_, d_ = (torch.from_numpy(a).to(dev) for a in (me.eps, me.B, me.dip))
    ttm = {"workload": "medium CVS-ADC(2): ncore %d, nval %d, nvirt %d, naux %d, %d roots, "
                       "residual 1e-6, inputs resident" % (
                           wm["ncore"], wm["nval"], wm["nvirt"], wm["naux"], wm["nroots"])}
    rm = {}
    for p in ("slice4", "fp64_slice7") + (("fp64",) if args.ttr_medium_fp64 else ()):
        rm[p], ttm[p] = solve_entry(e_, B_, d_, wm, p, conv=1e-6)
    for p in rm:
        if p != "slice4":
            ttm["max_abs_root_diff_slice4_vs_%s_Eh" % p] = float(np.abs(rm["slice4"] - rm[p]).max())
            ttm["speedup_slice4_vs_%s" % p] = round(ttm[p]["s"] / ttm["slice4"]["s"], 2)
    ttm["roots_Eh"] = [round(float(x), 9) for x in rm["slice4"]]
    res["time_to_roots_medium"] = ttm
    del e_, B_, d_, me
    torch.cuda.empty_cache()
    return res


def _large_ttr(args, inst, dev, torch, solve_entry):
    """Time-to-roots on the large shape (the doubles-folded solver).  At the
    stated Cholesky scale (0.3) the large problem is far from perturbative:
    |M| is ~1e5 Eh against roots of ~7 Eh, so a residual of 1e-6 asks for
    ~1e-11 relative accuracy of every sigma and neither path gets there.
    The solves run on the companion instance of the same shape and seed at
    the size-aware physical scale (synth.physical_scale), whose roots are
    singles-dominated core excitations below the doubles."""
    res = {}
    if args.ttr_large:
        # the full-space subspace does not fit: the doubles-folded solver
        # runs (singles-space vectors only)
        wl = WORKLOADS["large"]
        sc = physical_scale(wl["nval"], wl["nvirt"])
        comp = make_instance(wl["ncore"], wl["nval"], wl["nvirt"], wl["naux"], seed=0, scale=sc)
        e_ = torch.from_numpy(comp.eps).to(dev)
        B_ = torch.from_numpy(comp.B).to(dev)
        del comp
        ttl = {"workload": "large CVS-ADC(2) shape: ncore %d, nval %d, nvirt %d, naux %d, %d "
                           "roots, residual 1e-6, inputs resident, no dipoles; companion "
                           "instance at the physical Cholesky scale %.5f (seed 0)" % (
                               wl["ncore"], wl["nval"], wl["nvirt"], wl["naux"], wl["nroots"],
                               sc)}
        rl = {}
        for p in args.ttr_large.split(","):
            rl[p], ttl[p] = solve_entry(e_, B_, None, wl, p.replace("_norefine", ""), conv=1e-6,
                                        refine=not p.endswith("_norefine"))
        # every entry against the FP64-class (7-slice) solve
        ref_key = "fp64_slice7"
        for p in rl:
            if p != ref_key and ref_key in rl:
                ttl["max_abs_root_diff_%s_vs_%s_Eh" % (p, ref_key)] = float(
                    np.abs(rl[p] - rl[ref_key]).max())
                ttl["speedup_%s_vs_%s" % (p, ref_key)] = round(ttl[ref_key]["s"] / ttl[p]["s"], 2)
        ttl["roots_Eh"] = {p: [round(float(x), 9) for x in r] for p, r in rl.items()}
        res["time_to_roots_large"] = ttl
        del e_, B_
        torch.cuda.empty_cache()
    return res


# ------------------------------------------------------- reference arm

def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return
    w = WORKLOADS[WORKLOAD]
    inst = make_instance(w["ncore"], w["nval"], w["nvirt"], w["naux"], seed=0)
    # one step = one unit of the oracle's sigma: a valence spinor's coupling
    # block on a slice of rows, sized to a few seconds
    smp = OracleSigmaSample(inst, max(1, w["nvirt"] // 24))
    for _ in range(args.warmup):
        smp.unit()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        smp.unit()
    dt = time.perf_counter() - t0
    v = smp.rate(dt / args.steps)
    try:
        import threadpoolctl

        cores = max(i.get("num_threads", 1) for i in threadpoolctl.threadpool_info()) or os.cpu_count()
    except Exception:
        cores = os.cpu_count()
    cb = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
          "sample": "oracle matrix-free sigma of the %s workload, one vector: each step one "
                    "unit (a valence spinor's <ab||cj> coupling block on %d rows of the "
                    "first virtual index, %d units per sigma), scaled, plus one whole-vector "
                    "doubles unpack and pack (%.1f s)" % (WORKLOAD, smp.rows, smp.units,
                                                           smp.t_vector)}
    out = {"metric": METRIC, "value": round(v, 8), "unit": UNIT, "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": round(dt / args.steps * 1e3, 1), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
           "config": workload_config("fp64 (CPU oracle)"), "impl": "reference",
           "cpu_baseline": cb,
           "e2e": {"value": round(v, 8), "unit": UNIT, "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_profile_gemm(args):
    """One complex GEMM of 4096 x 4096 x 4096 (operands 268 MB each, larger
    than L2) in the given precision, repeated 3 times: the small case the
    ncu capture of the tensor-core kernel uses."""
    import torch

    import paper_2604_27451_gb300 as pkg

    ctx = pkg.Context(0)
    g = torch.Generator(device="cuda").manual_seed(3)
    A = torch.randn(4096, 4096, dtype=torch.complex128, device="cuda", generator=g)
    Bm = torch.randn(4096, 4096, dtype=torch.complex128, device="cuda", generator=g)
    for _ in range(3):
        ctx.zgemm(A, Bm, args.precision)
    torch.cuda.synchronize()
    print(json.dumps({"profile_gemm": "4096^3", "precision": args.precision}))


def run_batched(args):
    """The batched workload: the first K of the 48 ragged instances (ncore 6,
    nval U{20..80}, nvirt U{100..400}, naux 5 nvirt, 4 roots, seeds 1000+i),
    solved through cvsadc_solve_batched with one lane and with four."""
    import torch

    import paper_2604_27451_gb300 as pkg
    from synth import batched_shapes

    shapes = batched_shapes(48)[: args.batched]
    insts = []
    for sh in shapes:
        inst = make_instance(sh["ncore"], sh["nval"], sh["nvirt"], sh["naux"], seed=sh["seed"])
        insts.append(dict(eps=torch.from_numpy(inst.eps).cuda(),
                          B=torch.from_numpy(inst.B).cuda(), dip=None,
                          ncore=sh["ncore"], nval=sh["nval"], nvirt=sh["nvirt"]))
        del inst
    ctx = pkg.Context(0)
    out = {"metric": "batched CVS-ADC(2) instances/s", "unit": "instances/s",
           "config": {"workload": "first %d of 48 ragged instances: ncore 6, nval U{20..80}, "
                                  "nvirt U{100..400}, naux 5 nvirt, 4 roots, residual 1e-6, "
                                  "SLICE4 + refinement, inputs resident" % len(shapes),
                      "shapes": [(s["nval"], s["nvirt"], s["naux"]) for s in shapes]}}
    omegas = {}
    for lanes in (1, 4):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = ctx.solve_batched(insts, 4, precision="slice4", conv=1e-6, lanes=lanes)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        omegas[lanes] = np.array([r["omega"].cpu().numpy() for r in res])
        out["lanes_%d" % lanes] = {
            "s": round(dt, 3), "value": round(len(insts) / dt, 4),
            "status": [r["status"] for r in res],
            "iterations": [r["info"]["iterations"] for r in res],
            "t_total_s": [round(r["info"]["t_total_ms"] / 1e3, 2) for r in res]}
    out["speedup_4_lanes"] = round(out["lanes_1"]["s"] / out["lanes_4"]["s"], 3)
    out["max_abs_root_diff_lanes"] = float(np.abs(omegas[1] - omegas[4]).max())
    ctx.close()
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="slice4",
                    choices=["slice4", "fp64_slice7", "bf16x3", "fp64"])
    ap.add_argument("--core-only", action="store_true",
                    help="only the timed sigma steps (used for profiling)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--batched", type=int, default=0,
                    help="time K instances of the batched workload instead")
    ap.add_argument("--ttr-medium-fp64", action="store_true",
                    help="also time the FP64 solve of the medium workload (minutes)")
    ap.add_argument("--ttr-large", default="",
                    help="comma-separated precisions whose full solve of the large "
                         "workload is timed (e.g. slice4,fp64_slice7; a _norefine "
                         "suffix skips the FP64-class continuation)")
    ap.add_argument("--ttr-large-only", action="store_true",
                    help="after the timed steps, only the --ttr-large solves")
    ap.add_argument("--profile-gemm", action="store_true",
                    help="run one 4096^3 complex GEMM three times (ncu case)")
    args = ap.parse_args()
    if args.profile_gemm:
        run_profile_gemm(args)
    elif args.batched:
        run_batched(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
