#!/usr/bin/env python3
"""Throughput of DSBlockCG on one GB300: (rhs x shift) systems solved per second.

A step is one complete solve (sigma_j I + D^H D) X_j = B, j = 1..12, for
12 right-hand sides on a 16^3 x 32 lattice (Wilson, kappa = 0.125, smooth
random SU(3) links), to a true FP64 relative residual <= 1e-8 for every
(rhs, shift): FP32 storage of fields and links, FP32 arithmetic on them,
IEEE FP64 block coefficients, deflation, shift recurrences, true residuals
and restarts (reliable updates).  Inputs are resident in HBM when the timed
region starts and the working set of one block step (~9 GB) is far larger
than L2.  The double-float form of the reliable updates (an opt-in of the
library) is timed beside it over the same number of steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  With N > 1 (launched by torch.distributed.run)
every rank solves its own replica; the value is all ranks' systems divided by
the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "w2_16x16x16x32"
METRIC = "(rhs×shift) systems/s at true residual 1e-8; D†D stencil GB/s vs HBM peak"
UNIT = "systems/s"
KCLASS = ["dslash", "gram", "update", "shift", "small", "residual", "other"]


# Conventional Wilson-Dirac flop count per site and field for one D
# application: 1320 for the eight hops (spin projection, SU(3) multiply,
# reconstruction, accumulation) plus 48 for the diagonal term.
WILSON_FLOP_PER_SITE = 1368


def fp64_alu_peak_tflops(sm_mhz):
    """FP64 FMA peak of a GB300 from unit counts and the SM clock: 152 SMs,
    each with 4 sub-partitions that retire one warp-wide (32-lane) FP64
    instruction every 64 cycles, i.e. 2 FP64 FMA (4 flop) per SM per clock."""
    return 152 * 2 * 2 * float(sm_mhz) * 1e6 / 1e12


def fp32_alu_peak_tflops(sm_mhz):
    """FP32 FMA peak of a GB300 from unit counts and the SM clock: 152 SMs x
    128 FP32 lanes, one FMA (2 flop) per lane per clock.  The packed FMA
    (fma.rn.f32x2) the shift update uses halves the instructions per FMA; it
    is counted against this same per-lane rate."""
    return 152 * 128 * 2 * float(sm_mhz) * 1e6 / 1e12


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def workload_config(wl, storage, reliable="FP64"):
    return {
        "workload": (f"{WORKLOAD}: Wilson D^H D on {'x'.join(map(str, wl['dims']))}, kappa {wl['kappa']}, "
                     f"m={wl['B'].shape[0]} Z2 RHS, s={len(wl['sigma'])} shifts "
                     f"{wl['sigma'][0]:.0e}..{wl['sigma'][-1]:.0e}, true residual <= {wl['tol']:.0e}, "
                     f"{storage} storage + {reliable} reliable updates and m x m work"),
        "lattice": list(wl["dims"]), "m": int(wl["B"].shape[0]), "s": int(len(wl["sigma"])),
        "tol": wl["tol"], "storage": storage,
        "l2": "no flush: one block step streams ~9 GB, far above the 129 MB L2",
    }


# ----------------------------------------------------------------- clocks --
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.dev)], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    rows.append(dict(sm=float(parts[1]), smax=float(parts[2]),
                                     power=float(parts[3]) if parts[3] not in ("[N/A]", "") else 0.0,
                                     hw=parts[5], hwt=parts[6], swt=parts[7], swp=parts[8]))
                except ValueError:
                    continue
        os.unlink(self.path)
        if not rows:
            return None
        reasons = set()
        for r in rows:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                              ("swt", "sw_thermal_slowdown"), ("swp", "sw_power_cap")):
                if r[key].lower() == "active":
                    reasons.add(name)
        loaded = [r["sm"] for r in rows]
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(r["smax"] for r in rows),
                "power_w_max": max(r["power"] for r in rows), "samples": len(rows),
                "reasons": sorted(reasons)}


# --------------------------------------------------------------- traffic --
def ncu_traffic(kclass):
    """DRAM bytes / algorithmic bytes of a kernel class from the committed ncu
    summary, or None when the summary is missing or the kernel source changed."""
    path = os.path.join(ROOT, "profiles", "traffic.md")
    if not os.path.exists(path):
        return None
    src_hash = kernel_source_hash()
    for line in open(path):
        m = re.match(r"\|\s*" + kclass + r"\s*\|\s*([0-9.eE+]+)\s*\|\s*([0-9a-f]+)\s*\|", line)
        if m and m.group(2) == src_hash:
            return float(m.group(1))
    return None


def strip_comments(src):
    """C/C++ source without // and /* */ comments and with whitespace runs
    collapsed (string literals in the kernels hold no comment markers)."""
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    src = re.sub(r"//[^\n]*", " ", src)
    return " ".join(src.split())


def kernel_source_hash():
    """Hash of the device-code sources (every csrc file but the host
    orchestration in solver.cu), comments and whitespace removed: a change
    to the code invalidates the committed ncu figures, one to a comment does
    not."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1205_0359_gb300", "csrc")
    for name in sorted(os.listdir(csrc)):
        if name.endswith((".cu", ".cuh", ".h")) and name != "solver.cu":
            with open(os.path.join(csrc, name), encoding="utf-8") as f:
                h.update(name.encode())
                h.update(strip_comments(f.read()).encode())
    return h.hexdigest()[:12]


# ------------------------------------------------------------ CPU oracle --
def oracle_sample(wl, vectors, total_vectors):
    """Time the FP64 oracle (numpy band-Lanczos DSBlockCG) on the same workload
    for `vectors` Lanczos vectors and scale to a whole solve of
    `total_vectors` vectors.  Returns (systems/s, cores used, seconds)."""
    from oracle import wilson as W
    from oracle.dsbcg import dsbcg as oracle_dsbcg
    U, k, dims = wl["U"], wl["kappa"], wl["dims"]
    Aop = lambda v: W.A_vec(U, k, dims, v)
    c0, t0 = time.process_time(), time.perf_counter()
    oracle_dsbcg(Aop, wl["B"], wl["sigma"], wl["tol"], freeze=False, stop_after_vectors=vectors)
    wall = time.perf_counter() - t0
    cpu = time.process_time() - c0
    per_vec = wall / vectors
    systems = wl["B"].shape[0] * len(wl["sigma"])
    return systems / (per_vec * total_vectors), max(1, round(cpu / wall)), wall, per_vec


# ------------------------------------------------------- replica timing --
def max_over_ranks(x, world, device):
    """The largest of a per-rank float over the process group (the job is as
    slow as its slowest replica); x itself at world size 1."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(world, m, s, solves, seconds):
    """Whole-job (rhs x shift) systems/s of `world` independent replicas that
    each ran `solves` solves of m x s systems in `seconds` (the slowest's)."""
    return world * m * s * solves / seconds


# ------------------------------------------------------------- our arm --
def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_1205_0359_gb300 import dsbcg, synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wl = synth.make_workload(WORKLOAD, dims=args.lattice)
    m, s = wl["B"].shape[0], len(wl["sigma"])
    n = wl["B"].shape[1]
    stream = torch.cuda.current_stream(dev)
    ctx = dsbcg.Context(wl["dims"], torch.from_numpy(wl["U"]).to(dev), wl["kappa"], stream=stream)
    B = torch.from_numpy(wl["B"]).to(dev)
    X = torch.empty((s, m, n), dtype=torch.complex128, device=dev)

    def solve(storage=args.storage, Bx=B, Xx=X, fp64res=True):
        _, st = ctx.solve(Bx, wl["sigma"], wl["tol"], storage=storage, out=Xx, fp64_residuals=fp64res)
        return st

    for _ in range(args.warmup):
        solve()
    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    stats = [solve() for _ in range(args.steps)]
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms_total = max_over_ranks(ev0.elapsed_time(ev1), world, dev)
    ms_step = ms_total / args.steps
    value = replica_value(world, m, s, args.steps, ms_total / 1e3)
    maxrel = max(float(st["true_relres"].max()) for st in stats)
    ok = all(st["code"] == 0 for st in stats) and maxrel <= wl["tol"]
    Xmix = X.clone()                       # the headline solution, for the FP64 comparison

    # per-kernel breakdown: one more solve with the library's per-launch CUDA
    # events on (restarts then run one at a time, so that each class's event
    # time is its own); its result is bitwise the same as the timed solves'
    ctx.set_profiling(True)
    prof_steps = 1
    stats = [solve() for _ in range(prof_steps)]
    ctx.set_profiling(False)

    kms = {q: sum(st["kernel_ms"][q] for st in stats) for q in KCLASS}
    kby = {q: sum(st["kernel_bytes"][q] for st in stats) for q in KCLASS}
    kla = {q: sum(st["kernel_launches"][q] for st in stats) for q in KCLASS}
    kfl = {q: sum(st["kernel_flops"][q] for st in stats) for q in KCLASS}
    peak, peak_kind = load_peaks()
    kernels = {}
    for q in KCLASS:
        if kms[q] > 0:
            gbs = kby[q] / (kms[q] / 1e3) / 1e9
            kernels[q] = {"ms_per_step": kms[q] / prof_steps, "launches_per_step": kla[q] / prof_steps,
                          "GB_per_step": kby[q] / prof_steps / 1e9, "GBps": gbs,
                          "frac_of_hbm": gbs / peak}
            if kfl[q] > 0:
                kernels[q]["TFLOPs"] = kfl[q] / (kms[q] / 1e3) / 1e12
    # HBM-bound classes in the reduced-precision storage; the true-residual
    # class runs the FP64 stencil, which is bound by the FP64 pipe, and the
    # shift update (P_j, X_j on chip over a chunk of steps) by the FP32 FMA pipe
    hbm_bound = [q for q in ("dslash", "gram", "update") if q in kernels]
    dom = max(hbm_bound, key=lambda q: kms[q])
    clk_mhz = (clk or {}).get("sm_mhz") or 2070.0

    def roof(q):
        achieved = kby[q] / (kms[q] / 1e3) / 1e9
        ratio = ncu_traffic(q)
        per_launch = kby[q] / kla[q] if kla[q] else 0.0
        return {"kernel": q, "bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                "unit": "GB/s", "frac": round(achieved / peak, 4),
                "traffic": (None if ratio is None else round(ratio * per_launch / 1e9, 4)),
                "traffic_unit": "GB per launch",
                "algorithmic_GB_per_launch": round(kby[q] / kla[q] / 1e9, 4) if kla[q] else None,
                "peak_source": f"{peak_kind} HBM copy bandwidth"}

    def residual_roof():
        """FP64 true residuals r = b - sigma x - A x: each call applies D and
        D^H to its fields (FP64 stencil, 1368 flop per site and field each)
        plus a streaming residual kernel; the class's flops over its event
        time against the FP64 ALU peak at the sampled SM clock."""
        calls = kla["residual"] / 4.0                 # 2 stencils + residual + column reduction
        V = wl["B"].shape[1] // 12
        nfields = (kby["residual"] / 16.0 - 72.0 * V * calls) / (8.0 * wl["B"].shape[1])
        flop = 2.0 * WILSON_FLOP_PER_SITE * V * nfields
        ach = flop / (kms["residual"] / 1e3) / 1e12
        pk = fp64_alu_peak_tflops(clk_mhz)
        return {"kernel": "residual (FP64 stencil D, D^H + r = b - sigma x - A x)", "bound": "alu",
                "achieved": round(ach, 4), "peak": round(pk, 4), "unit": "TFLOP/s", "frac": round(ach / pk, 4),
                "traffic": None, "flop_per_solve": flop, "fields_per_solve": round(nfields, 1),
                "ms_per_solve": round(kms["residual"], 3),
                "peak_source": f"derived: 152 SMs x 2 FP64 FMA/clock x 2 flop x {clk_mhz:.0f} MHz (sampled)"}

    def shift_roof():
        """Shift update over chunks of block steps: X_j += P_j Ut_j and
        P_j <- V_{k+1} - P_j Lh_j for every active shift and step, 8 flop per
        complex multiply-add (the library's count from the block widths of
        every step), against the FP32 FMA peak at the sampled SM clock."""
        ach = kfl["shift"] / (kms["shift"] / 1e3) / 1e12
        pk = fp32_alu_peak_tflops(clk_mhz)
        return {"kernel": "shift (chunked per-shift update, packed FP32 FMA)", "bound": "alu",
                "achieved": round(ach, 3), "peak": round(pk, 3), "unit": "TFLOP/s", "frac": round(ach / pk, 4),
                "traffic": None, "flop_per_solve": kfl["shift"], "ms_per_solve": round(kms["shift"], 3),
                "peak_source": f"derived: 152 SMs x 128 FP32 FMA/clock x 2 flop x {clk_mhz:.0f} MHz (sampled)"}

    alu = [q for q in ("residual", "shift") if q in kernels and (q == "residual" or kfl[q] > 0)]
    top = max(hbm_bound + alu, key=lambda q: kms[q])
    top_roof = {"residual": residual_roof, "shift": shift_roof}.get(top, lambda: roof(top))
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": workload_config(wl, args.storage),
        "valid": ok, "max_true_relres": maxrel,
        "solver": {"block_steps": stats[-1]["block_steps"], "restarts": stats[-1]["restarts"],
                   "mvms": stats[-1]["mvms"], "deflations": stats[-1]["deflations"]},
        "roofline": top_roof(),
        "hbm_roofline": roof(dom),
        "stencil_roofline": roof("dslash"),
        "kernels": kernels,
        "kernels_from": "one extra solve with per-launch CUDA events (restarts serialised)",
        # launches per solve are the same with and without the events
        "gpu_launches": int(round(sum(kla.values()) / prof_steps * args.steps)),
    }
    if "residual" in kernels:
        line["residual_roofline"] = residual_roof()
    if "shift" in alu:
        line["shift_roofline"] = shift_roof()
    if clk is not None:
        line["clocks"] = clk
    ctx.set_profiling(False)

    # e2e: the same solve through the C ABI with pinned host buffers
    Bh = torch.empty((m, n), dtype=torch.complex128, pin_memory=True)
    Bh.copy_(torch.from_numpy(wl["B"]))
    Xh = torch.empty((s, m, n), dtype=torch.complex128, pin_memory=True)
    solve(Bx=Bh, Xx=Xh)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        solve(Bx=Bh, Xx=Xh)
    torch.cuda.synchronize(dev)
    e2e_s = max_over_ranks((time.perf_counter() - t0) / args.steps, world, dev)
    line["e2e"] = {"value": round(replica_value(world, m, s, 1, e2e_s), 3), "unit": UNIT,
                   "h2d_bytes_per_step": int(Bh.numel() * 16), "d2h_bytes_per_step": int(Xh.numel() * 16)}

    # the same mixed solve with the library's opt-in double-float reliable
    # updates and m x m work (dsbcg_params.fp64_residuals = 0), timed over
    # the same number of steps as the headline
    if rank == 0 and not args.no_df32:
        for _ in range(args.warmup):
            solve(fp64res=False)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        stf = [solve(fp64res=False) for _ in range(args.steps)]
        e1.record(stream)
        torch.cuda.synchronize(dev)
        tf = e0.elapsed_time(e1) / 1e3 / args.steps
        line["double_float_reliable_updates"] = {
            "value": round(m * s / tf, 3), "unit": UNIT, "ms_per_step": round(tf * 1e3, 1), "steps": args.steps,
            "block_steps": stf[-1]["block_steps"], "restarts": stf[-1]["restarts"],
            "max_true_relres": float(max(st["true_relres"].max() for st in stf)),
            "note": ("FP32 storage; true residuals, solution accumulation and m x m work in double-float "
                     "(48-bit significands on the FP32 pipes), the library's opt-in")}

    # gauge-link force of the gradient workload (16^3 x 32, m = s = 8, FP32):
    # dsbcg_force on device X and adjoint Lambda, whole call and force kernel
    if rank == 0 and not args.no_force:
        wf = synth.make_workload("w4_force_16x16x16x32")
        fctx = dsbcg.Context(wf["dims"], torch.from_numpy(wf["U"]).to(dev), wf["kappa"], stream=stream)
        fm, fs = wf["B"].shape[0], len(wf["sigma"])
        fn = wf["B"].shape[1]
        g = torch.Generator(device=dev).manual_seed(44)
        Xf = torch.randn((fs, fm, fn), dtype=torch.complex128, device=dev, generator=g)
        Lf = torch.randn((fs, fm, fn), dtype=torch.complex128, device=dev, generator=g)
        dU = fctx.force(Xf, Lf, wf["weights"], storage="fp32")
        torch.cuda.synchronize(dev)
        nfr = 3
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(nfr):
            fctx.force(Xf, Lf, wf["weights"], storage="fp32", out=dU)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        call_ms = e0.elapsed_time(e1) / nfr
        fctx.set_profiling(True)
        fctx.read_profile()
        fctx.force(Xf, Lf, wf["weights"], storage="fp32", out=dU)
        kst, _ = fctx.read_profile()
        fctx.set_profiling(False)
        nf = fs * fm
        V = fn // 12
        # force kernel: four FP32 fields of nf spinors in, 36 FP64 link entries per site out
        fbytes = 4.0 * nf * fn * 8 + V * 36 * 16
        kms = kst.get("other", 0.0)
        line["force"] = {
            "workload": "w4_force 16x16x16x32, m=8, s=8, FP32 storage",
            "ms_per_call": round(call_ms, 3), "kernel_ms": round(kms, 3),
            "kernel_GBps": round(fbytes / (kms / 1e3) / 1e9, 1) if kms > 0 else None,
            "kernel_frac_of_hbm": round(fbytes / (kms / 1e3) / 1e9 / peak, 4) if kms > 0 else None,
            "note": "call = pack X and Lambda to FP32, D on both, force kernel, dU out (device buffers)"}
        fctx.close()
        del Xf, Lf, dU

    def leg(key, fn):
        """An optional leg: its error is recorded in the line, never raised."""
        try:
            line[key] = fn()
        except Exception as e:                   # noqa: BLE001 - a failed leg must not cost the line
            line[key] = {"error": repr(e)[:400]}
        torch.cuda.synchronize(dev)
        torch.cuda.empty_cache()

    if rank == 0 and not args.no_compare:
        leg("comparison", lambda: run_comparison(dev, stream))
        leg("comparison_near_critical", lambda: run_comparison(dev, stream, name="cmp_critical_16x16x16x16"))
    clk_mhz = (clk or {}).get("sm_mhz") or 2070.0
    if rank == 0 and not args.no_w3:
        leg("w3_precision_ladder", lambda: run_w3_ladder(dev, stream, peak, clk_mhz))
    if rank == 0 and not args.no_schur:
        leg("schur_operator", lambda: run_schur(dev, stream, wl, value / world, stats[-1]))
    if rank == 0 and args.sweeps:
        line["sweeps"] = run_sweeps(dev, stream)

    fp64_mvms = None
    if rank == 0 and not args.no_fp64:
        X64 = torch.empty_like(X)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st64 = solve(storage="fp64", Xx=X64)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        t64 = e0.elapsed_time(e1) / 1e3
        fp64_mvms = st64["mvms"]
        # per-(rhs, shift) error of the headline (mixed) solution against the
        # plain FP64 solution; both meet tol in their own FP64 true residual
        err = (torch.linalg.vector_norm(Xmix - X64, dim=-1) / torch.linalg.vector_norm(X64, dim=-1)).cpu().numpy()
        line["fp64_plain"] = {"value": round(m * s / t64, 4), "unit": UNIT, "ms_per_step": round(t64 * 1e3, 1),
                              "block_steps": st64["block_steps"], "restarts": st64["restarts"],
                              "max_true_relres": float(st64["true_relres"].max()),
                              "mixed_over_fp64": round(value / world / (m * s / t64), 2),
                              "mixed_error_vs_fp64": {"max": float(err.max()),
                                                      "per_pair": [[float(f"{v:.3e}") for v in r] for r in err]}}
        del X64
        # the FP64 stencil is bound by the FP64 pipe, not by HBM: time its D
        # launches (library CUDA events) on the workload's m fields
        try:
            ctx.set_profiling(True)
            ctx.apply("A", B, storage="fp64")
            ctx.read_profile()
            reps = 3
            for _ in range(reps):
                ctx.apply("A", B, storage="fp64")
            kms64, kl64 = ctx.read_profile()
            ms_launch = kms64["dslash"] / kl64["dslash"]
            V = n // 12
            flop = WILSON_FLOP_PER_SITE * V * m
            sm_mhz = (clk or {}).get("sm_mhz") or 2070.0
            peak64 = fp64_alu_peak_tflops(sm_mhz)
            ach = flop / (ms_launch / 1e3) / 1e12
            gb = (2.0 * m * n * 16 + 36.0 * V * 16) / 1e9
            line["fp64_plain"]["stencil_roofline"] = {
                "kernel": "dslash (FP64)", "bound": "alu", "achieved": round(ach, 4), "peak": round(peak64, 4),
                "unit": "TFLOP/s", "frac": round(ach / peak64, 4), "ms_per_launch": round(ms_launch, 4),
                "flop_per_launch": flop, "hbm_GBps": round(gb / (ms_launch / 1e3), 1),
                "peak_source": f"derived: 152 SMs x 2 FP64 FMA/clock x 2 flop x {sm_mhz:.0f} MHz"}
        except Exception as e:           # the FP64 stencil figure must not cost the bench line
            line["fp64_plain"]["stencil_roofline"] = {"error": repr(e)[:300]}
        finally:
            ctx.set_profiling(False)
    if rank == 0 and world == 1 and not args.no_cpu:
        total_vec = fp64_mvms if fp64_mvms else stats[-1]["mvms"]
        v, cores, wall, per_vec = oracle_sample(wl, args.cpu_vectors, total_vec)
        line["cpu_baseline"] = {
            "value": round(v, 6), "unit": UNIT, "cores": cores, "host_cores": os.cpu_count(), "kind": "oracle",
            "sample": (f"numpy FP64 oracle, first {args.cpu_vectors} band-Lanczos vectors of the same "
                       f"workload ({wall:.1f} s, {per_vec:.2f} s/vector), scaled to the "
                       f"{total_vec} single-vector A applications of the FP64 GPU solve")}
    ctx.close()
    del X, Xmix, B
    torch.cuda.empty_cache()
    # the 32^3 x 64 workload needs most of the device: run it alone
    if rank == 0 and not args.no_w5:
        leg("w5_full_size", lambda: run_w5(dev, stream, peak, clk_mhz, fp64=not args.no_fp64))
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ------------------------------------------------------- reference arm --
def run_comparison(dev, stream, name="cmp_16x16x16x16", storage="fp64", dims=None, m=None, s=None):
    """The paper's algorithm comparison (Sec. 4, Table 1) on the same kernels:
    CG = one solve per (rhs, shift), block CG = one solve per shift with all
    right-hand sides, shifted CG = one solve per right-hand side with all
    shifts, DSBlockCG = one joint solve.  Returns mvms, block steps and GPU
    time per algorithm, and their ratios to DSBlockCG."""
    import torch
    from paper_1205_0359_gb300 import dsbcg, synth
    wl = synth.make_workload(name, dims=dims, m=m, s=s)
    ctx = dsbcg.Context(wl["dims"], torch.from_numpy(wl["U"]).to(dev), wl["kappa"], stream=stream)
    B = torch.from_numpy(wl["B"]).to(dev)
    sig = np.asarray(wl["sigma"])
    m, s = B.shape[0], sig.size
    plans = {
        "CG": [(slice(i, i + 1), [j]) for i in range(m) for j in range(s)],
        "BlockCG": [(slice(0, m), [j]) for j in range(s)],
        "shiftedCG": [(slice(i, i + 1), list(range(s))) for i in range(m)],
        "DSBlockCG": [(slice(0, m), list(range(s)))],
    }
    out = {}
    for alg, runs in plans.items():
        rows, shifts = runs[0]                                # warm-up (workspace of this shape)
        ctx.solve(B[rows].contiguous(), sig[shifts], wl["tol"], storage=storage)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        mv = steps = 0
        worst = 0.0
        for rows, shifts in runs:
            _, st = ctx.solve(B[rows].contiguous(), sig[shifts], wl["tol"], storage=storage)
            mv += st["mvms"]
            steps += st["block_steps"]
            worst = max(worst, float(st["true_relres"].max()))
        e1.record(stream)
        torch.cuda.synchronize(dev)
        out[alg] = {"mvms": int(mv), "block_steps": int(steps), "ms": round(e0.elapsed_time(e1), 2),
                    "solves": len(runs), "max_true_relres": worst}
    ref = out["DSBlockCG"]
    for alg in out:
        out[alg]["mvms_ratio"] = round(out[alg]["mvms"] / ref["mvms"], 3)
        out[alg]["time_ratio"] = round(out[alg]["ms"] / ref["ms"], 3)
    ctx.close()
    return {"workload": f"{name}: Wilson D^H D on {'x'.join(map(str, wl['dims']))}, kappa {wl['kappa']}, "
                        f"m={m} Gaussian RHS, "
                        f"s={s} shifts {sig[0]:.0e}..{sig[-1]:.0e}, tol {wl['tol']:.0e}, {storage} storage",
            "algorithms": out}


def _timed_solve(ctx, B, sig, tol, storage, X, dev, stream):
    """One solve timed with CUDA events on the stream, after a one-step
    warm-up solve of the same shape (workspace and restart lanes allocated,
    links packed for the precision)."""
    import torch
    ctx.solve(B, sig, tol, storage=storage, out=X, max_block_steps=1, raise_on_error=False)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    _, st = ctx.solve(B, sig, tol, storage=storage, out=X)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    return st, e0.elapsed_time(e1)


def _stencil_rate(ctx, B, storage, m, n, peak, clk_mhz):
    """D on the m fields of B in `storage` (dsbcg_apply), the stencil launch
    timed by the library's CUDA events: GB/s of its algorithmic bytes (fields
    in and out, links once) against the HBM peak, and TFLOP/s (1368 flop per
    site and field)."""
    eb = {"fp64": 16, "fp32": 8, "bf16": 4, "fp16": 4}[storage]
    V = n // 12
    ctx.set_profiling(True)
    ctx.apply("D", B, storage=storage)
    ctx.read_profile()
    reps = 5
    for _ in range(reps):
        ctx.apply("D", B, storage=storage)
    kms, kl = ctx.read_profile()
    ctx.set_profiling(False)
    ms = kms["dslash"] / kl["dslash"]
    gb = (2.0 * m * n * eb + 36.0 * V * eb) / 1e9
    out = {"ms_per_launch": round(ms, 4), "GBps": round(gb / (ms / 1e3), 1),
           "frac_of_hbm": round(gb / (ms / 1e3) / peak, 4),
           "TFLOPs": round(WILSON_FLOP_PER_SITE * V * m / (ms / 1e3) / 1e12, 3)}
    if storage == "fp64":
        pk = fp64_alu_peak_tflops(clk_mhz)
        out["bound"] = "alu"
        out["frac_of_fp64_peak"] = round(out["TFLOPs"] / pk, 4)
    else:
        out["bound"] = "hbm"
    return out


def run_w3_ladder(dev, stream, peak, clk_mhz):
    """The storage-precision ladder on 24^3 x 48 (m = s = 8, shifts 1e-4..1,
    tol 1e-8): per storage (FP64, FP32, BF16, FP16; the last three inside
    FP64 reliable updates) systems/s, the stencil's GB/s and roofline
    fraction, and the per-(rhs, shift) error against the FP64-storage
    solution."""
    import torch
    from paper_1205_0359_gb300 import dsbcg, synth
    wl = synth.make_workload("w3_24x24x24x48")
    m, s, n = wl["B"].shape[0], len(wl["sigma"]), wl["B"].shape[1]
    ctx = dsbcg.Context(wl["dims"], torch.from_numpy(wl["U"]).to(dev), wl["kappa"], stream=stream)
    B = torch.from_numpy(wl["B"]).to(dev)
    X64 = torch.empty((s, m, n), dtype=torch.complex128, device=dev)
    X = torch.empty_like(X64)
    out = {"workload": (f"w3_24x24x24x48: Wilson D^H D, kappa {wl['kappa']}, m={m} Gaussian RHS, s={s} shifts "
                        f"{wl['sigma'][0]:.0e}..{wl['sigma'][-1]:.0e}, tol {wl['tol']:.0e}"), "storages": {}}
    n64 = None
    for storage in ("fp64", "fp32", "bf16", "fp16"):
        dst = X64 if storage == "fp64" else X
        st, ms = _timed_solve(ctx, B, wl["sigma"], wl["tol"], storage, dst, dev, stream)
        row = {"systems_per_s": round(m * s / (ms / 1e3), 3), "ms_per_solve": round(ms, 1),
               "block_steps": st["block_steps"], "restarts": st["restarts"],
               "max_true_relres": float(st["true_relres"].max()), "valid": st["code"] == 0,
               "stencil": _stencil_rate(ctx, B, storage, m, n, peak, clk_mhz)}
        if storage == "fp64":
            n64 = torch.linalg.vector_norm(X64, dim=-1)
        else:
            err = (torch.linalg.vector_norm(X - X64, dim=-1) / n64).cpu().numpy()
            row["error_vs_fp64_storage"] = {"max": float(err.max()),
                                            "per_pair": [[float(f"{v:.3e}") for v in r] for r in err]}
        out["storages"][storage] = row
    ctx.close()
    del X, X64, B
    return out


def run_schur(dev, stream, wl, full_value, full_stats):
    """The even-odd preconditioned operator on the headline lattice: the
    same shifts and tolerance for sigma_j + Ahat on the odd sites, with the
    odd-site half of the headline right-hand sides (FP32 storage, FP64
    reliable updates, one timed solve after a one-step warm-up).  Ahat is a
    different operator from A, so this compares cost, not solutions."""
    import torch
    from paper_1205_0359_gb300 import dsbcg
    Lx, Ly, Lz, Lt = wl["dims"]
    t, z, y, x = np.meshgrid(np.arange(Lt), np.arange(Lz), np.arange(Ly), np.arange(Lx), indexing="ij")
    odd = np.nonzero(((x + y + z + t) % 2).reshape(-1) == 1)[0]
    m, s = wl["B"].shape[0], len(wl["sigma"])
    Bh = np.ascontiguousarray(wl["B"].reshape(m, -1, 12)[:, odd, :].reshape(m, -1))
    ctx = dsbcg.Context(wl["dims"], torch.from_numpy(wl["U"]).to(dev), wl["kappa"], stream=stream)
    ctx.set_operator("schur")
    B = torch.from_numpy(Bh).to(dev)
    X = torch.empty((s, m, B.shape[1]), dtype=torch.complex128, device=dev)
    st, ms = _timed_solve(ctx, B, wl["sigma"], wl["tol"], "fp32", X, dev, stream)
    ctx.close()
    del X, B
    value = m * s / (ms / 1e3)
    return {"workload": "the headline lattice, shifts and tol; sigma_j + Dhat^H Dhat on the odd sites, "
                        "Dhat = 1 - kappa^2 H_oe H_eo, odd-site half of the headline right-hand sides",
            "systems_per_s": round(value, 3), "ms_per_solve": round(ms, 1), "block_steps": st["block_steps"],
            "restarts": st["restarts"], "max_true_relres": float(st["true_relres"].max()), "valid": st["code"] == 0,
            "full_operator": {"systems_per_s": round(full_value, 3), "block_steps": full_stats["block_steps"],
                              "restarts": full_stats["restarts"]},
            "schur_over_full": round(value / full_value, 3)}


def run_w5(dev, stream, peak, clk_mhz, fp64=True):
    """32^3 x 64, m = 16 (b_16 = b_1 + 1e-9 noise), s = 8 shifts 1e-5..1,
    tol 1e-8 (~140 GB of HBM in FP32 storage): mixed precision (FP32 storage,
    FP64 reliable updates) against the plain FP64 form, one timed solve each,
    and the FP32 stencil's roofline fraction."""
    import torch
    from paper_1205_0359_gb300 import dsbcg, synth
    wl = synth.make_workload("w5_32x32x32x64")
    m, s, n = wl["B"].shape[0], len(wl["sigma"]), wl["B"].shape[1]
    out = {"workload": (f"w5_32x32x32x64: Wilson D^H D, kappa {wl['kappa']}, m={m} Gaussian RHS with "
                        f"b_16 = b_1 + 1e-9 noise, s={s} shifts {wl['sigma'][0]:.0e}..{wl['sigma'][-1]:.0e}, "
                        f"tol {wl['tol']:.0e}")}
    B = torch.from_numpy(wl["B"]).to(dev)
    X = torch.empty((s, m, n), dtype=torch.complex128, device=dev)
    for storage in (("fp32", "fp64") if fp64 else ("fp32",)):
        ctx = dsbcg.Context(wl["dims"], torch.from_numpy(wl["U"]).to(dev), wl["kappa"], stream=stream)
        # the stencil first: dsbcg_apply's temporaries would not fit beside
        # the solver's workspace
        stencil = _stencil_rate(ctx, B, storage, m, n, peak, clk_mhz)
        torch.cuda.empty_cache()
        st, ms = _timed_solve(ctx, B, wl["sigma"], wl["tol"], storage, X, dev, stream)
        out[storage] = {"systems_per_s": round(m * s / (ms / 1e3), 4), "ms_per_solve": round(ms, 1),
                        "block_steps": st["block_steps"], "restarts": st["restarts"],
                        "deflations": st["deflations"], "max_true_relres": float(st["true_relres"].max()),
                        "valid": st["code"] == 0, "stencil": stencil}
        ctx.close()
        torch.cuda.empty_cache()
    if fp64:
        out["mixed_over_fp64"] = round(out["fp32"]["systems_per_s"] / out["fp64"]["systems_per_s"], 2)
    del X, B
    return out


def run_sweeps(dev, stream, storage="fp64"):
    """The paper's two sweeps (Sec. 4, Figs. 2 and 3), DSBlockCG against
    shifted CG (one solve per right-hand side with all shifts) on the same
    kernels: 16^4 with m = 4 and a growing number of shifts spread over
    1e-6..1e-1, and 12^4 with s = 10 shifts and a growing number of
    right-hand sides.  Each point: mvms and GPU time of both, and the ratios
    DSBlockCG / shifted CG the figures plot."""
    import dataclasses
    import torch
    from paper_1205_0359_gb300 import dsbcg, synth

    def timed(ctx, B, sig, tol):
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, st = ctx.solve(B, sig, tol, storage=storage)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return st, e0.elapsed_time(e1)

    def point(ctx, B, sig, tol):
        ctx.solve(B, sig, tol, storage=storage)                        # warm-up, this shape
        st, t_dsb = timed(ctx, B, sig, tol)
        mv_sh, t_sh = 0, 0.0
        ctx.solve(B[0:1].contiguous(), sig, tol, storage=storage)
        for i in range(B.shape[0]):
            st1, t1 = timed(ctx, B[i:i + 1].contiguous(), sig, tol)
            mv_sh += st1["mvms"]
            t_sh += t1
        return {"dsb_mvms": int(st["mvms"]), "shifted_mvms": int(mv_sh), "dsb_ms": round(t_dsb, 2),
                "shifted_ms": round(t_sh, 2), "mvms_ratio": round(st["mvms"] / mv_sh, 3),
                "time_ratio": round(t_dsb / t_sh, 3)}

    base = synth.WORKLOADS["cmp_16x16x16x16"]
    out = {"shift_sweep": {}, "rhs_sweep": {}}
    d = synth.make_workload(base, m=4)
    ctx = dsbcg.Context(d["dims"], torch.from_numpy(d["U"]).to(dev), d["kappa"], stream=stream)
    B = torch.from_numpy(d["B"]).to(dev)
    for s in (1, 2, 4, 7, 10):
        sig = synth.log_shifts(1e-6, 1e-1, s) if s > 1 else np.array([1e-6])
        out["shift_sweep"][str(s)] = point(ctx, B, sig, base.tol)
    ctx.close()
    wl12 = dataclasses.replace(base, name="cmp_12x12x12x12", dims=(12, 12, 12, 12), m=12, s=10,
                               shifts=tuple(synth.log_shifts(1e-6, 1e-1, 10)))
    d = synth.make_workload(wl12)
    ctx = dsbcg.Context(d["dims"], torch.from_numpy(d["U"]).to(dev), d["kappa"], stream=stream)
    Ball = torch.from_numpy(d["B"]).to(dev)
    for m in (1, 2, 4, 6, 8, 12):
        out["rhs_sweep"][str(m)] = point(ctx, Ball[:m].contiguous(), np.asarray(d["sigma"]), base.tol)
    ctx.close()
    out["workload"] = (f"16^4 (m = 4, s = 1..10) and 12^4 (s = 10, m = 1..12), kappa {base.kappa}, "
                       f"shifts 1e-6..1e-1, tol {base.tol:.0e}, {storage} storage")
    return out


def run_reference(args):
    """The FP64 CPU oracle on the host cores, as the reference implementation."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_1205_0359_gb300 import synth
    wl = synth.make_workload(WORKLOAD)
    m, s = wl["B"].shape[0], len(wl["sigma"])
    # whole-solve vector count of an FP64 DSBlockCG on this workload (block
    # steps x m), as measured by the FP64 GPU form; used to scale each sample
    total_vec = args.ref_total_vectors
    for _ in range(args.warmup):
        oracle_sample(wl, args.ref_vectors, total_vec)
    vals, walls, cores = [], [], 1
    for _ in range(args.steps):
        v, cores, wall, _ = oracle_sample(wl, args.ref_vectors, total_vec)
        vals.append(v)
        walls.append(wall)
    value = float(np.mean(vals))
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * float(np.mean(walls)), 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(wl, "fp32"),
        "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": cores, "host_cores": os.cpu_count(),
                         "kind": "oracle",
                         "sample": (f"each step: numpy FP64 oracle for {args.ref_vectors} band-Lanczos vectors, "
                                    f"scaled to a {total_vec}-vector solve")},
        "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--storage", default="fp32", choices=["fp32", "bf16", "fp16", "fp64"])
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 comparison solve")
    ap.add_argument("--no-df32", action="store_true", help="skip the double-float reliable-update form")
    ap.add_argument("--no-w3", action="store_true", help="skip the 24^3 x 48 storage-precision ladder")
    ap.add_argument("--no-w5", action="store_true", help="skip the 32^3 x 64 workload (mixed and plain FP64)")
    ap.add_argument("--no-schur", action="store_true", help="skip the even-odd (Schur) operator leg")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle sample")
    ap.add_argument("--no-force", action="store_true", help="skip the gauge-force timing")
    ap.add_argument("--sweeps", action="store_true",
                    help="also run the paper's shift and right-hand-side sweeps (DSBlockCG vs shifted CG)")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the paper's algorithm comparison (CG, block CG, shifted CG, DSBlockCG)")
    ap.add_argument("--cpu-vectors", type=int, default=4)
    ap.add_argument("--ref-vectors", type=int, default=1)
    # single-vector A applications of a whole FP64 solve of the workload (the
    # plain FP64 GPU form measured 1488 on 16^3 x 32, m = s = 12); the main
    # line's cpu_baseline scales its sample by the same count
    ap.add_argument("--ref-total-vectors", type=int, default=1488)
    ap.add_argument("--lattice", type=lambda t: tuple(int(x) for x in t.split(",")), default=None,
                    help="Lx,Ly,Lz,Lt to resize the workload (profiling of smaller cases)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
