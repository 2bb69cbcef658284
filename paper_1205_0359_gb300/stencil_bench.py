"""Time the Wilson stencil on its own: D (or D^H, A) on m fields through
dsbcg_apply, each stencil launch timed by the library's CUDA events.

    python -m paper_1205_0359_gb300.stencil_bench --lattice 16,16,16,32 --fields 12 --storage fp32

Prints one JSON line: milliseconds per stencil launch, GB/s of its algorithmic
bytes (m fields in, m out, the links once; 12-real links counted as 24 V
entries when the field is in SU(3)), the fraction of the HBM peak (the
measured copy bandwidth in MEASURED_PEAKS.json if present) and TFLOP/s (1368
flop per site and field).  Only the fields and the links live on the device
(about 0.5 GB at 16^3 x 32 with 12 FP32 fields), so the tool also serves as
a small, self-contained target for profilers.  Inputs: the seeded SU(3)
links and Gaussian fields of the package's input generators.
"""
from __future__ import annotations

import argparse
import json
import os

import numpy as np
import torch

from . import dsbcg, synth

BYTES = {"fp64": 16, "fp32": 8, "bf16": 4, "fp16": 4, "df32": 16}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--lattice", default="16,16,16,32")
    ap.add_argument("--fields", type=int, default=12)
    ap.add_argument("--storage", default="fp32", choices=sorted(BYTES))
    ap.add_argument("--op", default="D", choices=["D", "Ddag", "A"])
    ap.add_argument("--kappa", type=float, default=0.125)
    ap.add_argument("--eps", type=float, default=0.5)
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--operator", default="normal", choices=["normal", "schur"])
    args = ap.parse_args(argv)
    dims = tuple(int(x) for x in args.lattice.split(","))
    dev = torch.device("cuda")
    rng = np.random.Generator(np.random.PCG64(1205))
    U = synth.su3_links(dims, args.eps, rng)
    ctx = dsbcg.Context(dims, torch.from_numpy(U).to(dev), args.kappa)
    if args.operator == "schur":
        ctx.set_operator("schur")
    F = torch.from_numpy(synth.gaussian_rhs(ctx.n, args.fields, rng)).to(dev)
    out = torch.empty_like(F)
    ctx.set_profiling(True)
    ctx.apply(args.op, F, storage=args.storage, out=out)          # links packed, warm
    ctx.read_profile()
    for _ in range(args.reps):
        ctx.apply(args.op, F, storage=args.storage, out=out)
    kms, kl = ctx.read_profile()
    ctx.close()
    V = int(np.prod(dims))
    launches = kl["dslash"]
    ms = kms["dslash"] / launches
    per_launch_ops = launches / args.reps                          # stencil launches per apply
    sites = V if args.operator == "normal" else V // 2
    eb = BYTES[args.storage]
    # the half-lattice passes of the Schur operator read the 18-real links and,
    # in every second pass, a source field (2.5 fields per field on average)
    link_entries = 24 if (args.storage in ("fp32", "bf16", "fp16") and args.operator == "normal") else 36
    fields_rw = 2.0 if args.operator == "normal" else 2.5
    gb = (fields_rw * args.fields * 12 * sites * eb + link_entries * V * eb) / 1e9
    peak = 6795.8
    p = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            peak = float(json.load(f)["hbm_gbs"])
    line = {"lattice": list(dims), "fields": args.fields, "storage": args.storage, "op": args.op,
            "operator": args.operator, "stencil_launches_per_apply": per_launch_ops,
            "ms_per_launch": round(ms, 4), "GB_per_launch": round(gb, 4),
            "GBps": round(gb / (ms / 1e3), 1), "frac_of_hbm": round(gb / (ms / 1e3) / peak, 4),
            "TFLOPs": round(1368.0 * sites * args.fields / (ms / 1e3) / 1e12, 3),
            "note": ("bytes: fields in and out once per launch, the links once (12-real for the reduced storages "
                     "of the normal operator, the generated field being in SU(3))")}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
