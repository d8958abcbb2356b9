"""Micro-benchmark of the inner-loop stencil kernel on a synthetic field.

    python -m paper_1601_04587_gb300.hopbench --lattice 32 24 24 24 --ncol 12 --precision fp32 --iters 20

Times the Schur-complement hopping kernel (v = p - kappa^2 H_eo tmp with the
fused (rh, v) partials) on the whole lattice with CUDA events and prints the
average launch time, the kernel's algorithmic bytes and the bandwidth they
imply.  Small enough to run under ncu.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--lattice", type=int, nargs=4, default=[32, 24, 24, 24])
    ap.add_argument("--ncol", type=int, default=12)
    ap.add_argument("--precision", default="fp32", choices=["fp64", "fp32", "fp16", "bf16"])
    ap.add_argument("--iters", type=int, default=20)
    ap.add_argument("--kappa", type=float, default=0.14)
    ap.add_argument("--tile-sites", type=int, default=0)
    ap.add_argument("--tile-cols", type=int, default=0)
    args = ap.parse_args()

    import torch

    import paper_1601_04587_gb300 as ddp
    import synth

    L = tuple(args.lattice)
    U = synth.gauge_field_torch(L, seed=synth.SEED_GAUGE, device="cuda")
    ctx = ddp.ddp_create(0, torch.cuda.current_stream().cuda_stream)
    if args.tile_sites:
        ddp.ddp_set_param(ctx, "tile_sites", args.tile_sites)
    if args.tile_cols:
        ddp.ddp_set_param(ctx, "tile_cols", args.tile_cols)
    gid = ddp.ddp_load_gauge(ctx, U, L, ddp.DDP_BC_ANTIPERIODIC)
    did = ddp.ddp_set_domain(ctx, gid, (0, 0, 0, 0), L)
    ms, nbytes = ddp.ddp_time_hop(ctx, did, args.kappa, args.ncol, ddp.PRECISIONS[args.precision], args.iters)
    ddp.ddp_destroy(ctx)
    print(json.dumps({"lattice": L, "ncol": args.ncol, "precision": args.precision, "ms_per_launch": ms,
                      "algorithmic_bytes": nbytes, "GBps": nbytes / ms / 1e6,
                      "tile_sites": args.tile_sites, "tile_cols": args.tile_cols}))


if __name__ == "__main__":
    main()
