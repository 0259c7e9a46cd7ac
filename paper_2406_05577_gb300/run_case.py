"""Runs one transform case with its launch configuration given explicitly,
for profiling and for reproducing measurements:

    python -m paper_2406_05577_gb300.run_case --grid 160 --radius 40 --bands 8 \\
        --direction roundtrip --precision fp32 --plane-schedule 1 --repeat 3

Builds the library if needed, creates the plan (cutoff sphere, k = 0,
band-major), applies the given settings (or --autotune), executes it
--repeat times on seeded synthetic coefficients (complex Gaussian) and
prints the plan's launch configuration, the mean event time per execute and
the relative L2 error of the round trip against N0 N1 N2 times the input
(G -> r -> G) as one JSON line. Nothing here is timed for the benchmark.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--grid", type=int, nargs="+", required=True, help="N (cubic) or N0 N1 N2")
    ap.add_argument("--radius", type=float, required=True)
    ap.add_argument("--bands", type=int, default=8)
    ap.add_argument("--direction", default="roundtrip", choices=["roundtrip", "g2r", "r2g", "apply"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64", "mixed"])
    ap.add_argument("--plane-schedule", type=int, default=None, help="0 default, 1 alternative")
    ap.add_argument("--stick-schedule", type=int, default=None, help="0 default, 1 alternative")
    ap.add_argument("--prefetch", type=int, default=None, help="0, 1 or 2")
    ap.add_argument("--slab-buffers", type=int, default=None, help="1 or 2")
    ap.add_argument("--pdl", type=int, default=None, help="0 or 1")
    ap.add_argument("--chunk", type=int, default=0, help="max bands per launch (0: the plan's default)")
    ap.add_argument("--autotune", action="store_true", help="autotune instead of the settings above")
    ap.add_argument("--repeat", type=int, default=3)
    args = ap.parse_args(argv)

    import torch
    import fftb_inputs as fi
    from paper_2406_05577_gb300 import build
    build.build()
    from paper_2406_05577_gb300 import fftb

    n = tuple(args.grid * 3) if len(args.grid) == 1 else tuple(args.grid)
    plan = fftb.Plan(n, args.direction, args.precision, radius=args.radius, bands=[args.bands],
                     max_chunk_bands=args.chunk)
    if args.autotune:
        plan.autotune(3)
    else:
        if args.plane_schedule is not None or args.stick_schedule is not None:
            plan.set_radix_schedule(args.plane_schedule or 0, args.stick_schedule or 0)
        if args.prefetch is not None:
            plan.set_prefetch(args.prefetch)
        if args.slab_buffers is not None:
            plan.set_slab_buffers(args.slab_buffers)
        if args.pdl is not None:
            plan.set_pdl(bool(args.pdl))
    info = plan.info
    cd = plan.complex_dtype
    g = plan.sphere(0)
    vol = n[0] * n[1] * n[2]
    if args.direction == "r2g":
        x = torch.from_numpy(fi.complex_gaussian((args.bands * vol,), 7)).to(cd).cuda()
        out = torch.empty(info["sphere_elems"], dtype=cd, device="cuda")
    else:
        x = torch.from_numpy(fi.complex_gaussian((args.bands, len(g)), 7).reshape(-1)).to(cd).cuda()
        out = torch.empty(info["cube_elems"] if args.direction == "g2r" else info["sphere_elems"], dtype=cd,
                          device="cuda")
    cube = torch.empty(info["cube_elems"], dtype=cd, device="cuda") if args.direction == "roundtrip" else None
    if args.direction == "apply":
        v = fi.gaussian_potential(n, 32, 4.0, seed=4)
        vd = torch.from_numpy(v.astype(np.float64 if args.precision == "fp64" else np.float32)).cuda()
        plan.set_potential(vd)
    plan.execute(x, out, cube)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(args.repeat):
        plan.execute(x, out, cube)
    b.record()
    torch.cuda.synchronize()
    plan.check()
    res = {"grid": list(n), "radius": args.radius, "bands": args.bands, "direction": args.direction,
           "precision": args.precision, "ms_per_execute": a.elapsed_time(b) / max(args.repeat, 1),
           "info": {k: v for k, v in info.items()}}
    if args.direction == "roundtrip":
        res["rel_l2_roundtrip"] = (torch.linalg.vector_norm(out - vol * x) / torch.linalg.vector_norm(vol * x)).item()
    print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
