"""Run one operation of the library on a seeded synthetic cell (for profilers and quick checks).

  python -m paper_2412_01695_gb300.run_case --op hpsi --cfg 2 --precision fp32 --reps 3
  python -m paper_2412_01695_gb300.run_case --op davidson --cfg 1 --precision fp64
  python -m paper_2412_01695_gb300.run_case --op sternheimer --cfg 4 --nk 64

Cells 1-4 are the synthetic cells of the generator (synth.CONFIGS); --nk takes the first
nk points of the grid (default: all).  The timed repetitions run inside the NVTX range
"run_case" (plan creation, which times candidate launch shapes, is outside it).  Prints one JSON line with the CUDA-event time of
each repetition.  No result is checked here (the tests do that).
"""
from __future__ import annotations

import argparse
import json

import numpy as np


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--op", default="hpsi", choices=["hpsi", "davidson", "sternheimer"])
    ap.add_argument("--cfg", type=int, default=2)
    ap.add_argument("--nk", type=int, default=0)
    ap.add_argument("--nb", type=int, default=0)
    ap.add_argument("--precision", default="fp32", choices=["fp64", "fp32", "fp32_c128"])
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--max-iter", type=int, default=100, help="Davidson iterations")
    args = ap.parse_args()

    import torch
    from . import pwk, synth

    nkfull = int(np.prod(synth.CONFIGS[args.cfg]["mp"]))
    sub = None if args.nk in (0, nkfull) else list(range(args.nk))
    prob = synth.make_config(args.cfg, k_subset=sub, nb=args.nb or None)
    plan = pwk.plan_from_problem(prob)
    prec = pwk.PRECISIONS[args.precision]
    times = []
    # the repetitions sit in an NVTX range "run_case" (profilers can select exactly them)
    torch.cuda.nvtx.range_push("run_case")
    if args.op == "hpsi":
        dt = torch.complex64 if args.precision == "fp32" else torch.complex128
        x = torch.from_numpy(prob.psi).cuda().to(dt)
        y = torch.empty_like(x)
        for _ in range(args.reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            pwk.hpsi_batched(plan, prec, x, y, prob.nb)
            b.record()
            torch.cuda.synchronize()
            times.append(a.elapsed_time(b))
        extra = {}
    elif args.op == "davidson":
        mode = pwk.PWK_FP64 if args.precision == "fp64" else pwk.PWK_FP32_C128
        for _ in range(args.reps):
            psi = torch.from_numpy(prob.psi).cuda()
            eig = torch.zeros((prob.nk, prob.nb), dtype=torch.float64, device="cuda")
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            rc, iters, notc, napply = pwk.davidson_batched(plan, mode, psi, eig, prob.nb, 1e-10,
                                                           1e-5, args.max_iter, 0)
            b.record()
            torch.cuda.synchronize()
            times.append(a.elapsed_time(b))
        extra = {"unconverged": int(rc), "iters_max": int(iters.max()), "napply": napply.tolist(),
                 "iters_percentiles": np.percentile(iters, [50, 90, 99, 100]).tolist(),
                 "slowest_k": int(np.argmax(iters))}
    else:
        raise SystemExit("sternheimer: see tests/test_sternheimer_gpu.py for input preparation")
    torch.cuda.nvtx.range_pop()
    shape = plan.launch_shape(pwk.PRECISIONS[args.precision])
    print(json.dumps({"op": args.op, "cfg": args.cfg, "nk": prob.nk, "nb": prob.nb,
                      "precision": args.precision, "ms": times, "launch_shape": shape, **extra}))
    plan.close()


if __name__ == "__main__":
    main()
