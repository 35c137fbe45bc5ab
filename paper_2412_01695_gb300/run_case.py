"""Run one operation of the library on a seeded synthetic cell (for profilers and quick checks).

  python -m paper_2412_01695_gb300.run_case --op hpsi --cfg 2 --precision fp32 --reps 3
  python -m paper_2412_01695_gb300.run_case --op davidson --cfg 1 --precision fp64
  python -m paper_2412_01695_gb300.run_case --op sternheimer --cfg 4 --nk 256 --precision fp32_c128

Cells 1-4 are the synthetic cells of the generator (synth.CONFIGS); --nk takes the first
nk points of the grid (default: all).  The timed repetitions run inside the NVTX range
"run_case" (plan creation, which times candidate launch shapes, is outside it).  Prints one JSON line with the CUDA-event time of
each repetition.  No result is checked here (the tests do that).
"""
from __future__ import annotations

import argparse
import json

import numpy as np


def sternheimer_block(nk: int, dev, stream, nocc: int = 12, nbx: int = 16):
    """Inputs of a batched Sternheimer solve on the first nk k-points of the DFPT cell (cell 4):
    plans of the k and k+q blocks, the nbx lowest bands of both by the batched FP64 Davidson,
    the nocc occupied ones, alpha_k = 2 (spread of the occupied levels) (>= 0.01 Ry) and the
    perturbation dv(r).  Returns a dict."""
    import torch
    from . import pwk, synth
    ks = list(range(nk))
    pk = synth.make_config(4, k_subset=ks, nb=nbx)
    pq = synth.make_config(4, k_subset=ks, shift_q=True, nb=nbx)
    plan_k = pwk.plan_from_problem(pk, device=dev)
    plan_q = pwk.plan_from_problem(pq, device=dev)

    def lowest(plan, pr):
        psi = torch.from_numpy(pr.psi[:, :nbx].copy()).to(dev)
        eig = torch.zeros((pr.nk, nbx), dtype=torch.float64, device=dev)
        pwk.davidson_batched(plan, pwk.PWK_FP64, psi, eig, nbx, 1e-10, 1e-5, 300, 0, stream)
        return eig, psi

    eps_k, psi_k = lowest(plan_k, pk)
    eps_q, psi_q = lowest(plan_q, pq)
    e_all = torch.cat([eps_k[:, :nocc], eps_q[:, :nocc]], dim=1)
    alpha = torch.clamp(2.0 * (e_all.max(dim=1).values - e_all.min(dim=1).values), min=0.01).contiguous()
    return {"pk": pk, "pq": pq, "plan_k": plan_k, "plan_q": plan_q, "nocc": nocc,
            "psi_k": psi_k[:, :nocc].contiguous(), "psi_q": psi_q[:, :nocc].contiguous(),
            "eps_k": eps_k, "eps_q": eps_q, "ek": eps_k[:, :nocc].contiguous(), "alpha": alpha,
            "dv": torch.from_numpy(synth.dv_for(4)).to(dev)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--op", default="hpsi", choices=["hpsi", "davidson", "sternheimer"])
    ap.add_argument("--cfg", type=int, default=2)
    ap.add_argument("--nk", type=int, default=0)
    ap.add_argument("--nb", type=int, default=0)
    ap.add_argument("--precision", default="fp32", choices=["fp64", "fp32", "fp32_c128"])
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--max-iter", type=int, default=100, help="Davidson iterations")
    ap.add_argument("--projector-path", type=int, default=0,
                    help="0: CUDA-core projections, 1: tensor cores where they apply")
    args = ap.parse_args()

    import torch
    from . import pwk, synth

    if args.op == "sternheimer":
        return run_sternheimer(args)
    nkfull = int(np.prod(synth.CONFIGS[args.cfg]["mp"]))
    sub = None if args.nk in (0, nkfull) else list(range(args.nk))
    prob = synth.make_config(args.cfg, k_subset=sub, nb=args.nb or None)
    plan = pwk.plan_from_problem(prob)
    plan.set_projector_path(args.projector_path)
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
    torch.cuda.nvtx.range_pop()
    shape = plan.launch_shape(pwk.PRECISIONS[args.precision])
    print(json.dumps({"op": args.op, "cfg": args.cfg, "nk": prob.nk, "nb": prob.nb,
                      "precision": args.precision, "ms": times, "launch_shape": shape, **extra}))
    plan.close()


def run_sternheimer(args):
    """--op sternheimer: the DFPT cell (cell 4), the first --nk k-points (default 256), 12
    occupied bands, solved to a true residual of 1e-10; --precision fp64 runs the FP64 CG,
    anything else the mixed mode."""
    import torch
    from . import pwk
    if args.cfg != 4:
        raise SystemExit("sternheimer runs on the DFPT cell: --cfg 4")
    nk = args.nk or 256
    stream = torch.cuda.current_stream()
    blk = sternheimer_block(nk, torch.device("cuda"), stream)
    mode = pwk.PWK_FP64 if args.precision == "fp64" else pwk.PWK_FP32_C128
    nocc = blk["nocc"]
    times = []
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("run_case")
    for _ in range(args.reps):
        dpsi = torch.zeros((nk, nocc, blk["pq"].npw_max), dtype=torch.complex128, device="cuda")
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        rc, iters, resid = pwk.sternheimer_cg_batched(blk["plan_q"], blk["plan_k"], mode, blk["psi_k"],
                                                      blk["ek"], blk["psi_q"], nocc, blk["alpha"],
                                                      blk["dv"], dpsi, 1e-10, 500, stream)
        b.record()
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
    torch.cuda.nvtx.range_pop()
    print(json.dumps({"op": "sternheimer", "cfg": 4, "nk": nk, "nocc": nocc, "precision": args.precision,
                      "ms": times, "pairs_above_tol": int(rc), "iters_max": int(iters.max()),
                      "iters_mean": float(iters.mean()), "max_true_residual": float(resid.max())}))
    blk["plan_k"].close()
    blk["plan_q"].close()


if __name__ == "__main__":
    main()
