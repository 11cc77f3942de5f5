"""Batched form of the chi0 chain: many systems of uneven sizes set up once
as chi0 plans (gw_chi0_plan_*) and launched together as one CUDA graph.

    python -m paper_1607_02859_gb300.batch [--count 16] [--prec fp32] [--reps 3]

prints one JSON line: the batch's replay time and effective TFLOP/s (the
algorithmic flops of every system's chi0 evaluation over the replay time),
and each system's relative Frobenius difference from the FP64 path of the same
library (for systems whose FP64 evaluation is cheap), with the systems' sizes.
"""
from __future__ import annotations

import argparse
import json
import math

import numpy as np

from . import gw, inputs


def chi0_flops(n_r, n_b, n_tau, n_chi):
    """Algorithmic flops of one chi0(i omega) evaluation (complex MAC = 8 flops)."""
    return (n_tau * 8.0 * n_r * n_r * n_b                                # G_occ, G_unocc (Eqs. Green_occ/unocc)
            + n_tau * (n_r + n_chi) * 5.0 * n_r * math.log2(n_r)         # row and column transforms
            + n_tau * n_tau * 4.0 * n_chi * n_chi                         # cosine transform
            + n_tau * 6.0 * n_r * n_r)                                     # chi = -2 G_occ conj(G_unocc)


def main(argv=None):
    import torch
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--count", type=int, default=16)
    ap.add_argument("--seed", type=int, default=4)
    ap.add_argument("--prec", default="fp32", choices=["fp32", "f16x3", "bf16x3"])
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--fp64-max-flops", type=float, default=2e12,
                    help="compare with the FP64 path only for systems below this many flops")
    args = ap.parse_args(argv)
    ctx = gw.Context(0)
    problems = inputs.batch_mix(args.count, args.seed)
    systems = []
    for p in problems:
        grid = gw.make_grid(p.n, p.lattice)
        gvec, fidx = gw.g_set(grid, p.n_chi)
        mats = gw.fit_transform(p.tau, p.omega, p.x_min, p.x_max, p.n_x, p.ridge)
        psi = torch.from_numpy(np.ascontiguousarray(p.psi)).to("cuda", dtype=gw.cdtype(args.prec))
        out = torch.empty((len(p.tau), p.n_chi, p.n_chi), dtype=gw.cdtype(args.prec), device="cuda")
        plan = gw.Chi0Plan(ctx, grid, p.n_b, p.eps, p.n_occ, p.mu, p.tau, mats["C"], fidx, args.prec)
        systems.append(dict(p=p, grid=grid, fidx=fidx, mats=mats, psi=psi, out=out, plan=plan,
                            flops=chi0_flops(p.n_r, p.n_b, len(p.tau), p.n_chi)))
    for s in systems:                         # first launches outside the capture
        s["plan"].launch(s["psi"], s["out"])
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        for s in systems:
            s["plan"].launch(s["psi"], s["out"])
    graph.replay()
    torch.cuda.synchronize()
    for s in systems:
        s["plan"].status()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.reps):
        graph.replay()
    e1.record(stream)
    e1.synchronize()
    t = e0.elapsed_time(e1) / 1e3 / args.reps
    total = sum(s["flops"] for s in systems)
    rows = []
    for s in systems:
        p = s["p"]
        row = {"system": p.name, "n_chi": p.n_chi, "gflop": s["flops"] / 1e9}
        if s["flops"] <= args.fp64_max_flops:
            psi64 = torch.from_numpy(np.ascontiguousarray(p.psi)).to("cuda", dtype=torch.complex128)
            ref = torch.empty(s["out"].shape, dtype=torch.complex128, device="cuda")
            gw.chi0_omega(ctx, s["grid"], psi64, p.eps, p.n_occ, p.mu, p.tau, s["mats"]["C"], s["fidx"], "fp64", ref)
            got = s["out"].to(torch.complex128)
            row["rel_err_vs_fp64"] = (torch.linalg.vector_norm(got - ref) / torch.linalg.vector_norm(ref)).item()
            del ref, psi64
        rows.append(row)
    print(json.dumps({"batch": len(systems), "prec": args.prec, "replay_ms": t * 1e3, "tflops": total / t / 1e12,
                      "gflop_total": total / 1e9, "systems": rows}))
    for s in systems:
        s["plan"].close()
    ctx.close()


if __name__ == "__main__":
    main()
