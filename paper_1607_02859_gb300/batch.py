"""Batched form of the hot path: many systems of uneven sizes through the whole
chain -- chi0(i omega), W~ (with optional refinement), W~(i tau), Sigma_nn(i
omega) -- planned once and launched together as one CUDA graph
(gw_batch_plan / gw_batch_launch / gw_batch_wait).  The rows per r-block of
each system's chi0 pass come from the r-block autotuner (one tuning per
distinct system shape, cached in a JSON file).

    python -m paper_1607_02859_gb300.batch [--count 48] [--prec fp32] [--reps 3]
                                            [--fp64-max-nr 4096]

prints one JSON line: the replay time and effective TFLOP/s of the whole batch
(the algorithmic flops of every system's chain over the replay time) and, for
the systems with N_r <= --fp64-max-nr, each system's largest difference in meV
from the same batch run through the library's FP64 path.  With --stages the
same chains run once more call by call with the library's per-kernel timing
(a graph replay cannot carry it), and the line adds each kernel family's device
time, work and fraction of the measured peaks (MEASURED_PEAKS.json).  (The comparison with
the FP64 oracle is in the GPU tests, tests/test_gpu_batch.py.)
"""
from __future__ import annotations

import argparse
import json
import math
import types

import numpy as np

from . import autotune, gw, inputs


def chain_flops(n_r, n_b, n_tau, n_chi, n_n):
    """Algorithmic flops of one system's chain (complex MAC = 8 flops), as in the bench's model."""
    lg = math.log2(n_r)
    return (2 * n_tau * 8.0 * n_r * n_r * n_b                            # G_occ, G_unocc for chi and again for Sigma
            + n_tau * (2 * n_r + 2 * n_chi) * 5.0 * n_r * lg             # row and column transforms, both passes
            + 2 * n_tau * n_tau * 4.0 * n_chi * n_chi                    # cosine transform and its inverse
            + n_tau * 4.0 * n_chi ** 3                                   # screening
            + n_tau * 2 * 8.0 * n_r * n_r * n_n                          # (G o W~) psi_n
            + n_tau * 3 * 6.0 * n_r * n_r)                               # real-space products


def family_stages(ctx, systems, prec):
    """Every system's chain through the direct entry points with per-kernel timing on:
    {family: launches, ms, work, unit and the fraction of the measured peak that bounds it}."""
    import os
    import torch
    peaks = {}
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "..", "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except OSError:
        pass
    hbm = peaks.get("hbm_gbs")
    tc = peaks.get("bf16_tflops_sustained")
    alu = 152 * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    torch.cuda.synchronize()
    ctx.set_timing(True)
    for s in systems:
        gw.chi0_omega(ctx, s["grid"], s["psi"], s["eps"], s["n_occ"], s["mu"], s["tau"], s["C"], s["fft_index"],
                      prec, s["chi_w"], r_block=s["r_block"])
        gw.screen_W(ctx, s["grid"], s["gvec"], prec, s["chi_w"], s["chi_w"], resid=False, refine=s["refine"])
        gw.tau_to_omega(ctx, gw.CT, s["Cinv"], s["chi_w"], s["w_tau"], prec)
        gw.sigma_diag(ctx, s["grid"], s["psi"], s["eps"], s["n_occ"], s["mu"], s["bands"], s["tau"], s["omega"],
                      s["C"], s["S"], s["w_tau"], s["fft_index"], prec)
    torch.cuda.synchronize()
    out = {}
    split = 3.0 if prec in ("f16x3", "bf16x3") else None
    for fam, (n, ms, work, is_bytes) in ctx.kernel_stats().items():
        if not n:
            continue
        rate = work / (ms / 1e3)
        row = {"launches": n, "ms": ms, "work": work, "unit": "B" if is_bytes else "flop"}
        if is_bytes and hbm:
            row["frac_of_hbm"] = rate / 1e9 / hbm
        elif fam in ("green_tc", "cgemm_tc") and tc and split:
            row["frac_of_split_tensor"] = rate / 1e12 / (tc / split)
        elif fam == "cgemm_exact" and tc:
            row["frac_of_sliced_tensor"] = rate / 1e12 / (tc / 15.0)
        elif not is_bytes:
            row["frac_of_fp32_alu"] = rate / 1e12 / alu
        out[fam] = row
    ctx.set_timing(False)
    return out


def main(argv=None):
    import torch
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--count", type=int, default=48)
    ap.add_argument("--seed", type=int, default=4)
    ap.add_argument("--prec", default="fp32", choices=["fp32", "f16x3", "bf16x3", "fp64"])
    ap.add_argument("--refine", type=int, default=0)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--tune-cache", default="", help="JSON file for the r-block autotuner (empty: no cache)")
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--fp64-max-nr", type=int, default=4096)
    ap.add_argument("--stages", action="store_true", help="per-kernel-family times of the chains, call by call")
    args = ap.parse_args(argv)
    ctx = gw.Context(0)
    problems = inputs.batch_mix(args.count, args.seed)
    dt = gw.cdtype(args.prec)
    systems, meta, tuned = [], [], {}
    for p in problems:
        grid = gw.make_grid(p.n, p.lattice)
        gvec, fidx = gw.g_set(grid, p.n_chi)
        g = gw.mp2_grids(len(p.tau), p.x_min, p.x_max)            # optimised time / frequency grids
        p = inputs.on_grids(p, g["tau"], g["omega"], 0.0)
        mats = gw.fit_transform(p.tau, p.omega, p.x_min, p.x_max, p.n_x, p.ridge)
        psi = torch.from_numpy(np.ascontiguousarray(p.psi)).to("cuda", dtype=dt)
        shape = (len(p.tau), p.n_chi, p.n_chi)
        rb = 0
        if not args.no_tune:
            k = (p.n, p.n_b, len(p.tau), p.n_chi)
            if k not in tuned:
                sysv = types.SimpleNamespace(grid=grid, n_b=p.n_b, n_occ=p.n_occ, tau=p.tau, n_chi=p.n_chi,
                                             prec=args.prec, psi=psi, eps=p.eps, mu=p.mu, mats=mats, fidx=fidx)
                tuned[k] = autotune.tune(ctx, sysv, cache_path=args.tune_cache or None)[0]
            rb = tuned[k]
        systems.append(dict(grid=grid, psi=psi, eps=p.eps, n_occ=p.n_occ, mu=p.mu, tau=p.tau, omega=p.omega,
                            C=mats["C"], S=mats["S"], Cinv=mats["Cinv"], gvec=gvec, fft_index=fidx, bands=p.bands,
                            r_block=rb, refine=args.refine, chi_w=torch.empty(shape, dtype=dt, device="cuda"),
                            w_tau=torch.empty(shape, dtype=dt, device="cuda")))
        meta.append((p, mats, rb))
    batch = gw.Batch(ctx, systems, args.prec)
    batch.launch()                                # first launch (also loads the modules)
    sig, status = batch.wait()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.reps):
        batch.launch()
    e1.record(stream)
    e1.synchronize()
    sig, status = batch.wait()
    t = e0.elapsed_time(e1) / 1e3 / args.reps
    batch.close()
    stages = family_stages(ctx, systems, args.prec) if args.stages else None
    # the small systems again through the FP64 path, as one more batch
    small = [i for i, (p, _, _) in enumerate(meta) if p.n_r <= args.fp64_max_nr and args.prec != "fp64"]
    ref = {}
    if small:
        sys64 = []
        for i in small:
            s = dict(systems[i])
            s["psi"] = s["psi"].to(torch.complex128)
            s["chi_w"] = torch.empty(s["chi_w"].shape, dtype=torch.complex128, device="cuda")
            s["w_tau"] = torch.empty(s["w_tau"].shape, dtype=torch.complex128, device="cuda")
            s["r_block"] = 0
            sys64.append(s)
        b64 = gw.Batch(ctx, sys64, "fp64")
        b64.launch()
        s64, _ = b64.wait()
        b64.close()
        ref = dict(zip(small, s64))
    total = 0.0
    rows = []
    for i, ((p, mats, rb), s_iw, st) in enumerate(zip(meta, sig, status)):
        f = chain_flops(p.n_r, p.n_b, len(p.tau), p.n_chi, len(p.bands))
        total += f
        row = {"system": p.name, "n_chi": p.n_chi, "gflop": f / 1e9, "r_block": rb, "status": st}
        if i in ref:
            row["max_dsigma_meV_vs_fp64"] = float(np.max(np.abs(s_iw - ref[i]))) / 3.674932e-5
        rows.append(row)
    line = {"batch": len(systems), "prec": args.prec, "refine": args.refine, "replay_ms": t * 1e3,
            "tflops": total / t / 1e12, "gflop_total": total / 1e9, "systems": rows}
    if stages is not None:
        line["kernels"] = stages
    print(json.dumps(line))
    ctx.close()


if __name__ == "__main__":
    main()
