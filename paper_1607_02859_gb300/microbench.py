"""Microbenchmarks of single kernel families through the C ABI, for profiling
and tuning: each prints one JSON line with the family's per-launch time (the
library's own CUDA-event timing of its launches), its algorithmic bytes or
flops per launch, and the fraction of the measured HBM copy bandwidth or
tensor-core rate.

    python -m paper_1607_02859_gb300.microbench row --n 36 --n-chi 8192 --rows 2048
        spatial row transform of Eqs. FFTX1 / FFTW (second step) over a block of
        rows of the n^3 grid, both directions (gw_rr_to_GG_fft, stage 1);
        algorithmic bytes per row: the N_r grid values and the n_chi G-set values,
        each read or written once.
    python -m paper_1607_02859_gb300.microbench sliced --n 2048 --levels 4
        the exact sliced complex product of the refinement residual
        (gw_zgemm_sliced); flops 8 n^3 per product.
    python -m paper_1607_02859_gb300.microbench pwchi --n 36 --bands 256 --n-chi 2048 --tau 2
        chi0 through the plane-wave form of G (gw_chi0_omega_pw) on an n^3 cell
        whose orbitals span the lowest `bands` plane waves: the call's time and
        the row pass's share (its launches are the row-transform family).

Inputs are seeded Gaussian; --reps timed launches follow one untimed launch."""
from __future__ import annotations

import argparse
import json
import os

import numpy as np

from . import gw

HERE = os.path.dirname(os.path.abspath(__file__))


def measured_peaks():
    try:
        with open(os.path.join(HERE, "..", "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def row(args, ctx):
    import torch
    n = (args.n, args.n, args.n)
    lattice = np.eye(3) * (args.n * 10.26 / 12)
    grid = gw.make_grid(n, lattice)
    _, idx = gw.g_set(grid, args.n_chi)
    nr = args.n ** 3
    cdt = torch.complex64 if args.prec == "fp32" else torch.complex128
    g = torch.Generator(device="cuda").manual_seed(5)
    real = torch.empty((args.rows, nr), dtype=cdt, device="cuda")
    real.real.normal_(generator=g)
    real.imag.normal_(generator=g)
    rec = torch.empty((args.rows, args.n_chi), dtype=cdt, device="cuda")
    hbm = measured_peaks().get("hbm_gbs")
    out = []
    for direction, src, dst in ((1, real, rec), (-1, rec, real)):
        gw.rr_to_GG_fft(ctx, grid, direction, 1, idx, args.prec, 0, args.rows, src, dst)   # warm-up
        torch.cuda.synchronize()
        ctx.set_timing(True)
        for _ in range(args.reps):
            gw.rr_to_GG_fft(ctx, grid, direction, 1, idx, args.prec, 0, args.rows, src, dst)
        torch.cuda.synchronize()
        launches, ms, work, _ = ctx.kernel_stats()["row_fft"]
        ctx.set_timing(False)
        calls = args.reps
        gbs = work / (ms / 1e3) / 1e9 if ms > 0 else float("nan")
        out.append({"kernel": "row_fft", "direction": direction, "grid": list(n), "n_chi": args.n_chi,
                    "rows": args.rows, "prec": args.prec, "launches_per_call": launches // calls,
                    "ms_per_call": ms / calls, "bytes_per_call": work / calls, "GB/s": gbs,
                    "frac_of_hbm": gbs / hbm if hbm else None, "hbm_peak_gbs": hbm})
    return out


def sliced(args, ctx):
    import torch
    g = torch.Generator(device="cuda").manual_seed(6)
    A = torch.randn((args.n, args.n), dtype=torch.complex128, device="cuda", generator=g)
    B = torch.randn((args.n, args.n), dtype=torch.complex128, device="cuda", generator=g)
    C = torch.empty_like(A)
    gw.zgemm_sliced(ctx, A, B, C, args.levels)
    torch.cuda.synchronize()
    ctx.set_timing(True)
    for _ in range(args.reps):
        gw.zgemm_sliced(ctx, A, B, C, args.levels)
    torch.cuda.synchronize()
    launches, ms, work, _ = ctx.kernel_stats()["cgemm_exact"]
    ctx.set_timing(False)
    pairs = (args.levels + 1) * (args.levels + 2) // 2
    tf = work / (ms / 1e3) / 1e12 if ms > 0 else float("nan")
    peak = measured_peaks().get("bf16_tflops")
    sliced_peak = peak / pairs if peak else None        # fp16 rate equal to bf16; one product per slice pair
    return [{"kernel": "cgemm_exact", "n": args.n, "levels": args.levels, "pairs": pairs,
             "ms_per_launch": ms / max(launches, 1), "TFLOP/s": tf,
             "frac_of_sliced_tensor": tf / sliced_peak if sliced_peak else None}]


def pwchi(args, ctx):
    import torch
    from . import inputs
    n = (args.n, args.n, args.n)
    p = inputs.tiny(seed=47, n=n, a=(args.n * 10.26 / 12,) * 3, n_occ=args.bands // 8,
                    n_unocc=args.bands - args.bands // 8, n_tau=args.tau, n_chi=args.n_chi)
    grid = gw.make_grid(p.n, p.lattice)
    _, fidx = gw.g_set(grid, p.n_chi)
    _, pw = gw.g_set(grid, p.n_b)
    mats = gw.fit_transform(p.tau, p.omega, p.x_min, p.x_max, p.n_x, p.ridge)
    psi = torch.from_numpy(p.psi).to("cuda", dtype=torch.complex64)
    chi = torch.empty((len(p.tau), p.n_chi, p.n_chi), dtype=torch.complex64, device="cuda")
    gw.chi0_omega_pw(ctx, grid, psi, p.eps, p.n_occ, p.mu, p.tau, mats["C"], fidx, pw, args.prec, chi)
    torch.cuda.synchronize()
    ctx.set_timing(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.reps):
        gw.chi0_omega_pw(ctx, grid, psi, p.eps, p.n_occ, p.mu, p.tau, mats["C"], fidx, pw, args.prec, chi)
    e1.record()
    torch.cuda.synchronize()
    stats = ctx.kernel_stats()
    ctx.set_timing(False)
    rows = {k: {"launches": v[0] // args.reps, "ms": v[1] / args.reps} for k, v in stats.items() if v[0]}
    return [{"kernel": "chi0_omega_pw", "grid": list(n), "bands": p.n_b, "n_chi": p.n_chi, "tau": len(p.tau),
             "prec": args.prec, "ms_per_call": e0.elapsed_time(e1) / args.reps, "families": rows}]


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    sub = ap.add_subparsers(dest="what", required=True)
    r = sub.add_parser("row")
    r.add_argument("--n", type=int, default=36)
    r.add_argument("--n-chi", type=int, default=8192)
    r.add_argument("--rows", type=int, default=2048)
    r.add_argument("--prec", default="fp32", choices=["fp32", "fp64"])
    r.add_argument("--reps", type=int, default=5)
    s = sub.add_parser("sliced")
    s.add_argument("--n", type=int, default=2048)
    s.add_argument("--levels", type=int, default=4)
    s.add_argument("--reps", type=int, default=3)
    c = sub.add_parser("pwchi")
    c.add_argument("--n", type=int, default=36)
    c.add_argument("--bands", type=int, default=256)
    c.add_argument("--n-chi", type=int, default=2048)
    c.add_argument("--tau", type=int, default=2)
    c.add_argument("--prec", default="f16x3", choices=["fp32", "f16x3", "bf16x3"])
    c.add_argument("--reps", type=int, default=2)
    args = ap.parse_args(argv)
    ctx = gw.Context(0)
    for line in {"row": row, "sliced": sliced, "pwchi": pwchi}[args.what](args, ctx):
        print(json.dumps(line))
    ctx.close()


if __name__ == "__main__":
    main()
