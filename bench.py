#!/usr/bin/env python
"""Benchmark of the space-time GW hot path on synthetic Si-like inputs.

One step = the whole hot path through the C ABI on one seeded system:
chi0(i omega) (gw_chi0_omega: G formation, chi = -2 G_occ o conj(G_unocc), row
and column FFTs, cosine transform), screening (gw_screen_W), inverse cosine
transform (gw_tau_to_omega), the diagonal self-energy with its Thiele
continuation (gw_sigma_diag), the linearised QP energies and spectral
functions (gw_qp_energies) and Sigma back on the imaginary time axis
(gw_sigma_to_tau).  The metric is the effective TFLOP/s of the
method's algorithmic work (flop model below) divided by the device time.
--sigma matrix replaces the last two calls by the full self-energy matrix over
the same bands (gw_sigma_matrix).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gw|reference]
                  [--prec fp32|fp64|f16x3|bf16x3] [--workload si64|si8|mid|gamma_toy|k8448]
                  [--sigma diag|matrix]

N > 1 (under torchrun): independent replicas, one per GPU (the path is not
sharded); value = the work of all ranks / the slowest rank's time.
--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "chi0+Sigma_nn effective TFLOP/s"
ACCURACY = {
    "f16x3": "G, Sigma and screening contractions as 3 fp16 split products on tcgen05 (fp32 accumulate); refinement "
             "residual as exact fp16 slice products (30 bits of the row/column maxima, summed as FP32 hi/lo pairs); "
             "tested at this size against the FP64 oracle: chi0(i omega) within 3e-6 relative (sampled rows, all "
             "bands; 1.9e-6 measured), refined W~ against the dense solve within 2e-7, Sigma_nn within 1 meV",
    "fp32": "all steps FP32 on CUDA cores; tested: chi0(i omega) within 1e-6 relative, Sigma_nn within 1 meV",
    "fp64": "all steps FP64 on CUDA cores",
    "bf16x3": "3 bf16 split products on tcgen05; tested: chi0 within 2e-5 relative, Sigma_nn within 1 meV",
}
N_REAL = 64          # real frequencies of the continued Sigma_nn(omega)
E2E_STEPS = 3        # steps of the end-to-end pass
SLICE_PAIRS = 15     # fp16 slice-pair products of the refinement's residual product (levels 4)
FLUSH_BYTES = 512 << 20


def flop_model(n_r, n_b, n_tau, n_chi, n_n):
    """Algorithmic flops of one pass of the hot path (complex MAC = 8 flops)."""
    lg = math.log2(n_r)
    f = {
        # G_occ and G_unocc, once for chi and once again for Sigma (Eqs. Green_occ/unocc)
        "green": 2 * n_tau * 8.0 * n_r * n_r * n_b,
        # chi rows, chi columns, W~ columns, W~ rows: 5 N log2 N per transform
        "fft": n_tau * (2 * n_r + 2 * n_chi) * 5.0 * n_r * lg,
        # forward and inverse cosine transform, real weight x complex data
        "ct": 2 * n_tau * n_tau * 4.0 * n_chi * n_chi,
        # eps~ = L L^H, L^{-1}, L^{-H} L^{-1}: N^3/2 complex MACs per frequency
        "dyson": n_tau * 4.0 * n_chi ** 3,
        # (G o W~) psi_n for the occupied and unoccupied parts
        "sigma": n_tau * 2 * 8.0 * n_r * n_r * n_n,
        # real-space products chi = -2 G_occ conj(G_unocc) and G o W~ (6 flops each)
        "hadamard": n_tau * 3 * 6.0 * n_r * n_r,
    }
    f["total"] = sum(f.values())
    return f


def sm_peak_fp32(sm_mhz, n_sm=152):
    return n_sm * 128 * 2 * sm_mhz * 1e6 / 1e12


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    def __init__(self, index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), "--query-gpu=" + q, "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": []}
        if self.p is None:
            return out
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if sm:
            out = {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                   "samples": len(sm)}
        return out


# DRAM bytes per launch of a kernel family from an ncu capture (profiles/), valid
# only for the kernel source it was taken on: the sha1 of those files is checked
# at run time and a mismatch reports null.
MEASURED_TRAFFIC = {
    # green_tc on the 36^3 workload: ncu DRAM bytes per algorithmic flop of the two modes on the
    # k8448 case (same kernel and K; 3.49e-6 for the chi pass, 3.07e-6 for the fused Sigma
    # pass, equal flop shares in the step) times the step's 2.12e12 flops per launch; the
    # 36^3 launches, with 2-5x more tiles, reuse more in L2, so this is an upper estimate
    ("si64", "f16x3", "green_tc"): {
        "bytes_per_launch": 6.96e9,
        "sources": {"paper_1607_02859_gb300/csrc/gw_tc.cu": "6d1061d1b8c170b6b869627d5056bace4943b6de",
                    "paper_1607_02859_gb300/csrc/gw_tcgen05.cuh": "9b50b7a589cc5e99cff2a95e30ffc334ce4d64ad"},
        "profile": "profiles/green_tc_k8448_f16x3.md",
    },
}


def measured_traffic(workload, prec, family):
    """Bytes per launch recorded for this kernel, or None if none was recorded or its source changed."""
    import hashlib
    rec = MEASURED_TRAFFIC.get((workload, prec, family))
    if rec is None:
        return None
    root = os.path.dirname(os.path.abspath(__file__))
    for path, sha in rec["sources"].items():
        try:
            with open(os.path.join(root, path), "rb") as f:
                if hashlib.sha1(f.read()).hexdigest() != sha:
                    return None
        except OSError:
            return None
    return rec["bytes_per_launch"]


def max_over_ranks(x, dist=None, device="cuda"):
    """The largest x over the ranks of the process group (x itself without one)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, flops_per_step, steps, seconds):
    """Whole-job TFLOP/s: every rank's work over the slowest rank's time."""
    return world * flops_per_step * steps / seconds / 1e12


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        return {}


# ---------------------------------------------------------------------- reference arm (CPU oracle)

SAMPLE_SOLVE = 3072
SAMPLE_G_FLOPS = 2.8e12     # G-row work of one sample: ~10 s of the FP64 oracle on 16 host cores


def sample_rows(p):
    """Rows of the bounded oracle sample: about SAMPLE_G_FLOPS of G formation (1536 rows at si8,
    89 at si64)."""
    return int(min(1536, max(16, SAMPLE_G_FLOPS // (8.0 * p.n_r * p.n_b * len(p.tau)))))


def oracle_sample(p, rows=None, n_solve=SAMPLE_SOLVE):
    """Time the FP64 oracle on a bounded slice of the workload: G_occ/G_unocc rows and the
    real-space chi product for `rows` rows at every tau, plus one screening solve of size
    n_solve.  Returns (flops, seconds) under the same flop model."""
    from oracle import chi as ochi  # noqa: F401  (oracle only in this leg)
    from oracle import green as ogr
    from oracle import screen as osc
    rows = sample_rows(p) if rows is None else rows
    rr = np.arange(rows)
    t0 = time.perf_counter()
    for tau in p.tau:
        go = ogr.green_occ_rows(p.psi, p.eps, p.n_occ, p.mu, tau, rr)
        gu = ogr.green_unocc_rows(p.psi, p.eps, p.n_occ, p.mu, tau, rr)
        _ = -2.0 * go * gu.conj()
    rng = np.random.default_rng(0)
    a = rng.standard_normal((n_solve, 64)) + 1j * rng.standard_normal((n_solve, 64))
    chi = -(a @ a.conj().T) / n_solve
    osc.screen_one(chi, np.full(n_solve, 0.5))
    dt = time.perf_counter() - t0
    flops = len(p.tau) * 8.0 * rows * p.n_r * p.n_b + len(p.tau) * 6.0 * rows * p.n_r + 4.0 * n_solve ** 3
    return flops, dt


def cpu_cores():
    try:
        from threadpoolctl import threadpool_info
        n = max((i.get("num_threads") or 0) for i in threadpool_info())
        if n:
            return n
    except Exception:
        pass
    return os.cpu_count()


def run_reference(args, p, workload):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    for _ in range(args.warmup):
        oracle_sample(p, rows=32, n_solve=512)
    tot_f, tot_t = 0.0, 0.0
    for _ in range(args.steps):
        f, t = oracle_sample(p)
        tot_f += f
        tot_t += t
    val = tot_f / tot_t / 1e12
    sample = ("FP64 numpy oracle: G_occ/G_unocc rows + chi product for %d of %d rows at all %d tau, plus one %d^2 "
              "screening solve" % (sample_rows(p), p.n_r, len(p.tau), SAMPLE_SOLVE))
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "TFLOP/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload,
            "cpu_baseline": {"value": val, "unit": "TFLOP/s", "cores": cpu_cores(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": val, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------- GPU arm

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gw", choices=["gw", "reference"])
    ap.add_argument("--prec", default="f16x3", choices=["fp32", "fp64", "f16x3", "bf16x3"])
    ap.add_argument("--workload", default="si64", choices=["si8", "mid", "gamma_toy", "si64", "k8448"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-breakdown", action="store_true", help="skip the per-stage pass")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end pass")
    ap.add_argument("--refine", type=int, default=None,
                    help="refinement steps of the screening solve (default: 1 on si64, whose recipe asks for it, else 0)")
    ap.add_argument("--r-block", type=int, default=None,
                    help="rows per r-block of the chi0 pass (default: 4096 on si64, as its recipe streams chi0, "
                         "else the library's default)")
    ap.add_argument("--g-form", default="rr", choices=["rr", "pw"],
                    help="G of the chi0 and Sigma passes: rr = real-space contraction on the tensor cores "
                         "(N_r^2 N_b per tau); pw = plane-wave form over the orbitals' plane waves, then "
                         "transforms (gw_chi0_omega_pw, gw_sigma_diag_pw)")
    ap.add_argument("--sigma", default="diag", choices=["diag", "matrix"],
                    help="diag: Sigma_nn, continuation and QP energies; matrix: the full Sigma_nm(i omega)")
    args = ap.parse_args()

    from paper_1607_02859_gb300 import inputs
    refine = args.refine if args.refine is not None else (1 if args.workload == "si64" else 0)
    r_block = args.r_block if args.r_block is not None else (4096 if args.workload == "si64" else 0)
    p = getattr(inputs, args.workload)()
    n_tau = len(p.tau)
    grids = "log-spaced tau in [0.05, 40], omega_k = 1/tau_(N-1-k), weight ridge 1e-6 (the workload's given grid)"
    if args.workload != "gamma_toy" and args.impl == "gw":
        # optimised (MP2 minimax) time and frequency grids from the library's host setup
        from paper_1607_02859_gb300 import gw as _gw
        g = _gw.mp2_grids(n_tau, p.x_min, p.x_max)
        p = inputs.on_grids(p, g["tau"], g["omega"], 0.0)
        grids = "MP2 minimax tau/omega grids (gw_mp2_grids), weights fitted without ridge"
    elif args.workload != "gamma_toy":
        grids = "MP2 minimax tau/omega grids"
    workload = {"workload": "%s: %dx%dx%d grid (N_r=%d), %d+%d %s bands, %d tau/i omega, chi0 %dx%d, Sigma_nn for %d bands"
                % (args.workload, *p.n, p.n_r, p.n_occ, p.n_b - p.n_occ, "real" if p.real else "complex", n_tau,
                   p.n_chi, p.n_chi, len(p.bands)),
                "prec": args.prec, "sigma": args.sigma, "grids": grids, "refine_iters": refine,
                "r_block": r_block if r_block > 0 else "library default (2048)",
                "g_form": {"rr": "real-space G contraction (tcgen05)",
                           "pw": "plane-wave G over the orbitals' N_b plane waves, then transforms"}[args.g_form],
                "l2": "per-step working set > 40 GB >> 129 MB L2; L2 also flushed between steps",
                "accuracy": ACCURACY.get(args.prec, "")}
    if args.impl == "reference":
        run_reference(args, p, workload)
        return

    import torch
    from paper_1607_02859_gb300 import gw

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    ctx = gw.Context(local)
    grid = gw.make_grid(p.n, p.lattice)
    gvec, fidx = gw.g_set(grid, p.n_chi)                                      # product host setup
    # the synthetic orbitals span the lowest N_b plane waves e^{+i G.r}
    pw_index = gw.g_set(grid, p.n_b)[1] if args.g_form == "pw" else None
    mats = gw.fit_transform(p.tau, p.omega, p.x_min, p.x_max, p.n_x, p.ridge)
    dt = gw.cdtype(args.prec)
    psi_h = torch.from_numpy(p.psi.astype(np.complex128)).to(dt).pin_memory()
    psi = psi_h.to("cuda", non_blocking=False)
    chi_w = torch.empty((n_tau, p.n_chi, p.n_chi), dtype=dt, device="cuda")
    w_tau = torch.empty_like(chi_w)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    w_real = np.linspace(-1.0, 1.0, N_REAL)
    eps_n = p.eps[p.bands]
    vstat = eps_n.copy()          # synthetic static part: bare exchange - <V_xc> taken as 0
    stream = torch.cuda.current_stream()

    def step(psi_dev, events=None):
        def mark(i):
            if events is not None:
                events[i].record(stream)
        mark(0)
        if args.g_form == "pw":
            gw.chi0_omega_pw(ctx, grid, psi_dev, p.eps, p.n_occ, p.mu, p.tau, mats["C"], fidx, pw_index, args.prec,
                             chi_w)
        else:
            gw.chi0_omega(ctx, grid, psi_dev, p.eps, p.n_occ, p.mu, p.tau, mats["C"], fidx, args.prec, chi_w,
                          r_block=r_block)
        mark(1)
        gw.screen_W(ctx, grid, gvec, args.prec, chi_w, chi_w, resid=False, refine=refine)
        mark(2)
        gw.tau_to_omega(ctx, gw.CT, mats["Cinv"], chi_w, w_tau, args.prec)
        mark(3)
        if args.sigma == "matrix":
            out = gw.sigma_matrix(ctx, grid, psi_dev, p.eps, p.n_occ, p.mu, p.bands, p.tau, p.omega, mats["C"],
                                  mats["S"], w_tau, fidx, args.prec)
            mark(4)
            mark(5)
            mark(6)
            return out
        if args.g_form == "pw":
            out = gw.sigma_diag_pw(ctx, grid, psi_dev, p.eps, p.n_occ, p.mu, p.bands, p.tau, p.omega, mats["C"],
                                   mats["S"], w_tau, fidx, pw_index, args.prec, w_real=w_real)
        else:
            out = gw.sigma_diag(ctx, grid, psi_dev, p.eps, p.n_occ, p.mu, p.bands, p.tau, p.omega, mats["C"],
                                mats["S"], w_tau, fidx, args.prec, w_real=w_real)
        mark(4)
        out["qp"] = gw.qp_energies(ctx, p.omega, out["sigma_iw"], eps_n, p.mu, vstat, w=w_real + p.mu)
        mark(5)
        out["back_to_tau"] = gw.sigma_to_tau(ctx, out["sigma_iw"], mats["Cinv"], mats["Sinv"])
        mark(6)
        return out

    for _ in range(args.warmup):
        out = step(psi)
        if not np.all(np.isfinite(out["sigma_iw"])):
            raise RuntimeError("Sigma(i omega) of the warm-up step is not finite")
    torch.cuda.synchronize()

    fl = flop_model(p.n_r, p.n_b, n_tau, p.n_chi, len(p.bands))
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    l0 = ctx.launches
    times = []
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step(psi)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
    torch.cuda.synchronize()
    launches = (ctx.launches - l0) // max(args.steps, 1)
    clocks = sampler.stop()
    t_dev = max_over_ranks(float(np.sum(times)), dist)
    if dist is not None:
        dist.barrier()
    value = job_value(world, fl["total"], args.steps, t_dev)

    # per-stage breakdown and the dominant stage's roofline (same stream, CUDA events)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(7)]
    flush.zero_()
    if args.no_breakdown:
        for e in ev:
            e.record(stream)
    else:
        step(psi, ev)
    torch.cuda.synchronize()
    stage_ms = {name: ev[i].elapsed_time(ev[i + 1]) for i, name in
                enumerate(["chi0_omega", "screen_W", "inverse_ct", "sigma_" + args.sigma, "qp_energies",
                           "sigma_to_tau"])}
    if args.sigma == "matrix":
        del stage_ms["qp_energies"], stage_ms["sigma_to_tau"]
    # per-kernel device time and algorithmic work (library events on the launch stream)
    peaks = measured_peaks()
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    tc_peak = peaks.get("bf16_tflops_sustained", 1716.4)      # fp16 dense = bf16 dense rate
    hbm_peak = peaks.get("hbm_gbs", 6785.5)
    kernels = {}
    if not args.no_breakdown:
        flush.zero_()
        torch.cuda.synchronize()
        ctx.set_timing(True)
        step(psi)
        torch.cuda.synchronize()
        for fam, (n_l, ms, work, is_bytes) in ctx.kernel_stats().items():
            if n_l:
                kernels[fam] = {"launches": n_l, "ms": ms, "work": work, "unit": "B" if is_bytes else "flop"}
                rate = work / (ms / 1e3)
                if is_bytes:
                    kernels[fam]["frac_of_hbm"] = rate / 1e9 / hbm_peak
                elif fam in ("green_tc", "cgemm_tc"):
                    kernels[fam]["frac_of_split_tensor"] = rate / 1e12 / (tc_peak / 3.0)
                elif fam == "cgemm_exact":
                    kernels[fam]["frac_of_sliced_tensor"] = rate / 1e12 / (tc_peak / SLICE_PAIRS)
                elif fam in ("row_pw", "cgemm_simt"):
                    kernels[fam]["frac_of_fp32_alu"] = rate / 1e12 / sm_peak_fp32(sm_max)
        ctx.set_timing(False)
    roof = None
    if kernels:
        dom = max(kernels, key=lambda k: kernels[k]["ms"])
        k = kernels[dom]
        if k["unit"] == "B":
            ach = k["work"] / (k["ms"] / 1e3) / 1e9
            roof = {"bound": "hbm", "unit": "GB/s", "peak": hbm_peak,
                    "peak_source": "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"}
        elif dom in ("green_tc", "cgemm_tc"):
            ach = k["work"] / (k["ms"] / 1e3) / 1e12
            roof = {"bound": "tensor", "unit": "TFLOP/s", "peak": tc_peak / 3.0,
                    "peak_source": "measured sustained bf16 dense peak %.1f TFLOP/s (fp16 rate equal) / 3 split "
                                   "products per algorithmic flop" % tc_peak}
        elif dom == "cgemm_exact":
            ach = k["work"] / (k["ms"] / 1e3) / 1e12
            roof = {"bound": "tensor", "unit": "TFLOP/s", "peak": tc_peak / SLICE_PAIRS,
                    "peak_source": "measured sustained bf16 dense peak %.1f TFLOP/s (fp16 rate equal) / %d exact "
                                   "slice-pair products per algorithmic flop" % (tc_peak, SLICE_PAIRS)}
        else:
            ach = k["work"] / (k["ms"] / 1e3) / 1e12
            roof = {"bound": "alu", "unit": "TFLOP/s", "peak": sm_peak_fp32(sm_max),
                    "peak_source": "FP32 CUDA-core peak 152 SM x 128 lanes x 2 flop x %.0f MHz" % sm_max}
        traffic = measured_traffic(args.workload, args.prec, dom)
        roof.update({"kernel": dom, "launches": k["launches"], "achieved": ach, "frac": ach / roof["peak"],
                     "traffic": traffic, "share_of_step": k["ms"] / (1e3 * t_dev / args.steps)})
        if traffic is not None:
            roof["traffic_source"] = ("ncu dram__bytes_read.sum + dram__bytes_write.sum per launch, %s"
                                      % MEASURED_TRAFFIC[(args.workload, args.prec, dom)]["profile"])

    # end to end through the public API: orbitals copied from pinned host memory every step,
    # Sigma read back to the host inside the call; at most E2E_STEPS steps (a step of the
    # 36^3 workload takes ~10 s)
    e_times = []
    e_steps = 0 if args.no_e2e else min(args.steps, E2E_STEPS)
    for _ in range(e_steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        psi_dev = psi_h.to("cuda", non_blocking=True)
        step(psi_dev)
        e1.record(stream)
        e1.synchronize()
        e_times.append(e0.elapsed_time(e1) / 1e3)
    t_e2e = max_over_ranks(float(np.sum(e_times)) if e_times else float("nan"), dist)
    e2e = {"value": job_value(world, fl["total"], max(e_steps, 1), t_e2e), "unit": "TFLOP/s", "steps": e_steps,
           "h2d_bytes_per_step": int(psi_h.numel() * psi_h.element_size()),
           "d2h_bytes_per_step": int(len(p.bands) * (3 * n_tau + N_REAL) * 16 + len(p.bands) * (48 + 8 * N_REAL)
                                     + 2 * len(p.bands) * n_tau * 8
                                     if args.sigma == "diag" else len(p.bands) ** 2 * 3 * n_tau * 16)}

    line = {"metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_dev / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": {"fp64": "f64", "fp32": "f32", "f16x3": "f16x3->f32", "bf16x3": "bf16x3->f32"}[args.prec],
            "data": "synthetic", "config": dict(workload, parallelism="replicas x%d" % world),
            "stage_ms": stage_ms, "kernels": kernels, "flops_per_step": fl, "roofline": roof, "e2e": e2e,
            "gpu_launches": int(launches),
            "clocks": clocks}
    if rank == 0 and not args.no_cpu_baseline:
        f, t = oracle_sample(p)
        line["cpu_baseline"] = {"value": f / t / 1e12, "unit": "TFLOP/s", "cores": cpu_cores(), "kind": "oracle",
                                "sample": "FP64 numpy oracle: G rows + chi product for %d of %d rows at all %d tau, plus "
                                          "one %d^2 screening solve (%.1f s)" % (sample_rows(p), p.n_r, n_tau, SAMPLE_SOLVE, t)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
