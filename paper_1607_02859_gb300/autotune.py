"""r-block autotuner for the chi0(i omega) pipeline.

gw_chi0_omega walks the real-space rows r in blocks of r_block rows: each block
holds 2 x r_block x N_r Green's-function slabs in the scratch arena (and, on the
tensor-core path, the split operands).  Larger blocks feed the GEMMs and the row
FFTs bigger batches; smaller ones keep the working set in L2 and leave device
memory to concurrent requests.  The tuner times chi0_omega for each candidate
whose scratch fits the given budget (CUDA events on the launching stream, after
one warm-up call) and keeps the fastest per (grid, bands, tau points, G set,
precision, device) in a JSON cache.
"""
from __future__ import annotations

import json
import os

from . import gw

DEFAULT_CANDIDATES = (256, 512, 1024, 2048, 4096, 8192)


def key(grid_n, n_b, n_occ, n_tau, n_chi, prec, device_name):
    return "%dx%dx%d/b%d/o%d/t%d/g%d/%s/%s" % (tuple(grid_n) + (n_b, n_occ, n_tau, n_chi, prec, device_name))


def feasible(grid, n_b, n_occ, n_tau, n_chi, prec, candidates=DEFAULT_CANDIDATES, budget_bytes=None):
    """Candidates (clipped to N_r, deduplicated) whose chi0 scratch fits the budget."""
    n_r = int(grid.n[0] * grid.n[1] * grid.n[2])
    out = []
    for rb in sorted({min(int(c), n_r) for c in candidates if int(c) > 0}):
        need = gw.workspace_size(grid, n_b, n_occ, n_tau, n_chi, 1, prec, rb)[0]
        if budget_bytes is None or need <= budget_bytes:
            out.append(rb)
    return out


def load(path):
    if path and os.path.exists(path):
        with open(path) as f:
            return json.load(f)
    return {}


def store(path, cache):
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tune(ctx, system, candidates=DEFAULT_CANDIDATES, budget_bytes=None, cache_path=None, reps=2):
    """Best r_block for a registered serve.System; cached when cache_path is given.
    Returns (r_block, {r_block: ms})."""
    import torch
    dev = system.psi.device
    k = key(system.grid.n, system.n_b, system.n_occ, len(system.tau), system.n_chi, system.prec,
            torch.cuda.get_device_name(dev))
    cache = load(cache_path)
    if k in cache:
        return int(cache[k]["r_block"]), {int(a): b for a, b in cache[k]["ms"].items()}
    cands = feasible(system.grid, system.n_b, system.n_occ, len(system.tau), system.n_chi, system.prec, candidates,
                     budget_bytes)
    if not cands:
        raise ValueError("no r_block candidate fits the budget")
    chi = torch.empty((len(system.tau), system.n_chi, system.n_chi), dtype=gw.cdtype(system.prec), device=dev)
    st = torch.cuda.current_stream(dev)
    times = {}
    for rb in cands:
        def call():
            gw.chi0_omega(ctx, system.grid, system.psi, system.eps, system.n_occ, system.mu, system.tau,
                          system.mats["C"], system.fidx, system.prec, chi, r_block=rb)
        call()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        e0.record(st)
        for _ in range(reps):
            call()
        e1.record(st)
        e1.synchronize()
        times[rb] = e0.elapsed_time(e1) / reps
    best = min(times, key=times.get)
    if cache_path:
        cache[k] = {"r_block": best, "ms": {str(a): b for a, b in times.items()}}
        store(cache_path, cache)
    return best, times
