"""chi0 plans (gw_chi0_plan_*): a plan launch equals gw_chi0_omega, and the
launches of several uneven systems captured in one CUDA graph and replayed
give the same results as the direct calls."""
import time

import numpy as np
import pytest

from oracle import pipeline as opipe
from paper_1607_02859_gb300 import gw, inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import os
    if not os.path.exists(gw.LIB_PATH):
        from paper_1607_02859_gb300 import build
        build.build()
    c = gw.Context(0)
    yield c
    c.close()


SYSTEMS = [("gamma_toy", inputs.gamma_toy, "fp32"),
           ("tiny_c", lambda: inputs.tiny(seed=71), "f16x3"),
           ("ragged", lambda: inputs.tiny(seed=72, n=(8, 6, 10), a=(7.0, 6.0, 8.0), n_occ=6, n_unocc=42, n_tau=8),
            "fp32")]


def setup_system(ctx, make, prec):
    p = make()
    s = opipe.setup(p)
    grid = gw.make_grid(p.n, p.lattice)
    psi = torch.from_numpy(np.ascontiguousarray(p.psi)).to("cuda", dtype=gw.cdtype(prec))
    shape = (len(p.tau), len(s["fft_index"]), len(s["fft_index"]))
    direct = torch.empty(shape, dtype=gw.cdtype(prec), device="cuda")
    gw.chi0_omega(ctx, grid, psi, p.eps, p.n_occ, p.mu, p.tau, s["C"], s["fft_index"], prec, direct)
    plan = gw.Chi0Plan(ctx, grid, p.n_b, p.eps, p.n_occ, p.mu, p.tau, s["C"], s["fft_index"], prec)
    return dict(p=p, s=s, grid=grid, psi=psi, direct=direct, plan=plan,
                out=torch.empty(shape, dtype=gw.cdtype(prec), device="cuda"))


def rel(a, b):
    return (torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b)).item()


def test_plan_launch_equals_call(ctx):
    for name, make, prec in SYSTEMS:
        d = setup_system(ctx, make, prec)
        d["plan"].launch(d["psi"], d["out"])
        d["plan"].status()
        assert rel(d["out"], d["direct"]) < 1e-7, name
        d["plan"].close()


def test_uneven_systems_in_one_graph(ctx):
    ds = [setup_system(ctx, make, prec) for _, make, prec in SYSTEMS]
    for d in ds:                      # first launches outside the capture
        d["plan"].launch(d["psi"], d["out"])
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        for d in ds:
            d["plan"].launch(d["psi"], d["out"])
    for d in ds:
        d["out"].zero_()
    graph.replay()
    torch.cuda.synchronize()
    for (name, _, _), d in zip(SYSTEMS, ds):
        d["plan"].status()
        assert rel(d["out"], d["direct"]) < 1e-7, name
    # one graph launch for the whole batch against the per-system calls
    reps = 5
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        graph.replay()
    torch.cuda.synchronize()
    t_graph = (time.perf_counter() - t0) / reps
    t0 = time.perf_counter()
    for _ in range(reps):
        for d in ds:
            gw.chi0_omega(ctx, d["grid"], d["psi"], d["p"].eps, d["p"].n_occ, d["p"].mu, d["p"].tau, d["s"]["C"],
                          d["s"]["fft_index"], d["plan"].prec, d["out"])
    torch.cuda.synchronize()
    t_call = (time.perf_counter() - t0) / reps
    print("3 systems: one graph replay %.2f ms, direct calls %.2f ms" % (t_graph * 1e3, t_call * 1e3))
    for d in ds:
        d["plan"].close()
