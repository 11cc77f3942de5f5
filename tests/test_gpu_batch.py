"""The whole hot path of several uneven systems as one CUDA-graph launch
(gw_batch_plan / gw_batch_launch / gw_batch_wait): every system's
Sigma_nn(i omega) against the FP64 oracle chain (chi0 -> W~ -> W~(tau) ->
Sigma), replays reproduce the first launch to rounding (the fused self-energy
sums its r-block partials with atomics, whose order varies), and the plan
refuses to replay once the context's arena has moved."""
import numpy as np
import pytest

from oracle import pipeline as opipe
from paper_1607_02859_gb300 import gw, inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
MEV = 3.674932e-5


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


MAKERS = [lambda: inputs.tiny(seed=81),
          lambda: inputs.tiny(seed=82, n=(8, 6, 10), a=(7.0, 6.0, 8.0), n_occ=6, n_unocc=42, n_tau=8),
          lambda: inputs.tiny(seed=83, n=(12, 12, 12), a=(9.0, 9.0, 9.0), n_occ=24, n_unocc=120, n_tau=6, n_chi=300)]


@pytest.fixture(scope="module")
def problems():
    out = []
    for make in MAKERS:
        p = make()
        ref = opipe.run(p)
        out.append((p, ref))
    return out


def system(p, s, prec, refine=0):
    dt = gw.cdtype(prec)
    shape = (len(p.tau), len(s["fft_index"]), len(s["fft_index"]))
    return dict(grid=gw.make_grid(p.n, p.lattice), psi=torch.from_numpy(np.ascontiguousarray(p.psi)).to("cuda", dtype=dt),
                eps=p.eps, n_occ=p.n_occ, mu=p.mu, tau=p.tau, omega=p.omega, C=s["C"], S=s["S"], Cinv=s["Cinv"],
                gvec=s["gvecs"], fft_index=s["fft_index"], bands=p.bands, refine=refine,
                chi_w=torch.empty(shape, dtype=dt, device="cuda"), w_tau=torch.empty(shape, dtype=dt, device="cuda"))


@pytest.mark.parametrize("prec,refine", [("fp32", 0), ("f16x3", 1), ("fp64", 0)])
def test_batch_matches_oracle(ctx, problems, prec, refine):
    systems = [system(p, ref["setup"], prec, refine) for p, ref in problems]
    b = gw.Batch(ctx, systems, prec)
    b.launch()
    sig, status = b.wait(timeout_ms=60000)
    assert status == [0] * len(problems)
    tol = 1e-9 if prec == "fp64" else MEV
    for (p, ref), got in zip(problems, sig):
        err = float(np.max(np.abs(got - ref["sigma_iw"])))
        print("%s %s: max |dSigma(i omega)| = %.2e Ha" % (p.name, prec, err))
        assert err < tol, (p.name, err)
    # a replay gives the same results (the graph keeps every pointer and table);
    # the self-energy's r-block partials are summed by atomics in varying order,
    # so equal up to rounding of the working precision
    b.launch()
    sig2, status2 = b.wait(timeout_ms=60000)
    assert status2 == [0] * len(problems)
    rel = 1e-12 if prec == "fp64" else 1e-5
    for a, c in zip(sig, sig2):
        assert np.max(np.abs(a - c)) <= rel * np.max(np.abs(a)) + 1e-12
    b.close()


def test_batch_refuses_a_moved_arena(ctx, problems):
    p, ref = problems[0]
    b = gw.Batch(ctx, [system(p, ref["setup"], "fp32")], "fp32")
    ctx.reserve(ctx.scratch_bytes + (64 << 20))           # grows (reallocates) the arena
    with pytest.raises(gw.GwError) as e:
        b.launch()
    assert e.value.status == 1
    b.close()


def test_batch_wait_before_launch(ctx, problems):
    p, ref = problems[0]
    b = gw.Batch(ctx, [system(p, ref["setup"], "fp32")], "fp32")
    with pytest.raises(gw.GwError):
        b.wait(timeout_ms=10)
    b.close()
