"""The request server on the device: every request of a concurrent mix (several
slots, each with its own context and stream, systems of different sizes and
both request kinds) returns what the same request returns when run alone, and
the chain's Sigma_nn(i omega) agrees with the FP64 oracle within 1 meV."""
import numpy as np
import pytest

from oracle import pipeline as opl
from oracle import qp as oqp
from paper_1607_02859_gb300 import gw, inputs, serve

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
MEV = 3.674932e-5


@pytest.fixture(scope="module")
def built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import os
    if not os.path.exists(gw.LIB_PATH):
        from paper_1607_02859_gb300 import build
        build.build()


@pytest.mark.parametrize("prec", ["fp32", "f16x3"])
def test_mix_matches_alone(built, prec):
    systems = [serve.register(inputs.gamma_toy(), prec),
               serve.register(inputs.tiny(seed=21, n=(8, 8, 8), n_occ=6, n_unocc=40, n_tau=8), prec)]
    alone = {}
    slot = serve.GpuSlot(0, keep_chi=True)
    try:
        for i, s in enumerate(systems):
            for kind in ("chi0", "sigma"):
                r = serve.Request(s, kind)
                alone[(i, kind)] = slot.run(r)
    finally:
        slot.close()
    srv = serve.Server(3, 8 << 30, keep_chi=True)
    try:
        mix = []
        rng = np.random.default_rng(3)
        for _ in range(12):
            i = int(rng.integers(0, 2))
            kind = ("chi0", "sigma")[int(rng.integers(0, 2))]
            mix.append((i, kind, srv.submit(systems[i], kind)))
        srv.drain(timeout=300)
        assert srv.max_concurrent >= 2
        for i, kind, r in mix:
            assert r.error == "", r.error
            ref = alone[(i, kind)]
            if kind == "chi0":
                d = (torch.linalg.vector_norm(r.result - ref) / torch.linalg.vector_norm(ref)).item()
                assert d < 1e-6, d
            else:
                d = np.max(np.abs(r.result["sigma_iw"] - ref["sigma_iw"]))
                assert d < 1e-3 * MEV, d
                d = np.max(np.abs(r.result["qp"]["e_qp"] - ref["qp"]["e_qp"]))
                assert d < 1e-3 * MEV, d
        st = srv.stats()
        assert st["requests"] == 12 and st["p99_ms"] >= st["p50_ms"] > 0
    finally:
        srv.close()
    # the served chain against the oracle's FP64 chain on the toy system
    p = inputs.gamma_toy()
    ref = opl.run(p)
    got = alone[(0, "sigma")]["sigma_iw"]
    assert np.max(np.abs(got - ref["sigma_iw"])) < MEV
    eps_n = p.eps[p.bands]
    e_ref = oqp.linearized(ref["sigma_iw"], p.omega, eps_n, p.mu, eps_n)[0]
    assert np.max(np.abs(alone[(0, "sigma")]["qp"]["e_qp"] - e_ref)) < MEV
