"""FP64 refinement of the screening solve (gw_screen_W_refine, Eq. W_correlated):
the working-precision factorisation followed by Newton-Schulz steps on
X = eps~^{-1} - 1 with FP64 residuals.  The oracle solves the same input the
GPU receives (chi0 rounded to the working precision), so the comparison
measures the solve alone."""
import numpy as np
import pytest

from oracle import pipeline as opipe
from oracle import screen as osc
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


@pytest.fixture(scope="module")
def toy():
    p = inputs.gamma_toy()
    s = opipe.setup(p)
    chi_ref, _ = opipe.chi0_omega(p, s)
    return p, s, chi_ref


def relf(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("prec", ["fp32", "f16x3", "fp64"])
def test_refinement_reaches_working_precision(ctx, toy, prec):
    p, s, chi_ref = toy
    grid = gw.make_grid(p.n, p.lattice)
    chi_in = chi_ref.astype(np.complex128 if prec == "fp64" else np.complex64)
    w_ref = osc.screen(chi_in.astype(np.complex128), s["vhalf"])
    chi_d = torch.from_numpy(np.ascontiguousarray(chi_in)).to("cuda")
    w0 = torch.zeros_like(chi_d)
    r0 = gw.screen_W(ctx, grid, s["gvecs"], prec, chi_d, w0)
    w2 = torch.zeros_like(chi_d)
    r2 = gw.screen_W(ctx, grid, s["gvecs"], prec, chi_d, w2, refine=2)
    e0 = relf(w0.cpu().numpy().astype(np.complex128), w_ref)
    e2 = relf(w2.cpu().numpy().astype(np.complex128), w_ref)
    print("%s: W~ error %.2e -> %.2e, residual %.2e -> %.2e" % (prec, e0, e2, r0.max(), r2.max()))
    if prec == "fp64":
        # the residual bound of an FP64 solve
        assert np.all(r2 < 1e-12) and e2 < 1e-12
    else:
        # refined X is exact to FP64 before it is rounded into the FP32 W~
        assert e2 < 1e-6 and np.all(r2 < 1e-6)
        assert e2 <= e0 * 1.01
    # in place (chi_w and w_w the same buffer) gives the same W~
    w3 = chi_d.clone()
    gw.screen_W(ctx, grid, s["gvecs"], prec, w3, w3, resid=False, refine=2)
    assert torch.equal(w3, w2)


def test_refine_argument_checks(ctx, toy):
    p, s, chi_ref = toy
    grid = gw.make_grid(p.n, p.lattice)
    chi_d = torch.from_numpy(chi_ref[:1].astype(np.complex64)).to("cuda")
    with pytest.raises(gw.GwError):
        gw.screen_W(ctx, grid, s["gvecs"], "fp32", chi_d, chi_d.clone(), refine=9)
