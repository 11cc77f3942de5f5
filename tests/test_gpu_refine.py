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


def test_zgemm_sliced_exact_on_integers(ctx):
    """Integer components below 64 are one exact slice each, so with every K block's
    sum below 2^24 the tensor-core product must equal the exact integer product:
    checks the exactness of the FP32 accumulation in tensor memory, the K blocks
    (K = 2500 complex = 5000 real: two blocks), ragged tiles and the complex
    mapping."""
    rng = np.random.default_rng(5)
    M, K, N = 300, 2500, 200
    a = rng.integers(-50, 51, (M, K)) + 1j * rng.integers(-50, 51, (M, K))
    b = rng.integers(-50, 51, (K, N)) + 1j * rng.integers(-50, 51, (K, N))
    ar, ai = a.real.astype(np.int64), a.imag.astype(np.int64)
    br, bi = b.real.astype(np.int64), b.imag.astype(np.int64)
    ref = (ar @ br - ai @ bi) + 1j * (ar @ bi + ai @ br)          # exact in int64
    A = torch.from_numpy(a).to("cuda")
    B = torch.from_numpy(b).to("cuda")
    C = torch.full((M, N), 7.0 + 0j, dtype=torch.complex128, device="cuda")
    gw.zgemm_sliced(ctx, A, B, C, levels=1)
    got = C.cpu().numpy()
    assert np.array_equal(got, ref.astype(np.complex128))


@pytest.mark.parametrize("levels", [3, 5])
def test_zgemm_sliced_accuracy(ctx, levels):
    """Gaussian matrices with rows and columns of magnitudes spread over four
    decades, against numpy's FP64 product.  The slice pairs dropped (a + b >
    levels, each below 2^(e_i + f_j - 6 (a+b) - 1)) and the slicing rest bound
    each element's error by 4 (levels + 2) 2^(-6(levels+1)) K max|A_i.| max|B_.j|."""
    rng = np.random.default_rng(6 + levels)
    M, K, N = 520, 3000, 390
    a = (rng.standard_normal((M, K)) + 1j * rng.standard_normal((M, K))) * 10.0 ** rng.uniform(-2, 2, (M, 1))
    b = (rng.standard_normal((K, N)) + 1j * rng.standard_normal((K, N))) * 10.0 ** rng.uniform(-2, 2, (1, N))
    ref = a @ b
    C = torch.empty((M, N), dtype=torch.complex128, device="cuda")
    gw.zgemm_sliced(ctx, torch.from_numpy(a).to("cuda"), torch.from_numpy(b).to("cuda"), C, levels=levels)
    err = np.abs(C.cpu().numpy() - ref)
    amax = np.max(np.maximum(np.abs(a.real), np.abs(a.imag)), axis=1)
    bmax = np.max(np.maximum(np.abs(b.real), np.abs(b.imag)), axis=0)
    scale = 4.0 * (levels + 2) * 2.0 ** (-6 * (levels + 1)) * K * np.outer(amax, bmax)
    print("levels %d: max err / bound %.2e, relative Frobenius error %.2e"
          % (levels, np.max(err / scale), np.linalg.norm(err) / np.linalg.norm(ref)))
    assert np.max(err / scale) < 1.0
    # a plain split GEMM with FP32 accumulation would be near 1e-6 here
    assert np.linalg.norm(err) / np.linalg.norm(ref) < (1e-6 if levels == 3 else 1e-9)


def test_zgemm_sliced_argument_checks(ctx):
    A = torch.zeros((4, 4), dtype=torch.complex128, device="cuda")
    with pytest.raises(gw.GwError) as e:
        gw.zgemm_sliced(ctx, A, A, A.clone(), levels=0)
    assert e.value.status == 1
    with pytest.raises(ValueError):
        gw.zgemm_sliced(ctx, A.to(torch.complex64), A, A.clone())
