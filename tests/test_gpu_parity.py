"""GPU parity: every C-ABI call against the FP64 oracle on the same seeded
inputs, at sizes the oracle finishes in seconds (several FFT pencils and GEMM
tiles, ragged row blocks, a truncated G sphere, real and complex orbitals).

Tolerances: FP64 path ~1e-10 relative; FP32 path 1e-6 relative Frobenius on
chi0(i omega) (the stated target), and 1 meV = 3.675e-5 Ha absolute on every
Sigma_nn(i omega_k)."""
import numpy as np
import pytest

from oracle import chi as ochi
from oracle import green as ogr
from oracle import gvec as ogv
from oracle import pipeline as opipe
from oracle import screen as osc
from oracle import sigma as osg
from paper_1607_02859_gb300 import gw, inputs

pytestmark = pytest.mark.gpu
MEV = 3.674932e-5
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


def relf(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def to_dev(x, prec):
    return torch.from_numpy(np.ascontiguousarray(x)).to(device="cuda", dtype=gw.cdtype(prec))


def host(t):
    return t.detach().cpu().numpy().astype(np.complex128)


PROBLEMS = {
    "tiny_c": lambda: inputs.tiny(seed=21),
    "tiny_r": lambda: inputs.tiny(seed=22, n=(6, 4, 6), a=(6.0, 5.0, 6.5), n_occ=4, n_unocc=12, real=True),
    "ragged": lambda: inputs.tiny(seed=23, n=(8, 6, 10), a=(7.0, 6.0, 8.0), n_occ=6, n_unocc=42, n_tau=8),
    "sphere": lambda: inputs.tiny(seed=24, n=(8, 8, 8), a=(7.0, 7.0, 7.0), n_occ=5, n_unocc=35, n_tau=7,
                                  n_chi=123),
}
TOL = {"fp64": 1e-10, "fp32": 1e-6}


@pytest.fixture(scope="module", params=list(PROBLEMS))
def case(request):
    p = PROBLEMS[request.param]()
    s = opipe.setup(p)
    return request.param, p, s


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_green_tau_rows(ctx, case, prec):
    name, p, s = case
    grid = gw.make_grid(p.n, p.lattice)
    psi = to_dev(p.psi, prec)
    r0, rows = 3, p.n_r - 7                          # ragged: not a multiple of any tile
    for tau in (p.tau[0], p.tau[-1]):
        go = torch.zeros((rows, p.n_r), dtype=gw.cdtype(prec), device="cuda")
        gu = torch.zeros_like(go)
        gw.green_tau(ctx, grid, psi, p.eps, p.n_occ, p.mu, tau, r0, rows, prec, go, gu)
        rr = np.arange(r0, r0 + rows)
        ref_o = ogr.green_occ_rows(p.psi, p.eps, p.n_occ, p.mu, tau, rr)
        ref_u = ogr.green_unocc_rows(p.psi, p.eps, p.n_occ, p.mu, tau, rr)
        assert relf(host(go), ref_o) < 10 * TOL[prec]
        assert relf(host(gu), ref_u) < 10 * TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_chi0_rtau_and_fused(ctx, case, prec):
    name, p, s = case
    grid = gw.make_grid(p.n, p.lattice)
    psi = to_dev(p.psi, prec)
    tau = p.tau[1]
    go = torch.zeros((p.n_r, p.n_r), dtype=gw.cdtype(prec), device="cuda")
    gu = torch.zeros_like(go)
    gw.green_tau(ctx, grid, psi, p.eps, p.n_occ, p.mu, tau, 0, p.n_r, prec, go, gu)
    chi = torch.zeros_like(go)
    gw.chi0_rtau(ctx, go, gu, chi, prec)
    ref = ochi.chi_rr(ogr.green_occ(p.psi, p.eps, p.n_occ, p.mu, tau), ogr.green_unocc(p.psi, p.eps, p.n_occ, p.mu, tau))
    assert relf(host(chi), ref) < 10 * TOL[prec]
    chi2 = torch.zeros((p.n_r - 5, p.n_r), dtype=gw.cdtype(prec), device="cuda")
    gw.chi0_rtau_fused(ctx, grid, psi, p.eps, p.n_occ, p.mu, tau, 5, p.n_r - 5, prec, chi2)
    assert relf(host(chi2), ref[5:]) < 10 * TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_spatial_transforms(ctx, case, prec):
    name, p, s = case
    grid = gw.make_grid(p.n, p.lattice)
    gv, idx = s["gvecs"], s["fft_index"]
    nchi = len(idx)
    rng = np.random.default_rng(7)
    rows, r0 = min(p.n_r, 37), 11
    x = rng.standard_normal((rows, p.n_r)) + 1j * rng.standard_normal((rows, p.n_r))
    out = torch.zeros((rows, nchi), dtype=gw.cdtype(prec), device="cuda")
    gw.rr_to_GG_fft(ctx, grid, +1, 1, idx, prec, r0, rows, to_dev(x, prec), out)
    assert relf(host(out), ochi.rows_to_g(x, gv, p.n)) < 10 * TOL[prec]
    X = rng.standard_normal((p.n_r, nchi)) + 1j * rng.standard_normal((p.n_r, nchi))
    out2 = torch.zeros((nchi, nchi), dtype=gw.cdtype(prec), device="cuda")
    gw.rr_to_GG_fft(ctx, grid, +1, 2, idx, prec, 0, p.n_r, to_dev(X, prec), out2)
    assert relf(host(out2), ochi.cols_to_g(X, gv, p.n, p.lattice)) < 10 * TOL[prec]
    W = rng.standard_normal((nchi, nchi)) + 1j * rng.standard_normal((nchi, nchi))
    out3 = torch.zeros((p.n_r, nchi), dtype=gw.cdtype(prec), device="cuda")
    gw.rr_to_GG_fft(ctx, grid, -1, 2, idx, prec, 0, p.n_r, to_dev(W, prec), out3)
    ref3 = osc.w_rows_to_r(W, gv, p.n)
    assert relf(host(out3), ref3) < 10 * TOL[prec]
    out4 = torch.zeros((rows, p.n_r), dtype=gw.cdtype(prec), device="cuda")
    gw.rr_to_GG_fft(ctx, grid, -1, 1, idx, prec, r0, rows, to_dev(ref3[r0:r0 + rows], prec), out4)
    assert relf(host(out4), osc.w_cols_to_r(ref3[r0:r0 + rows], gv, p.n, p.lattice)) < 10 * TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_tau_to_omega(ctx, case, prec):
    name, p, s = case
    rng = np.random.default_rng(8)
    n = len(p.tau)
    f = rng.standard_normal((n, 333)) + 1j * rng.standard_normal((n, 333))
    out = torch.zeros((n, 333), dtype=gw.cdtype(prec), device="cuda")
    gw.tau_to_omega(ctx, gw.CT, s["C"], to_dev(f, prec), out, prec)
    assert relf(host(out), s["C"] @ f) < 10 * TOL[prec]
    gw.tau_to_omega(ctx, gw.ST, s["S"], to_dev(f, prec), out, prec)
    assert relf(host(out), 1j * (s["S"] @ f)) < 10 * TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_chi0_omega(ctx, case, prec):
    name, p, s = case
    grid = gw.make_grid(p.n, p.lattice)
    chi_ref, _ = opipe.chi0_omega(p, s)
    nchi = len(s["fft_index"])
    for rb in (0, 29):                                # default and a ragged r-block
        out = torch.zeros((len(p.tau), nchi, nchi), dtype=gw.cdtype(prec), device="cuda")
        gw.chi0_omega(ctx, grid, to_dev(p.psi, prec), p.eps, p.n_occ, p.mu, p.tau, s["C"], s["fft_index"], prec,
                      out, r_block=rb)
        assert relf(host(out), chi_ref) < TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_screen_W(ctx, case, prec):
    name, p, s = case
    grid = gw.make_grid(p.n, p.lattice)
    chi_ref, _ = opipe.chi0_omega(p, s)
    w_ref = osc.screen(chi_ref, s["vhalf"])
    chi_d = to_dev(chi_ref, prec)
    w_d = torch.zeros_like(chi_d)
    res = gw.screen_W(ctx, grid, s["gvecs"], prec, chi_d, w_d)
    # W~ is an intermediate: FP32 Cholesky error ~ cond(eps~) * sqrt(N) * 6e-8
    wtol = 1e-10 if prec == "fp64" else 1e-5
    assert relf(host(w_d), w_ref) < wtol
    assert np.all(res < wtol)
    gw.screen_W(ctx, grid, s["gvecs"], prec, chi_d, chi_d, resid=False)     # in place
    assert relf(host(chi_d), w_ref) < wtol


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_sigma_diag(ctx, case, prec):
    name, p, s = case
    grid = gw.make_grid(p.n, p.lattice)
    chi_ref, _ = opipe.chi0_omega(p, s)
    wt, _ = opipe.w_tau(p, s, chi_ref)
    su, so = opipe.sigma_from_w(p, s, wt)
    sig_ref = osg.sigma_iw(su, so, s["C"], s["S"])
    wr = np.linspace(-0.6, 0.6, 7)
    ref_real = opipe.continue_sigma(p, sig_ref, wr)
    out = gw.sigma_diag(ctx, grid, to_dev(p.psi, prec), p.eps, p.n_occ, p.mu, p.bands, p.tau, p.omega, s["C"],
                        s["S"], to_dev(wt, prec), s["fft_index"], prec, w_real=wr)
    if prec == "fp64":
        assert np.max(np.abs(out["sigma_unocc"] - su)) < 1e-12
        assert np.max(np.abs(out["sigma_occ"] - so)) < 1e-12
        assert np.max(np.abs(out["sigma_iw"] - sig_ref)) < 1e-11
        assert np.max(np.abs(out["sigma_real"] - ref_real) / np.abs(ref_real)) < 1e-6
    else:
        assert np.max(np.abs(out["sigma_iw"] - sig_ref)) < MEV
        assert np.max(np.abs(out["sigma_iw"] - sig_ref)) < 1e-3 * np.max(np.abs(sig_ref))


def test_screen_rejects_non_positive_definite(ctx):
    """chi with a large positive eigenvalue makes eps~ indefinite: GW_ERR_NUMERIC, context still usable."""
    p = PROBLEMS["tiny_c"]()
    grid = gw.make_grid(p.n, p.lattice)
    gv, _ = gw.g_set(grid, p.n_r)
    vh = gw.coulomb_sqrt(grid, gv)
    u = np.zeros(p.n_r, dtype=complex)
    u[1] = 1.0
    chi = (50.0 / vh[1] ** 2) * np.outer(u, u.conj())[None]
    d = to_dev(chi, "fp64")
    out = torch.zeros_like(d)
    with pytest.raises(gw.GwError) as e:
        gw.screen_W(ctx, grid, gv, "fp64", d, out)
    assert e.value.status == 5
    gw.screen_W(ctx, grid, gv, "fp64", torch.zeros_like(d), out)       # still usable
    assert float(out.abs().max()) == 0.0


def test_argument_errors(ctx):
    p = PROBLEMS["tiny_c"]()
    grid = gw.make_grid(p.n, p.lattice)
    psi = to_dev(p.psi, "fp32")
    g = torch.zeros((4, p.n_r), dtype=torch.complex64, device="cuda")
    with pytest.raises(gw.GwError) as e:                               # mu outside the gap
        gw.green_tau(ctx, grid, psi, p.eps, p.n_occ, p.eps[p.n_occ] + 0.1, 1.0, 0, 4, "fp32", g, g)
    assert e.value.status == 1
    with pytest.raises(gw.GwError) as e:                               # rows beyond N_r
        gw.green_tau(ctx, grid, psi, p.eps, p.n_occ, p.mu, 1.0, p.n_r - 2, 4, "fp32", g, g)
    assert e.value.status == 2
    gw.green_tau(ctx, grid, psi, p.eps, p.n_occ, p.mu, 1.0, 0, 0, "fp32", g, g)   # empty: no-op
    bad = gw.make_grid((10, 10, 10), p.lattice)
    with pytest.raises(gw.GwError) as e:
        gw.rr_to_GG_fft(ctx, bad, 1, 1, np.arange(10), "fp32", 0, 1, g, g)
    assert e.value.status == 7


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_gamma_toy_end_to_end(ctx, prec):
    """The 12^3 real-orbital Gamma toy through the whole chain on the GPU."""
    p = inputs.gamma_toy()
    ref = opipe.run(p, w_real=np.linspace(-0.5, 0.5, 5))
    s = ref["setup"]
    grid = gw.make_grid(p.n, p.lattice)
    psi = to_dev(p.psi, prec)
    n = len(p.tau)
    chi_w = torch.zeros((n, p.n_chi, p.n_chi), dtype=gw.cdtype(prec), device="cuda")
    gw.chi0_omega(ctx, grid, psi, p.eps, p.n_occ, p.mu, p.tau, s["C"], s["fft_index"], prec, chi_w)
    assert relf(host(chi_w), ref["chi_w"]) < TOL[prec]
    gw.screen_W(ctx, grid, s["gvecs"], prec, chi_w, chi_w, resid=False)
    w_tau = torch.zeros_like(chi_w)
    gw.tau_to_omega(ctx, gw.CT, s["Cinv"], chi_w, w_tau, prec)
    assert relf(host(w_tau), ref["W_tau"]) < (1e-9 if prec == "fp64" else 1e-5)
    out = gw.sigma_diag(ctx, grid, psi, p.eps, p.n_occ, p.mu, p.bands, p.tau, p.omega, s["C"], s["S"], w_tau,
                        s["fft_index"], prec, w_real=np.linspace(-0.5, 0.5, 5))
    err = np.max(np.abs(out["sigma_iw"] - ref["sigma_iw"]))
    assert err < (1e-9 if prec == "fp64" else MEV)
