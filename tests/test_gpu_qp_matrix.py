"""GPU parity of the full self-energy matrix (gw_sigma_matrix) and of the
linearised QP energies and spectral functions (gw_qp_energies) against the
FP64 oracle on the same seeded inputs.

Tolerances: FP64 paths ~1e-11 Ha on Sigma and 1e-6 relative on continued
values (Thiele's recursion amplifies rounding-order differences); FP32 and
fp16x3 1 meV = 3.675e-5 Ha on every Sigma_nm(i omega_k), and 1 meV on E_QP
through the chain."""
import numpy as np
import pytest

from oracle import pipeline as opipe
from oracle import qp as oqp
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


def to_dev(x, prec):
    return torch.from_numpy(np.ascontiguousarray(x)).to(device="cuda", dtype=gw.cdtype(prec))


# ---------------------------------------------------------------- Sigma_nm

PROBLEMS = {
    # 4 bands: one partial 16 x 16 tile, one band chunk
    "tiny_c": (lambda: inputs.tiny(seed=61), None),
    "tiny_r": (lambda: inputs.tiny(seed=62, n=(6, 4, 6), a=(6.0, 5.0, 6.5), n_occ=4, n_unocc=12, real=True), None),
    # 20 bands: 2 x 2 tiles with ragged edges, three band chunks of the contraction
    "ragged20": (lambda: inputs.tiny(seed=63, n=(8, 6, 10), a=(7.0, 6.0, 8.0), n_occ=6, n_unocc=42, n_tau=8),
                 np.r_[0:6, 6:48:3][:20]),
    # the degenerate 1 x 1 matrix
    "one_band": (lambda: inputs.tiny(seed=64), np.array([3])),
}


@pytest.fixture(scope="module", params=list(PROBLEMS))
def case(request):
    make, bands = PROBLEMS[request.param]
    p = make()
    if bands is not None:
        p.bands = np.asarray(bands)
    s = opipe.setup(p)
    chi_ref, _ = opipe.chi0_omega(p, s)
    wt, _ = opipe.w_tau(p, s, chi_ref)
    dv = p.volume / p.n_r
    n = len(p.tau)
    nb = len(p.bands)
    su = np.empty((nb, nb, n), dtype=complex)
    so = np.empty((nb, nb, n), dtype=complex)
    for j, t in enumerate(p.tau):
        wrr = osc.w_rr(wt[j], s["gvecs"], p.n, p.lattice)
        su[:, :, j], so[:, :, j] = osg.sigma_matrix_tau(p.psi, p.eps, p.n_occ, p.mu, t, wrr, p.bands, dv)
    return request.param, p, s, wt, su, so, osg.sigma_matrix_iw(su, so, s["C"], s["S"])


@pytest.mark.parametrize("prec", ["fp64", "fp32", "f16x3"])
def test_sigma_matrix(ctx, case, prec):
    name, p, s, wt, su, so, sig_ref = case
    grid = gw.make_grid(p.n, p.lattice)
    psi = to_dev(p.psi, prec)
    out = gw.sigma_matrix(ctx, grid, psi, p.eps, p.n_occ, p.mu, p.bands, p.tau, p.omega, s["C"], s["S"],
                          to_dev(wt, prec), s["fft_index"], prec)
    err = np.max(np.abs(out["sigma_iw"] - sig_ref))
    if prec == "fp64":
        assert np.max(np.abs(out["sigma_unocc"] - su)) < 1e-12
        assert np.max(np.abs(out["sigma_occ"] - so)) < 1e-12
        assert err < 1e-11
    else:
        assert err < MEV
        assert err < (1e-3 if prec == "fp32" else 1e-4) * np.max(np.abs(sig_ref))
    # the off-diagonal part is really there, Hermitian in (n, m) at every tau
    if len(p.bands) > 1:
        off = out["sigma_unocc"][~np.eye(len(p.bands), dtype=bool)]
        assert np.max(np.abs(off)) > 1e-3 * np.max(np.abs(out["sigma_unocc"]))
    herm = np.max(np.abs(out["sigma_unocc"] - out["sigma_unocc"].conj().transpose(1, 0, 2)))
    assert herm < (1e-13 if prec == "fp64" else 1e-5) * np.max(np.abs(out["sigma_unocc"]))
    # its diagonal is gw_sigma_diag's result
    d = gw.sigma_diag(ctx, grid, psi, p.eps, p.n_occ, p.mu, p.bands, p.tau, p.omega, s["C"], s["S"],
                      to_dev(wt, prec), s["fft_index"], prec)
    diag = np.einsum("nnk->nk", out["sigma_iw"])
    tol = 1e-12 if prec == "fp64" else 1e-6
    assert np.max(np.abs(diag - d["sigma_iw"])) < tol * np.max(np.abs(d["sigma_iw"])) + 1e-15


@pytest.mark.parametrize("which", ["matrix", "diag"])
def test_sigma_back_to_tau(ctx, case, which):
    """gw_sigma_to_tau inverts the CT + ST (Eqs. INV_CT_FFT, INV_ST_FFT): from the
    oracle's Sigma(i omega) it returns the oracle's Sigma_unocc(tau) and
    Sigma_occ(-tau), and the GPU's own round trip returns gw_sigma_matrix's."""
    name, p, s, wt, su, so, sig_ref = case
    if which == "diag":
        sig_ref = np.einsum("nnk->nk", sig_ref)
        su, so = np.einsum("nnk->nk", su).real, np.einsum("nnk->nk", so).real
    bu, bo = gw.sigma_to_tau(ctx, sig_ref, s["Cinv"], s["Sinv"])
    ou, oo = osg.sigma_tau_from_iw(sig_ref, s["Cinv"], s["Sinv"])
    scale = max(np.max(np.abs(su)), np.max(np.abs(so)))
    tol = 1e-13 * np.linalg.cond(s["S"]) * scale
    assert np.max(np.abs(bu - ou)) < tol and np.max(np.abs(bo - oo)) < tol
    assert np.max(np.abs(bu - su)) < 10 * tol and np.max(np.abs(bo - so)) < 10 * tol


def test_sigma_matrix_argument_errors(ctx):
    p = inputs.tiny(seed=61)
    s = opipe.setup(p)
    grid = gw.make_grid(p.n, p.lattice)
    psi = to_dev(p.psi, "fp32")
    w = torch.zeros((len(p.tau), p.n_r, p.n_r), dtype=torch.complex64, device="cuda")
    with pytest.raises(gw.GwError) as e:                                # more than 256 bands
        gw.sigma_matrix(ctx, grid, psi, p.eps, p.n_occ, p.mu, np.zeros(257, dtype=np.int32), p.tau, p.omega,
                        s["C"], s["S"], w, s["fft_index"], "fp32")
    assert e.value.status == 2
    with pytest.raises(gw.GwError) as e:                                # band out of range
        gw.sigma_matrix(ctx, grid, psi, p.eps, p.n_occ, p.mu, [0, p.n_b], p.tau, p.omega, s["C"], s["S"], w,
                        s["fft_index"], "fp32")
    assert e.value.status == 1


# ---------------------------------------------------------------- QP energies

def _pole_sigma(rng, n_n, omega):
    """Seeded causal pole sums on the nodes i omega, as many poles as nodes (so
    that no entry is a rational function the approximant reproduces early)."""
    k = len(omega)
    out = np.empty((n_n, k), dtype=complex)
    for b in range(n_n):
        e = rng.uniform(-2, 2, k)
        eta = 0.05 * rng.uniform(0.5, 1.5, k)
        r = 0.1 * rng.uniform(0.1, 1.0, k)
        out[b] = sum(ri / (1j * omega - (ei - 1j * hi)) for ri, ei, hi in zip(r, e, eta))
    return out


@pytest.mark.parametrize("n_n,n,n_w", [(37, 8, 1001), (5, 16, 257), (3, 1, 11), (64, 12, 0)])
def test_qp_energies_parity(ctx, n_n, n, n_w):
    """Same Sigma(i omega) into both: the continuation amplifies a relative
    perturbation of 1e-15 in Sigma to ~1e-8 Ha in E at 16 nodes (measured on
    the oracle), so rounding-order differences allow 1e-7 Ha and 1e-5 relative."""
    rng = np.random.default_rng(100 + n_n)
    omega = np.geomspace(0.02, 30.0, n)
    sig = _pole_sigma(rng, n_n, omega)
    eps = rng.uniform(-1, 1, n_n)
    vstat = eps + rng.uniform(-0.2, 0.2, n_n)
    mu = 0.05
    w = np.linspace(-1.5, 1.5, n_w) if n_w else None
    out = gw.qp_energies(ctx, omega, sig, eps, mu, vstat, w)
    e, z, se, ds = oqp.linearized(sig, omega, eps, mu, vstat)
    assert np.max(np.abs(out["e_qp"] - e)) < 1e-7
    assert np.max(np.abs(out["z"] - z) / np.abs(z)) < 1e-5
    assert np.max(np.abs(out["sigma_eps"] - se) / np.abs(se)) < 1e-5
    assert np.max(np.abs(out["dsigma"] - ds) / (np.abs(ds) + 1e-12)) < 1e-5
    if n_w:
        a = oqp.spectral(sig, omega, eps, mu, vstat, w)
        assert np.max(np.abs(out["spectral"] - a)) < 1e-5 * np.max(np.abs(a))
    else:
        assert "spectral" not in out


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_qp_through_the_chain(ctx, prec):
    """gamma_toy: Sigma_nn(i omega) from the GPU chain, then E_QP, Z and A on the
    GPU, against the oracle chain and the oracle's QP step."""
    p = inputs.gamma_toy()
    ref = opipe.run(p)
    s = ref["setup"]
    grid = gw.make_grid(p.n, p.lattice)
    psi = to_dev(p.psi, prec)
    n = len(p.tau)
    chi_w = torch.zeros((n, p.n_chi, p.n_chi), dtype=gw.cdtype(prec), device="cuda")
    gw.chi0_omega(ctx, grid, psi, p.eps, p.n_occ, p.mu, p.tau, s["C"], s["fft_index"], prec, chi_w)
    gw.screen_W(ctx, grid, s["gvecs"], prec, chi_w, chi_w, resid=False)
    w_tau = torch.zeros_like(chi_w)
    gw.tau_to_omega(ctx, gw.CT, s["Cinv"], chi_w, w_tau, prec)
    sig = gw.sigma_diag(ctx, grid, psi, p.eps, p.n_occ, p.mu, p.bands, p.tau, p.omega, s["C"], s["S"], w_tau,
                        s["fft_index"], prec)["sigma_iw"]
    eps = p.eps[p.bands]
    vstat = eps + 0.01          # a static shift standing in for Sigma_x - V_xc
    w = np.linspace(-0.8, 0.6, 141)
    out = gw.qp_energies(ctx, p.omega, sig, eps, p.mu, vstat, w)
    e, z, _, _ = oqp.linearized(ref["sigma_iw"], p.omega, eps, p.mu, vstat)
    a = oqp.spectral(ref["sigma_iw"], p.omega, eps, p.mu, vstat, w)
    tol = 1e-7 if prec == "fp64" else MEV
    assert np.max(np.abs(out["e_qp"] - e)) < tol
    assert np.all((out["z"] > 0) & (out["z"] <= 1))
    assert np.max(np.abs(out["z"] - z)) < (1e-6 if prec == "fp64" else 1e-3)
    assert np.max(np.abs(out["spectral"] - a)) < (1e-5 if prec == "fp64" else 1e-2) * np.max(a)


def test_qp_breakdown_and_argument_errors(ctx):
    omega = np.array([1.0, 2.0, 3.0])
    bad = np.array([[1.0, 2.0, 1.0], [0.5, 0.4, 0.3]], dtype=complex)    # entry 0: vanishing difference
    with pytest.raises(gw.GwError) as e:
        gw.qp_energies(ctx, omega, bad, [0.0, 0.0], 0.0, [0.0, 0.0])
    assert e.value.status == 5 and "entry 0" in e.value.message
    ok = gw.qp_energies(ctx, omega, bad[1:], [0.0], 0.0, [0.0])             # the context is still usable
    assert np.isfinite(ok["e_qp"]).all()
    for om, err in ((np.array([1.0, -2.0, 3.0]), 1), (np.array([1.0, 1.0, 3.0]), 1)):
        with pytest.raises(gw.GwError) as e:
            gw.qp_energies(ctx, om, bad[1:], [0.0], 0.0, [0.0])
        assert e.value.status == err
    with pytest.raises(gw.GwError) as e:
        gw.qp_energies(ctx, np.geomspace(0.1, 10, 33), np.ones((1, 33)), [0.0], 0.0, [0.0])
    assert e.value.status == 2


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("n", [6, 8, 11])
def test_inverse_sine_kind(ctx, prec, n):
    """gw_tau_to_omega with GW_IST: out[j] = -i sum_k M[j][k] in[k] (Eq. INV_ST_FFT),
    on the register-resident sizes (6, 8) and the generic kernel (11)."""
    rng = np.random.default_rng(n)
    m = rng.standard_normal((n, n))
    x = rng.standard_normal((n, 1000)) + 1j * rng.standard_normal((n, 1000))
    out = torch.zeros((n, 1000), dtype=gw.cdtype(prec), device="cuda")
    gw.tau_to_omega(ctx, gw.IST, m, to_dev(x, prec), out, prec)
    ref = -1j * (m @ x)
    err = np.max(np.abs(out.cpu().numpy() - ref)) / np.max(np.abs(ref))
    assert err < (1e-14 if prec == "fp64" else 1e-6)
