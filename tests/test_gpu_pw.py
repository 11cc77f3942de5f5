"""chi0(G,G',i omega) and Sigma_nn(i omega) with G through its plane-wave form
(gw_chi0_omega_pw, gw_sigma_diag_pw).  chi0:
the G formation over the orbitals' plane-wave set, its column transform over
the grid, and the row pass that expands G_occ and G_unocc over R', multiplies
them (Eq. chi_rr) and transforms onto chi's G set (Eq. FFTX1).  Checked against
the FP64 oracle chain on the small cases (every precision), against the
pair sum on sampled rows at 36^3 (the thread-block-cluster row pass), and
for its refusals: orbitals outside the plane-wave set, and a grid whose two
expanded rows do not fit a cluster.  Sigma: the oracle chain's W~ on the small
cases, a sparse W~ at 36^3 against the conventional route."""
import numpy as np
import pytest

from oracle import chi as ochi
from oracle import grids as ogrids
from oracle import gvec as ogv
from oracle import pipeline as opipe
from oracle import sigma as osg
from paper_1607_02859_gb300 import gw, inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
TOL = {"fp64": 1e-12, "fp32": 1e-6, "f16x3": 5e-6, "bf16x3": 2e-5}


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


def support(p):
    """FFT positions of the plane waves e^{+i g.r} in any orbital (numpy, test side)."""
    w = np.zeros(int(np.prod(p.n)))
    for v in p.psi:
        w += np.abs(np.fft.fftn(v.reshape(p.n)).reshape(-1)) ** 2
    return np.flatnonzero(w > 1e-20 * w.max()).astype(np.int32)


def dev(x, prec):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda", dtype=gw.cdtype(prec))


CASES = {
    "tiny_c": lambda: inputs.tiny(seed=41),
    "ragged": lambda: inputs.tiny(seed=43, n=(8, 6, 10), a=(7.0, 6.0, 8.0), n_occ=6, n_unocc=42, n_tau=8),
    "gamma_toy_real": lambda: inputs.gamma_toy(),
    "k_multi": lambda: inputs.tiny(seed=44, n=(12, 12, 12), a=(9.0, 9.0, 9.0), n_occ=40, n_unocc=180, n_tau=6,
                                   n_chi=400),
}


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
    p = CASES[request.param]()
    s = opipe.setup(p)
    chi_ref, _ = opipe.chi0_omega(p, s)
    return request.param, p, s, chi_ref


@pytest.mark.parametrize("prec", ["fp64", "fp32", "f16x3", "bf16x3"])
def test_pw_chi0_omega_matches_oracle(ctx, case, prec):
    name, p, s, chi_ref = case
    grid = gw.make_grid(p.n, p.lattice)
    pw = support(p)
    n = len(p.tau)
    chi = torch.empty((n, p.n_chi, p.n_chi), dtype=gw.cdtype(prec), device="cuda")
    gw.chi0_omega_pw(ctx, grid, dev(p.psi, prec), p.eps, p.n_occ, p.mu, p.tau, s["C"], s["fft_index"], pw, prec, chi)
    got = chi.cpu().numpy().astype(np.complex128)
    err = float(np.linalg.norm(got - chi_ref) / np.linalg.norm(chi_ref))
    print("%s %s (n_pw %d of %d): chi0(i omega) relative error %.2e" % (name, prec, len(pw), p.n_r, err))
    assert err < TOL[prec], err


def test_pw_rejects_orbitals_outside_the_set(ctx):
    p = CASES["tiny_c"]()
    s = opipe.setup(p)
    grid = gw.make_grid(p.n, p.lattice)
    pw = support(p)
    outside = np.setdiff1d(np.arange(p.n_r), pw)[0]
    psi = p.psi.copy()
    r = np.arange(p.n_r)
    # a small component on a plane wave outside the set (its FFT position `outside`)
    idx3 = np.array(np.unravel_index(r, p.n)).T
    o3 = np.array(np.unravel_index(outside, p.n))
    phase = np.exp(2j * np.pi * (idx3 @ (o3 / np.array(p.n))))
    psi[3] = psi[3] + 1e-2 * np.abs(psi[3]).max() * phase
    chi = torch.empty((len(p.tau), p.n_chi, p.n_chi), dtype=torch.complex128, device="cuda")
    with pytest.raises(gw.GwError) as e:
        gw.chi0_omega_pw(ctx, grid, dev(psi, "fp64"), p.eps, p.n_occ, p.mu, p.tau, s["C"], s["fft_index"], pw,
                         "fp64", chi)
    assert e.value.status == 1 and "band 3" in e.value.message


def test_pw_unsupported_grid_is_refused(ctx):
    """FP64 rows of 36^3: two expanded rows do not fit a cluster's shared memory."""
    p = inputs.tiny(seed=45, n=(36, 36, 36), a=(20.0, 20.0, 20.0), n_occ=4, n_unocc=28, n_tau=6, n_chi=64)
    mats = ogrids.transform_matrices(p.tau, p.omega, p.x_min, p.x_max, p.n_x, p.ridge)
    grid = gw.make_grid(p.n, p.lattice)
    idx = ogv.fft_index(ogv.g_set(p.n, p.n_chi), p.n)
    pw = ogv.fft_index(ogv.g_set(p.n, p.n_b), p.n)
    chi = torch.empty((len(p.tau), p.n_chi, p.n_chi), dtype=torch.complex128, device="cuda")
    with pytest.raises(gw.GwError) as e:
        gw.chi0_omega_pw(ctx, grid, dev(p.psi, "fp64"), p.eps, p.n_occ, p.mu, p.tau, mats["C"], idx, pw, "fp64", chi)
    assert e.value.status == 7


@pytest.fixture(scope="module")
def g36():
    p = inputs.tiny(seed=46, n=(36, 36, 36), a=(20.52, 20.52, 20.52), n_occ=16, n_unocc=240, n_tau=6, n_chi=2048)
    gv = ogv.g_set(p.n, p.n_chi)
    idx = ogv.fft_index(gv, p.n)
    mats = ogrids.transform_matrices(p.tau, p.omega, p.x_min, p.x_max, p.n_x, p.ridge)
    rows = sorted(np.random.default_rng(17).choice(p.n_chi, 10, replace=False).tolist())
    ref_tau = ochi.chi_rows_pair(p.psi, p.eps, p.n_occ, p.tau, rows, p.n, p.lattice, idx, None)
    return p, idx, mats, rows, ref_tau


@pytest.mark.parametrize("prec", ["fp32", "f16x3"])
def test_pw_chi0_36cube_rows(ctx, g36, prec):
    """36^3 (the cluster row pass: four CTAs per row, two expanded rows each) on
    sampled G rows with every band, against the pair sum (Eq. CHI_g_it)."""
    p, idx, mats, rows, ref_tau = g36
    grid = gw.make_grid(p.n, p.lattice)
    pw = ogv.fft_index(ogv.g_set(p.n, p.n_b), p.n)      # the orbitals' plane waves: the lowest N_b
    n = len(p.tau)
    chi = torch.empty((n, p.n_chi, p.n_chi), dtype=torch.complex64, device="cuda")
    gw.chi0_omega_pw(ctx, grid, dev(p.psi, prec), p.eps, p.n_occ, p.mu, p.tau, np.eye(n), idx, pw, prec, chi)
    got = chi[:, rows, :].cpu().numpy().astype(np.complex128)
    err_tau = float(np.linalg.norm(got - ref_tau) / np.linalg.norm(ref_tau))
    ref = ochi.ct(ref_tau, mats["C"])
    gw.chi0_omega_pw(ctx, grid, dev(p.psi, prec), p.eps, p.n_occ, p.mu, p.tau, mats["C"], idx, pw, prec, chi)
    got = chi[:, rows, :].cpu().numpy().astype(np.complex128)
    err = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    print("36^3 plane-wave chi0 %s: chi0(i tau) %.2e, chi0(i omega) %.2e" % (prec, err_tau, err))
    assert err_tau < TOL[prec] and err < TOL[prec], (err_tau, err)


MEV = 3.674932e-5
SIG_TOL = {"fp64": 1e-10, "fp32": MEV, "f16x3": MEV, "bf16x3": MEV}


@pytest.mark.parametrize("prec", ["fp64", "fp32", "f16x3", "bf16x3"])
def test_pw_sigma_diag_matches_oracle(ctx, case, prec):
    """Sigma_nn(i omega) through the plane-wave G (gw_sigma_diag_pw) for the
    oracle chain's W~(tau), against the oracle's Sigma (Eqs. Sigma_occ,
    Sigma_rr, cos_sin_sigma), and equal to gw_sigma_diag's result."""
    name, p, s, chi_ref = case
    grid = gw.make_grid(p.n, p.lattice)
    pw = support(p)
    wt, _ = opipe.w_tau(p, s, chi_ref)
    su, so = opipe.sigma_from_w(p, s, wt)
    ref = osg.sigma_iw(su, so, s["C"], s["S"])
    out = gw.sigma_diag_pw(ctx, grid, dev(p.psi, prec), p.eps, p.n_occ, p.mu, p.bands, p.tau, p.omega, s["C"],
                           s["S"], dev(wt, prec), s["fft_index"], pw, prec)
    err = float(np.max(np.abs(out["sigma_iw"] - ref)))
    print("%s %s: plane-wave Sigma_nn(i omega) max error %.2e Ha" % (name, prec, err))
    assert err < SIG_TOL[prec], err
    assert np.max(np.abs(out["sigma_unocc"] - su)) < 1e-4 * np.max(np.abs(su)) + 1e-12
    assert np.max(np.abs(out["sigma_occ"] - so)) < 1e-4 * np.max(np.abs(so)) + 1e-12


@pytest.mark.parametrize("prec", ["fp32", "f16x3"])
def test_pw_sigma_36cube_sparse_w(ctx, g36, prec):
    """36^3 (cluster rows with three expanded functions): Sigma_nn for a W~ with a
    few nonzero (G, G') entries, every band in the sums, against the conventional
    route of the oracle."""
    p, idx, mats, rows, ref_tau = g36
    grid = gw.make_grid(p.n, p.lattice)
    pw = ogv.fft_index(ogv.g_set(p.n, p.n_b), p.n)
    n = len(p.tau)
    base = [(3, 3, -0.9, 0.25), (40, 40, -0.5, 0.6), (3, 40, 0.1 + 0.05j, 0.4), (40, 3, 0.1 - 0.05j, 0.4),
            (900, 900, -0.3, 1.1)]
    entries = [(a, b, p.volume * c * np.exp(-om * p.tau)) for (a, b, c, om) in base]
    w = torch.zeros((n, p.n_chi, p.n_chi), dtype=torch.complex64, device="cuda")
    for (a, b, v) in entries:
        for j in range(n):
            w[j, a, b] = complex(v[j])
    su, so = osg.sigma_pair_sparse(p.psi, p.eps, p.n_occ, p.mu, p.tau, entries, p.n, p.lattice, idx, p.bands)
    ref = osg.sigma_iw(su, so, mats["C"], mats["S"])
    out = gw.sigma_diag_pw(ctx, grid, dev(p.psi, prec), p.eps, p.n_occ, p.mu, p.bands, p.tau, p.omega, mats["C"],
                           mats["S"], w, idx, pw, prec)
    err = float(np.max(np.abs(out["sigma_iw"] - ref)))
    print("36^3 plane-wave Sigma_nn %s (sparse W~): max error %.2e Ha" % (prec, err))
    assert err < MEV and err < 1e-4 * np.max(np.abs(ref)), err
