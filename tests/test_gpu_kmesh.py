"""chi0 on a Gamma-centred k mesh (gw_chi0_omega_kmesh) against the k-mesh
oracle: the stripe route of Sec. II.A (Eqs. FFT_G1, FFT_G2), pinned to the
Gamma-point chi of the supercell in tests/test_oracle_kmesh.py, followed by
the cosine transform (Eq. CTX)."""
import numpy as np
import pytest

from oracle import chi as ochi
from oracle import grids as ogrids
from oracle import gvec as ogv
from oracle import kmesh as okm
from paper_1607_02859_gb300 import gw, inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
TOL = {"fp64": 1e-12, "fp32": 1e-6, "f16x3": 5e-6}


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


def reference(p, gv, C):
    per_tau = np.array([okm.chi_q_tau(p.psi_k, p.eps_k, p.n_occ, p.mu, t, p.n, p.nk, p.lattice, gv) for t in p.tau])
    return np.stack([ochi.ct(per_tau[:, q], C) for q in range(p.n_k)])        # [N_q][n][n_chi][n_chi]


CASES = {
    "6^3_k2x2x2": dict(n=(6, 6, 6), a=(6.0, 6.5, 7.0), nk=(2, 2, 2), n_occ=4, n_unocc=20, n_tau=4, seed=61, n_chi=None),
    "4^3_k3x3x3_partial": dict(n=(4, 4, 4), a=(5.0, 5.5, 6.0), nk=(3, 3, 3), n_occ=3, n_unocc=13, n_tau=4, seed=62,
                               n_chi=40),
    # the largest mesh the library takes: 64 k points (16^3 supercell)
    "4^3_k4x4x4_max": dict(n=(4, 4, 4), a=(5.0, 5.5, 6.0), nk=(4, 4, 4), n_occ=2, n_unocc=10, n_tau=4, seed=66,
                           n_chi=None),
}


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
    kw = dict(CASES[request.param])
    p = inputs.kmesh_problem(**kw)
    gv = ogv.g_set(p.n, p.n_chi)
    mats = ogrids.transform_matrices(p.tau, p.omega, p.x_min, p.x_max, p.n_x, p.ridge)
    return request.param, p, gv, mats, reference(p, gv, mats["C"])


@pytest.mark.parametrize("prec", ["fp32", "f16x3", "fp64"])
def test_chi0_kmesh(ctx, case, prec):
    name, p, gv, mats, ref = case
    grid = gw.make_grid(p.n, p.lattice)
    dt = gw.cdtype(prec)
    psi = torch.from_numpy(np.ascontiguousarray(p.psi_k)).to("cuda", dtype=dt)
    out = torch.zeros((p.n_k, len(p.tau), p.n_chi, p.n_chi), dtype=dt, device="cuda")
    gw.chi0_omega_kmesh(ctx, grid, p.nk, psi, p.eps_k, p.n_occ, p.mu, p.tau, mats["C"], gv, prec, out)
    got = out.cpu().numpy().astype(np.complex128)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    per_q = [np.linalg.norm(got[q] - ref[q]) / np.linalg.norm(ref[q]) for q in range(p.n_k)]
    print("%s %s: %.2e (worst q %.2e)" % (name, prec, err, max(per_q)))
    assert err < TOL[prec] and max(per_q) < 3 * TOL[prec]


def test_chi0_kmesh_12cube_k4x4x4(ctx):
    """A 12^3 cell on a 4 x 4 x 4 mesh (the meshes of the batched configuration):
    64 k points and a 48^3 supercell, rows of 110 592 points through the
    two-pass row transform; sampled q and G rows against the stripe oracle."""
    p = inputs.kmesh_problem(n=(12, 12, 12), a=(10.26, 10.26, 10.26), nk=(4, 4, 4), n_occ=2, n_unocc=10, n_tau=2,
                             seed=67, n_chi=60)
    gv = ogv.g_set(p.n, p.n_chi)
    mats = ogrids.transform_matrices(p.tau, p.omega, p.x_min, p.x_max, p.n_x, p.ridge)
    qs, rows = [0, 21, 63], [0, 7, 33, 59]
    ref_t = []
    for t in p.tau:
        go, gu = okm.green_stripe(p.psi_k, p.eps_k, p.n_occ, p.mu, t, p.n, p.nk)
        ref_t.append(okm.chi_q_rows(-2.0 * go * gu.conj(), p.n, p.nk, p.lattice, gv, qs, rows))
        del go, gu
    ref_t = np.array(ref_t)                                                    # [tau][q][rows][n_chi]
    ref = np.einsum("kj,jqrg->qkrg", mats["C"], ref_t)                         # [q][omega][rows][n_chi]
    grid = gw.make_grid(p.n, p.lattice)
    for prec in ("fp32", "f16x3"):
        dt = gw.cdtype(prec)
        psi = torch.from_numpy(np.ascontiguousarray(p.psi_k)).to("cuda", dtype=dt)
        out = torch.zeros((p.n_k, len(p.tau), p.n_chi, p.n_chi), dtype=dt, device="cuda")
        gw.chi0_omega_kmesh(ctx, grid, p.nk, psi, p.eps_k, p.n_occ, p.mu, p.tau, mats["C"], gv, prec, out)
        got = out[qs][:, :, rows, :].cpu().numpy().astype(np.complex128)
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        print("12^3 on 4x4x4 (48^3 supercell) %s: sampled rows %.2e" % (prec, err))
        assert err < TOL[prec], err
        del psi, out
        torch.cuda.empty_cache()


def test_kmesh_argument_checks(ctx, case):
    name, p, gv, mats, ref = case
    grid = gw.make_grid(p.n, p.lattice)
    psi = torch.from_numpy(np.ascontiguousarray(p.psi_k)).to("cuda", dtype=torch.complex64)
    out = torch.zeros((p.n_k, len(p.tau), p.n_chi, p.n_chi), dtype=torch.complex64, device="cuda")
    with pytest.raises(gw.GwError):       # a supercell grid the library does not compile (6 x 5 = 30)
        gw.chi0_omega_kmesh(ctx, grid, (1, 1, 5), psi, p.eps_k, p.n_occ, p.mu, p.tau, mats["C"], gv, "fp32", out)
    with pytest.raises(gw.GwError):       # mu outside a gap
        gw.chi0_omega_kmesh(ctx, grid, p.nk, psi, p.eps_k, p.n_occ, 5.0, p.tau, mats["C"], gv, "fp32", out)
    with pytest.raises(gw.GwError) as e:  # more than 64 k points (checked before any array is read)
        gw.chi0_omega_kmesh(ctx, grid, (5, 4, 4), psi, p.eps_k, p.n_occ, p.mu, p.tau, mats["C"], gv, "fp32", out)
    assert e.value.status == 2


@pytest.mark.parametrize("prec", ["fp32", "f16x3", "fp64"])
def test_sigma_kmesh(ctx, prec):
    from oracle import sigma as osg
    p = inputs.kmesh_problem(n=(6, 6, 6), a=(6.0, 6.5, 7.0), nk=(2, 2, 2), n_occ=4, n_unocc=20, n_tau=4, seed=63)
    gv = ogv.g_set(p.n, 60)
    mats = ogrids.transform_matrices(p.tau, p.omega, p.x_min, p.x_max, p.n_x, p.ridge)
    rng = np.random.default_rng(64)
    nc = len(gv)
    w = np.zeros((p.n_k, len(p.tau), nc, nc), dtype=np.complex128)
    for q in range(p.n_k):                     # Hermitian negative W~_q(tau) decaying with tau
        a = rng.standard_normal((nc, nc)) + 1j * rng.standard_normal((nc, nc))
        for j, t in enumerate(p.tau):
            w[q, j] = -0.02 * p.volume * (a @ a.conj().T) / nc * np.exp(-0.7 * t)
    bands = [(3, 0), (4, 1), (2, 5), (5, 7)]
    su = np.zeros((len(bands), len(p.tau)))
    so = np.zeros_like(su)
    for j, t in enumerate(p.tau):
        ws = okm.w_stripe(w[:, j], p.n, p.nk, p.lattice, gv)
        su[:, j], so[:, j] = okm.sigma_k_tau(p.psi_k, p.eps_k, p.n_occ, p.mu, t, ws, p.n, p.nk, p.lattice, bands)
    ref = osg.sigma_iw(su, so, mats["C"], mats["S"])
    dt = gw.cdtype(prec)
    grid = gw.make_grid(p.n, p.lattice)
    psi = torch.from_numpy(np.ascontiguousarray(p.psi_k)).to("cuda", dtype=dt)
    w_d = torch.from_numpy(w).to("cuda", dtype=dt)
    out = gw.sigma_diag_kmesh(ctx, grid, p.nk, psi, p.eps_k, p.n_occ, p.mu, bands, p.tau, p.omega, mats["C"],
                              mats["S"], w_d, gv, prec)
    err = np.max(np.abs(out["sigma_iw"] - ref))
    scale = np.max(np.abs(ref))
    print("sigma k mesh %s: max |dSigma| %.2e Ha (max |Sigma| %.2e)" % (prec, err, scale))
    # the bars of the Gamma-point Sigma tests: FP64 to rounding, the others within 1 meV and 1e-4 relative
    assert np.max(np.abs(out["sigma_unocc"] - su)) < (1e-11 if prec == "fp64" else 1e-4) * np.max(np.abs(su))
    assert err < (1e-11 * scale if prec == "fp64" else min(1e-4 * scale, 3.674932e-5))


@pytest.mark.parametrize("prec", ["fp32", "f16x3"])
def test_kmesh_chain_to_sigma(ctx, prec):
    """chi0_q -> W~_q (gw_screen_W per q on the supercell G triples q + nk g) ->
    W~_q(tau) -> Sigma_nk, against the same chain in the oracle; Sigma within 1 meV."""
    from oracle import screen as osc
    from oracle import sigma as osg
    p = inputs.kmesh_problem(n=(6, 6, 6), a=(6.0, 6.5, 7.0), nk=(2, 2, 2), n_occ=4, n_unocc=20, n_tau=4, seed=65)
    gv = ogv.g_set(p.n, 60)
    nc = len(gv)
    mats = ogrids.transform_matrices(p.tau, p.omega, p.x_min, p.x_max, p.n_x, p.ridge)
    ns = tuple(np.asarray(p.n) * np.asarray(p.nk))
    lat_s = p.lattice * np.asarray(p.nk)[:, None]
    gs_all = okm.supercell_gvecs(gv, p.nk)
    bands = [(3, 0), (4, 6), (2, 3)]
    # oracle chain
    chi_w = reference(p, gv, mats["C"])                                   # [N_q][n][nc][nc]
    w_tau = np.empty_like(chi_w)
    for q in range(p.n_k):
        vh = ogv.v_sqrt(gs_all[q * nc:(q + 1) * nc], lat_s)
        w_tau[q] = osc.inverse_ct(osc.screen(chi_w[q], vh), mats["Cinv"])
    su = np.zeros((len(bands), len(p.tau)))
    so = np.zeros_like(su)
    for j, t in enumerate(p.tau):
        ws = okm.w_stripe(w_tau[:, j], p.n, p.nk, p.lattice, gv)
        su[:, j], so[:, j] = okm.sigma_k_tau(p.psi_k, p.eps_k, p.n_occ, p.mu, t, ws, p.n, p.nk, p.lattice, bands)
    ref = osg.sigma_iw(su, so, mats["C"], mats["S"])
    # GPU chain
    dt = gw.cdtype(prec)
    grid = gw.make_grid(p.n, p.lattice)
    grid_s = gw.make_grid(ns, lat_s)
    psi = torch.from_numpy(np.ascontiguousarray(p.psi_k)).to("cuda", dtype=dt)
    chi = torch.empty((p.n_k, len(p.tau), nc, nc), dtype=dt, device="cuda")
    gw.chi0_omega_kmesh(ctx, grid, p.nk, psi, p.eps_k, p.n_occ, p.mu, p.tau, mats["C"], gv, prec, chi)
    wt = torch.empty_like(chi)
    for q in range(p.n_k):
        gw.screen_W(ctx, grid_s, gs_all[q * nc:(q + 1) * nc], prec, chi[q], chi[q], resid=False)
        gw.tau_to_omega(ctx, gw.CT, mats["Cinv"], chi[q], wt[q], prec)
    out = gw.sigma_diag_kmesh(ctx, grid, p.nk, psi, p.eps_k, p.n_occ, p.mu, bands, p.tau, p.omega, mats["C"],
                              mats["S"], wt, gv, prec)
    err = np.max(np.abs(out["sigma_iw"] - ref))
    print("k-mesh chain %s: max |dSigma| %.2e Ha (max |Sigma| %.2e)" % (prec, err, np.max(np.abs(ref))))
    assert err < 3.674932e-5
