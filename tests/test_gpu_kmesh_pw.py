"""chi0 on a Gamma-centred k mesh with G_k through its plane-wave form
(gw_chi0_omega_kmesh_pw) against the oracle of that form: coefficients of the
cell-periodic parts, G_k(g, k+g') (Eqs. G1_unocc_k, G1_occ_k), the stripe by
Eqs. FFT_G1 and FFT_G2 (pinned to the real-space stripe in
tests/test_oracle_kmesh.py), chi_q and the cosine transform (Eq. CTX).  Also
its refusals: orbitals outside the plane-wave set, and a supercell whose two
expanded rows do not fit a thread-block cluster."""
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


def support(p):
    """Cell FFT positions of the plane waves in any exp(-i k.r) psi_nk (test side)."""
    c = okm.pw_coefficients_k(p.psi_k, p.n, p.nk)
    w = np.sum(np.abs(c) ** 2, axis=(0, 1))
    return np.flatnonzero(w > 1e-20 * w.max()).astype(np.int32)


CASES = {
    "6^3_k2x2x2": dict(n=(6, 6, 6), a=(6.0, 6.5, 7.0), nk=(2, 2, 2), n_occ=4, n_unocc=20, n_tau=4, seed=71, n_chi=None),
    "4^3_k3x3x3_partial": dict(n=(4, 4, 4), a=(5.0, 5.5, 6.0), nk=(3, 3, 3), n_occ=3, n_unocc=13, n_tau=4, seed=72,
                               n_chi=40),
    "4^3_k4x4x4": dict(n=(4, 4, 4), a=(5.0, 5.5, 6.0), nk=(4, 4, 4), n_occ=2, n_unocc=10, n_tau=4, seed=73,
                       n_chi=None),
}


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
    p = inputs.kmesh_problem(**CASES[request.param])
    gv = ogv.g_set(p.n, p.n_chi)
    pw = support(p)
    mats = ogrids.transform_matrices(p.tau, p.omega, p.x_min, p.x_max, p.n_x, p.ridge)
    per_tau = np.array([okm.chi_q_tau_pw(p.psi_k, p.eps_k, p.n_occ, p.mu, t, p.n, p.nk, p.lattice, gv, pw_index=pw)
                        for t in p.tau])
    ref = np.stack([ochi.ct(per_tau[:, q], mats["C"]) for q in range(p.n_k)])
    return request.param, p, gv, pw, mats, ref


def run(ctx, p, gv, pw, C, prec, psi_k=None):
    grid = gw.make_grid(p.n, p.lattice)
    dt = gw.cdtype(prec)
    psi = torch.from_numpy(np.ascontiguousarray(p.psi_k if psi_k is None else psi_k)).to("cuda", dtype=dt)
    out = torch.zeros((p.n_k, len(p.tau), len(gv), len(gv)), dtype=dt, device="cuda")
    gw.chi0_omega_kmesh_pw(ctx, grid, p.nk, psi, p.eps_k, p.n_occ, p.mu, p.tau, C, gv, pw, prec, out)
    return out.cpu().numpy().astype(np.complex128)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "f16x3"])
def test_chi0_kmesh_pw_matches_oracle(ctx, case, prec):
    name, p, gv, pw, mats, ref = case
    got = run(ctx, p, gv, pw, mats["C"], prec)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    per_q = [np.linalg.norm(got[q] - ref[q]) / np.linalg.norm(ref[q]) for q in range(p.n_k)]
    print("%s %s (n_pw %d of %d): %.2e (worst q %.2e)" % (name, prec, len(pw), p.n_r, err, max(per_q)))
    assert err < TOL[prec] and max(per_q) < 3 * TOL[prec]


def test_chi0_kmesh_pw_rejects_orbitals_outside_the_set(ctx):
    p = inputs.kmesh_problem(**CASES["6^3_k2x2x2"])
    gv = ogv.g_set(p.n, p.n_chi)
    pw = support(p)
    mats = ogrids.transform_matrices(p.tau, p.omega, p.x_min, p.x_max, p.n_x, p.ridge)
    outside = np.setdiff1d(np.arange(p.n_r), pw)[0]
    idx3 = np.array(np.unravel_index(np.arange(p.n_r), p.n)).T
    o3 = np.array(np.unravel_index(outside, p.n))
    psi_k = p.psi_k.copy()
    # band 5 at k index 3 gains a component on a plane wave outside the set
    psi_k[3, 5] = psi_k[3, 5] + 1e-2 * np.abs(psi_k[3, 5]).max() * np.exp(2j * np.pi * (idx3 @ (o3 / np.array(p.n))))
    with pytest.raises(gw.GwError) as e:
        run(ctx, p, gv, pw, mats["C"], "fp64", psi_k=psi_k)
    assert e.value.status == 1 and "band 5" in e.value.message


def test_chi0_kmesh_pw_refuses_supercells_beyond_a_cluster(ctx):
    """A 12^3 cell on a 4 x 4 x 4 mesh: rows of the 48^3 supercell do not fit."""
    p = inputs.kmesh_problem(n=(12, 12, 12), a=(10.26, 10.26, 10.26), nk=(4, 4, 4), n_occ=2, n_unocc=10, n_tau=2,
                             seed=74, n_chi=60)
    gv = ogv.g_set(p.n, p.n_chi)
    pw = ogv.fft_index(ogv.g_set(p.n, p.n_b), p.n)
    mats = ogrids.transform_matrices(p.tau, p.omega, p.x_min, p.x_max, p.n_x, p.ridge)
    with pytest.raises(gw.GwError) as e:
        run(ctx, p, gv, pw, mats["C"], "fp32")
    assert e.value.status == 7
