"""Full-size checks at the benchmark workload (24^3 grid, 16+1008 bands, 16 tau,
chi0 13824 x 13824) in the launch configuration bench.py times, for the FP32
CUDA-core path and the fp16 x 3 tensor-core path.

The oracle cannot run the whole chain at this size, so:
  * chi0(i tau) and chi0(i omega) are checked on sampled rows G (all G', all
    tau / omega) against the Adler-Wiser pair sum (Eq. CHI_g_it), followed by
    the cosine transform (Eq. CTX) for i omega;
  * the screening is checked through its residual |eps~ X - chi~| / |chi~|,
    a property that holds at any size;
  * Sigma_nn(i omega) is checked for a synthetic W~ with a few nonzero
    entries, against the pair route restricted to those entries.
Each test holds ~50 GB of device memory at most."""
import numpy as np
import pytest

from oracle import chi as ochi
from oracle import grids as ogrids
from oracle import gvec as ogv
from oracle import sigma as osg
from paper_1607_02859_gb300 import gw, inputs

pytestmark = pytest.mark.gpu
MEV = 3.674932e-5
torch = pytest.importorskip("torch")
CHI_TOL = {"fp32": 1e-6, "f16x3": 5e-6}


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
def si8():
    p = inputs.si8()
    gv = ogv.g_set(p.n, p.n_chi)
    idx = ogv.fft_index(gv, p.n)
    mats = ogrids.transform_matrices(p.tau, p.omega, p.x_min, p.x_max, p.n_x, p.ridge)
    return p, gv, idx, mats


@pytest.mark.parametrize("prec", ["fp32", "f16x3"])
def test_si8_chi0_rows_and_screening(ctx, si8, prec):
    p, gv, idx, mats = si8
    grid = gw.make_grid(p.n, p.lattice)
    psi = torch.from_numpy(p.psi).to("cuda", dtype=torch.complex64)
    n = len(p.tau)
    chi = torch.empty((n, p.n_chi, p.n_chi), dtype=torch.complex64, device="cuda")
    # rows drawn uniformly: the ratio of the sampled error and signal norms
    # estimates the relative Frobenius error of the whole [N][N_chi][N_chi]
    rows = sorted(np.random.default_rng(12).choice(p.n_chi, 24, replace=False).tolist())
    ref_tau = ochi.chi_rows_pair(p.psi, p.eps, p.n_occ, p.tau, rows, p.n, p.lattice, idx)
    ref = ochi.ct(ref_tau, mats["C"])

    # chi0(G,G',i tau): the same launch with the transform set to the identity
    gw.chi0_omega(ctx, grid, psi, p.eps, p.n_occ, p.mu, p.tau, np.eye(n), idx, prec, chi)
    got = chi[:, rows, :].cpu().numpy().astype(np.complex128)
    err_tau = np.linalg.norm(got - ref_tau) / np.linalg.norm(ref_tau)
    per_tau = [float(np.linalg.norm(got[j] - ref_tau[j]) / np.linalg.norm(ref_tau[j])) for j in range(n)]
    print("chi0(i tau) sampled-row relative error %.3e; per tau %s" % (err_tau, " ".join("%.1e" % x for x in per_tau)))
    assert err_tau < CHI_TOL[prec], (err_tau, per_tau)

    # chi0(i omega).  Independent relative errors e_j of the chi0(tau_j) reach
    # chi0(i omega) as sum_j C_kj e_j chi0(tau_j); with weights |C_kj| ~ 10^2 of
    # both signs the factor
    #     A = sqrt(sum_kj C_kj^2 |chi0(tau_j)|^2) / |chi0(i omega)|
    # is ~20 here, so FP32 rounding of chi0(tau) alone puts chi0(i omega) near
    # 1e-6.  The transform must add nothing beyond that propagation.
    gw.chi0_omega(ctx, grid, psi, p.eps, p.n_occ, p.mu, p.tau, mats["C"], idx, prec, chi)
    got = chi[:, rows, :].cpu().numpy().astype(np.complex128)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    per = [float(np.linalg.norm(got[k] - ref[k]) / np.linalg.norm(ref[k])) for k in range(n)]
    tn2 = np.array([np.linalg.norm(ref_tau[j]) ** 2 for j in range(n)])
    amp = np.sqrt((mats["C"] ** 2 * tn2[None, :]).sum()) / np.linalg.norm(ref)
    bound = max(CHI_TOL[prec], 2.0 * amp * max(per_tau))
    print("chi0(i omega) sampled-row relative error %.3e (amplification %.1f, bound %.2e); per omega %s"
          % (err, amp, bound, " ".join("%.1e" % x for x in per)))
    assert err < bound, (err, bound, per)
    # Hermiticity of the computed matrix on the sampled rows
    cols = chi[:, :, rows].cpu().numpy().astype(np.complex128)
    herm = np.linalg.norm(np.conj(np.transpose(cols, (0, 2, 1))) - got) / np.linalg.norm(got)
    assert herm < bound
    res = gw.screen_W(ctx, grid, gv, prec, chi, chi, resid=True)
    assert np.all(res < (1e-5 if prec == "fp32" else 2e-5)), res
    del chi
    torch.cuda.empty_cache()


@pytest.mark.parametrize("prec", ["fp32", "f16x3"])
def test_si8_sigma_sparse_w(ctx, si8, prec):
    p, gv, idx, mats = si8
    grid = gw.make_grid(p.n, p.lattice)
    psi = torch.from_numpy(p.psi).to("cuda", dtype=torch.complex64)
    n = len(p.tau)
    vol = p.volume
    # W~(G,G',tau) = sum_p -B_p exp(-Om_p tau) on a few (G, G') entries, Hermitian
    base = [(5, 5, -0.9, 0.25), (40, 40, -0.5, 0.6), (5, 40, 0.1 + 0.05j, 0.4), (40, 5, 0.1 - 0.05j, 0.4),
            (700, 700, -0.3, 1.1)]
    w = torch.zeros((n, p.n_chi, p.n_chi), dtype=torch.complex64, device="cuda")
    entries = [(a, b, vol * c * np.exp(-om * p.tau)) for (a, b, c, om) in base]
    for (a, b, v) in entries:
        for j in range(n):
            w[j, a, b] = complex(v[j])
    su, so = osg.sigma_pair_sparse(p.psi, p.eps, p.n_occ, p.mu, p.tau, entries, p.n, p.lattice, idx, p.bands)
    ref = osg.sigma_iw(su, so, mats["C"], mats["S"])
    out = gw.sigma_diag(ctx, grid, psi, p.eps, p.n_occ, p.mu, p.bands, p.tau, p.omega, mats["C"], mats["S"], w, idx,
                        prec)
    assert np.max(np.abs(out["sigma_unocc"] - su)) < 1e-4 * np.max(np.abs(su))
    assert np.max(np.abs(out["sigma_occ"] - so)) < 1e-4 * np.max(np.abs(so))
    err = np.max(np.abs(out["sigma_iw"] - ref))
    assert err < MEV, err
    assert err < 1e-4 * np.max(np.abs(ref))
    del w
    torch.cuda.empty_cache()
