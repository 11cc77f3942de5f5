"""Full-size checks at the 24^3 workload (16+1008 bands, 16 tau/omega on the
optimised grids, chi0 13824 x 13824) in the launch configuration bench.py times
for it, for the FP32 CUDA-core path and the fp16 x 3 tensor-core path.

The oracle cannot run the whole chain at this size, so:
  * chi0(i tau) and chi0(i omega) are checked on sampled rows G (all G', all
    tau / omega) against the Adler-Wiser pair sum (Eq. CHI_g_it), followed by
    the cosine transform (Eq. CTX) for i omega;
  * the screening (Eqs. die, W_correlated) runs on seeded chi0-shaped
    matrices of the full size N_chi = 13824, against the oracle's dense solve;
  * Sigma_nn(i omega) is checked for a synthetic W~ with a few nonzero
    entries, against the pair route restricted to those entries.
Each test holds ~50 GB of device memory at most."""
import os

import numpy as np
import pytest

from oracle import chi as ochi
from oracle import grids as ogrids
from oracle import gvec as ogv
from oracle import screen as osc
from oracle import sigma as osg
from paper_1607_02859_gb300 import gw, inputs

pytestmark = pytest.mark.gpu
MEV = 3.674932e-5
torch = pytest.importorskip("torch")
# relative Frobenius error of chi0(i omega) and chi0(i tau): the FP32 path meets the 1e-6 bar; the
# fp16 x 3 path adds the truncating FP32 accumulation of the tensor cores, about (3 products x 8 K16
# steps per 128-wide accumulation block) x 2^-24 = 1.4e-6 relative, and 2^-22 from the dropped lo x lo
# products: 3e-6 at any number of bands (blocks are summed in round-to-nearest FP32)
CHI_TOL = {"fp32": 1e-6, "f16x3": 3e-6}
CHI_TAU_TOL = {"fp32": 1e-6, "f16x3": 3e-6}
W_TOL = {"fp32": 2e-5, "f16x3": 5e-5}            # relative Frobenius of W~ against the FP64 solve
WORKERS = os.cpu_count()


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    if not os.path.exists(gw.LIB_PATH):
        from paper_1607_02859_gb300 import build
        build.build()
    c = gw.Context(0)
    yield c
    c.close()


def optimised(p):
    """The workload on the oracle's optimised (MP2 minimax) grids, weights without ridge."""
    g = ogrids.mp2_grids(len(p.tau), p.x_min, p.x_max)
    return inputs.on_grids(p, g["tau"], g["omega"], 0.0)


def transform_report(mats, ref_tau, ref_w):
    n = mats["C"].shape[0]
    tn2 = np.array([np.linalg.norm(ref_tau[j]) ** 2 for j in range(n)])
    amp = np.sqrt((mats["C"] ** 2 * tn2[None, :]).sum()) / np.linalg.norm(ref_w)
    return ("amplification A %.2f, max_k sum_j |C_kj| %.1f, cond(S) %.2e, fit error cos %.1e sin %.1e"
            % (amp, np.abs(mats["C"]).sum(1).max(), np.linalg.cond(mats["S"]), mats["fit_err_cos"],
               mats["fit_err_sin"]))


def chi_rows_check(ctx, p, idx, mats, prec, rows, ref_tau):
    """chi0(i tau) (identity transform) and chi0(i omega) on sampled rows against the pair sum."""
    grid = gw.make_grid(p.n, p.lattice)
    psi = torch.from_numpy(p.psi).to("cuda", dtype=torch.complex64)
    n = len(p.tau)
    ref = ochi.ct(ref_tau, mats["C"])
    chi = torch.empty((n, p.n_chi, p.n_chi), dtype=torch.complex64, device="cuda")
    gw.chi0_omega(ctx, grid, psi, p.eps, p.n_occ, p.mu, p.tau, np.eye(n), idx, prec, chi)
    got = chi[:, rows, :].cpu().numpy().astype(np.complex128)
    err_tau = np.linalg.norm(got - ref_tau) / np.linalg.norm(ref_tau)
    gw.chi0_omega(ctx, grid, psi, p.eps, p.n_occ, p.mu, p.tau, mats["C"], idx, prec, chi)
    got = chi[:, rows, :].cpu().numpy().astype(np.complex128)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    per = [float(np.linalg.norm(got[k] - ref[k]) / np.linalg.norm(ref[k])) for k in range(n)]
    cols = chi[:, :, rows].cpu().numpy().astype(np.complex128)
    herm = np.linalg.norm(np.conj(np.transpose(cols, (0, 2, 1))) - got) / np.linalg.norm(got)
    print("%s %s: chi0(i tau) %.3e, chi0(i omega) %.3e (per omega %s), Hermiticity %.1e; %s"
          % (p.name, prec, err_tau, err, " ".join("%.1e" % x for x in per), herm,
             transform_report(mats, ref_tau, ref)))
    del chi, psi
    torch.cuda.empty_cache()
    return err_tau, err, herm


def scaled_screening_input(n_chi, vhalf, strengths, seed):
    """inputs.screening_chi scaled so that the largest |eigenvalue| of
    chi~ = v^1/2 chi v^1/2 is each given strength (eps~ spectrum in [1, 1 + s])."""
    chi = inputs.screening_chi(n_chi, n_w=len(strengths), seed=seed)
    rng = np.random.default_rng(seed + 1)
    for w, s in enumerate(strengths):
        x = rng.standard_normal(n_chi) + 1j * rng.standard_normal(n_chi)
        lam = 1.0
        for _ in range(40):                       # power iteration on the NSD chi~
            y = vhalf * (chi[w] @ (vhalf * x))
            lam = np.linalg.norm(y) / np.linalg.norm(x)
            x = y / np.linalg.norm(y)
        chi[w] *= s / lam
    return chi


def screen_check(ctx, grid, gv, chi_h, w_ref, prec, refine=0):
    chi = torch.from_numpy(chi_h).to("cuda", dtype=torch.complex64)
    w = torch.empty_like(chi)
    res = gw.screen_W(ctx, grid, gv, prec, chi, w, resid=True, refine=refine)
    got = w.cpu().numpy().astype(np.complex128)
    errs = [float(np.linalg.norm(got[k] - w_ref[k]) / np.linalg.norm(w_ref[k])) for k in range(len(w_ref))]
    del chi, w
    torch.cuda.empty_cache()
    return errs, res


@pytest.fixture(scope="module")
def si8():
    p = optimised(inputs.si8())
    gv = ogv.g_set(p.n, p.n_chi)
    idx = ogv.fft_index(gv, p.n)
    mats = ogrids.transform_matrices(p.tau, p.omega, p.x_min, p.x_max, p.n_x, p.ridge)
    return p, gv, idx, mats


@pytest.fixture(scope="module")
def si8_rows(si8):
    p, gv, idx, mats = si8
    # rows drawn uniformly: the ratio of the sampled error and signal norms
    # estimates the relative Frobenius error of the whole [N][N_chi][N_chi]
    rows = sorted(np.random.default_rng(12).choice(p.n_chi, 24, replace=False).tolist())
    return rows, ochi.chi_rows_pair(p.psi, p.eps, p.n_occ, p.tau, rows, p.n, p.lattice, idx, WORKERS)


@pytest.mark.parametrize("prec", ["fp32", "f16x3"])
def test_si8_chi0_rows(ctx, si8, si8_rows, prec):
    p, gv, idx, mats = si8
    rows, ref_tau = si8_rows
    err_tau, err, herm = chi_rows_check(ctx, p, idx, mats, prec, rows, ref_tau)
    assert err_tau < CHI_TAU_TOL[prec], err_tau
    assert err < CHI_TOL[prec], err
    assert herm < CHI_TOL[prec], herm


@pytest.fixture(scope="module")
def si8_screen(si8):
    p, gv, idx, mats = si8
    vh = ogv.v_sqrt(gv, p.lattice)
    chi = scaled_screening_input(p.n_chi, vh, [8.0, 0.05], seed=61)
    return chi, np.stack([osc.screen_one(c, vh) for c in chi])


@pytest.mark.parametrize("prec", ["fp32", "f16x3"])
def test_si8_screen_vs_oracle(ctx, si8, si8_screen, prec):
    """W~ at N_chi = 13824 (27 screening panels of 512) against the FP64 dense solve, at a
    strongly screened (|chi~| = 8) and a weakly screened (|chi~| = 0.05) frequency."""
    p, gv, idx, mats = si8
    chi, w_ref = si8_screen
    errs, res = screen_check(ctx, gw.make_grid(p.n, p.lattice), gv, chi, w_ref, prec)
    print("si8 screening %s: W~ relative error %s, residual probe %s" % (prec, errs, res))
    assert max(errs) < W_TOL[prec], errs


def test_si8_screen_refined(ctx, si8, si8_screen):
    """One refinement step of the f16x3 solve at N_chi = 13824 (the residual
    product as exact fp16 slice products on the tensor cores)."""
    p, gv, idx, mats = si8
    chi, w_ref = si8_screen
    errs, res = screen_check(ctx, gw.make_grid(p.n, p.lattice), gv, chi, w_ref, "f16x3", refine=1)
    print("si8 screening f16x3 + 1 refinement step: W~ relative error %s, residual probe %s" % (errs, res))
    # one step squares the solve's ~5e-6 error and the 30-bit residual bounds X to ~1e-9: what is
    # left is W~'s FP32 storage (~6e-8); 2e-7 separates that from a residual product gone wrong
    assert max(errs) < 2e-7, errs


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
    su, so = osg.sigma_pair_sparse(p.psi, p.eps, p.n_occ, p.mu, p.tau, entries, p.n, p.lattice, idx, p.bands,
                                   WORKERS)
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
