"""The 36^3 grid of the 64-atom cell (rows of 46656 points: too long for
shared memory, so the row transform takes two passes through HBM), at a band
count, G set and tau count the oracle checks in seconds: 16+240 bands, 2048 G,
4 tau.  chi0(G,G',i tau) on sampled rows against the pair sum (Eq. CHI_g_it),
the public row transform in both directions against numpy's FFT, and Sigma for
a sparse W~ against the conventional route."""
import numpy as np
import pytest

from oracle import chi as ochi
from oracle import grids as ogrids
from oracle import gvec as ogv
from oracle import sigma as osg
from paper_1607_02859_gb300 import gw, inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
MEV = 3.674932e-5
TAU_TOL = {"fp32": 1e-6, "f16x3": 5e-6}


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
def g36():
    p = inputs.make_problem((36, 36, 36), 20.52, 16, 240, (-0.5, 0.0), (0.03, 5.0), 0.015, 4, 31,
                            n_bands_sigma=4, n_chi=2048, pin_edges=True, name="g36_reduced")
    gv = ogv.g_set(p.n, p.n_chi)
    idx = ogv.fft_index(gv, p.n)
    mats = ogrids.transform_matrices(p.tau, p.omega, p.x_min, p.x_max, p.n_x, p.ridge)
    return p, gv, idx, mats


@pytest.mark.parametrize("prec", ["fp32", "f16x3"])
def test_chi0_tau_rows(ctx, g36, prec):
    p, gv, idx, mats = g36
    grid = gw.make_grid(p.n, p.lattice)
    psi = torch.from_numpy(p.psi).to("cuda", dtype=torch.complex64)
    n = len(p.tau)
    chi = torch.empty((n, p.n_chi, p.n_chi), dtype=torch.complex64, device="cuda")
    gw.chi0_omega(ctx, grid, psi, p.eps, p.n_occ, p.mu, p.tau, np.eye(n), idx, prec, chi)
    rows = sorted(np.random.default_rng(36).choice(p.n_chi, 12, replace=False).tolist())
    ref = ochi.chi_rows_pair(p.psi, p.eps, p.n_occ, p.tau, rows, p.n, p.lattice, idx)
    got = chi[:, rows, :].cpu().numpy().astype(np.complex128)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    print("36^3 chi0(i tau) %s: %.2e" % (prec, err))
    assert err < TAU_TOL[prec]


@pytest.mark.parametrize("n,n_chi,prec", [(36, 2048, "fp32"), (36, 8192, "fp32"), (36, 2048, "fp64"),
                                          (48, 4096, "fp32")])
@pytest.mark.parametrize("direction", [1, -1])
def test_row_transform_large_rows(ctx, n, n_chi, prec, direction):
    """Rows longer than one CTA's shared memory: 36^3 and 48^3 FP32 rows are
    split over a thread-block cluster, FP64 36^3 rows take two passes."""
    shape = (n, n, n)
    lattice = np.eye(3) * (n * 10.26 / 12)
    volume = float(np.linalg.det(lattice))
    idx = ogv.fft_index(ogv.g_set(shape, n_chi), shape)
    grid = gw.make_grid(shape, lattice)
    rng = np.random.default_rng(7 + direction + n + n_chi)
    rows = 5
    nr = n ** 3
    cdt = torch.complex64 if prec == "fp32" else torch.complex128
    if direction > 0:
        x = rng.standard_normal((rows, nr)) + 1j * rng.standard_normal((rows, nr))
        # X(r,G') = sum_R' x(r,R') exp(+i G'.R')  (Eq. FFTX1)
        ref = np.stack([nr * np.fft.ifftn(v.reshape(shape)).reshape(-1)[idx] for v in x])
        out = torch.empty((rows, n_chi), dtype=cdt, device="cuda")
    else:
        x = rng.standard_normal((rows, n_chi)) + 1j * rng.standard_normal((rows, n_chi))
        # W(r,R') = (1/Omega) sum_G' W(r,G') exp(-i G'.R')  (second step of Eq. FFTW)
        ref = []
        for v in x:
            y = np.zeros(nr, dtype=np.complex128)
            y[idx] = v
            ref.append(np.fft.fftn(y.reshape(shape)).reshape(-1) / volume)
        ref = np.stack(ref)
        out = torch.empty((rows, nr), dtype=cdt, device="cuda")
    inp = torch.from_numpy(x).to("cuda", dtype=cdt)
    gw.rr_to_GG_fft(ctx, grid, direction, 1, idx, prec, 0, rows, inp, out)
    got = out.cpu().numpy().astype(np.complex128)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err < (1e-6 if prec == "fp32" else 1e-13), err


def test_sigma_sparse_w(ctx, g36):
    p, gv, idx, mats = g36
    grid = gw.make_grid(p.n, p.lattice)
    psi = torch.from_numpy(p.psi).to("cuda", dtype=torch.complex64)
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
    out = gw.sigma_diag(ctx, grid, psi, p.eps, p.n_occ, p.mu, p.bands, p.tau, p.omega, mats["C"], mats["S"], w, idx,
                        "f16x3")
    err = np.max(np.abs(out["sigma_iw"] - ref))
    assert err < MEV and err < 1e-4 * np.max(np.abs(ref)), err
