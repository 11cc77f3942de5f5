"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these re-types an oracle formula: each compares the oracle with a
closed form, a brute-force loop written independently (Cartesian vectors, the
reciprocal lattice, pure-Python sums), an exact identity between two different
routes, or an invariant.  All run on the CPU in a few seconds.
"""
import itertools

import numpy as np
import pytest

from oracle import chi as ochi
from oracle import green as ogr
from oracle import grids as ogrids
from oracle import gvec as ogv
from oracle import pipeline as opipe
from oracle import screen as osc
from oracle import sigma as osg
from oracle import thiele as oth
from paper_1607_02859_gb300 import inputs


def _cart_r(n, lattice):
    """Cartesian grid points, r index = (i1*n2+i2)*n3+i3."""
    pts = []
    for i1, i2, i3 in itertools.product(range(n[0]), range(n[1]), range(n[2])):
        f = np.array([i1 / n[0], i2 / n[1], i3 / n[2]])
        pts.append(f @ lattice)
    return np.array(pts)


def _cart_g(g, lattice):
    # reciprocal vectors from the defining relation a_d . b_e = 2 pi delta
    a = np.asarray(lattice, dtype=float)
    b = np.zeros((3, 3))
    vol = np.dot(a[0], np.cross(a[1], a[2]))
    b[0] = 2 * np.pi * np.cross(a[1], a[2]) / vol
    b[1] = 2 * np.pi * np.cross(a[2], a[0]) / vol
    b[2] = 2 * np.pi * np.cross(a[0], a[1]) / vol
    return np.asarray(g, dtype=float) @ b


@pytest.fixture(scope="module")
def tiny_c():
    return inputs.tiny(seed=5)


@pytest.fixture(scope="module")
def tiny_r():
    return inputs.tiny(seed=6, n=(6, 4, 6), a=(6.0, 5.0, 6.5), n_occ=4, n_unocc=12, real=True)


# ---------------------------------------------------------------- inputs

def test_orbitals_orthonormal(tiny_c, tiny_r):
    for p in (tiny_c, tiny_r):
        dv = p.volume / p.n_r
        ov = dv * p.psi.conj() @ p.psi.T
        assert np.allclose(ov, np.eye(p.n_b), atol=1e-12)
    assert np.allclose(tiny_r.psi.imag, 0)


# ---------------------------------------------------------------- G set and index map

def test_fft_index_matches_numpy_fft():
    """The index map puts exp(+iG.r) where numpy's inverse FFT puts a delta."""
    n = (6, 4, 10)
    gv = ogv.g_set(n, 60)
    idx = ogv.fft_index(gv, n)
    pm = ogv.phase_matrix(gv, n, +1.0)
    for j in (0, 7, 31, 59):
        d = np.zeros(n, dtype=complex)
        d.reshape(-1)[idx[j]] = 1.0
        ref = np.fft.ifftn(d).reshape(-1) * np.prod(n)
        assert np.allclose(pm[j], ref, atol=1e-12)
    assert len(set(idx.tolist())) == len(idx)


def test_gset_is_the_sphere():
    n = (8, 8, 8)
    gv = ogv.g_set(n, 100)
    r2 = (gv ** 2).sum(1)
    assert np.all(np.diff(r2) >= 0)
    # every grid point not taken is at least as far out as the last one taken
    ax = [range(-(m // 2), m - m // 2) for m in n]
    allp = np.array(list(itertools.product(*ax)))
    taken = {tuple(x) for x in gv}
    rest = np.array([x for x in allp if tuple(x) not in taken])
    assert (rest ** 2).sum(1).min() >= r2.max()
    assert tuple(gv[0]) == (0, 0, 0)


def test_coulomb_sqrt_closed_form():
    lat = np.diag([6.0, 5.0, 6.5])
    gv = np.array([[0, 0, 0], [1, 0, 0], [0, -2, 1], [1, 1, 1]])
    v = ogv.v_sqrt(gv, lat)
    assert v[0] == 0.0
    for g, val in zip(gv[1:], v[1:]):
        gc = 2 * np.pi * np.array(g) / np.array([6.0, 5.0, 6.5])
        assert abs(val ** 2 - 4 * np.pi / gc.dot(gc)) < 1e-12


# ---------------------------------------------------------------- Green's functions

def test_green_completeness_at_tau0(tiny_c):
    """Bands span the lowest N_b plane waves, so G_occ(0)+G_unocc(0) is the projector
    (1/Omega) sum_p exp(iG_p.(r-r'))."""
    p = tiny_c
    g = ogr.green_occ(p.psi, p.eps, p.n_occ, p.mu, 0.0) + \
        ogr.green_unocc(p.psi, p.eps, p.n_occ, p.mu, 0.0)
    ax = [range(-(m // 2), m - m // 2) for m in p.n]
    pts = sorted(itertools.product(*ax), key=lambda t: (t[0] ** 2 + t[1] ** 2 + t[2] ** 2, t))
    basis = np.array(pts[:p.n_b])
    rc = _cart_r(p.n, p.lattice)
    gc = _cart_g(basis, p.lattice)
    ph = np.exp(1j * rc @ gc.T)                     # [N_r][N_b]
    proj = ph @ ph.conj().T / p.volume
    assert np.allclose(g, proj, atol=1e-12)


def test_green_brute_force_time_dependence(tiny_c):
    p = tiny_c
    tau = 0.7
    go = ogr.green_occ(p.psi, p.eps, p.n_occ, p.mu, tau)
    gu = ogr.green_unocc(p.psi, p.eps, p.n_occ, p.mu, tau)
    for (r, rp) in [(0, 5), (17, 17), (100, 3)]:
        so = 0j
        su = 0j
        for b in range(p.n_b):
            term = p.psi[b, r] * np.conj(p.psi[b, rp])
            if b < p.n_occ:
                so += term * np.exp(-abs(p.eps[b] - p.mu) * tau)   # occupied: eps < mu
            else:
                su += term * np.exp(-abs(p.eps[b] - p.mu) * tau)
        assert abs(go[r, rp] - so) < 1e-14
        assert abs(gu[r, rp] - su) < 1e-14
    assert np.allclose(go, go.conj().T)
    assert np.allclose(gu, gu.conj().T)


# ---------------------------------------------------------------- chi

def test_chi_brute_force_transform(tiny_c):
    """One chi(G,G',tau) element by explicit Cartesian sums over r and r'."""
    p = tiny_c
    gv = ogv.g_set(p.n, p.n_r)
    tau = 0.9
    go = ogr.green_occ(p.psi, p.eps, p.n_occ, p.mu, tau)
    gu = ogr.green_unocc(p.psi, p.eps, p.n_occ, p.mu, tau)
    xrr = ochi.chi_rr(go, gu)
    full = ochi.chi_gg(xrr, gv, p.n, p.lattice)
    rc = _cart_r(p.n, p.lattice)
    dv = p.volume / p.n_r
    for (j, jp) in [(0, 0), (3, 11), (40, 2), (100, 100)]:
        gj = _cart_g(gv[j], p.lattice)
        gjp = _cart_g(gv[jp], p.lattice)
        ref = 0j
        for r in range(p.n_r):
            # chi(r,r') = -2 G_occ(r,r') G_unocc(r',r), each by an explicit band sum
            row = np.zeros(p.n_r, dtype=complex)
            for b in range(p.n_occ):
                row += p.psi[b, r] * p.psi[b].conj() * np.exp((p.eps[b] - p.mu) * tau)
            rowu = np.zeros(p.n_r, dtype=complex)
            for b in range(p.n_occ, p.n_b):
                rowu += p.psi[b] * np.conj(p.psi[b, r]) * np.exp(-(p.eps[b] - p.mu) * tau)
            x = -2.0 * row * rowu
            ref += np.exp(-1j * gj @ rc[r]) * np.sum(x * np.exp(1j * rc @ gjp))
        ref *= dv * dv / p.volume
        assert abs(full[j, jp] - ref) < 1e-12 * max(1.0, abs(ref))


@pytest.mark.parametrize("which", ["complex", "real"])
def test_chi_gg_equals_pair_sum(which, tiny_c, tiny_r):
    """Exact time-domain identity: GG product in real space, transformed, equals the
    Adler-Wiser pair sum over (occ, unocc) (Eqs. chi_rr -> CHI_g_it)."""
    p = tiny_c if which == "complex" else tiny_r
    gv = ogv.g_set(p.n, p.n_r)
    m = ochi.pair_matrix_elements(p.psi, p.n_occ, gv, p.n, p.lattice)
    for tau in (0.05, 1.3, 11.0):
        go = ogr.green_occ(p.psi, p.eps, p.n_occ, p.mu, tau)
        gu = ogr.green_unocc(p.psi, p.eps, p.n_occ, p.mu, tau)
        a = ochi.chi_gg(ochi.chi_rr(go, gu), gv, p.n, p.lattice)
        b = ochi.chi_pair(p.psi, p.eps, p.n_occ, p.mu, tau, gv, p.n, p.lattice, m=m)
        assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(b)


def test_chi_invariants(tiny_c, tiny_r):
    """chi(G,G',tau) Hermitian and NSD; real orbitals give chi(G,G') = chi(-G,-G')^*;
    chi(i omega) NSD wherever the fitted kernel sum_j C_kj exp(-D tau_j) is positive."""
    for p in (tiny_c, tiny_r):
        s = opipe.setup(p)
        chi_w, chit = opipe.chi0_omega(p, s)
        for x in list(chit) + list(chi_w):
            assert np.allclose(x, x.conj().T, atol=1e-14 * np.abs(x).max())
        for x in chit:
            ev = np.linalg.eigvalsh(x)
            assert ev.max() <= 1e-12 * abs(ev.min())
        d = (p.eps[p.n_occ:, None] - p.eps[None, :p.n_occ]).ravel()
        kern = s["C"] @ np.exp(-np.outer(p.tau, d))
        assert kern.min() > 0
        for x in chi_w:
            ev = np.linalg.eigvalsh(x)
            assert ev.max() <= 1e-12 * abs(ev.min())
    p = tiny_r
    gv = ogv.g_set(p.n, p.n_r)
    s = opipe.setup(p)
    x = opipe.chi_tau(p, s, 1)
    pos = {tuple(g): i for i, g in enumerate(gv)}
    n = np.array(p.n)
    for j in range(0, p.n_r, 7):
        for jp in range(0, p.n_r, 5):
            mg = tuple(((-gv[j] + n // 2) % n) - n // 2)
            mgp = tuple(((-gv[jp] + n // 2) % n) - n // 2)
            assert abs(x[j, jp] - np.conj(x[pos[mg], pos[mgp]])) < 1e-13


# ---------------------------------------------------------------- CT / ST weights

def test_ct_st_approach_lorentzians_as_grid_refines():
    """The discrete CT/ST of exp(-x tau) approach 2x/(x^2+w^2) and 2w/(x^2+w^2)
    (the integrals named in Eqs. cos_error_function / sin_error_function)."""
    x_lo, x_hi = 0.05, 4.0
    errs = []
    for n in (6, 12, 24):
        tau = np.geomspace(0.1 / x_hi, 3.0 / x_lo, n)
        om = 1.0 / tau[::-1]
        m = ogrids.transform_matrices(tau, om, x_lo, x_hi, n_x=1500)
        x = np.geomspace(x_lo, x_hi, 333)            # off the fit's sample points
        e = np.exp(-np.outer(tau, x))
        lc = 2 * x[None, :] / (x[None, :] ** 2 + om[:, None] ** 2)
        ls = 2 * om[:, None] / (x[None, :] ** 2 + om[:, None] ** 2)
        ec = np.max(np.abs(m["C"] @ e - lc) / lc)
        es = np.max(np.abs(m["S"] @ e - ls) / ls)
        errs.append((ec, es))
        assert np.allclose(m["C"] @ m["Cinv"], np.eye(n), atol=1e-9)
    assert errs[2][0] < errs[1][0] < errs[0][0]
    assert errs[2][1] < errs[0][1]
    assert errs[2][0] < 1e-2 and errs[2][1] < 2e-2


# ---------------------------------------------------------------- screening

def test_screen_sherman_morrison():
    """chi = -alpha u u^H has the closed-form W~ = -alpha (v^1/2 u~)(v^1/2 u~)^H/(1+alpha|u~|^2)."""
    rng = np.random.default_rng(3)
    nchi = 30
    vh = rng.uniform(0.1, 2.0, nchi)
    vh[0] = 0.0
    u = rng.standard_normal(nchi) + 1j * rng.standard_normal(nchi)
    alpha = 0.7
    chi = -alpha * np.outer(u, u.conj())
    w = osc.screen_one(chi, vh)
    ut = vh * u
    ref = -alpha * np.outer(vh * ut, (vh * ut).conj()) / (1 + alpha * np.vdot(ut, ut).real)
    assert np.allclose(w, ref, atol=1e-13)


def test_screen_invariants(tiny_c):
    p = tiny_c
    s = opipe.setup(p)
    chi_w, _ = opipe.chi0_omega(p, s)
    for c in chi_w:
        ct = s["vhalf"][:, None] * c * s["vhalf"][None, :]
        ev = np.linalg.eigvalsh(np.eye(len(ct)) - ct)
        assert ev.min() >= 1 - 1e-12                 # eps~ >= 1
        w = osc.screen_one(c, s["vhalf"])
        assert np.allclose(w, w.conj().T, atol=1e-14)
        assert np.linalg.eigvalsh(w).max() <= 1e-12   # W~(i omega) NSD
        # residual of the Dyson solve
        x = w / np.where(np.outer(s["vhalf"], s["vhalf"]) == 0, 1, np.outer(s["vhalf"], s["vhalf"]))
        res = (np.eye(len(ct)) - ct) @ x - ct
        assert np.linalg.norm(res) <= 1e-12 * max(1, np.linalg.norm(ct))


def test_w_to_real_space_diagonal_and_round_trip(tiny_c):
    p = tiny_c
    gv = ogv.g_set(p.n, p.n_r)
    rng = np.random.default_rng(4)
    wdiag = rng.standard_normal(p.n_r)
    wr = osc.w_rr(np.diag(wdiag).astype(complex), gv, p.n, p.lattice)
    rc = _cart_r(p.n, p.lattice)
    gc = _cart_g(gv, p.lattice)
    for (r, rp) in [(0, 0), (5, 30), (77, 2)]:
        ref = np.sum(wdiag * np.exp(1j * gc @ (rc[r] - rc[rp]))) / p.volume
        assert abs(wr[r, rp] - ref) < 1e-12
    a = rng.standard_normal((p.n_r, p.n_r)) + 1j * rng.standard_normal((p.n_r, p.n_r))
    back = ochi.chi_gg(osc.w_rr(a, gv, p.n, p.lattice), gv, p.n, p.lattice)
    assert np.allclose(back, a, atol=1e-11)


# ---------------------------------------------------------------- self-energy

def test_sigma_spacetime_equals_pair_route(tiny_c):
    p = tiny_c
    gv = ogv.g_set(p.n, p.n_r)
    rng = np.random.default_rng(8)
    a = rng.standard_normal((p.n_r, 12)) + 1j * rng.standard_normal((p.n_r, 12))
    wgg = -(a @ a.conj().T) * 0.01
    dv = p.volume / p.n_r
    wrr = osc.w_rr(wgg, gv, p.n, p.lattice)
    for tau in (0.1, 2.0):
        su, so = osg.sigma_tau(p.psi, p.eps, p.n_occ, p.mu, tau, wrr, p.bands, dv)
        pu, po = osg.sigma_pair_tau(p.psi, p.eps, p.n_occ, p.mu, tau, wgg, gv, p.n,
                                    p.lattice, p.bands)
        assert np.allclose(su, pu, rtol=1e-11, atol=1e-14)
        assert np.allclose(so, po, rtol=1e-11, atol=1e-14)


@pytest.mark.parametrize("n_tau", [8, 16])
def test_sigma_single_pole_closed_form(n_tau):
    """W~(r,r',tau) = -B u(r)u^*(r') exp(-Om|tau|) with u a plane wave gives
    Sigma_nn(i w) = sum_m B |<n|u|m>|^2 / (i w - E_m -+ Om), - for unoccupied m and
    + for occupied m (E_m = eps_m - mu).  The discrete CT+ST reproduces it to within
    the weight fit error of each Lorentzian."""
    p = inputs.tiny(seed=9, n_tau=n_tau)
    gv = ogv.g_set(p.n, p.n_r)
    big_b, om = 0.8, 0.3
    g0 = 5
    p.x_min = min(p.x_min, om)
    s = opipe.setup(p)
    wt = np.zeros((n_tau, p.n_r, p.n_r), dtype=complex)
    for j, t in enumerate(p.tau):
        wt[j, g0, g0] = -big_b * p.volume * np.exp(-om * t)
    su, so = opipe.sigma_from_w(p, s, wt)
    sig = osg.sigma_iw(su, so, s["C"], s["S"])
    rc = _cart_r(p.n, p.lattice)
    u = np.exp(1j * rc @ _cart_g(gv[g0], p.lattice))
    dv = p.volume / p.n_r
    for b, n_ in enumerate(p.bands):
        exact = np.zeros(n_tau, dtype=complex)
        bound = np.zeros(n_tau)
        for m in range(p.n_b):
            mel = dv * np.sum(p.psi[n_].conj() * u * p.psi[m])
            em = p.eps[m] - p.mu
            x = em + om if m >= p.n_occ else om - em
            sgn = -1.0 if m >= p.n_occ else 1.0
            exact += big_b * abs(mel) ** 2 / (1j * p.omega - em + sgn * om)
            # |B|M|^2| times half the Lorentzian magnitudes times the fit errors
            lc = 2 * x / (x ** 2 + p.omega ** 2)
            ls = 2 * p.omega / (x ** 2 + p.omega ** 2)
            bound += big_b * abs(mel) ** 2 * 0.5 * (s["fit_err_cos"] * lc + s["fit_err_sin"] * ls)
        assert np.all(np.abs(sig[b] - exact) <= 1.05 * bound + 1e-14)
        assert np.max(np.abs(sig[b] - exact)) < 0.02 * np.max(np.abs(exact))


# ---------------------------------------------------------------- Thiele

def test_thiele_interpolates_and_reproduces_rational():
    """P_N(z_j) = f_j (Eq. pade2); a rational f with N/2 poles is reproduced off the
    nodes (continuation is ill-conditioned, so the real-axis check uses N = 8)."""
    rng = np.random.default_rng(10)
    for n, xoff, tol in ((8, 0.0, 1e-7), (12, 0.5, 1e-7)):
        z = 1j * np.geomspace(0.01, 30, n)
        poles = rng.uniform(-2, 2, n // 2) - 0.05j * rng.uniform(0.5, 1.5, n // 2)
        res = rng.uniform(0.1, 1.0, n // 2)

        def f(x):
            return sum(r / (x - e) for r, e in zip(res, poles))

        a = oth.coefficients(z, f(z))
        assert np.allclose(oth.evaluate(a, z, z), f(z), rtol=1e-12)
        x = np.linspace(-3, 3, 41) + 1j * xoff
        err = np.abs(oth.evaluate(a, z, x) - f(x)) / np.abs(f(x))
        assert err.max() < tol


def test_thiele_breakdown_raises():
    z = 1j * np.array([1.0, 2.0, 3.0])
    with pytest.raises(oth.ThieleBreakdown):
        oth.coefficients(z, np.array([1.0, 2.0, 1.0]))


def test_fft_pair_elements_and_rows_match_dense_definitions(tiny_c):
    """The FFT-based pair matrix elements and chi rows used for full-size sampled
    checks equal the dense-phase-matrix definitions."""
    p = tiny_c
    gv = ogv.g_set(p.n, p.n_r)
    idx = ogv.fft_index(gv, p.n)
    dense = ochi.pair_matrix_elements(p.psi, p.n_occ, gv, p.n, p.lattice)      # [Nu][No][Nchi]
    for i in range(p.n_occ):
        m = ochi.pair_matrix_elements_fft(p.psi, i, np.arange(p.n_occ, p.n_b), p.n, p.lattice, idx)
        assert np.allclose(m, dense[:, i, :], atol=1e-13)
    rows = [0, 5, 77]
    taus = [0.1, 2.0]
    got = ochi.chi_rows_pair(p.psi, p.eps, p.n_occ, taus, rows, p.n, p.lattice, idx)
    for j, t in enumerate(taus):
        full = ochi.chi_pair(p.psi, p.eps, p.n_occ, p.mu, t, gv, p.n, p.lattice, m=dense)
        assert np.allclose(got[j], full[rows], atol=1e-14)


def test_sparse_pair_sigma_matches_dense(tiny_c):
    p = tiny_c
    gv = ogv.g_set(p.n, p.n_r)
    idx = ogv.fft_index(gv, p.n)
    taus = [0.2, 3.0]
    entries = [(3, 3, [-0.4, -0.3]), (10, 10, [-0.2, -0.1]), (3, 10, [0.05 + 0.02j, 0.01j]),
               (10, 3, [0.05 - 0.02j, -0.01j])]
    a = osg.sigma_pair_sparse(p.psi, p.eps, p.n_occ, p.mu, taus, entries, p.n, p.lattice, idx, p.bands)
    for t, tau in enumerate(taus):
        w = np.zeros((p.n_r, p.n_r), dtype=complex)
        for j, jp, v in entries:
            w[j, jp] = v[t]
        b = osg.sigma_pair_tau(p.psi, p.eps, p.n_occ, p.mu, tau, w, gv, p.n, p.lattice, p.bands)
        assert np.allclose(a[0][:, t], b[0], atol=1e-14)
        assert np.allclose(a[1][:, t], b[1], atol=1e-14)
