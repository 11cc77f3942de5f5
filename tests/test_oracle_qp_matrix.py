"""Pins of the oracle's QP energies, spectral functions (Sec. II.E.2, Eqs.
QP, GWQP, Z, A) and full self-energy matrix (Eq. Sigma_occ_reduce for a pair
of bands) against closed forms, invariants and an independent route."""
import numpy as np
import pytest

from oracle import gvec as ogv
from oracle import pipeline as opipe
from oracle import qp as oqp
from oracle import screen as osc
from oracle import sigma as osg
from oracle import thiele as oth
from paper_1607_02859_gb300 import inputs


@pytest.fixture(scope="module")
def tiny_c():
    return inputs.tiny(seed=5)


def _poles(rng, n):
    """A causal sum of poles: residues > 0, poles below the real axis."""
    e = rng.uniform(-2, 2, n)
    eta = 0.05 * rng.uniform(0.5, 1.5, n)
    r = rng.uniform(0.1, 1.0, n)
    return r, e - 1j * eta


def _f(r, poles, x):
    return sum(ri / (x - pi) for ri, pi in zip(r, poles))


def _df(r, poles, x):
    return sum(-ri / (x - pi) ** 2 for ri, pi in zip(r, poles))


# ---------------------------------------------------------------- Thiele derivative

def test_derivative_of_reproduced_rational_is_its_closed_form():
    """A rational f with N/2 poles is reproduced by the N-point approximant, so
    the approximant's derivative is f' = -sum r_p / (x - p)^2 on the real axis."""
    rng = np.random.default_rng(21)
    n = 8
    r, p = _poles(rng, n // 2)
    z = 1j * np.geomspace(0.01, 30, n)
    a = oth.coefficients(z, _f(r, p, z))
    x = np.linspace(-3, 3, 61).astype(complex)
    d = oth.derivative(a, z, x)
    assert np.max(np.abs(d - _df(r, p, x)) / np.abs(_df(r, p, x))) < 1e-5


def test_derivative_matches_central_difference_of_the_fraction():
    """For data the approximant does not reproduce (random values at 12
    nodes), its derivative still equals a central difference of itself."""
    rng = np.random.default_rng(22)
    z = 1j * np.geomspace(0.05, 20, 12)
    f = rng.standard_normal(12) + 1j * rng.standard_normal(12)
    a = oth.coefficients(z, f)
    x = np.linspace(-1.5, 1.5, 13) + 0.3j
    h = 1e-5
    fd = (oth.evaluate(a, z, x + h) - oth.evaluate(a, z, x - h)) / (2 * h)
    d = oth.derivative(a, z, x)
    assert np.max(np.abs(d - fd) / np.abs(d)) < 1e-6


# ---------------------------------------------------------------- QP energies

@pytest.mark.parametrize("n_nodes", [3, 4])
def test_linear_self_energy_makes_the_linearisation_exact(n_nodes):
    """Sigma(omega) = s0 + s1 (omega - mu) is reproduced by Thiele at 3 or 4
    nodes; then Eq. QP is exact, and the linearised E equals the root of
    E = v + Re Sigma(E): E = (v + Re s0 - s1 mu) / (1 - s1), Z = 1/(1 - s1),
    whatever the expansion point eps; the spectral function peaks there too."""
    s0, s1, v, mu = -0.12 + 0.03j, -0.27, 0.41, 0.02
    omega = np.geomspace(0.05, 4.0, n_nodes)
    sig = (s0 + s1 * 1j * omega)[None, :]
    e_exact = (v + s0.real - s1 * mu) / (1 - s1)
    for eps in (-0.3, 0.0, 0.25):
        e, zf, s_eps, ds = oqp.linearized(sig, omega, [eps], mu, [v])
        assert abs(zf[0] - 1 / (1 - s1)) < 1e-12
        assert abs(e[0] - e_exact) < 1e-12
        assert abs(ds[0] - s1) < 1e-12
        assert abs(s_eps[0] - (s0 + s1 * (eps - mu))) < 1e-12
        # with Im Sigma constant, A peaks at the same root
        w = np.linspace(e_exact - 0.05, e_exact + 0.05, 100001)
        a = oqp.spectral(sig, omega, [eps], mu, [v], w)[0]
        assert abs(w[np.argmax(a)] - e_exact) <= w[1] - w[0]


def test_qp_of_a_pole_self_energy():
    """Sigma a sum of poles (reproduced at 8 nodes): Sigma(eps - mu) and its
    derivative are the closed forms, and E_n = eps_n + Z_n (v_n + Re Sigma - eps_n)."""
    rng = np.random.default_rng(23)
    omega = np.geomspace(0.01, 30, 8)
    mu = 0.1
    sig, eps, v, ref = [], [], [], []
    for b in range(3):
        r, p = _poles(rng, 4)
        sig.append(_f(r, p, 1j * omega))
        eps.append(rng.uniform(-1, 1))
        v.append(eps[-1] + rng.uniform(-0.2, 0.2))
        x = eps[-1] - mu
        ref.append((_f(r, p, x), _df(r, p, x)))
    e, zf, s_eps, ds = oqp.linearized(np.array(sig), omega, eps, mu, v)
    for b in range(3):
        assert abs(s_eps[b] - ref[b][0]) < 1e-6 * abs(ref[b][0])
        assert abs(ds[b] - ref[b][1]) < 1e-5 * abs(ref[b][1])
        z_ref = 1 / (1 - ref[b][1].real)
        assert abs(zf[b] - z_ref) < 1e-5 * abs(z_ref)
        assert abs(e[b] - (eps[b] + z_ref * (v[b] + ref[b][0].real - eps[b]))) < 1e-5


# ---------------------------------------------------------------- spectral function

def test_constant_self_energy_gives_a_unit_lorentzian():
    """DeltaSigma = c - i gamma constant: A is a Lorentzian centred at eps + c,
    height 1/(pi gamma), full width 2 gamma at half maximum, unit area."""
    s0, v, eps, mu = -0.05 - 0.02j, 0.3, 0.1, 0.0
    sig = np.array([[s0]])
    omega = np.array([1.0])
    centre, gam = v + s0.real, abs(s0.imag)
    w = np.linspace(centre - 400 * gam, centre + 400 * gam, 400001)
    a = oqp.spectral(sig, omega, [eps], mu, [v], w)[0]
    k = np.argmax(a)
    assert abs(w[k] - centre) < 2 * (w[1] - w[0])
    assert abs(a[k] - 1 / (np.pi * gam)) < 1e-6 * a[k]
    half = w[a >= 0.5 * a[k]]
    assert abs((half[-1] - half[0]) - 2 * gam) < 4 * (w[1] - w[0])
    area = np.sum(a) * (w[1] - w[0])
    assert abs(area - 1) < 2e-3               # tails beyond 400 gamma hold 1.6e-3


def test_spectral_sum_rule_for_a_causal_self_energy():
    """Poles of Sigma below the real axis with positive residues make
    G = 1/(omega - eps - DeltaSigma) analytic above it and ~1/omega, so the
    area under A = |Im G|/pi is 1 (up to the truncated tails)."""
    rng = np.random.default_rng(24)
    r, p = _poles(rng, 4)
    r *= 0.1
    omega = np.geomspace(0.01, 30, 8)
    sig = _f(r, p, 1j * omega)[None, :]
    w = np.linspace(-60, 60, 1_200_001)
    a = oqp.spectral(sig, omega, [0.2], 0.0, [0.25], w)[0]
    area = np.sum(a) * (w[1] - w[0])
    assert abs(area - 1) < 5e-3


# ---------------------------------------------------------------- self-energy matrix

def test_matrix_spacetime_equals_pair_route(tiny_c):
    """Off-diagonal elements by the space-time route equal the conventional
    route (the pair-density quadratic form) for a random Hermitian W~."""
    p = tiny_c
    gv = ogv.g_set(p.n, p.n_r)
    rng = np.random.default_rng(25)
    a = rng.standard_normal((p.n_r, 12)) + 1j * rng.standard_normal((p.n_r, 12))
    wgg = -(a @ a.conj().T) * 0.01
    dv = p.volume / p.n_r
    wrr = osc.w_rr(wgg, gv, p.n, p.lattice)
    bands = np.array([0, 3, p.n_occ, p.n_occ + 2, p.n_b - 1])
    for tau in (0.1, 2.0):
        su, so = osg.sigma_matrix_tau(p.psi, p.eps, p.n_occ, p.mu, tau, wrr, bands, dv)
        pu, po = osg.sigma_matrix_pair_tau(p.psi, p.eps, p.n_occ, p.mu, tau, wgg, gv, p.n, p.lattice, bands)
        scale = np.max(np.abs(su)) + np.max(np.abs(so))
        assert np.max(np.abs(su - pu)) < 1e-11 * scale
        assert np.max(np.abs(so - po)) < 1e-11 * scale
        assert np.max(np.abs(su.imag)) > 1e-3 * scale        # a complex case
        # Hermitian, and the diagonal is the diagonal route's value
        assert np.allclose(su, su.conj().T, atol=1e-13 * scale)
        assert np.allclose(so, so.conj().T, atol=1e-13 * scale)
        du, do = osg.sigma_tau(p.psi, p.eps, p.n_occ, p.mu, tau, wrr, bands, dv)
        assert np.allclose(np.diag(su).real, du, rtol=1e-12, atol=1e-15)
        assert np.allclose(np.diag(so).real, do, rtol=1e-12, atol=1e-15)


def test_matrix_single_pole_closed_form():
    """W~(r,r',tau) = -B u(r)u^*(r') exp(-Om|tau|), u a plane wave:
    Sigma_nm(i w) = sum_l B M_nl conj(M_ml) / (i w - E_l -+ Om) with
    M_nl = dV sum_r psi_n^* u psi_l (- for unoccupied l, + for occupied), to
    within the weight fit error of each Lorentzian."""
    n_tau = 12
    p = inputs.tiny(seed=9, n_tau=n_tau)
    gv = ogv.g_set(p.n, p.n_r)
    big_b, om, g0 = 0.8, 0.3, 5
    p.x_min = min(p.x_min, om)
    s = opipe.setup(p)
    dv = p.volume / p.n_r
    bands = np.array([0, 2, p.n_occ + 1])
    su = np.empty((3, 3, n_tau), dtype=complex)
    so = np.empty((3, 3, n_tau), dtype=complex)
    for j, t in enumerate(p.tau):
        wgg = np.zeros((p.n_r, p.n_r), dtype=complex)
        wgg[g0, g0] = -big_b * p.volume * np.exp(-om * t)
        wrr = osc.w_rr(wgg, gv, p.n, p.lattice)
        su[:, :, j], so[:, :, j] = osg.sigma_matrix_tau(p.psi, p.eps, p.n_occ, p.mu, t, wrr, bands, dv)
    sig = osg.sigma_matrix_iw(su, so, s["C"], s["S"])
    idx = ogv.fft_index(gv, p.n)
    u = np.zeros(p.n_r, dtype=complex)
    u[idx[g0]] = 1.0
    u = np.fft.ifftn(u.reshape(p.n)).reshape(-1) * p.n_r          # exp(i G0 . r) on the grid
    m = dv * (p.psi.conj() @ (u[:, None] * p.psi.T))              # M[n, l]
    for i, bn in enumerate(bands):
        for k, bm in enumerate(bands):
            exact = np.zeros(n_tau, dtype=complex)
            bound = np.zeros(n_tau)
            for l in range(p.n_b):
                w_nl = big_b * m[bn, l] * np.conj(m[bm, l])
                el = p.eps[l] - p.mu
                x = el + om if l >= p.n_occ else om - el
                sgn = -1.0 if l >= p.n_occ else 1.0
                exact += w_nl / (1j * p.omega - el + sgn * om)
                lc = 2 * x / (x ** 2 + p.omega ** 2)
                ls = 2 * p.omega / (x ** 2 + p.omega ** 2)
                bound += abs(w_nl) * 0.5 * (s["fit_err_cos"] * lc + s["fit_err_sin"] * ls)
            assert np.all(np.abs(sig[i, k] - exact) <= 1.05 * bound + 1e-14)


# ---------------------------------------------------------------- inverse transforms

def test_inverse_sine_transform_and_sigma_round_trip():
    """Eq. INV_ST_FFT: Sinv S = S Sinv = 1; Sigma(i omega) of random Hermitian
    Sigma_unocc(tau), Sigma_occ(-tau) matrices (and of real diagonals) goes
    back to them through the Hermitian / anti-Hermitian split."""
    p = inputs.tiny(seed=9, n_tau=12)
    s = opipe.setup(p)
    n = len(p.tau)
    eye = np.eye(n)
    assert np.max(np.abs(s["Sinv"] @ s["S"] - eye)) < 1e-9
    assert np.max(np.abs(s["S"] @ s["Sinv"] - eye)) < 1e-9
    rng = np.random.default_rng(26)

    def herm(k):
        a = rng.standard_normal((k, k, n)) + 1j * rng.standard_normal((k, k, n))
        return a + a.conj().transpose(1, 0, 2)

    su, so = herm(5), herm(5)
    back_u, back_o = osg.sigma_tau_from_iw(osg.sigma_matrix_iw(su, so, s["C"], s["S"]), s["Cinv"], s["Sinv"])
    assert np.max(np.abs(back_u - su)) < 1e-9 * np.max(np.abs(su))
    assert np.max(np.abs(back_o - so)) < 1e-9 * np.max(np.abs(so))
    du, do = rng.standard_normal((4, n)), rng.standard_normal((4, n))
    bu, bo = osg.sigma_tau_from_iw(osg.sigma_iw(du, do, s["C"], s["S"]), s["Cinv"], s["Sinv"])
    assert np.max(np.abs(bu - du)) < 1e-9 * np.max(np.abs(du))
    assert np.max(np.abs(bo - do)) < 1e-9 * np.max(np.abs(do))
