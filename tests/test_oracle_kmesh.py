"""Pins of the k-mesh oracle (oracle/kmesh.py) against the Gamma-point oracle,
which tests/test_oracle_pins.py pins to the paper: the stripe route on a
Gamma-centred k mesh must give the q-diagonal blocks of the supercell's
Gamma-point chi, whose blocks q != q' vanish; a 1 x 1 x 1 mesh is the Gamma
point itself."""
import numpy as np

from oracle import chi as ochi
from oracle import green as ogr
from oracle import gvec as ogv
from oracle import kmesh as okm
from paper_1607_02859_gb300 import inputs


def supercell_chi(p, gv, tau):
    psi_s, eps_s, no_s = okm.supercell_orbitals(p.psi_k, p.eps_k, p.n_occ, p.n, p.nk)
    ns = tuple(np.asarray(p.n) * np.asarray(p.nk))
    lat_s = p.lattice * np.asarray(p.nk)[:, None]
    x = ochi.chi_rr(ogr.green_occ(psi_s, eps_s, no_s, p.mu, tau), ogr.green_unocc(psi_s, eps_s, no_s, p.mu, tau))
    return ochi.chi_gg(x, okm.supercell_gvecs(gv, p.nk), ns, lat_s)


def test_stripe_route_equals_supercell_gamma_point():
    p = inputs.kmesh_problem(n=(4, 4, 4), a=(5.0, 5.5, 6.0), nk=(2, 2, 1), n_occ=3, n_unocc=9, n_tau=2, seed=52)
    gv = ogv.g_set(p.n, 40)
    tau = p.tau[1]
    cq = okm.chi_q_tau(p.psi_k, p.eps_k, p.n_occ, p.mu, tau, p.n, p.nk, p.lattice, gv)
    cs = supercell_chi(p, gv, tau)
    nq, nc = p.n_k, len(gv)
    scale = np.linalg.norm(cs)
    for a in range(nq):
        for b in range(nq):
            blk = cs[a * nc:(a + 1) * nc, b * nc:(b + 1) * nc]
            if a == b:
                assert np.linalg.norm(blk - cq[a]) < 1e-12 * scale
            else:
                assert np.linalg.norm(blk) < 1e-12 * scale


def test_single_k_is_gamma_point():
    p = inputs.kmesh_problem(n=(4, 4, 4), nk=(1, 1, 1), n_occ=3, n_unocc=9, n_tau=2, seed=53)
    gv = ogv.g_set(p.n, 64)
    tau = p.tau[0]
    cq = okm.chi_q_tau(p.psi_k, p.eps_k, p.n_occ, p.mu, tau, p.n, p.nk, p.lattice, gv)
    x = ochi.chi_rr(ogr.green_occ(p.psi_k[0], p.eps_k[0], p.n_occ, p.mu, tau),
                    ogr.green_unocc(p.psi_k[0], p.eps_k[0], p.n_occ, p.mu, tau))
    ref = ochi.chi_gg(x, gv, p.n, p.lattice)
    assert np.linalg.norm(cq[0] - ref) < 1e-12 * np.linalg.norm(ref)


def test_chi_q_hermitian_and_negative_semidefinite():
    p = inputs.kmesh_problem(n=(4, 4, 4), nk=(2, 1, 2), n_occ=3, n_unocc=9, n_tau=2, seed=54)
    gv = ogv.g_set(p.n, 32)
    cq = okm.chi_q_tau(p.psi_k, p.eps_k, p.n_occ, p.mu, p.tau[0], p.n, p.nk, p.lattice, gv)
    for c in cq:
        assert np.linalg.norm(c - c.conj().T) < 1e-12 * np.linalg.norm(c)
        assert np.linalg.eigvalsh(0.5 * (c + c.conj().T)).max() < 1e-12 * np.linalg.norm(c)


def test_sigma_stripe_equals_supercell_gamma_point():
    from oracle import sigma as osg
    p = inputs.kmesh_problem(n=(4, 4, 4), a=(5.0, 5.5, 6.0), nk=(2, 1, 2), n_occ=3, n_unocc=9, n_tau=2, seed=55)
    gv = ogv.g_set(p.n, 24)
    rng = np.random.default_rng(56)
    w_q = []
    for _ in range(p.n_k):                       # Hermitian W~_q of moderate size
        a = rng.standard_normal((len(gv), len(gv))) + 1j * rng.standard_normal((len(gv), len(gv)))
        w_q.append(-(a @ a.conj().T) * 0.05)
    w_q = np.array(w_q)
    tau = p.tau[0]
    w_s = okm.w_stripe(w_q, p.n, p.nk, p.lattice, gv)
    bands = [(2, 0), (3, 1), (4, 3)]
    su, so = okm.sigma_k_tau(p.psi_k, p.eps_k, p.n_occ, p.mu, tau, w_s, p.n, p.nk, p.lattice, bands)
    # the same system as a Gamma-point problem of the supercell
    psi_s, eps_s, no_s = okm.supercell_orbitals(p.psi_k, p.eps_k, p.n_occ, p.n, p.nk)
    ns = tuple(np.asarray(p.n) * np.asarray(p.nk))
    lat_s = p.lattice * np.asarray(p.nk)[:, None]
    gs = okm.supercell_gvecs(gv, p.nk)
    nc = len(gv)
    w_full = np.zeros((len(gs), len(gs)), dtype=np.complex128)
    for q in range(p.n_k):
        w_full[q * nc:(q + 1) * nc, q * nc:(q + 1) * nc] = w_q[q]
    pm = ogv.phase_matrix(gs, ns, -1.0)                     # exp(-i Gs.R)
    w_rr = pm.conj().T @ w_full @ pm / abs(np.linalg.det(lat_s))
    # supercell band index of (b, k): occupied (k outer, b inner), then unoccupied
    def sband(b, k):
        return k * p.n_occ + b if b < p.n_occ else p.n_k * p.n_occ + k * (p.n_b - p.n_occ) + (b - p.n_occ)
    dv = abs(np.linalg.det(p.lattice)) / p.n_r
    ref_u, ref_o = osg.sigma_tau(psi_s, eps_s, no_s, p.mu, tau, w_rr, [sband(b, k) for b, k in bands], dv)
    scale = max(np.abs(ref_u).max(), np.abs(ref_o).max())
    assert np.abs(su - ref_u).max() < 1e-11 * scale
    assert np.abs(so - ref_o).max() < 1e-11 * scale
    # and the stripe of W~ is the supercell's W~ restricted to rows in the cell
    pos0 = okm.supercell_index(p.n, p.nk)[0]
    assert np.linalg.norm(w_s - w_rr[pos0]) < 1e-12 * np.linalg.norm(w_rr)


# ---------------------------------------------- plane-wave form of G_k (Sec. II.B)

def _support(c_k):
    """FFT positions where any band at any k has a plane-wave coefficient."""
    w = np.sum(np.abs(c_k) ** 2, axis=(0, 1))
    return np.flatnonzero(w > 1e-20 * w.max())


def test_pw_form_gives_the_real_space_stripe():
    """Coefficients, G_k(g, k+g') (Eqs. G1_unocc_k, G1_occ_k) and Eqs. FFT_G1,
    FFT_G2 give the stripe that the Bloch extension of the real-space Green's
    functions gives, for both Green's functions."""
    p = inputs.kmesh_problem(n=(4, 4, 4), a=(5.0, 5.5, 6.0), nk=(2, 1, 2), n_occ=3, n_unocc=9, n_tau=2, seed=57)
    for tau in p.tau:
        go, gu = okm.green_stripe(p.psi_k, p.eps_k, p.n_occ, p.mu, tau, p.n, p.nk)
        po, pu = okm.green_stripe_pw(p.psi_k, p.eps_k, p.n_occ, p.mu, tau, p.n, p.nk)
        assert np.linalg.norm(po - go) < 1e-12 * np.linalg.norm(go)
        assert np.linalg.norm(pu - gu) < 1e-12 * np.linalg.norm(gu)


def test_inverse_transforms_give_the_pw_form():
    """Eqs. INV_FFT_G1, INV_FFT_G2 applied to the real-space stripe give
    G_k(g, k+g') / N_k for every k: the ket over the supercell carries the N_k
    that the cell-normalised stripe (1/N_k) takes back."""
    p = inputs.kmesh_problem(n=(4, 4, 2), a=(5.0, 5.5, 3.5), nk=(2, 2, 2), n_occ=3, n_unocc=7, n_tau=2, seed=58)
    tau = p.tau[1]
    c_k = okm.pw_coefficients_k(p.psi_k, p.n, p.nk)
    go, gu = okm.green_stripe(p.psi_k, p.eps_k, p.n_occ, p.mu, tau, p.n, p.nk)
    for which, g_s in (("occ", go), ("unocc", gu)):
        ref = okm.green_k_pw(c_k, p.eps_k, p.n_occ, p.mu, tau, p.nk, which) / p.n_k
        got = okm.inv_fft_g1_g2(g_s, p.n, p.nk)
        assert np.linalg.norm(got - ref) < 1e-12 * np.linalg.norm(ref)


def test_pw_form_at_gamma_is_the_two_sided_dft():
    """A 1 x 1 x 1 mesh: G(g, g') is the cell DFT of G(r, r') over r and its
    inverse-signed DFT over r' (numpy's FFT on each side)."""
    p = inputs.kmesh_problem(n=(4, 3, 5), a=(5.0, 4.0, 6.0), nk=(1, 1, 1), n_occ=3, n_unocc=9, n_tau=2, seed=59)
    tau = p.tau[0]
    c_k = okm.pw_coefficients_k(p.psi_k, p.n, p.nk)
    for which, f in (("occ", ogr.green_occ), ("unocc", ogr.green_unocc)):
        g_rr = f(p.psi_k[0], p.eps_k[0], p.n_occ, p.mu, tau).reshape(p.n + p.n)
        ref = np.fft.ifftn(np.fft.fftn(g_rr, axes=(0, 1, 2)), axes=(3, 4, 5)) * p.n_r
        got = okm.green_k_pw(c_k, p.eps_k, p.n_occ, p.mu, tau, p.nk, which)[0]
        assert np.linalg.norm(got - ref.reshape(p.n_r, p.n_r)) < 1e-12 * np.linalg.norm(ref)


def test_pw_form_needs_only_the_orbitals_plane_waves():
    """The memory-lean point of Sec. II.B: G_k(g, g') vanishes outside the
    orbitals' plane-wave set (here the lowest N_b plane waves, fewer than the
    grid points), and the transforms over that set alone give the same stripe
    and the same chi_q."""
    p = inputs.kmesh_problem(n=(4, 4, 4), a=(5.0, 5.5, 6.0), nk=(2, 2, 1), n_occ=3, n_unocc=9, n_tau=2, seed=60)
    tau = p.tau[0]
    c_k = okm.pw_coefficients_k(p.psi_k, p.n, p.nk)
    pw = _support(c_k)
    assert len(pw) == p.n_b < p.n_r
    out = np.setdiff1d(np.arange(p.n_r), pw)
    for which in ("occ", "unocc"):
        gk = okm.green_k_pw(c_k, p.eps_k, p.n_occ, p.mu, tau, p.nk, which)
        assert np.abs(gk[:, out, :]).max() < 1e-12 * np.abs(gk).max()
        assert np.abs(gk[:, :, out]).max() < 1e-12 * np.abs(gk).max()
    full = okm.green_stripe_pw(p.psi_k, p.eps_k, p.n_occ, p.mu, tau, p.n, p.nk)
    lean = okm.green_stripe_pw(p.psi_k, p.eps_k, p.n_occ, p.mu, tau, p.n, p.nk, pw_index=pw)
    for a, b in zip(full, lean):
        assert np.linalg.norm(a - b) < 1e-12 * np.linalg.norm(a)
    gv = ogv.g_set(p.n, 30)
    ref = okm.chi_q_tau(p.psi_k, p.eps_k, p.n_occ, p.mu, tau, p.n, p.nk, p.lattice, gv)
    got = okm.chi_q_tau_pw(p.psi_k, p.eps_k, p.n_occ, p.mu, tau, p.n, p.nk, p.lattice, gv, pw_index=pw)
    assert np.linalg.norm(got - ref) < 1e-12 * np.linalg.norm(ref)
