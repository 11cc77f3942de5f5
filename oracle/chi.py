"""Polarizability chi0 (Secs. II.B and II.C steps (i)-(ii)).  Oracle only.

Real space, imaginary time (Eqs. chi_GG, chi_rr), spin-degenerate factor 2,
index order chi(r,r') = -2 G_occ(r,r') G_unocc(r',r):

    chi(r,r',tau) = -2 G_occ(r,r',tau) G_unocc(r',r,tau)

For complex orbitals this is the complex conjugate (equivalently, the
transpose) of the tau > 0 slice as printed in Eq. chi_rr; both are Hermitian
and negative semidefinite after the transform below, and they coincide for
real orbitals.

Reciprocal space (Eqs. FFTX1, FFTX2 with the normalisation chosen so that the
dielectric matrix reads eps = 1 - v chi with v = 4 pi / |G|^2):

    chi(G,G',tau) = (dV^2 / Omega) sum_r sum_r' exp(-i G.r) chi(r,r') exp(+i G'.r')

written here as dense phase matrices (a direct DFT, not an FFT algorithm).
"""
import numpy as np

from . import gvec as _gv


def chi_rr(g_occ, g_unocc):
    """Eq. chi_rr in the order chi(r,r') = -2 G_occ(r,r') G_unocc(r',r), spin factor 2."""
    return -2.0 * g_occ * g_unocc.T


def rows_to_g(x_rr, gvecs, n):
    """Eq. FFTX1: X(r,G') = sum_R' x(r,R') exp(+i G'.R') for the G' of the set."""
    pm = _gv.phase_matrix(gvecs, n, -1.0)          # exp(-i G.r)
    return x_rr @ pm.conj().T


def cols_to_g(x_rg, gvecs, n, lattice):
    """Eq. FFTX2 with the dV^2/Omega factor: chi(G,G') = dV^2/Omega sum_r exp(-iG.r) X(r,G')."""
    vol = abs(np.linalg.det(lattice))
    dv = vol / int(np.prod(n))
    pm = _gv.phase_matrix(gvecs, n, -1.0)
    return (dv * dv / vol) * (pm @ x_rg)


def chi_gg(x_rr, gvecs, n, lattice):
    """Both steps at once: (dV^2/Omega) P x P^H with P[j][r] = exp(-i G_j.r)."""
    return cols_to_g(rows_to_g(x_rr, gvecs, n), gvecs, n, lattice)


def pair_matrix_elements(psi, n_occ, gvecs, n, lattice):
    """M_ai(G) = dV sum_r exp(-i G.r) psi_a^*(r) psi_i(r): the matrix elements
    <psi_a| e^{-iG.r} |psi_i> of Eq. CHI_g_it, shape [N_unocc][N_occ][N_chi]."""
    vol = abs(np.linalg.det(lattice))
    dv = vol / int(np.prod(n))
    pm = _gv.phase_matrix(gvecs, n, -1.0)           # [N_chi][N_r]
    occ = psi[:n_occ]
    un = psi[n_occ:]
    prod = un.conj()[:, None, :] * occ[None, :, :]   # [Nu][No][N_r]
    return dv * prod @ pm.T


def chi_pair(psi, eps, n_occ, mu, tau, gvecs, n, lattice, m=None):
    """Adler-Wiser pair form in imaginary time (Eq. CHI_g_it):
    chi(G,G',tau) = -(2/Omega) sum_{i,a} exp(-(eps_a - eps_i) tau) M_ai(G) M_ai(G')^*."""
    vol = abs(np.linalg.det(lattice))
    if m is None:
        m = pair_matrix_elements(psi, n_occ, gvecs, n, lattice)
    w = np.exp(-(eps[n_occ:, None] - eps[None, :n_occ]) * tau)   # [Nu][No]
    mm = m.reshape(-1, m.shape[-1])
    return -(2.0 / vol) * (mm.T * w.reshape(-1)) @ mm.conj()


def ct(f_tau, C):
    """Eq. CTX: F(i omega_k) = sum_j C_kj F(i tau_j) over the leading axis."""
    return np.tensordot(C, f_tau, axes=(1, 0))


def fftn_batch(x, workers=None):
    """3-D DFT over the last three axes, sum_r x(r) exp(-2 pi i k.r / n): numpy's
    FFT, or scipy's with `workers` threads (the same transform) when given."""
    if workers:
        import scipy.fft
        return scipy.fft.fftn(x, axes=(1, 2, 3), workers=workers)
    return np.fft.fftn(x, axes=(1, 2, 3))


def pair_matrix_elements_fft(psi, i, a_bands, n, lattice, fft_index, workers=None):
    """M_ai(G) of Eq. CHI_g_it for one occupied band i and the bands a_bands, at
    the G-set grid positions fft_index, with an FFT as the transform step:
    fftn(x)[k] = sum_r x(r) exp(-2 pi i k.r / n) = sum_r exp(-i G.r) x(r)."""
    vol = abs(np.linalg.det(lattice))
    dv = vol / int(np.prod(n))
    prod = psi[a_bands].conj() * psi[i][None, :]              # [Na][N_r]
    f = fftn_batch(prod.reshape(len(a_bands), *n), workers).reshape(len(a_bands), -1)
    return dv * f[:, fft_index]


def chi_rows_pair(psi, eps, n_occ, taus, rows, n, lattice, fft_index, workers=None):
    """Rows `rows` (G-set indices) of chi(G,G',tau) for every tau, by the pair
    sum of Eq. CHI_g_it: [N_tau][len(rows)][N_chi]."""
    vol = abs(np.linalg.det(lattice))
    un = np.arange(n_occ, psi.shape[0])
    out = np.zeros((len(taus), len(rows), len(fft_index)), dtype=np.complex128)
    taus = np.asarray(taus, dtype=np.float64)
    for i in range(n_occ):
        m = pair_matrix_elements_fft(psi, i, un, n, lattice, fft_index, workers)   # [Nu][N_chi]
        mr = m[:, rows]                                                    # [Nu][rows]
        w = np.exp(-np.outer(taus, eps[n_occ:] - eps[i]))                 # [N_tau][Nu]
        # sum over a of exp(-(eps_a - eps_i) tau_j) M_ai(G_row) M_ai(G')^*, all tau in one product
        lhs = (w[:, None, :] * mr.T[None, :, :]).reshape(len(taus) * len(rows), -1)
        out += (lhs @ m.conj()).reshape(len(taus), len(rows), -1)
    return -(2.0 / vol) * out
