"""Correlation self-energy, diagonal and full matrix (Sec. II.D).  Oracle only.

Space-time route (Eq. Sigma_rr, first term of Eq. Sigma_occ_reduce; the PAW
one-centre terms are out of scope).  With G_occ/G_unocc as in green.py and
W~ even in tau,

    Sigma_unocc_nn(tau)  = + dV^2 sum_{r,r'} psi_n^*(r) G_unocc(r,r',tau) W~(r,r',tau) psi_n(r')
    Sigma_occ_nn(-tau)   = - dV^2 sum_{r,r'} psi_n^*(r) G_occ(r,r',tau)   W~(r,r',tau) psi_n(r')

(the paper's overline/underline Sigma = -G W~ with its overline-G = -G_unocc).
Both quadratic forms are real (G o W~ is Hermitian); their real parts are kept.

Even/odd split and transform (Eqs. cos_sin_sigma_matrix1/2, sigma_r_w,
cos_sin_sigma1/2):

    Sigma^c(tau) = (Sigma_unocc(tau) + Sigma_occ(-tau)) / 2
    Sigma^s(tau) = (Sigma_unocc(tau) - Sigma_occ(-tau)) / 2
    Sigma(i omega_k) = sum_j C_kj Sigma^c(tau_j) + i sum_j S_kj Sigma^s(tau_j)
"""
import numpy as np

from . import chi as _chi
from . import green as _gr


def sigma_tau(psi, eps, n_occ, mu, tau, w_rr, bands, dv):
    """(Sigma_unocc_nn(tau), Sigma_occ_nn(-tau)) for the listed bands at one tau."""
    gu = _gr.green_unocc(psi, eps, n_occ, mu, tau)
    go = _gr.green_occ(psi, eps, n_occ, mu, tau)
    hu = gu * w_rr
    ho = go * w_rr
    su = np.empty(len(bands))
    so = np.empty(len(bands))
    for b, n_ in enumerate(bands):
        p = psi[n_]
        su[b] = (dv * dv * (p.conj() @ hu @ p)).real
        so[b] = -(dv * dv * (p.conj() @ ho @ p)).real
    return su, so


def sigma_pair_tau(psi, eps, n_occ, mu, tau, w_gg, gvecs, n, lattice, bands):
    """Conventional route: Sigma_unocc_nn(tau) = (1/Omega) sum_{m unocc}
    exp(-(eps_m-mu) tau) a_nm^H W~ a_nm with a_nm(G) = dV sum_r exp(-iG.r)
    psi_m^*(r) psi_n(r); Sigma_occ_nn(-tau) likewise over occupied m with
    exp(+(eps_m-mu) tau) and a minus sign.  Same quantity as sigma_tau."""
    from . import gvec as _gv
    vol = abs(np.linalg.det(lattice))
    dv = vol / int(np.prod(n))
    pm = _gv.phase_matrix(gvecs, n, -1.0)
    su = np.empty(len(bands))
    so = np.empty(len(bands))
    for b, n_ in enumerate(bands):
        a = dv * (psi.conj() * psi[n_][None, :]) @ pm.T      # [N_b][N_chi]
        q = np.einsum("mg,gh,mh->m", a.conj(), w_gg, a).real / vol
        fu = np.exp(-(eps[n_occ:] - mu) * tau)
        fo = np.exp((eps[:n_occ] - mu) * tau)
        su[b] = (fu * q[n_occ:]).sum()
        so[b] = -(fo * q[:n_occ]).sum()
    return su, so


def sigma_iw(s_unocc, s_occ, C, S):
    """Sigma_nn(i omega_k) from [N_n][N_tau] arrays via CT + ST."""
    sc = 0.5 * (s_unocc + s_occ)
    ss = 0.5 * (s_unocc - s_occ)
    return sc @ C.T + 1j * (ss @ S.T)


def sigma_pair_sparse(psi, eps, n_occ, mu, taus, entries, n, lattice, fft_index, bands, workers=None):
    """The conventional route of sigma_pair_tau for a W~(G,G',tau) with only a
    few nonzero entries, given as (j, j', values) with G-set indices j, j' and
    one value per tau:
    Sigma_unocc_nn(tau) = (1/Omega) sum_{m unocc} exp(-(eps_m-mu) tau)
                          sum_(j,j') conj(a_nm(G_j)) W~_jj'(tau) a_nm(G_j'),
    Sigma_occ_nn(-tau) likewise over occupied m with exp(+(eps_m-mu) tau) and a
    minus sign; a_nm(G) = dV sum_r exp(-iG.r) psi_m^*(r) psi_n(r).
    Returns ([N_n][N_tau], [N_n][N_tau])."""
    vol = abs(np.linalg.det(lattice))
    dv = vol / int(np.prod(n))
    taus = np.atleast_1d(np.asarray(taus, dtype=np.float64))
    idx = sorted({e[0] for e in entries} | {e[1] for e in entries})
    pos = {j: k for k, j in enumerate(idx)}
    su = np.empty((len(bands), len(taus)))
    so = np.empty((len(bands), len(taus)))
    for b, n_ in enumerate(bands):
        prod = psi.conj() * psi[n_][None, :]
        f = _chi.fftn_batch(prod.reshape(psi.shape[0], *n), workers).reshape(psi.shape[0], -1)
        a = dv * f[:, np.asarray(fft_index)[idx]]                  # [N_b][len(idx)]
        for t, tau in enumerate(taus):
            q = np.zeros(psi.shape[0])
            for (j, jp, vals) in entries:
                val = np.atleast_1d(vals)[t]
                q += (np.conj(a[:, pos[j]]) * val * a[:, pos[jp]]).real
            q /= vol
            su[b, t] = (np.exp(-(eps[n_occ:] - mu) * tau) * q[n_occ:]).sum()
            so[b, t] = -(np.exp((eps[:n_occ] - mu) * tau) * q[:n_occ]).sum()
    return su, so


# ---------------------------------------------------------------- full matrix
# Matrix elements Sigma_nm = <psi_n|Sigma|psi_m> of the same operators: the
# paper's Eq. Sigma_occ_reduce written for a pair of bands (n, m) instead of
# (n, n).  G o W~ is Hermitian in (r, r'), so the matrices are Hermitian and
# their diagonals are the real values above.  The even/odd split and CT+ST
# (Eqs. cos_sin_sigma, cos_sin_sigma1/2) act element by element on the
# complex matrices.

def sigma_matrix_tau(psi, eps, n_occ, mu, tau, w_rr, bands, dv):
    """(Su, So) [N_n][N_n] complex at one tau:
        Su_nm(tau)  = +dV^2 psi_n^H (G_unocc o W~) psi_m
        So_nm(-tau) = -dV^2 psi_n^H (G_occ o W~) psi_m"""
    gu = _gr.green_unocc(psi, eps, n_occ, mu, tau)
    go = _gr.green_occ(psi, eps, n_occ, mu, tau)
    p = psi[np.asarray(bands)]
    su = dv * dv * (p.conj() @ (gu * w_rr) @ p.T)
    so = -dv * dv * (p.conj() @ (go * w_rr) @ p.T)
    return su, so


def sigma_matrix_pair_tau(psi, eps, n_occ, mu, tau, w_gg, gvecs, n, lattice, bands):
    """Conventional route for the matrix: with a_nl(G) = dV sum_r exp(-iG.r)
    psi_l^*(r) psi_n(r),
        Su_nm(tau) = (1/Omega) sum_{l unocc} exp(-(eps_l-mu) tau) a_nl^H W~ a_ml
    and So_nm(-tau) likewise over occupied l with exp(+(eps_l-mu) tau) and a
    minus sign."""
    from . import gvec as _gv
    vol = abs(np.linalg.det(lattice))
    dv = vol / int(np.prod(n))
    pm = _gv.phase_matrix(gvecs, n, -1.0)
    a = [dv * (psi.conj() * psi[b][None, :]) @ pm.T for b in bands]     # each [N_b][N_chi]
    fu = np.exp(-(eps[n_occ:] - mu) * tau)
    fo = np.exp((eps[:n_occ] - mu) * tau)
    nb = len(bands)
    su = np.empty((nb, nb), dtype=np.complex128)
    so = np.empty((nb, nb), dtype=np.complex128)
    for i in range(nb):
        for k in range(nb):
            q = np.einsum("lg,gh,lh->l", a[i].conj(), w_gg, a[k]) / vol
            su[i, k] = (fu * q[n_occ:]).sum()
            so[i, k] = -(fo * q[:n_occ]).sum()
    return su, so


def sigma_matrix_iw(s_unocc, s_occ, C, S):
    """Sigma_nm(i omega_k) [N_n][N_n][N] from complex [N_n][N_n][N_tau] arrays:
    sum_j C_kj Sigma^c_nm(tau_j) + i sum_j S_kj Sigma^s_nm(tau_j)."""
    sc = 0.5 * (s_unocc + s_occ)
    ss = 0.5 * (s_unocc - s_occ)
    return sc @ C.T + 1j * (ss @ S.T)


def sigma_tau_from_iw(sig_iw, Cinv, Sinv):
    """Back to imaginary time (Eqs. INV_CT_FFT, INV_ST_FFT): the inverse of
    sigma_iw / sigma_matrix_iw.  Sigma(i omega) = C Sigma^c + i S Sigma^s with
    Sigma^c(tau), Sigma^s(tau) Hermitian in the band indices (real on the
    diagonal) and C, S real, so C Sigma^c is the Hermitian part of Sigma(i omega)
    and i S Sigma^s its anti-Hermitian part; then
        Sigma^c(tau_j) = sum_k Cinv_jk [Herm Sigma](i omega_k)
        Sigma^s(tau_j) = -i sum_k Sinv_jk [AntiHerm Sigma](i omega_k)
    and Sigma_unocc(tau) = Sigma^c + Sigma^s, Sigma_occ(-tau) = Sigma^c - Sigma^s.
    sig_iw is [N_n][N] (diagonal elements: Hermitian part = real part) or
    [N_n][N_n][N] (matrix).  Returns (Su, So) of the same shape."""
    sig = np.asarray(sig_iw)
    if sig.ndim == 2:
        herm, anti = sig.real.astype(np.complex128), 1j * sig.imag
    else:
        sh = sig.conj().transpose(1, 0, 2)
        herm, anti = 0.5 * (sig + sh), 0.5 * (sig - sh)
    sc = herm @ Cinv.T
    ss = -1j * (anti @ Sinv.T)
    su, so = sc + ss, sc - ss
    if sig.ndim == 2:
        return su.real, so.real
    return su, so
