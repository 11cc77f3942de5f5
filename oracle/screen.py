"""Screened interaction (Sec. II.C steps (iii)-(v)).  Oracle only.

With the symmetrised kernel v^{1/2}(G) = sqrt(4 pi)/|G| (Eq. bareV):

    chi~   = v^{1/2} chi v^{1/2}
    eps~   = 1 - chi~                          (Eq. die, symmetrised)
    W      = v^{1/2} eps~^{-1} v^{1/2}        (Eq. W_tot)
    W~     = W - v = v^{1/2} (eps~^{-1} - 1) v^{1/2}
           = v^{1/2} [eps~^{-1} chi~] v^{1/2}  (Eq. W_correlated)

The solve uses the LAPACK routine behind numpy.linalg.solve as one step.
"""
import numpy as np

from . import gvec as _gv


def screen_one(chi_w, vhalf):
    """W~(G,G',i omega) from chi(G,G',i omega) at one frequency."""
    ct = vhalf[:, None] * chi_w * vhalf[None, :]
    eps_t = np.eye(len(vhalf)) - ct
    x = np.linalg.solve(eps_t, ct)
    return vhalf[:, None] * x * vhalf[None, :]


def screen(chi_w, vhalf):
    return np.stack([screen_one(c, vhalf) for c in chi_w])


def inverse_ct(w_omega, Cinv):
    """Eq. CT_W: W~(i tau_j) = sum_k xi_jk cos(tau_j omega_k) W~(i omega_k)."""
    return np.tensordot(Cinv, w_omega, axes=(1, 0))


def w_rows_to_r(w_gg, gvecs, n):
    """First step of Eq. FFTW: W~(r,G') = sum_G exp(+i G.r) W~(G,G')."""
    pm = _gv.phase_matrix(gvecs, n, +1.0)            # exp(+i G.r), [N_chi][N_r]
    return pm.T @ w_gg


def w_cols_to_r(w_rg, gvecs, n, lattice):
    """Second step of Eq. FFTW with the 1/Omega of the inverse transform:
    W~(r,R') = (1/Omega) sum_G' W~(r,G') exp(-i G'.R')."""
    vol = abs(np.linalg.det(lattice))
    pm = _gv.phase_matrix(gvecs, n, -1.0)
    return (w_rg @ pm) / vol


def w_rr(w_gg, gvecs, n, lattice):
    """W~(r,R') = (1/Omega) sum_{G,G'} exp(iG.r) W~(G,G') exp(-iG'.R')."""
    return w_cols_to_r(w_rows_to_r(w_gg, gvecs, n), gvecs, n, lattice)
