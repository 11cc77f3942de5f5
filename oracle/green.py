"""Imaginary-time Green's functions (Sec. II.A.1).  Oracle only.

With energies measured from mu (the paper puts the Fermi level at zero),
Eqs. Green_occ and Green_unocc give, for tau > 0,

    G_occ(r,r',tau)   = sum_{i occ}   psi_i(r) psi_i^*(r') exp(+(eps_i - mu) tau)
    G_unocc(r,r',tau) = sum_{a unocc} psi_a(r) psi_a^*(r') exp(-(eps_a - mu) tau)

i.e. the paper's underline-G at -tau and minus its overline-G at +tau.  Both
decay because eps_i < mu < eps_a.
"""
import numpy as np


def green_occ(psi, eps, n_occ, mu, tau):
    """[N_r][N_r] complex: the band sum of Eq. Green_occ, written as a product."""
    s = np.exp((eps[:n_occ] - mu) * tau)
    p = psi[:n_occ]
    return (p.T * s) @ p.conj()


def green_unocc(psi, eps, n_occ, mu, tau):
    """[N_r][N_r] complex: the band sum of Eq. Green_unocc (sign dropped)."""
    s = np.exp(-(eps[n_occ:] - mu) * tau)
    p = psi[n_occ:]
    return (p.T * s) @ p.conj()


def green_occ_rows(psi, eps, n_occ, mu, tau, rows):
    """Rows r of G_occ only (for sampled checks at full size)."""
    s = np.exp((eps[:n_occ] - mu) * tau)
    p = psi[:n_occ]
    return (p[:, rows].T * s) @ p.conj()


def green_unocc_rows(psi, eps, n_occ, mu, tau, rows):
    s = np.exp(-(eps[n_occ:] - mu) * tau)
    p = psi[n_occ:]
    return (p[:, rows].T * s) @ p.conj()
