"""Quasiparticle energies and spectral functions from the continued
self-energy (Sec. II.E.2, Eqs. QP, GWQP, Z, A).  Oracle only: test
infrastructure, never imported by the product path.

Sigma_n(omega) is the correlation self-energy of band n continued to the real
axis by Thiele's approximant through the nodes z_k = i omega_k (thiele.py),
with the real frequency measured from mu, as in pipeline.continue_sigma.  The
frequency-independent part of the paper's Sigma_nk (bare exchange,
core-valence exchange) and <psi_n|T + V_ne + V_H|psi_n> are the caller's input
v_n, so that

    DeltaSigma_n(omega) = v_n + Sigma_n(omega - mu) - eps_n.

Linearised QP equation (Eq. QP expanded to first order around eps_n, then
solved for E; Eqs. GWQP and Z):

    Z_n   = 1 / (1 - d Re Sigma_n / d omega |_{eps_n})
    E_n   = eps_n + Z_n Re DeltaSigma_n(eps_n)

Spectral function (Eq. A):

    A_n(omega) = (1/pi) |Im DeltaSigma_n(omega)|
                 / ((omega - eps_n - Re DeltaSigma_n(omega))^2 + (Im DeltaSigma_n(omega))^2)
"""
import numpy as np

from . import thiele as _th


def _coeffs(sig_iw, omega):
    z = 1j * np.asarray(omega, dtype=np.float64)
    return z, [_th.coefficients(z, row) for row in np.atleast_2d(sig_iw)]


def linearized(sig_iw, omega, eps_n, mu, v_n):
    """(E_n, Z_n, Sigma_n(eps_n), dSigma_n/domega at eps_n) for every band;
    sig_iw [N_n][N] at the nodes i omega_k."""
    z, coeffs = _coeffs(sig_iw, omega)
    nb = len(coeffs)
    e_qp = np.empty(nb)
    zf = np.empty(nb)
    s_eps = np.empty(nb, dtype=np.complex128)
    ds = np.empty(nb, dtype=np.complex128)
    for b in range(nb):
        x = np.array([eps_n[b] - mu], dtype=np.complex128)
        s_eps[b] = _th.evaluate(coeffs[b], z, x)[0]
        ds[b] = _th.derivative(coeffs[b], z, x)[0]
        zf[b] = 1.0 / (1.0 - ds[b].real)
        e_qp[b] = eps_n[b] + zf[b] * (v_n[b] + s_eps[b].real - eps_n[b])
    return e_qp, zf, s_eps, ds


def spectral(sig_iw, omega, eps_n, mu, v_n, w):
    """A_n(w) [N_n][len(w)] at real energies w (absolute, same zero as eps)."""
    z, coeffs = _coeffs(sig_iw, omega)
    w = np.asarray(w, dtype=np.float64)
    out = np.empty((len(coeffs), len(w)))
    for b in range(len(coeffs)):
        s = _th.evaluate(coeffs[b], z, (w - mu).astype(np.complex128))
        d = v_n[b] + s - eps_n[b]
        out[b] = np.abs(d.imag) / np.pi / ((w - eps_n[b] - d.real) ** 2 + d.imag ** 2)
    return out
