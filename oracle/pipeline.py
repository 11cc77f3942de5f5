"""The whole hot path in the paper's order (Fig. 1 steps (1)-(11)).  Oracle only.

chi0(i omega) -> W~(i omega) -> W~(i tau) -> W~(r,r',tau) -> Sigma_nn(tau)
-> Sigma_nn(i omega) -> Sigma_nn(omega) by Thiele continuation.
"""
import numpy as np

from . import chi as _chi
from . import green as _gr
from . import grids as _grids
from . import gvec as _gv
from . import screen as _sc
from . import sigma as _sg
from . import thiele as _th


def setup(p):
    """Host setup of a problem: G set, index map, v^{1/2}, transform matrices."""
    gvecs = _gv.g_set(p.n, p.n_chi)
    mats = _grids.transform_matrices(p.tau, p.omega, p.x_min, p.x_max, p.n_x, p.ridge)
    return {"gvecs": gvecs, "fft_index": _gv.fft_index(gvecs, p.n),
            "vhalf": _gv.v_sqrt(gvecs, p.lattice), **mats}


def chi_tau(p, s, j):
    """chi(G,G',tau_j) through the real-space product and the spatial transform."""
    go = _gr.green_occ(p.psi, p.eps, p.n_occ, p.mu, p.tau[j])
    gu = _gr.green_unocc(p.psi, p.eps, p.n_occ, p.mu, p.tau[j])
    return _chi.chi_gg(_chi.chi_rr(go, gu), s["gvecs"], p.n, p.lattice)


def chi0_omega(p, s):
    """[N_omega][N_chi][N_chi] chi0(G,G',i omega_k) (Eq. CTX)."""
    chit = np.stack([chi_tau(p, s, j) for j in range(len(p.tau))])
    return _chi.ct(chit, s["C"]), chit


def w_tau(p, s, chi_w):
    """W~(G,G',i tau_j) from chi0(i omega): screening then inverse CT."""
    ww = _sc.screen(chi_w, s["vhalf"])
    return _sc.inverse_ct(ww, s["Cinv"]), ww


def sigma_from_w(p, s, wt, route="spacetime", m=None):
    """(Sigma_unocc, Sigma_occ) arrays [N_n][N_tau] from W~(G,G',tau)."""
    dv = p.volume / p.n_r
    nb = len(p.bands)
    su = np.empty((nb, len(p.tau)))
    so = np.empty((nb, len(p.tau)))
    for j in range(len(p.tau)):
        if route == "spacetime":
            wrr = _sc.w_rr(wt[j], s["gvecs"], p.n, p.lattice)
            su[:, j], so[:, j] = _sg.sigma_tau(p.psi, p.eps, p.n_occ, p.mu, p.tau[j], wrr,
                                               p.bands, dv)
        else:
            su[:, j], so[:, j] = _sg.sigma_pair_tau(p.psi, p.eps, p.n_occ, p.mu, p.tau[j],
                                                    wt[j], s["gvecs"], p.n, p.lattice,
                                                    p.bands)
    return su, so


def continue_sigma(p, sig_iw, w_real):
    """Sigma_nn(omega) at real frequencies (measured from mu) by Thiele continuation
    through the nodes z_k = i omega_k."""
    z = 1j * np.asarray(p.omega)
    out = np.empty((sig_iw.shape[0], len(w_real)), dtype=np.complex128)
    for b in range(sig_iw.shape[0]):
        a = _th.coefficients(z, sig_iw[b])
        out[b] = _th.evaluate(a, z, np.asarray(w_real, dtype=np.complex128))
    return out


def run(p, w_real=None):
    """End to end.  Returns a dict with every intermediate the GPU path exposes."""
    s = setup(p)
    chi_w, chit = chi0_omega(p, s)
    wt, ww = w_tau(p, s, chi_w)
    su, so = sigma_from_w(p, s, wt)
    sig = _sg.sigma_iw(su, so, s["C"], s["S"])
    out = {"setup": s, "chi_tau": chit, "chi_w": chi_w, "W_w": ww, "W_tau": wt,
           "sigma_unocc": su, "sigma_occ": so, "sigma_iw": sig}
    if w_real is not None:
        out["sigma_real"] = continue_sigma(p, sig, w_real)
    return out
