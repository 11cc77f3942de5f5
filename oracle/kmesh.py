"""k-point sampling: chi0 on a Gamma-centred k mesh through the supercell
stripe (Sec. II.A "Spatial fast Fourier transformation", Eqs. FFT_G1, FFT_G2 and
their inverses).  Oracle only (test infrastructure, not the product path).

Conventions.  The supercell S holds nk_1 x nk_2 x nk_3 cells; a point R = r + L
with r on the cell grid (i_1, i_2, i_3) and L = sum_d l_d a_d has supercell
grid index I_d = i_d + n_d l_d, linear ((I_1 nS_2 + I_2) nS_3 + I_3) with
nS_d = nk_d n_d.  k = sum_d (k_d / nk_d) b_d, k_d in [0, nk_d); q likewise.
A supercell reciprocal vector q + g is the integer triple m_d = k_d + nk_d g_d,
(q + g).R = 2 pi sum_d m_d I_d / nS_d.

Bloch orbitals satisfy psi_nk(r + L) = exp(i k.L) psi_nk(r), so the Green's
function on the stripe r in C, R' in S is
    G(r, r'+L, tau) = (1/N_k) sum_k exp(-i k.L) G_k(r, r', tau)
(the 1/N_k is the normalisation of the orbitals over S), chi(r, R') follows
the Gamma-point form chi(r, R') = -2 G_occ(r, R') conj(G_unocc(r, R')) (the
index order G_occ(r,r') G_unocc(r',r) of the spin-degenerate product), and
    chi_q(g, g') = (dV^2 / Omega) sum_{r in C} exp(-i(q+g).r)
                                  sum_{R' in S} chi(r, R') exp(+i(q+g').R'),
which is the q-diagonal block of the Gamma-point chi of the supercell (the
blocks q != q' vanish by translation symmetry; tests/test_oracle_kmesh.py).
"""
import numpy as np

from . import chi as _chi
from . import green as _gr


def k_list(nk):
    """Integer k_d triples in index order (k1*nk2 + k2)*nk3 + k3."""
    return np.array([(a, b, c) for a in range(nk[0]) for b in range(nk[1]) for c in range(nk[2])], dtype=np.int64)


def supercell_index(n, nk):
    """pos[l][r]: supercell grid index of r + L for cell point r and lattice vector l (index order of k_list)."""
    ls = k_list(nk)
    ns = np.asarray(n) * np.asarray(nk)
    i = np.stack(np.meshgrid(*[np.arange(nd) for nd in n], indexing="ij"), -1).reshape(-1, 3)
    out = np.empty((len(ls), len(i)), dtype=np.int64)
    for li, l in enumerate(ls):
        big = i + np.asarray(n) * l
        out[li] = (big[:, 0] * ns[1] + big[:, 1]) * ns[2] + big[:, 2]
    return out


def green_stripe(psi_k, eps_k, n_occ, mu, tau, n, nk):
    """G_occ and G_unocc on the stripe, [N_r][N_k N_r] (columns: supercell index of R')."""
    ks = k_list(nk)
    pos = supercell_index(n, nk)
    nr = int(np.prod(n))
    n_k = len(ks)
    # ph[l][k] = exp(-i k.L_l) / N_k; G_L = sum_k ph[l][k] G_k for every lattice vector L at once
    ph = np.exp(-2j * np.pi * (ks / np.asarray(nk)) @ ks.T).T / n_k
    go = np.zeros((nr, n_k * nr), dtype=np.complex128)
    gu = np.zeros((nr, n_k * nr), dtype=np.complex128)
    for which, out in (("occ", go), ("unocc", gu)):
        gk = np.stack([(_gr.green_occ if which == "occ" else _gr.green_unocc)(psi_k[ki], eps_k[ki], n_occ, mu, tau)
                       for ki in range(n_k)])                                   # [N_k][N_r][N_r]
        gl = (ph @ gk.reshape(n_k, -1)).reshape(n_k, nr, nr)                   # [N_L][N_r][N_r]
        for li in range(n_k):
            out[:, pos[li]] = gl[li]
    return go, gu


def chi_q(chi_s, n, nk, lattice, gvecs):
    """chi_q(g, g') for every q from chi(r, R') on the stripe: [N_q][N_chi][N_chi]."""
    n = np.asarray(n)
    nk = np.asarray(nk)
    ns = n * nk
    vol = abs(np.linalg.det(lattice))
    dv = vol / int(np.prod(n))
    i_cell = np.stack(np.meshgrid(*[np.arange(d) for d in n], indexing="ij"), -1).reshape(-1, 3)
    i_sup = np.stack(np.meshgrid(*[np.arange(d) for d in ns], indexing="ij"), -1).reshape(-1, 3)
    out = []
    for q in k_list(nk):
        m = q[None, :] + nk[None, :] * np.asarray(gvecs)               # [N_chi][3]
        p_row = np.exp(-2j * np.pi * (m / ns) @ i_cell.T)               # exp(-i(q+g).r), r in C
        p_col = np.exp(-2j * np.pi * (m / ns) @ i_sup.T)                # exp(-i(q+g').R'), R' in S
        out.append((dv * dv / vol) * (p_row @ chi_s @ p_col.conj().T))
    return np.array(out)


def chi_q_rows(chi_s, n, nk, lattice, gvecs, qs, rows):
    """chi_q(g_row, g') for the listed q (indices in k_list order) and G-set rows
    only, every g': the same sums as chi_q, [len(qs)][len(rows)][N_chi]."""
    n = np.asarray(n)
    nk = np.asarray(nk)
    ns = n * nk
    vol = abs(np.linalg.det(lattice))
    dv = vol / int(np.prod(n))
    i_cell = np.stack(np.meshgrid(*[np.arange(d) for d in n], indexing="ij"), -1).reshape(-1, 3)
    i_sup = np.stack(np.meshgrid(*[np.arange(d) for d in ns], indexing="ij"), -1).reshape(-1, 3)
    kl = k_list(nk)
    out = []
    for qi in qs:
        q = kl[qi]
        m = q[None, :] + nk[None, :] * np.asarray(gvecs)
        p_row = np.exp(-2j * np.pi * (m[rows] / ns) @ i_cell.T)
        p_col = np.exp(-2j * np.pi * (m / ns) @ i_sup.T)
        out.append((dv * dv / vol) * ((p_row @ chi_s) @ p_col.conj().T))
    return np.array(out)


def chi_q_tau(psi_k, eps_k, n_occ, mu, tau, n, nk, lattice, gvecs):
    """chi_q(g, g', tau) for every q, by the stripe route above."""
    go, gu = green_stripe(psi_k, eps_k, n_occ, mu, tau, n, nk)
    return chi_q(-2.0 * go * gu.conj(), n, nk, lattice, gvecs)


def supercell_orbitals(psi_k, eps_k, n_occ, n, nk):
    """The same system as a Gamma-point problem of the supercell: orbitals
    psi_nk(r + L) / sqrt(N_k) = exp(i k.L) psi_nk(r) / sqrt(N_k) on the supercell
    grid, occupied ones first.  Returns (psi_S [N_k N_b][N_S], eps_S, n_occ_S)."""
    ks = k_list(nk)
    pos = supercell_index(n, nk)
    n_k = len(ks)
    nr = int(np.prod(n))
    rows, eps = [], []
    for part in (slice(0, n_occ), slice(n_occ, psi_k.shape[1])):
        for ki, kv in enumerate(ks):
            for b in range(psi_k.shape[1])[part]:
                v = np.zeros(n_k * nr, dtype=np.complex128)
                for li, l in enumerate(ks):
                    v[pos[li]] = np.exp(2j * np.pi * np.sum(kv * l / np.asarray(nk))) * psi_k[ki, b]
                rows.append(v / np.sqrt(n_k))
                eps.append(eps_k[ki, b])
    return np.array(rows), np.array(eps), n_k * n_occ


def supercell_gvecs(gvecs, nk):
    """Integer triples m = k + nk g of the supercell for every q (outer) and g (inner)."""
    return np.concatenate([q[None, :] + np.asarray(nk)[None, :] * np.asarray(gvecs) for q in k_list(nk)])


def w_stripe(w_q, n, nk, lattice, gvecs):
    """W~(r, R') on the stripe from W~_q(g, g') for every q:
    (1/Omega_S) sum_q sum_{g,g'} exp(+i(q+g).r) W~_q(g,g') exp(-i(q+g').R')
    (Eq. FFTW on the supercell, whose W~ is block-diagonal in q)."""
    n = np.asarray(n)
    nk = np.asarray(nk)
    ns = n * nk
    vol_s = abs(np.linalg.det(lattice)) * int(np.prod(nk))
    i_cell = np.stack(np.meshgrid(*[np.arange(d) for d in n], indexing="ij"), -1).reshape(-1, 3)
    i_sup = np.stack(np.meshgrid(*[np.arange(d) for d in ns], indexing="ij"), -1).reshape(-1, 3)
    out = np.zeros((len(i_cell), len(i_sup)), dtype=np.complex128)
    for qi, q in enumerate(k_list(nk)):
        m = q[None, :] + nk[None, :] * np.asarray(gvecs)
        p_row = np.exp(2j * np.pi * i_cell @ (m / ns).T)       # exp(+i(q+g).r)   [N_r][N_chi]
        p_col = np.exp(-2j * np.pi * (m / ns) @ i_sup.T)       # exp(-i(q+g').R') [N_chi][N_S]
        out += p_row @ w_q[qi] @ p_col
    return out / vol_s


def bloch_extend(psi, kv, n, nk):
    """psi_nk(r + L) = exp(i k.L) psi_nk(r) on the supercell grid (cell normalisation)."""
    pos = supercell_index(n, nk)
    out = np.zeros(pos.size, dtype=np.complex128)
    for li, l in enumerate(k_list(nk)):
        out[pos[li]] = np.exp(2j * np.pi * np.sum(np.asarray(kv) * l / np.asarray(nk))) * psi
    return out


def sigma_k_tau(psi_k, eps_k, n_occ, mu, tau, w_s, n, nk, lattice, bands_nk):
    """(Sigma_unocc_nk(tau), Sigma_occ_nk(-tau)) for the (band, k index) pairs on
    the stripe (Eqs. Sigma_rr, Sigma_occ_reduce first term, with Bloch orbitals):
        Sigma_unocc = +dV^2 sum_{r in C} sum_{R' in S} psi*_nk(r) G_unocc(r,R') W~(r,R') psi_nk(R'),
    likewise occupied with a minus sign; real parts."""
    dv = abs(np.linalg.det(lattice)) / int(np.prod(n))
    go, gu = green_stripe(psi_k, eps_k, n_occ, mu, tau, n, nk)
    ks = k_list(nk)
    su = np.empty(len(bands_nk))
    so = np.empty(len(bands_nk))
    for i, (b, k) in enumerate(bands_nk):
        row = psi_k[k, b]
        col = bloch_extend(row, ks[k], n, nk)
        su[i] = (dv * dv * (row.conj() @ ((gu * w_s) @ col))).real
        so[i] = -(dv * dv * (row.conj() @ ((go * w_s) @ col))).real
    return su, so
