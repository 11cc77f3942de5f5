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


# ------------------------------------------------------------------ plane-wave form of G_k
# Sec. II.B keeps G_k in its plane-wave form and transforms it to the stripe
# only when needed.  With the bra-kets of Eq. notation_bra_ket,
#     <g|psi_ak>  = sum_{r in C}  exp(-i(k+g).r) psi_ak(r),
#     <psi_ak|G'> = sum_{R' in S} psi*_ak(R') exp(+i G'.R'),
# a Bloch orbital gives <psi_ak|G'> = N_k conj(<g'|psi_ak>) for G' = k + g' and
# zero for every other supercell vector (the sum over the cells L of
# exp(i(k'-k).L) is N_k delta_kk'), so G_k(g, G') lives on G' = k + g' only and
# is stored as an [N_r][N_r] block per k, g and g' in the cell's FFT order
# (exp(i g.r) on the cell grid depends on g modulo the grid).


def pw_coefficients_k(psi_k, n, nk):
    """<g|psi_ak> for every k, band and g of the cell's FFT grid (Eq.
    notation_bra_ket): the Bloch phase exp(-i k.r) applied, then the cell's
    discrete Fourier transform.  [N_k][N_b][N_r], g in FFT order."""
    n = np.asarray(n)
    nk = np.asarray(nk)
    i_cell = np.stack(np.meshgrid(*[np.arange(d) for d in n], indexing="ij"), -1).reshape(-1, 3)
    out = np.empty(psi_k.shape, dtype=np.complex128)
    for ki, kv in enumerate(k_list(nk)):
        ph = np.exp(-2j * np.pi * (i_cell @ (kv / (nk * n))))                 # exp(-i k.r), r in C
        x = (psi_k[ki] * ph[None, :]).reshape(-1, *n)
        out[ki] = np.fft.fftn(x, axes=(1, 2, 3)).reshape(psi_k.shape[1], -1)
    return out


def green_k_pw(c_k, eps_k, n_occ, mu, tau, nk, which):
    """G_k(g, k+g') in plane-wave form for every k (Eqs. G1_unocc_k, G1_occ_k),
    energies from mu and the signs of oracle.green:
        unocc: sum_{a unocc} <g|psi_ak> <psi_ak|k+g'> exp(-(eps_a - mu) tau)
        occ:   sum_{i occ}   <g|psi_ik> <psi_ik|k+g'> exp(+(eps_i - mu) tau)
    with <psi|k+g'> = N_k conj(<g'|psi>).  The unoccupied one is minus the
    paper's overline-G^(1)_k; the occupied one is the complex conjugate of its
    underline-G^*(1)_k (the same product in the index order of
    oracle.green.green_occ).  [N_k][N_r][N_r]."""
    n_k = int(np.prod(nk))
    out = np.empty((c_k.shape[0], c_k.shape[2], c_k.shape[2]), dtype=np.complex128)
    for ki in range(c_k.shape[0]):
        if which == "occ":
            s = np.exp((eps_k[ki, :n_occ] - mu) * tau)
            c = c_k[ki, :n_occ]
        else:
            s = np.exp(-(eps_k[ki, n_occ:] - mu) * tau)
            c = c_k[ki, n_occ:]
        out[ki] = (c.T * s) @ (n_k * c.conj())
    return out


def fft_g1_g2(gk_pw, n, nk, pw_index=None):
    """Eqs. FFT_G1 then FFT_G2 summed over k, as written (unnormalised sums):
        G(r, G')  = sum_g exp(+i(k+g).r) G_k(g, G')        r in C
        G(r, R')  = sum_{G'} G(r, G') exp(-i G'.R')         R' in S
    where G' runs over k + g' for the block of k.  pw_index (FFT positions)
    restricts g and g' to a plane-wave set; None takes the whole cell grid.
    [N_r][N_k N_r], columns in the supercell order of supercell_index."""
    n = np.asarray(n)
    nk = np.asarray(nk)
    ns = n * nk
    i_cell = np.stack(np.meshgrid(*[np.arange(d) for d in n], indexing="ij"), -1).reshape(-1, 3)
    i_sup = np.stack(np.meshgrid(*[np.arange(d) for d in ns], indexing="ij"), -1).reshape(-1, 3)
    sel = np.arange(int(np.prod(n))) if pw_index is None else np.asarray(pw_index)
    g = i_cell[sel]                                                            # FFT position = g mod n
    out = np.zeros((len(i_cell), len(i_sup)), dtype=np.complex128)
    for ki, kv in enumerate(k_list(nk)):
        m = kv[None, :] + nk[None, :] * g                                      # k + g as supercell triples
        to_r = np.exp(2j * np.pi * i_cell @ (m / ns).T)                        # exp(+i(k+g).r)   [N_r][n_pw]
        to_R = np.exp(-2j * np.pi * (m / ns) @ i_sup.T)                        # exp(-i(k+g').R') [n_pw][N_S]
        out += to_r @ gk_pw[ki][np.ix_(sel, sel)] @ to_R
    return out


def inv_fft_g1_g2(g_s, n, nk):
    """Eqs. INV_FFT_G1 then INV_FFT_G2, as written (unnormalised sums):
        G(r, G')    = sum_{R' in S} G(r, R') exp(+i G'.R')
        G_k(g, G')  = sum_{r in C} exp(-i(k+g).r) G(r, G')
    for G' = k + g' with every g, g' of the cell's FFT grid.  [N_k][N_r][N_r]."""
    n = np.asarray(n)
    nk = np.asarray(nk)
    ns = n * nk
    i_cell = np.stack(np.meshgrid(*[np.arange(d) for d in n], indexing="ij"), -1).reshape(-1, 3)
    i_sup = np.stack(np.meshgrid(*[np.arange(d) for d in ns], indexing="ij"), -1).reshape(-1, 3)
    out = []
    for kv in k_list(nk):
        m = kv[None, :] + nk[None, :] * i_cell
        from_R = np.exp(2j * np.pi * i_sup @ (m / ns).T)                       # exp(+i(k+g').R') [N_S][N_r]
        from_r = np.exp(-2j * np.pi * (m / ns) @ i_cell.T)                     # exp(-i(k+g).r)   [N_r][N_r]
        out.append(from_r @ (g_s @ from_R))
    return np.array(out)


def green_stripe_pw(psi_k, eps_k, n_occ, mu, tau, n, nk, pw_index=None):
    """G_occ and G_unocc on the stripe through the plane-wave form (Sec. II.B):
    coefficients, G_k(g, k+g') per k, then Eqs. FFT_G1, FFT_G2.  Each of the two
    transforms inverts an unnormalised bra-ket (a factor N_r from the cell
    transform of the coefficients) and the ket over S carries N_k, so the
    stripe of green_stripe (cell-normalised orbitals, 1/N_k) is the transformed
    sum divided by N_r^2 N_k^2.  [N_r][N_k N_r] each."""
    c_k = pw_coefficients_k(psi_k, n, nk)
    scale = 1.0 / (float(np.prod(n)) ** 2 * float(np.prod(nk)) ** 2)
    go = scale * fft_g1_g2(green_k_pw(c_k, eps_k, n_occ, mu, tau, nk, "occ"), n, nk, pw_index)
    gu = scale * fft_g1_g2(green_k_pw(c_k, eps_k, n_occ, mu, tau, nk, "unocc"), n, nk, pw_index)
    return go, gu


def chi_q_tau_pw(psi_k, eps_k, n_occ, mu, tau, n, nk, lattice, gvecs, pw_index=None):
    """chi_q(g, g', tau) for every q with G on the stripe taken from its
    plane-wave form (green_stripe_pw), then the stripe product and chi_q."""
    go, gu = green_stripe_pw(psi_k, eps_k, n_occ, mu, tau, n, nk, pw_index)
    return chi_q(-2.0 * go * gu.conj(), n, nk, lattice, gvecs)
