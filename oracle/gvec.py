"""Reciprocal lattice, the G set of chi/W and the bare Coulomb kernel.  Oracle only.

Grid convention: r index = (i1*n2 + i2)*n3 + i3, fractional position
(i1/n1, i2/n2, i3/n3); a G vector is an integer triple g with
G = sum_d g_d b_d, so G.r = 2 pi sum_d g_d i_d / n_d.
"""
import numpy as np


def reciprocal(lattice):
    """Rows b_d with a_d . b_e = 2 pi delta_de."""
    return 2.0 * np.pi * np.linalg.inv(np.asarray(lattice, dtype=np.float64)).T


def g_set(n, n_chi):
    """The N_chi lowest G: integer triples g_d in [-n_d/2, n_d/2), ordered by
    (g1^2+g2^2+g3^2, g1, g2, g3), the cutoff sphere of Eq. FFTX1 with a
    deterministic tie-break.  Written as a plain sort over all grid points."""
    pts = []
    for g1 in range(-(n[0] // 2), n[0] - n[0] // 2):
        for g2 in range(-(n[1] // 2), n[1] - n[1] // 2):
            for g3 in range(-(n[2] // 2), n[2] - n[2] // 2):
                pts.append((g1 * g1 + g2 * g2 + g3 * g3, g1, g2, g3))
    pts.sort()
    return np.array([p[1:] for p in pts[:n_chi]], dtype=np.int64)


def fft_index(gvecs, n):
    """Position of each g on the FFT grid: ((g1 mod n1)*n2 + g2 mod n2)*n3 + g3 mod n3."""
    g = np.asarray(gvecs) % np.asarray(n)
    return (g[:, 0] * n[1] + g[:, 1]) * n[2] + g[:, 2]


def cartesian(gvecs, lattice):
    return np.asarray(gvecs, dtype=np.float64) @ reciprocal(lattice)


def v_sqrt(gvecs, lattice):
    """sqrt of the bare Coulomb kernel, v(G,G') = 4 pi / (|G||G'|) (Eq. bareV,
    e = 1, Gamma point).  The G = 0 entry is set to 0: the paper gives no
    head/wings treatment for insulators, so head and wings of W~ are dropped."""
    gc = cartesian(gvecs, lattice)
    norm = np.sqrt((gc ** 2).sum(1))
    out = np.zeros(len(gc))
    nz = norm > 0
    out[nz] = np.sqrt(4.0 * np.pi) / norm[nz]
    return out


def phase_matrix(gvecs, n, sign):
    """P[j][r] = exp(sign * i G_j . r) over the grid, built axis by axis."""
    i = [np.arange(nd) for nd in n]
    g = np.asarray(gvecs)
    e = [np.exp(sign * 2j * np.pi * np.outer(g[:, d], i[d]) / n[d]) for d in range(3)]
    p = e[0][:, :, None, None] * e[1][:, None, :, None] * e[2][:, None, None, :]
    return p.reshape(len(g), -1)
