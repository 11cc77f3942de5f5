"""Seeded synthetic inputs for the space-time GW hot path.

This module only *draws* problems: Kohn-Sham-like orbitals on a real-space
grid, their eigenvalues, the chemical potential, the imaginary-time grid and
the list of bands whose self-energy is wanted.  It holds none of the method's
arithmetic (no Green's functions, transforms, weight fits or screening), so
both the FP64 oracle and the CUDA path can take their inputs from here.

Shapes follow the semiconductor cells of the paper (Si lattice constant
10.26 bohr, eight atoms per cubic cell, bands far above the occupied ones,
16-20 time points; Sec. III), at the sizes of the benchmark workloads:

* ``gamma_toy``  -- 12^3 grid, 16 occupied + 112 unoccupied *real* orbitals on
  the lowest 128 real plane-wave combinations, 8 log-spaced tau in [0.05, 40].
* ``si8``        -- 24^3 grid, 16 + 1008 complex orbitals on the lowest 1024
  plane waves, gap 0.04 Ha, 16 tau points.
* ``si64``       -- 36^3 grid, 128 + 4096 complex orbitals (64-atom cell).
* ``tiny``/``small`` -- reduced versions for tests.

Orbitals are psi_n(r) = Omega^{-1/2} sum_p U_pn phi_p(r) with U a seeded
random unitary (QR of a Gaussian matrix) and phi_p plane waves (or their
real cos/sin combinations), so that dV sum_r psi_n^* psi_m = delta_nm exactly
on the grid.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Problem:
    """One synthetic system.  Energies in Hartree, lengths in bohr."""

    n: tuple                 # FFT grid (n1, n2, n3); r index = (i1*n2+i2)*n3+i3
    lattice: np.ndarray      # 3x3, row d = lattice vector a_d
    psi: np.ndarray          # [N_b][N_r] complex128, band-major
    eps: np.ndarray          # [N_b] ascending
    n_occ: int
    mu: float
    tau: np.ndarray          # [N] ascending, > 0
    omega: np.ndarray        # [N] ascending, omega_k = 1 / tau_{N-1-k}
    bands: np.ndarray        # [N_n] band indices whose Sigma_nn is wanted
    n_chi: int               # size of the G set of chi / W
    x_min: float             # transition-energy window of the weight fit
    x_max: float
    n_x: int = 4000
    ridge: float = 1e-6
    real: bool = False
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n_r(self) -> int:
        return int(np.prod(self.n))

    @property
    def n_b(self) -> int:
        return self.psi.shape[0]

    @property
    def volume(self) -> float:
        return abs(float(np.linalg.det(self.lattice)))


def on_grids(p, tau, omega, ridge=0.0):
    """The same problem on other imaginary-time / frequency grids (for example
    the optimised grids of the method's host setup), with the ridge of the
    weight fit those grids want.  Pure data: no arithmetic on the grids."""
    import dataclasses
    return dataclasses.replace(p, tau=np.asarray(tau, dtype=np.float64).copy(),
                               omega=np.asarray(omega, dtype=np.float64).copy(), ridge=float(ridge))


def _sorted_lattice_points(n):
    """Integer triples g_d in [-n_d/2, n_d/2) ordered by (|g|^2, g1, g2, g3)."""
    ax = [np.arange(-(nd // 2), nd - nd // 2) for nd in n]
    g = np.stack(np.meshgrid(*ax, indexing="ij"), -1).reshape(-1, 3)
    key = (g ** 2).sum(1)
    order = np.lexsort((g[:, 2], g[:, 1], g[:, 0], key))
    return g[order]


def _plane_waves_on_grid(n, gs):
    """exp(2 pi i sum_d g_d i_d / n_d) on the grid, [len(gs)][N_r]."""
    i = [np.arange(nd) for nd in n]
    e = [np.exp(2j * np.pi * np.outer(gs[:, d], i[d]) / n[d]) for d in range(3)]
    pw = e[0][:, :, None, None] * e[1][:, None, :, None] * e[2][:, None, None, :]
    return pw.reshape(len(gs), -1)


def _real_basis(n, n_b):
    """Real basis {1, sqrt2 cos(G.r), sqrt2 sin(G.r)} over +-G pairs, truncated."""
    gs = _sorted_lattice_points(n)
    seen = set()
    rows = []
    for g in gs:
        t = tuple(int(x) for x in g)
        if t in seen:
            continue
        seen.add(t)
        seen.add(tuple(-x for x in t))
        pw = _plane_waves_on_grid(n, g[None, :])[0]
        if t == (0, 0, 0):
            rows.append(pw.real.copy())
        else:
            rows.append(np.sqrt(2.0) * pw.real)
            rows.append(np.sqrt(2.0) * pw.imag)
        if len(rows) >= n_b:
            break
    return np.array(rows[:n_b])


def make_problem(n, a, n_occ, n_unocc, eps_occ, eps_unocc, mu, n_tau, seed,
                 tau_range=None, n_bands_sigma=4, n_chi=None, real=False,
                 pin_edges=False, name=""):
    """Draw one problem.

    n: grid; a: cubic lattice constant (float) or 3 orthorhombic lengths.
    tau_range: (t0, t1) for log-spaced tau; default (0.1/D_max, 3/D_min) with
    D_min the gap and D_max the spectral width.
    """
    rng = np.random.default_rng(seed)
    n = tuple(int(x) for x in n)
    lengths = np.broadcast_to(np.asarray(a, dtype=float), (3,))
    lattice = np.diag(lengths)
    vol = float(np.prod(lengths))
    n_b = n_occ + n_unocc
    if real:
        basis = _real_basis(n, n_b)
        U, _ = np.linalg.qr(rng.standard_normal((n_b, n_b)))
        psi = (U.T @ basis) / np.sqrt(vol)
        psi = psi.astype(np.complex128)
    else:
        gs = _sorted_lattice_points(n)[:n_b]
        basis = _plane_waves_on_grid(n, gs)
        z = rng.standard_normal((n_b, n_b)) + 1j * rng.standard_normal((n_b, n_b))
        U, _ = np.linalg.qr(z)
        psi = (U.T @ basis) / np.sqrt(vol)
    eo = np.sort(rng.uniform(eps_occ[0], eps_occ[1], n_occ))
    eu = np.sort(rng.uniform(eps_unocc[0], eps_unocc[1], n_unocc))
    if pin_edges:
        eo[-1] = eps_occ[1]
        eu[0] = eps_unocc[0]
    eps = np.concatenate([eo, eu])
    gap = eu[0] - eo[-1]
    width = eps[-1] - eps[0]
    if tau_range is None:
        tau_range = (0.1 / width, 3.0 / gap)
    tau = np.geomspace(tau_range[0], tau_range[1], n_tau)
    omega = 1.0 / tau[::-1]
    half = n_bands_sigma // 2
    bands = np.arange(n_occ - half, n_occ - half + n_bands_sigma)
    x_min = float(np.min(np.abs(eps - mu)))
    x_max = float(width + np.max(np.abs(eps - mu)))
    return Problem(n=n, lattice=lattice, psi=psi, eps=eps, n_occ=n_occ, mu=float(mu),
                   tau=tau, omega=omega, bands=bands,
                   n_chi=int(np.prod(n)) if n_chi is None else int(n_chi),
                   x_min=x_min, x_max=x_max, real=real, name=name)


def gamma_toy(seed=1):
    """12^3, 16+112 real orbitals, mu=-0.04, 8 tau in [0.05,40]."""
    return make_problem((12, 12, 12), 10.26, 16, 112, (-0.6, -0.1), (0.02, 3.0), -0.04, 8,
                        seed, tau_range=(0.05, 40.0), n_bands_sigma=4, real=True,
                        name="gamma_toy_12^3_real_128b")


def si8(seed=2):
    """24^3, 16+1008 complex orbitals, gap 0.04 Ha (HOMO 0, LUMO 0.04), 16 tau."""
    return make_problem((24, 24, 24), 10.26, 16, 1008, (-0.5, 0.0), (0.04, 4.0), 0.02, 16,
                        seed, n_bands_sigma=8, pin_edges=True, name="si8_24^3_1024b")


def mid(seed=4):
    """16^3, 32+480 complex orbitals, 8 tau: the si8 recipe at a size whose
    per-step device footprint (~3.5 GB) suits a full profiler capture."""
    return make_problem((16, 16, 16), 10.26 * 16 / 24, 32, 480, (-0.5, 0.0), (0.04, 4.0), 0.02, 8,
                        seed, n_bands_sigma=8, pin_edges=True, name="mid_16^3_512b")


def si64(seed=3):
    """36^3, 128+4096 complex orbitals, chi on the lowest 8192 G, 20 tau."""
    return make_problem((36, 36, 36), 20.52, 128, 4096, (-0.5, 0.0), (0.03, 5.0), 0.015, 20,
                        seed, n_bands_sigma=32, n_chi=8192, pin_edges=True,
                        name="si64_36^3_4224b")


def k8448(seed=3):
    """The 36^3 workload's bands (128 + 4096, so K = 8448 real per G element) and
    energy windows on a 20^3 grid with 4 tau and chi on 2048 G: the G-formation
    kernels at their full K, on a device footprint that suits a profiler capture."""
    return make_problem((20, 20, 20), 20.52 * 20 / 36, 128, 4096, (-0.5, 0.0), (0.03, 5.0), 0.015, 4,
                        seed, n_bands_sigma=32, n_chi=2048, pin_edges=True, name="k8448_20^3_4224b")


def tiny(seed=11, n=(6, 6, 6), a=(6.0, 6.5, 7.0), n_occ=4, n_unocc=20, n_tau=6, real=False,
         n_chi=None):
    """Few-second case for the oracle: orthorhombic cell, ragged sizes allowed."""
    return make_problem(n, a, n_occ, n_unocc, (-0.6, -0.05), (0.05, 2.0), 0.0, n_tau, seed,
                        n_bands_sigma=4, real=real, n_chi=n_chi, pin_edges=True,
                        name="tiny_%dx%dx%d" % n)


def screening_chi(n_chi, n_w=2, rank=None, seed=60, decay=64.0):
    """Seeded Hermitian negative semidefinite matrices shaped like chi0(G,G',i omega)
    for screening tests at sizes where the oracle cannot form chi0 itself:
    chi_w = -B_w B_w^H / rank with B_w [n_chi][rank] complex Gaussian rows damped
    as (1 + j/decay)^-1 along the G-set index j (pair densities fall off with |G|).
    Returns [n_w][n_chi][n_chi] complex128; the caller scales each matrix to the
    screening strength it wants."""
    rng = np.random.default_rng(seed)
    rank = n_chi // 2 if rank is None else int(rank)
    damp = 1.0 / (1.0 + np.arange(n_chi) / float(decay))
    out = np.empty((n_w, n_chi, n_chi), dtype=np.complex128)
    for w in range(n_w):
        b = (rng.standard_normal((n_chi, rank)) + 1j * rng.standard_normal((n_chi, rank))) * damp[:, None]
        out[w] = -(b @ b.conj().T) / rank
    return out


def serve_mix(count=6, seed=40, n_chi_cap=1536):
    """Systems of uneven sizes for the request server: grid n^3 with n in
    {12, 16, 20} (cell a = n * 10.26 / 12), 128-512 complex bands (multiples of
    64, one eighth occupied), 8, 12 or 16 tau points, the G set capped at
    n_chi_cap, Sigma for 4 bands.  The si8 energy windows and gap."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.choice([12, 16, 20]))
        n_b = int(rng.choice(np.arange(128, 513, 64)))
        n_occ = n_b // 8
        n_tau = int(rng.choice([8, 12, 16]))
        out.append(make_problem((n, n, n), n * 10.26 / 12, n_occ, n_b - n_occ, (-0.5, 0.0), (0.04, 4.0), 0.02,
                                n_tau, seed + 1 + i, n_bands_sigma=4, n_chi=min(n ** 3, n_chi_cap),
                                pin_edges=True, name="mix%d_%d^3_%db_%dt" % (i, n, n_b, n_tau)))
    return out


@dataclass
class KmeshProblem:
    """A cell sampled on a Gamma-centred k mesh.  k index = (k1*nk2 + k2)*nk3 + k3
    for k = sum_d (k_d / nk_d) b_d, k_d in [0, nk_d)."""

    n: tuple
    lattice: np.ndarray
    nk: tuple
    psi_k: np.ndarray        # [N_k][N_b][N_r] complex128: Bloch orbitals exp(i k.r) u_nk(r) on the cell grid
    eps_k: np.ndarray        # [N_k][N_b], ascending per k
    n_occ: int
    mu: float
    tau: np.ndarray
    omega: np.ndarray
    n_chi: int
    x_min: float
    x_max: float
    n_x: int = 4000
    ridge: float = 1e-6
    name: str = ""

    @property
    def n_r(self) -> int:
        return int(np.prod(self.n))

    @property
    def n_k(self) -> int:
        return int(np.prod(self.nk))

    @property
    def n_b(self) -> int:
        return self.psi_k.shape[1]

    @property
    def volume(self) -> float:
        return abs(float(np.linalg.det(self.lattice)))


def kmesh_problem(n=(6, 6, 6), a=(6.0, 6.5, 7.0), nk=(2, 2, 2), n_occ=4, n_unocc=20, n_tau=4, seed=51,
                  eps_occ=(-0.6, -0.05), eps_unocc=(0.05, 2.0), mu=0.0, n_chi=None):
    """Seeded k-mesh system: for every k, N_b orthonormal Bloch orbitals
    exp(i k.r) sum_g U_k[g][n] exp(i g.r) / sqrt(Omega) over the lowest N_b plane
    waves g (U_k from QR of a complex Gaussian), eigenvalues uniform in the
    windows with the band edges pinned (gap eps_unocc[0] - eps_occ[1] at every k)."""
    rng = np.random.default_rng(seed)
    n = tuple(int(x) for x in n)
    nk = tuple(int(x) for x in nk)
    lengths = np.broadcast_to(np.asarray(a, dtype=float), (3,))
    lattice = np.diag(lengths)
    vol = float(np.prod(lengths))
    n_b = n_occ + n_unocc
    basis = _plane_waves_on_grid(n, _sorted_lattice_points(n)[:n_b])
    i = [np.arange(nd) for nd in n]
    psi_k, eps_k = [], []
    for k1 in range(nk[0]):
        for k2 in range(nk[1]):
            for k3 in range(nk[2]):
                kk = (k1, k2, k3)
                e = [np.exp(2j * np.pi * kk[d] * i[d] / (nk[d] * n[d])) for d in range(3)]
                bloch = (e[0][:, None, None] * e[1][None, :, None] * e[2][None, None, :]).reshape(-1)
                z = rng.standard_normal((n_b, n_b)) + 1j * rng.standard_normal((n_b, n_b))
                U, _ = np.linalg.qr(z)
                psi_k.append(bloch[None, :] * (U.T @ basis) / np.sqrt(vol))
                eo = np.sort(rng.uniform(eps_occ[0], eps_occ[1], n_occ))
                eu = np.sort(rng.uniform(eps_unocc[0], eps_unocc[1], n_unocc))
                eo[-1], eu[0] = eps_occ[1], eps_unocc[0]
                eps_k.append(np.concatenate([eo, eu]))
    eps_k = np.array(eps_k)
    gap = eps_unocc[0] - eps_occ[1]
    width = eps_k.max() - eps_k.min()
    tau = np.geomspace(0.1 / width, 3.0 / gap, n_tau)
    return KmeshProblem(n=n, lattice=lattice, nk=nk, psi_k=np.array(psi_k), eps_k=eps_k, n_occ=n_occ, mu=float(mu),
                        tau=tau, omega=1.0 / tau[::-1], n_chi=int(np.prod(n)) if n_chi is None else int(n_chi),
                        x_min=float(np.min(np.abs(eps_k - mu))), x_max=float(width + np.max(np.abs(eps_k - mu))),
                        name="kmesh_%dx%dx%d_k%dx%dx%d" % (n + nk))


def batch_mix(count=16, seed=4, n_chi_cap=2048):
    """Uneven systems for one batched launch: grid n^3 with n in {12, 16, 20, 24}
    (cell a = n * 10.26 / 12), 128-1024 complex bands in multiples of 8 (one
    eighth occupied), 8-16 tau, the G set capped at n_chi_cap, the si8 energy
    windows and gap."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.choice([12, 16, 20, 24]))
        n_b = int(rng.integers(16, 129)) * 8
        n_occ = n_b // 8
        n_tau = int(rng.integers(8, 17))
        out.append(make_problem((n, n, n), n * 10.26 / 12, n_occ, n_b - n_occ, (-0.5, 0.0), (0.04, 4.0), 0.02, n_tau,
                                seed + 100 + i, n_bands_sigma=4, n_chi=min(n ** 3, n_chi_cap), pin_edges=True,
                                name="batch%d_%d^3_%db_%dt" % (i, n, n_b, n_tau)))
    return out
