"""Nonuniform cosine/sine transform weights (Sec. II.A.3).  Oracle only.

The time grid tau_j and the frequency grid omega_k are inputs.  For every
omega_k separately the cosine weights gamma_kj are chosen so that

    sum_j gamma_kj cos(omega_k tau_j) exp(-x tau_j)  ~  2x / (x^2 + omega_k^2)

for all transition energies x in [x_min, x_max] (Eq. cos_error_function), and
the sine weights lambda_kj so that

    sum_j lambda_kj sin(omega_k tau_j) exp(-x tau_j)  ~  2 omega_k / (x^2 + omega_k^2)

(Eq. sin_error_function).  The paper only asks that the error be minimised on
the interval.  Reading taken here: the residual is divided by the target
(relative error), sampled at n_x log-spaced x, and minimised in the least
squares sense with a ridge term ridge^2 * n_x * |gamma_k|^2, which keeps the
weights of moderate size so that the transform does not amplify rounding.
"""
import numpy as np


def _fit_rows(tau, omega, x_min, x_max, n_x, ridge, trig):
    tau = np.asarray(tau, dtype=np.float64)
    omega = np.asarray(omega, dtype=np.float64)
    x = np.geomspace(x_min, x_max, n_x)
    n = len(tau)
    w = np.zeros((len(omega), n))
    worst = 0.0
    for k, wk in enumerate(omega):
        if trig == "cos":
            target = 2.0 * x / (x ** 2 + wk ** 2)
            basis = np.cos(wk * tau)[None, :] * np.exp(-np.outer(x, tau))
        else:
            target = 2.0 * wk / (x ** 2 + wk ** 2)
            basis = np.sin(wk * tau)[None, :] * np.exp(-np.outer(x, tau))
        a = basis / target[:, None]          # relative residual: a @ g - 1
        b = np.ones(n_x)
        a_aug = np.vstack([a, ridge * np.sqrt(n_x) * np.eye(n)])
        b_aug = np.concatenate([b, np.zeros(n)])
        g, *_ = np.linalg.lstsq(a_aug, b_aug, rcond=None)
        w[k] = g
        worst = max(worst, float(np.max(np.abs(a @ g - 1.0))))
    return w, worst


def cos_weights(tau, omega, x_min, x_max, n_x=4000, ridge=1e-6):
    """gamma_kj of Eq. CT_FFT fitted per Eq. cos_error_function.

    Returns (gamma, max relative error of the fitted Lorentzian on the x grid).
    """
    return _fit_rows(tau, omega, x_min, x_max, n_x, ridge, "cos")


def sin_weights(tau, omega, x_min, x_max, n_x=4000, ridge=1e-6):
    """lambda_kj of Eq. ST_FFT fitted per Eq. sin_error_function."""
    return _fit_rows(tau, omega, x_min, x_max, n_x, ridge, "sin")


def transform_matrices(tau, omega, x_min, x_max, n_x=4000, ridge=1e-6):
    """The stored matrices of the method.

    C[k][j]    = gamma_kj cos(omega_k tau_j)           (Eq. CT_FFT)
    S[k][j]    = lambda_kj sin(omega_k tau_j)          (Eq. ST_FFT; times i)
    Cinv[j][k] = xi_jk cos(tau_j omega_k) = C^{-1}     (Eq. INV_CT_FFT)
    Sinv[j][k] = zeta_jk sin(tau_j omega_k) = S^{-1}   (Eq. INV_ST_FFT; times -i)
    """
    tau = np.asarray(tau, dtype=np.float64)
    omega = np.asarray(omega, dtype=np.float64)
    gamma, err_c = cos_weights(tau, omega, x_min, x_max, n_x, ridge)
    lam, err_s = sin_weights(tau, omega, x_min, x_max, n_x, ridge)
    wt = np.outer(omega, tau)
    C = gamma * np.cos(wt)
    S = lam * np.sin(wt)
    Cinv = np.linalg.inv(C)
    Sinv = np.linalg.inv(S)
    return {"C": C, "S": S, "Cinv": Cinv, "Sinv": Sinv, "gamma": gamma, "lambda": lam,
            "fit_err_cos": err_c, "fit_err_sin": err_s}


# ---------------------------------------------------------------------------
# Optimised time and frequency grids (Sec. II.A.2).
#
# The paper takes tau_j and omega_k from the minimisation of the discretisation
# error of the direct MP2 energy in imaginary time and in imaginary frequency.
# For one transition energy x > 0 that energy needs 1/x, which both domains
# write as an integral of a squared propagator:
#
#   time:       1/x = int_{-inf}^{inf} dtau exp(-x|tau|)^2        ~ sum_j alpha_j exp(-2 x tau_j)
#   frequency:  1/x = int dw/(2 pi) (2x/(x^2+w^2))^2               ~ sum_k sigma_k (2x/(x^2+omega_k^2))^2
#
# Reading taken here: each grid (with its weights) minimises the largest
# relative error  |1 - x * sum(...)|  over x in [x_min, x_max] -- a minimax
# (Chebyshev) approximation, computed by the Remez exchange: the error of the
# best n-term approximation alternates 2n+1 times with equal magnitude, and
# Newton's method solves for the 2n parameters and that magnitude on a
# reference set of 2n+1 points, which is then moved to the extrema of the new
# error.  A good start for n terms comes from the n-1 term solution (the
# log-positions and log-weights resampled over the term index), starting
# from a scan for n = 1.  All work is on y = x / x_min in [1, R], R = x_max/x_min.
# ---------------------------------------------------------------------------

def _mp2_basis(kind, y, s):
    """phi_j(y) = y * (squared propagator of node j) and d phi_j / d s_j, s_j = log(node_j)."""
    v = np.exp(s)
    if kind == "time":
        e = np.exp(-2.0 * np.outer(y, v))
        phi = y[:, None] * e
        dphi = -2.0 * (y[:, None] ** 2) * v[None, :] * e
    else:
        d = y[:, None] ** 2 + v[None, :] ** 2
        phi = 4.0 * y[:, None] ** 3 / d ** 2
        dphi = -16.0 * y[:, None] ** 3 * v[None, :] ** 2 / d ** 3
    return phi, dphi


def mp2_relative_error(kind, y, logw, s):
    """1 - y sum_j w_j (squared propagator)_j(y): the relative error of the
    discretised 1/y (time: nodes tau_j, frequency: nodes omega_k)."""
    phi, _ = _mp2_basis(kind, np.asarray(y, dtype=np.float64), s)
    return 1.0 - phi @ np.exp(logw)


def _newton_on_reference(kind, p, ref, e0, iters=30):
    n = len(p) // 2
    sgn = (-1.0) ** np.arange(2 * n + 1)
    q = np.concatenate([p, [e0]])
    for _ in range(iters):
        w = np.exp(q[:n])
        phi, dphi = _mp2_basis(kind, ref, q[n:2 * n])
        f = 1.0 - phi @ w - sgn * q[-1]
        jac = np.hstack([-(phi * w), -(dphi * w), -sgn[:, None]])
        try:
            d = np.linalg.solve(jac, -f)
        except np.linalg.LinAlgError:
            return None
        step = min(1.0, 0.3 / max(float(np.max(np.abs(d[:2 * n]))), 1e-300))
        q = q + step * d
        if step == 1.0 and np.max(np.abs(f)) < 1e-14:
            break
    return q if np.all(np.isfinite(q)) else None


def _extrema(kind, p, ref, r, n_fine=4000):
    """The largest |error| in each run of equal sign on a log grid of [1, R]
    (plus the current reference), each interior one refined on a local grid."""
    n = len(p) // 2
    y = np.unique(np.concatenate([np.geomspace(1.0, r, n_fine), ref]))
    e = mp2_relative_error(kind, y, p[:n], p[n:])
    pos = []
    i = 0
    while i < len(y):
        j = i
        while j + 1 < len(y) and np.sign(e[j + 1]) == np.sign(e[i]):
            j += 1
        pos.append(i + int(np.argmax(np.abs(e[i:j + 1]))))
        i = j + 1
    if len(pos) != 2 * n + 1:
        return None
    out = y[pos].copy()
    for m in range(1, len(pos) - 1):
        k = pos[m]
        yy = np.geomspace(y[k - 1], y[k + 1], 41)
        out[m] = yy[int(np.argmax(np.abs(mp2_relative_error(kind, yy, p[:n], p[n:]))))]
    return out


def _remez(kind, p, ref, r, tol=1e-4, iters=40):
    n = len(p) // 2
    e0 = float(np.mean(np.abs(mp2_relative_error(kind, ref, p[:n], p[n:]))))
    for _ in range(iters):
        q = _newton_on_reference(kind, p, ref, e0)
        if q is None:
            break
        p, e0 = q[:2 * n], float(q[-1])
        new = _extrema(kind, p, ref, r)
        if new is None:
            break
        ref = new
        a = np.abs(mp2_relative_error(kind, ref, p[:n], p[n:]))
        if a.max() - a.min() < tol * a.max():
            break
    return p, ref


def _resample(v, m):
    return np.interp(np.linspace(0.0, 1.0, m), np.linspace(0.0, 1.0, len(v)), v)


def mp2_minimax(kind, n, r):
    """Best n-term approximation of 1/y on [1, r] (kind "time" or "frequency").
    Returns (nodes ascending, weights, largest relative error on a fine grid)."""
    y = np.geomspace(1.0, r, 2000)
    if kind == "time":
        scan = np.linspace(np.log(1e-3 / r), np.log(10.0), 400)
    else:
        scan = np.linspace(np.log(0.1), np.log(10.0 * r), 400)
    best = None
    for s in scan:
        phi, _ = _mp2_basis(kind, y, np.array([s]))
        a = 2.0 / (phi.max() + phi.min())                # the best single weight for this node
        err = float(np.max(np.abs(1.0 - a * phi[:, 0])))
        if best is None or err < best[0]:
            best = (err, np.array([np.log(a), s]))
    p = best[1]
    ref = np.array([1.0, np.sqrt(r), r])
    p, ref = _remez(kind, p, ref, r)
    for m in range(2, n + 1):
        logw, s = p[:m - 1], p[m - 1:]
        if m == 2:
            s_new = np.array([s[0] - 1.0, s[0] + 1.0])
            lw = np.full(2, logw[0] - s[0] - np.log(2.0)) + s_new
        else:
            s_new = _resample(s, m)
            lw = _resample(logw - s, m) + np.log((m - 1) / m) + s_new
        p = np.concatenate([lw, s_new])
        ref = np.exp(_resample(np.log(ref), 2 * m + 1))
        p, ref = _remez(kind, p, ref, r)
    order = np.argsort(p[n:])
    nodes = np.exp(p[n:][order])
    weights = np.exp(p[:n][order])
    err = float(np.max(np.abs(mp2_relative_error(kind, np.geomspace(1.0, r, 20000), p[:n], p[n:]))))
    return nodes, weights, err


def mp2_grids(n, x_min, x_max):
    """The n-point imaginary-time and imaginary-frequency grids (Sec. II.A.2)
    for transition energies in [x_min, x_max]:

    tau_j   minimise max_x |1 - x sum_j alpha_j exp(-2 x tau_j)|,
    omega_k minimise max_x |1 - x sum_k sigma_k (2x / (x^2 + omega_k^2))^2|.

    Returns a dict with tau, omega (ascending), alpha, sigma and the two
    largest relative errors err_time, err_frequency."""
    r = float(x_max) / float(x_min)
    t, a, et = mp2_minimax("time", n, r)
    w, sg, ew = mp2_minimax("frequency", n, r)
    return {"tau": t / x_min, "omega": w * x_min, "alpha": a / x_min, "sigma": sg / x_min,
            "err_time": et, "err_frequency": ew}
