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
