"""N-point Pade approximant by Thiele's reciprocal differences (Sec. II.E.1,
Eqs. pade1 and pade2).  Oracle only.

    P_N(z) = a_1 / (1 + a_2 (z - z_1) / (1 + ... a_N (z - z_{N-1}) / 1))

with the tail (z - z_N) g_{N+1}(z) of Eq. pade1 set to zero, and

    g_1(z_n) = f_n,
    g_p(z)   = (g_{p-1}(z_{p-1}) - g_{p-1}(z)) / ((z - z_{p-1}) g_{p-1}(z)),  p >= 2,
    a_p      = g_p(z_p).
"""
import numpy as np


class ThieleBreakdown(ArithmeticError):
    pass


def coefficients(z, f):
    z = np.asarray(z, dtype=np.complex128)
    n = len(z)
    g = np.array(f, dtype=np.complex128)          # g[m] holds g_p(z_m) for m >= p-1
    a = np.empty(n, dtype=np.complex128)
    a[0] = g[0]
    for p in range(1, n):
        prev = g[p - 1]
        for m in range(p, n):
            den = (z[m] - z[p - 1]) * g[m]
            if abs(den) < 1e-300:
                raise ThieleBreakdown("vanishing reciprocal difference")
            g[m] = (prev - g[m]) / den
        a[p] = g[p]
    return a


def evaluate(a, z, x):
    """Backward evaluation of the continued fraction at the points x."""
    x = np.asarray(x, dtype=np.complex128)
    t = np.ones_like(x)
    for p in range(len(a) - 1, 0, -1):
        if np.any(np.abs(t) < 1e-300):
            raise ThieleBreakdown("vanishing denominator")
        t = 1.0 + a[p] * (x - z[p - 1]) / t
    if np.any(np.abs(t) < 1e-300):
        raise ThieleBreakdown("vanishing denominator")
    return a[0] / t


def derivative(a, z, x):
    """dP_N/dz at the points x.  P_N is analytic away from its poles, so on the
    real axis this is also d/d omega.  Each backward step t <- 1 + a_p (x - z_{p-1}) / t
    is differentiated with the quotient rule,
        t' <- a_p / t - a_p (x - z_{p-1}) t' / t^2,
    starting from t = 1, t' = 0; finally P_N' = -a_1 t' / t^2."""
    x = np.asarray(x, dtype=np.complex128)
    t = np.ones_like(x)
    dt = np.zeros_like(x)
    for p in range(len(a) - 1, 0, -1):
        if np.any(np.abs(t) < 1e-300):
            raise ThieleBreakdown("vanishing denominator")
        dt = a[p] / t - a[p] * (x - z[p - 1]) * dt / (t * t)
        t = 1.0 + a[p] * (x - z[p - 1]) / t
    if np.any(np.abs(t) < 1e-300):
        raise ThieleBreakdown("vanishing denominator")
    return -a[0] * dt / (t * t)
