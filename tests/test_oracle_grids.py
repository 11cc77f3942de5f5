"""Pins of the optimised time and frequency grids (Sec. II.A.2) and the
library's host implementation against the oracle's.

The grids are Chebyshev (minimax) approximations of 1/x by sums of squared
propagators (direct MP2 energy in time and in frequency).  What fixes them
independently of the oracle's Remez code:
  * n = 1 by brute force: a scan over the single node with its best weight;
  * the alternation theorem: the best n-term sum's relative error takes its
    largest magnitude 2n+1 times with alternating signs, and nowhere exceeds it;
  * scale covariance: the grids of [a x_min, a x_max] are tau/a and a omega;
  * the nonuniform transform fitted on these grids approximates the closed-form
    Lorentzians (Eqs. cos_error_function, sin_error_function) better than on
    log-spaced grids of the same size, with smaller weights and a better
    conditioned sine matrix."""
import os

import numpy as np
import pytest

from oracle import grids as og
from paper_1607_02859_gb300 import gw, inputs


def _brute_single(kind, r):
    """Best single node by a coarse then a fine scan, its best weight in closed form."""
    y = np.geomspace(1.0, r, 20001)

    def err(v):
        if kind == "time":
            phi = y * np.exp(-2.0 * y * v)
        else:
            phi = y * (2.0 * y / (y ** 2 + v ** 2)) ** 2
        a = 2.0 / (phi.max() + phi.min())
        return float(np.max(np.abs(1.0 - a * phi)))

    lo, hi = (np.log(1e-4 / r), np.log(100.0)) if kind == "time" else (np.log(1e-2), np.log(100.0 * r))
    for _ in range(3):
        vs = np.linspace(lo, hi, 401)
        es = [err(np.exp(v)) for v in vs]
        k = int(np.argmin(es))
        step = vs[1] - vs[0]
        lo, hi = vs[k] - 2 * step, vs[k] + 2 * step
    return min(es)


@pytest.mark.parametrize("kind", ["time", "frequency"])
@pytest.mark.parametrize("r", [5.0, 60.0])
def test_single_term_brute_force(kind, r):
    _, _, err = og.mp2_minimax(kind, 1, r)
    assert abs(err - _brute_single(kind, r)) < 1e-5 * err


@pytest.mark.parametrize("kind", ["time", "frequency"])
@pytest.mark.parametrize("n,r", [(4, 30.0), (8, 422.0), (16, 422.0), (20, 699.0)])
def test_alternation(kind, n, r):
    nodes, weights, err = og.mp2_minimax(kind, n, r)
    y = np.geomspace(1.0, r, 200001)
    if kind == "time":
        phi = y[:, None] * np.exp(-2.0 * np.outer(y, nodes))
    else:
        phi = y[:, None] * (2.0 * y[:, None] / (y[:, None] ** 2 + nodes[None, :] ** 2)) ** 2
    e = 1.0 - phi @ weights
    emax = np.max(np.abs(e))
    assert emax < 1.001 * err
    # count the sign runs whose extreme reaches the maximum (within 1%)
    runs, i = [], 0
    while i < len(e):
        j = i
        while j + 1 < len(e) and np.sign(e[j + 1]) == np.sign(e[i]):
            j += 1
        runs.append(np.max(np.abs(e[i:j + 1])))
        i = j + 1
    assert len(runs) == 2 * n + 1
    assert min(runs) > 0.99 * emax
    # more terms, smaller error
    if n > 4:
        assert og.mp2_minimax(kind, n - 4, r)[2] > 10 * err


def test_scale_covariance():
    g1 = og.mp2_grids(10, 0.02, 4.0)
    g2 = og.mp2_grids(10, 0.06, 12.0)
    assert np.allclose(g2["tau"], g1["tau"] / 3.0, rtol=1e-8)
    assert np.allclose(g2["omega"], g1["omega"] * 3.0, rtol=1e-8)


@pytest.mark.parametrize("maker", ["si8", "si64"])
def test_optimised_grid_fits_better_than_log_grid(maker):
    """16 and 20 points (at 8 points the sine fit of the optimised grid is not
    better than the log grid's: 9.6e-2 against 5.7e-2)."""
    p = getattr(inputs, maker)() if maker != "si64" else None
    if p is None:
        n, x_min, x_max = 20, 0.015, 10.485          # si64 energy windows (x_min, x_max as for the others)
        tau_log = np.geomspace(0.1 / 5.5, 3.0 / 0.03, n)
    else:
        n, x_min, x_max = len(p.tau), p.x_min, p.x_max
        tau_log = p.tau
    g = og.mp2_grids(n, x_min, x_max)
    new = og.transform_matrices(g["tau"], g["omega"], x_min, x_max, 4000, 0.0)
    old = og.transform_matrices(tau_log, 1.0 / tau_log[::-1], x_min, x_max, 4000, 1e-6)
    assert new["fit_err_cos"] < old["fit_err_cos"]
    assert new["fit_err_sin"] < old["fit_err_sin"]
    assert np.linalg.cond(new["S"]) < np.linalg.cond(old["S"])
    # the cosine transform approaches the closed-form Lorentzian 2x/(x^2+w^2) of single transitions
    for x in (x_min * 1.5, 0.3, 2.0):
        got = new["C"] @ np.exp(-x * g["tau"])
        want = 2.0 * x / (x ** 2 + g["omega"] ** 2)
        assert np.max(np.abs(got / want - 1.0)) <= new["fit_err_cos"] * 1.0001


@pytest.fixture(scope="module")
def L():
    if not os.path.exists(gw.LIB_PATH):
        from paper_1607_02859_gb300 import build
        build.build()
    return gw.lib()


@pytest.mark.parametrize("n,x_min,x_max", [(1, 0.1, 5.0), (8, 0.02, 8.467), (16, 0.02, 8.449), (20, 0.015, 10.485),
                                           (12, 0.05, 2.5)])
def test_library_grids_match_oracle(L, n, x_min, x_max):
    lib_g = gw.mp2_grids(n, x_min, x_max)
    ref = og.mp2_grids(n, x_min, x_max)
    for key in ("tau", "omega", "alpha", "sigma"):
        assert np.allclose(lib_g[key], ref[key], rtol=1e-7, atol=0), key
    assert abs(lib_g["err_time"] - ref["err_time"]) < 1e-3 * ref["err_time"]
    assert abs(lib_g["err_frequency"] - ref["err_frequency"]) < 1e-3 * ref["err_frequency"]


def test_library_grid_errors(L):
    with pytest.raises(gw.GwError) as e:
        gw.mp2_grids(0, 0.1, 1.0)
    assert e.value.status == 2
    with pytest.raises(gw.GwError) as e:
        gw.mp2_grids(8, 1.0, 0.5)
    assert e.value.status == 1
