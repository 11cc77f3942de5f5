"""CPU checks of libgw.so: it loads, exports every symbol of include/gw.h, and its
host-side setup (G set, Coulomb kernel, transform weights) agrees with the
oracle.  No kernel is launched here."""
import os
import re

import numpy as np
import pytest

from oracle import grids as ogrids
from oracle import gvec as ogv
from paper_1607_02859_gb300 import gw, inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    if not os.path.exists(gw.LIB_PATH):
        from paper_1607_02859_gb300 import build
        build.build()
    return gw.lib()


def test_exports_match_header(L):
    hdr = open(os.path.join(ROOT, "include", "gw.h")).read()
    declared = set(re.findall(r"^\s*(?:gw_status|const char\*|unsigned long long|size_t|int)\s+(gw_\w+)\s*\(",
                              hdr, flags=re.M))
    assert declared == set(gw.EXPORTS)
    for name in declared:
        assert hasattr(L, name), name


def test_version(L):
    assert gw.lib().gw_version() == 101


@pytest.mark.parametrize("n,n_chi", [((6, 6, 6), 216), ((8, 6, 10), 120), ((12, 12, 12), 500), ((24, 24, 24), 13824)])
def test_g_set_bit_exact(L, n, n_chi):
    grid = gw.make_grid(n, np.diag([6.0, 7.0, 8.0]))
    gv, idx = gw.g_set(grid, n_chi)
    ref = ogv.g_set(n, n_chi)
    assert np.array_equal(gv, ref)
    assert np.array_equal(idx, ogv.fft_index(ref, n))


def test_coulomb_sqrt(L):
    lat = np.array([[6.0, 0.3, 0.0], [0.0, 7.0, 0.2], [0.1, 0.0, 8.0]])
    grid = gw.make_grid((8, 6, 10), lat)
    gv, _ = gw.g_set(grid, 200)
    v = gw.coulomb_sqrt(grid, gv)
    ref = ogv.v_sqrt(gv, lat)
    assert v[0] == 0.0
    assert np.allclose(v, ref, rtol=1e-13, atol=0)


@pytest.mark.parametrize("maker", ["gamma_toy", "si8", "tiny"])
def test_fit_transform_matches_oracle(L, maker):
    p = getattr(inputs, maker)()
    lib_m = gw.fit_transform(p.tau, p.omega, p.x_min, p.x_max, p.n_x, p.ridge)
    ref = ogrids.transform_matrices(p.tau, p.omega, p.x_min, p.x_max, p.n_x, p.ridge)
    for key in ("C", "S"):
        assert np.allclose(lib_m[key], ref[key], rtol=1e-7, atol=1e-9 * np.abs(ref[key]).max()), key
    assert np.allclose(lib_m["Cinv"] @ lib_m["C"], np.eye(len(p.tau)), atol=1e-9)
    assert np.allclose(lib_m["Sinv"] @ lib_m["S"], np.eye(len(p.tau)), atol=1e-9)
    # S is ill-conditioned (cond ~2e6 at 16 points): its 1e-12 difference between the two fits grows by cond(S)
    err = np.linalg.norm(lib_m["Sinv"] - ref["Sinv"]) / np.linalg.norm(ref["Sinv"])
    assert err < 1e-11 * np.linalg.cond(ref["S"])
    assert abs(lib_m["fit_err_cos"] - ref["fit_err_cos"]) < 1e-6
    assert abs(lib_m["fit_err_sin"] - ref["fit_err_sin"]) < 1e-6


def test_host_argument_errors(L):
    grid = gw.make_grid((7, 6, 6), np.eye(3) * 5)
    with pytest.raises(gw.GwError) as e:
        gw.g_set(grid, 10)
    assert e.value.status == 2            # GW_ERR_SHAPE: 7 is not a supported length
    with pytest.raises(gw.GwError) as e:
        gw.fit_transform([1.0, -1.0], [1.0, 2.0], 0.1, 1.0)
    assert e.value.status == 1            # GW_ERR_ARG: tau <= 0


def test_invert_transform(L):
    """gw_invert_transform (Eqs. INV_CT_FFT, INV_ST_FFT) on a well-conditioned
    matrix and its errors."""
    rng = np.random.default_rng(7)
    m = np.eye(12) + 0.1 * rng.standard_normal((12, 12))
    inv = gw.invert_transform(m)
    assert np.max(np.abs(inv @ m - np.eye(12))) < 1e-13
    with pytest.raises(gw.GwError) as e:
        gw.invert_transform(np.zeros((3, 3)))
    assert e.value.status == 5            # GW_ERR_NUMERIC: singular
    with pytest.raises(gw.GwError) as e:
        gw.invert_transform(np.eye(65))
    assert e.value.status == 2


def test_device_calls_reject_null_context(L):
    st = L.gw_chi0_rtau(None, 4, 4, 1, None, None, None, None)
    assert st == 1
    assert b"ctx" in L.gw_last_error(None)
    st = L.gw_chi0_omega_kmesh_pw(None, None, None, 0, 0, None, None, 0.0, 0, None, None, 0, None, 0, None, 0, None,
                                  None)
    assert st == 1
    assert b"ctx" in L.gw_last_error(None)


def test_ctx_create_without_gpu_fails_cleanly(L):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(gw.GwError) as e:
        gw.Context(0)
    assert e.value.status == 4            # GW_ERR_CUDA, no abort


def test_binding_checks_sizes_before_the_library():
    """The QP and back-to-tau bindings reject inconsistent shapes on the host,
    before any library or device call."""
    with pytest.raises(ValueError):
        gw.qp_energies(None, np.ones(4), np.ones((2, 4)), [0.0], 0.0, [0.0, 0.0])     # eps has 1 entry, not 2
    with pytest.raises(ValueError):
        gw.qp_energies(None, np.ones(3), np.ones((2, 4)), [0.0, 0.0], 0.0, [0.0, 0.0])  # 3 nodes, 4 values
    with pytest.raises(ValueError):
        gw.sigma_to_tau(None, np.ones((2, 3, 4)), np.eye(4), np.eye(4))               # not square in bands
