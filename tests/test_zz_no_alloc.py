"""The allocation-free spatial transform (gw_rr_to_GG_fft_noalloc) against the
regular entry point.

Some callers cannot allocate device memory at all (their memory pool owns the
GPU, or an allocation's implicit synchronisation is not acceptable in their
loop); this entry point keeps its index maps in a fixed array inside the
library instead of a context arena.  Two calls in a row with different grids
and G sets check that nothing from the previous call leaks into the next.
The file is named so that pytest collects it last."""
import numpy as np
import pytest

from paper_1607_02859_gb300 import gw, inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import os
    if not os.path.exists(gw.LIB_PATH):
        from paper_1607_02859_gb300 import build
        build.build()
    c = gw.Context(0)
    yield c
    c.close()


def _case(p, n_chi, seed):
    grid = gw.make_grid(p.n, p.lattice)
    _, idx = gw.g_set(grid, n_chi)
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((p.n_r, p.n_r)) + 1j * rng.standard_normal((p.n_r, p.n_r))
    return grid, idx, x


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_noalloc_matches_regular_entry_point(ctx, prec):
    dt = gw.cdtype(prec)
    cases = [(inputs.tiny(seed=31, n=(8, 6, 10), a=(7.0, 6.0, 8.0), n_occ=4, n_unocc=20), 150, 1),
             (inputs.tiny(seed=32), 216, 2)]
    for p, n_chi, seed in cases:                  # two calls in a row, different sizes
        grid, idx, x = _case(p, n_chi, seed)
        xd = torch.from_numpy(x).to("cuda", dtype=dt)
        rows, r0 = p.n_r - 3, 3
        # stage 1, forward: rows r0.. of x(r,R') -> X(r,G')
        a = torch.zeros((rows, n_chi), dtype=dt, device="cuda")
        b = torch.full((rows, n_chi), 7.0, dtype=dt, device="cuda")
        gw.rr_to_GG_fft(ctx, grid, +1, 1, idx, prec, r0, rows, xd[r0:], a)
        gw.rr_to_GG_fft_noalloc(grid, +1, 1, idx, prec, r0, rows, xd[r0:], b)
        torch.cuda.synchronize()
        assert torch.allclose(a, b, rtol=1e-6, atol=0)
        # stage 2, forward (the input is the work buffer: give each call its own copy)
        X = torch.from_numpy(x[:, :n_chi].copy()).to("cuda", dtype=dt)
        a2 = torch.zeros((n_chi, n_chi), dtype=dt, device="cuda")
        b2 = torch.full((n_chi, n_chi), 7.0, dtype=dt, device="cuda")
        gw.rr_to_GG_fft(ctx, grid, +1, 2, idx, prec, 0, p.n_r, X.clone(), a2)
        gw.rr_to_GG_fft_noalloc(grid, +1, 2, idx, prec, 0, p.n_r, X.clone(), b2)
        torch.cuda.synchronize()
        assert torch.allclose(a2, b2, rtol=1e-6, atol=0)
        # stage 2 and 1, backward
        W = torch.from_numpy(x[:n_chi, :n_chi].copy()).to("cuda", dtype=dt)
        a3 = torch.zeros((p.n_r, n_chi), dtype=dt, device="cuda")
        b3 = torch.full((p.n_r, n_chi), 7.0, dtype=dt, device="cuda")
        gw.rr_to_GG_fft(ctx, grid, -1, 2, idx, prec, 0, p.n_r, W, a3)
        gw.rr_to_GG_fft_noalloc(grid, -1, 2, idx, prec, 0, p.n_r, W, b3)
        a4 = torch.zeros((p.n_r, p.n_r), dtype=dt, device="cuda")
        b4 = torch.full((p.n_r, p.n_r), 7.0, dtype=dt, device="cuda")
        gw.rr_to_GG_fft(ctx, grid, -1, 1, idx, prec, 0, p.n_r, a3, a4)
        gw.rr_to_GG_fft_noalloc(grid, -1, 1, idx, prec, 0, p.n_r, b3, b4)
        torch.cuda.synchronize()
        assert torch.allclose(a3, b3, rtol=1e-6, atol=0)
        assert torch.allclose(a4, b4, rtol=1e-6, atol=1e-12)


def test_noalloc_rejects_invalid_sizes():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    grid24 = gw.make_grid((24, 24, 24), np.eye(3) * 10.26)
    _, idx = gw.g_set(grid24, 13824)
    x = torch.zeros((1, 13824), dtype=torch.complex64, device="cuda")
    gw.rr_to_GG_fft_noalloc(grid24, +1, 1, idx, "fp32", 0, 1, x, x.clone())     # n_chi + N_r at the capacity
    # the 36^3 grid is compiled, but its N_r alone is beyond the fixed map capacity
    grid36 = gw.make_grid((36, 36, 36), np.eye(3) * 20.52)
    _, idx36 = gw.g_set(grid36, 100)
    y = torch.zeros((1, 100), dtype=torch.complex64, device="cuda")
    z = torch.zeros((1, 46656), dtype=torch.complex64, device="cuda")
    with pytest.raises(gw.GwError) as e:
        gw.rr_to_GG_fft_noalloc(grid36, -1, 1, idx36, "fp32", 0, 1, y, z)
    assert e.value.status == 2
    assert "capacity" in str(e.value)


def test_noalloc_refuses_stream_capture():
    """The maps are copied from host memory that lives only for the call, so a
    call on a stream that is being captured must be refused and do nothing."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    p = inputs.tiny(seed=32)
    grid, idx, x = _case(p, 216, 3)
    xd = torch.from_numpy(x).to("cuda", dtype=torch.complex64)
    out = torch.zeros((p.n_r, 216), dtype=torch.complex64, device="cuda")
    flag = torch.zeros(1, device="cuda")
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    refused = None
    with torch.cuda.graph(g):
        flag.add_(1.0)                            # keep the captured graph non-empty
        try:
            gw.rr_to_GG_fft_noalloc(grid, +1, 1, idx, "fp32", 0, p.n_r, xd, out)
        except gw.GwError as err:
            refused = err
    assert refused is not None and refused.status == 7, refused
    assert "captured" in str(refused)
    g.replay()
    torch.cuda.synchronize()
    assert float(flag.item()) == 1.0
    assert float(out.abs().max().item()) == 0.0
    # the same call outside a capture works
    gw.rr_to_GG_fft_noalloc(grid, +1, 1, idx, "fp32", 0, p.n_r, xd, out)
    torch.cuda.synchronize()
    assert float(out.abs().max().item()) > 0.0
