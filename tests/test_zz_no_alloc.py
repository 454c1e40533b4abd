"""rte_cgs2_noalloc: the allocation-free Gram-Schmidt entry point.

It is meant for callers that cannot let a library allocate device memory (an
application that owns the device-memory budget through its own pool, or a
latency-critical loop where cudaMalloc is not allowed).  Its scratch lives in
a static device array shared by every call, so this test checks it against
the context-based rte_cgs2 on two calls in a row with different sizes: the
second call must not be disturbed by what the first left behind.  The file is
named to be collected last.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _ctx():
    from paper_2604_23265_gb300 import rte, workloads as W
    md = W.checkerboard_transport(2, I=19, M=8)      # n = 5776, several blocks, ragged tail
    return rte, rte.Context.from_medium(md)


def _case(n, k, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, k)))
    V = np.ascontiguousarray(Q.T)
    w = rng.standard_normal(n) + V.T @ rng.standard_normal(k) * 5.0
    return V, w


def test_noalloc_matches_cgs2_on_two_calls(lib):
    rte, ctx = _ctx()
    n = ctx.n
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call, (k, seed) in enumerate([(17, 1), (40, 2)]):
        V, w = _case(n, k, seed)
        Vd = torch.tensor(V.ravel(), dtype=torch.float64, device="cuda")
        w_ref = torch.tensor(w, dtype=torch.float64, device="cuda")
        h_ref = torch.zeros(k + 1, dtype=torch.float64, device="cuda")
        ctx.cgs2(Vd, k, w_ref, h_ref)
        w_new = torch.tensor(w, dtype=torch.float64, device="cuda")
        h_new = torch.zeros(k + 1, dtype=torch.float64, device="cuda")
        st = lib.rte_cgs2_noalloc(ctypes.c_void_p(Vd.data_ptr()), k, n,
                                  ctypes.c_void_p(w_new.data_ptr()),
                                  ctypes.c_void_p(h_new.data_ptr()), stream)
        assert st == rte.RTE_OK, lib.rte_last_error(None)
        torch.cuda.synchronize()
        hr, hn = h_ref.cpu().numpy(), h_new.cpu().numpy()
        np.testing.assert_allclose(hn, hr, rtol=1e-12, atol=1e-12, err_msg=f"call {call}")
        np.testing.assert_allclose(w_new.cpu().numpy(), w_ref.cpu().numpy(), rtol=0, atol=1e-12,
                                   err_msg=f"call {call}")
        # and against the definition: h = V^T w, w_out = (I - V V^T) w / norm
        np.testing.assert_allclose(hn[:k], V @ w, rtol=1e-12, atol=1e-12)
    ctx.close()


def _call(lib, rte, ctx, k, seed, stream):
    """One rte_cgs2_noalloc call against rte_cgs2 and against the definition."""
    n = ctx.n
    V, w = _case(n, k, seed)
    Vd = torch.tensor(V.ravel(), dtype=torch.float64, device="cuda")
    w_ref = torch.tensor(w, dtype=torch.float64, device="cuda")
    h_ref = torch.zeros(k + 1, dtype=torch.float64, device="cuda")
    ctx.cgs2(Vd, k, w_ref, h_ref)
    w_new = torch.tensor(w, dtype=torch.float64, device="cuda")
    h_new = torch.zeros(k + 1, dtype=torch.float64, device="cuda")
    st = lib.rte_cgs2_noalloc(ctypes.c_void_p(Vd.data_ptr()), k, n, ctypes.c_void_p(w_new.data_ptr()),
                              ctypes.c_void_p(h_new.data_ptr()), stream)
    assert st == rte.RTE_OK, lib.rte_last_error(None)
    torch.cuda.synchronize()
    hr, hn = h_ref.cpu().numpy(), h_new.cpu().numpy()
    np.testing.assert_allclose(hn, hr, rtol=1e-12, atol=1e-12, err_msg=f"n={n} k={k}")
    np.testing.assert_allclose(w_new.cpu().numpy(), w_ref.cpu().numpy(), rtol=0, atol=1e-12)
    np.testing.assert_allclose(hn[:k], V @ w, rtol=1e-12, atol=1e-12)
    p = w - V.T @ (V @ w)
    assert abs(hn[k] - np.linalg.norm(p)) <= 1e-12 * np.linalg.norm(w)


def test_noalloc_large_grids_then_small(lib):
    """A call on n >= 640 x 256 with k = 64 (one 128 KB block per SM), then a
    wide grid (k = 8, four blocks per SM, up to the array's 640 blocks of
    partial sums), then a small n: each equals rte_cgs2 and V^T w, so a
    smaller grid does not pick up the partial sums a larger one left."""
    from paper_2604_23265_gb300 import rte, workloads as W
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    big = rte.Context.from_medium(W.checkerboard_transport(3, I=64, M=32))      # n = 262,144
    assert big.n >= 640 * 256
    _call(lib, rte, big, 64, 11, stream)
    _call(lib, rte, big, 8, 12, stream)
    big.close()
    rte_, small = _ctx()
    _call(lib, rte, small, 5, 13, stream)
    small.close()


def test_noalloc_rejects_sizes_beyond_the_scratch(lib):
    from paper_2604_23265_gb300 import rte
    buf = torch.zeros(8, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(buf.data_ptr())
    st = lib.rte_cgs2_noalloc(p, 65, 8, p, p, None)
    assert st == rte.RTE_EINVAL
    assert b"k must be in [1, 64]" in lib.rte_last_error(None)
