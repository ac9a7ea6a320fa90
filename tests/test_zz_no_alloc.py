"""pdx_search_exact_noalloc, the search entry point for callers that cannot
allocate device memory during a search: callers whose device memory belongs
to another framework's allocator, or serving loops that must not allocate
after start-up. Its scratch is the library's static device array. These tests
call it through the C ABI and compare it with pdx_search_exact, which takes its
scratch from the stream-ordered allocator, on two calls in a row. The second
call runs on an array that still holds the first call's contents. The file
is named so that pytest collects it last."""
import ctypes

import numpy as np
import pytest

import pdx_synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_2503_04422_gb300 import build as pbuild
    pbuild.build()
    from paper_2503_04422_gb300 import pdx
    L = pdx.lib()
    L.pdx_search_exact_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                           ctypes.POINTER(pdx.pdx_search_opts), ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_void_p]
    L.pdx_search_exact_noalloc.restype = ctypes.c_int
    return torch, pdx, L


def _same_result(ref_d, ref_i, got_d, got_i, rtol=1e-5):
    """Equal up to the tolerance of the exact search: distances within rtol,
    ids equal except where the distance ties the k-th within rtol."""
    np.testing.assert_allclose(got_d, ref_d, rtol=rtol, atol=1e-6)
    for r in range(ref_i.shape[0]):
        if ref_i[r].tolist() == got_i[r].tolist():
            continue
        kth = ref_d[r, -1]
        for c in np.flatnonzero(ref_i[r] != got_i[r]):
            assert abs(ref_d[r, c] - kth) <= rtol * abs(kth) + 1e-6, f"row {r} col {c}"


@pytest.mark.parametrize("pruner", ["bond", "none"])
def test_noalloc_matches_allocating_entry_point_twice(env, pruner):
    torch, pdx, L = env
    x, q = pdx_synth.gaussian_mixture(pdx_synth.MixtureSpec(n=200_000, d=128, nq=256, n_centres=64, seed=21))
    ix = pdx.pdx_build_layout(torch.from_numpy(x).cuda())
    qd = torch.from_numpy(q).cuda()
    k = 10
    opts = pdx.search_opts(pruner=pruner)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    ref_d = torch.empty((256, k), dtype=torch.float32, device="cuda")
    ref_i = torch.empty((256, k), dtype=torch.int64, device="cuda")
    assert L.pdx_search_exact(ix.handle, qd.data_ptr(), 256, k, ctypes.byref(opts), ref_d.data_ptr(),
                              ref_i.data_ptr(), stream) == pdx.PDX_OK
    for call in range(2):
        od = torch.full((256, k), -7.0, dtype=torch.float32, device="cuda")
        oi = torch.full((256, k), -7, dtype=torch.int64, device="cuda")
        rc = L.pdx_search_exact_noalloc(ix.handle, qd.data_ptr(), 256, k, ctypes.byref(opts), od.data_ptr(),
                                        oi.data_ptr(), stream)
        assert rc == pdx.PDX_OK, pdx.pdx_last_error()
        torch.cuda.synchronize()
        _same_result(ref_d.cpu().numpy(), ref_i.cpu().numpy(), od.cpu().numpy(), oi.cpu().numpy())


def test_noalloc_rejects_oversize_and_host_buffers(env):
    torch, pdx, L = env
    x, q = pdx_synth.iid_normal(20_000, 32, 4096, seed=22)
    ix = pdx.pdx_build_layout(torch.from_numpy(x).cuda())
    qd = torch.from_numpy(q).cuda()
    k = 100
    od = torch.empty((4096, k), dtype=torch.float32, device="cuda")
    oi = torch.empty((4096, k), dtype=torch.int64, device="cuda")
    opts = pdx.search_opts(pruner="bond", start_vectors=8192)   # 4096 queries x 8192 START keys: > 32 MiB
    rc = L.pdx_search_exact_noalloc(ix.handle, qd.data_ptr(), 4096, k, ctypes.byref(opts), od.data_ptr(),
                                    oi.data_ptr(), None)
    assert rc == pdx.PDX_ERR_ARG
    assert "scratch" in pdx.pdx_last_error()
    hq = np.ascontiguousarray(q[:4])
    hd = np.empty((4, k), np.float32)
    hi = np.empty((4, k), np.int64)
    rc = L.pdx_search_exact_noalloc(ix.handle, hq.ctypes.data, 4, k, ctypes.byref(opts), hd.ctypes.data,
                                    hi.ctypes.data, None)
    assert rc == pdx.PDX_ERR_ARG
    assert "device memory" in pdx.pdx_last_error()
