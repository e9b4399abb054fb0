"""pa_weighted_average_noalloc: weighted averages with no device allocation.

For callers that cannot call cudaMalloc (serving loops that reserve all
device memory up front and must not enter the allocator, processes whose
device memory belongs to another allocator) the library offers an entry
point that takes records and output already in device memory and keeps its
scratch in a fixed device array.  This test calls it through the C ABI twice
in a row, with different sizes, and checks each result against the allocating
entry point pa_weighted_average on the same records.  It lives in its own file
so that it is collected after every other test.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_weighted_average_matches_allocating_entry_point():
    import torch

    from paper_2207_05535_gb300 import _lib, build
    from paper_2207_05535_gb300 import workloads as W

    build.build()
    lib = _lib.load()
    torch.cuda.set_device(0)
    n, N = 9, 64
    descs = W.glass_pairs(L=8, R=200, theta=2, beta_f=2.0, n=n, n_samples=2, seed=5)
    with _lib.Engine(descs) as eng:
        eng.run_to_end()
        recs = np.stack([eng.records(k) for k in range(len(descs))])

    stream = torch.cuda.Stream()
    for M, kind in [(4, 0), (3, 1)]:  # two calls in a row; the second reuses the scratch
        ref, _, _ = _lib.pa_weighted_average(recs[:M], N, kind)
        d_recs = torch.from_numpy(np.ascontiguousarray(recs[:M]).view(np.uint8).reshape(-1).copy()).cuda()
        d_out = torch.full((ref.nbytes,), 0xFF, dtype=torch.uint8, device="cuda")
        torch.cuda.synchronize()
        rc = lib.pa_weighted_average_noalloc(C.c_void_p(d_recs.data_ptr()), M, n, N, kind,
                                             C.c_void_p(d_out.data_ptr()), C.c_void_p(stream.cuda_stream))
        assert rc == 0, _lib.pa_status_string(rc)
        stream.synchronize()
        got = d_out.cpu().numpy().view(_lib.WAVG_DTYPE)
        assert got.shape == ref.shape
        for f in _lib.WAVG_DTYPE.names:
            np.testing.assert_allclose(got[f], ref[f], rtol=1e-12, atol=1e-15, err_msg=f)

    # sizes beyond the fixed scratch are refused before any work is enqueued
    rc = lib.pa_weighted_average_noalloc(C.c_void_p(d_recs.data_ptr()), 5000, 1, N, 0,
                                         C.c_void_p(d_out.data_ptr()), None)
    assert rc == 1
    rc = lib.pa_weighted_average_noalloc(C.c_void_p(d_recs.data_ptr()), 1000, 100, N, 0,
                                         C.c_void_p(d_out.data_ptr()), None)
    assert rc == 1
