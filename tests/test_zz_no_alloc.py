"""The allocation-free table sort against the regular table build (GPU).

fast_table_sort_static serves callers that cannot let the library allocate
device memory (hosts that reserve the GPU's memory for their own pools, or
cannot afford cudaMalloc's implicit synchronisation).  It must give exactly
the listing one table of fast_build_tables gives, call after call, although
every call reuses the same fixed scratch array.  Both calls are also
compared with the oracle's canonical table listing.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_1803_09835_gb300 import _build, _lib
    _build.build()
    assert torch.cuda.is_available()
    return _lib.load()


def _reference_table(keys_dev, n):
    """One table built by the regular entry point (b = 1, filter off)."""
    from paper_1803_09835_gb300 import _lib
    p = dict(D=8, K=1, b=1, r=1, kind=0, seed=1, v=1, excl=0, occ_num=0, occ_den=1)
    ctx = _lib.fast_create(p)
    tb = _lib.fast_build_tables(ctx, keys_dev, n)
    k, s, _ = _lib.fast_tables_view(tb)
    out = (k.cpu().numpy().view(np.uint32).copy(), s.cpu().numpy().view(np.uint32).copy())
    _lib.fast_tables_free(tb)
    _lib.fast_destroy(ctx)
    return out


def _call(lib, keys_dev, n):
    skey = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
    sid = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    st = lib.fast_table_sort_static(ctypes.c_void_p(keys_dev.data_ptr()), n, ctypes.c_void_p(skey.data_ptr()),
                                    ctypes.c_void_p(sid.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
    torch.cuda.synchronize()
    return st, skey[:n].cpu().numpy().view(np.uint32), sid[:n].cpu().numpy().view(np.uint32)


def test_static_scratch_sort_matches_table_build(lib):
    rng = np.random.default_rng(2024)
    # two calls in a row: a large one, then a smaller one with many equal keys,
    # so stale scratch from the first call would show in the second
    cases = [rng.integers(0, 2**32, 1 << 20, dtype=np.uint64).astype(np.uint32),
             rng.integers(0, 300, 54_321).astype(np.uint32)]
    for keys in cases:
        n = len(keys)
        kd = torch.from_numpy(keys.view(np.int32)).cuda()
        st, skey, sid = _call(lib, kd, n)
        assert st == 0
        want_k, want_s = _reference_table(kd, n)
        assert np.array_equal(skey, want_k) and np.array_equal(sid, want_s)
        # and against the oracle's canonical table listing (key, then id)
        ok, oid = oracle.table(keys)
        assert np.array_equal(skey, ok) and np.array_equal(sid, oid)


def test_static_scratch_sort_rejects_oversize(lib):
    from paper_1803_09835_gb300 import _lib
    kd = torch.zeros(8, dtype=torch.int32, device="cuda")
    st, _, _ = _call(lib, kd, 0)
    assert st == 0
    big = (1 << 20) + 1
    stream = torch.cuda.current_stream()
    st = lib.fast_table_sort_static(ctypes.c_void_p(kd.data_ptr()), big, ctypes.c_void_p(kd.data_ptr()),
                                    ctypes.c_void_p(kd.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
    assert st == _lib.FAST_EINVAL
