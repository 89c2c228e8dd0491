"""ctypes binding of libfast.so (include/fast.h).  Argument marshalling only.

Every function here has the name of the C entry point it calls and takes
torch tensors (device memory) or numpy arrays (host memory) in place of raw
pointers.  All work runs in the library's CUDA kernels; if the library is
missing or no GPU is present the calls raise -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfast.so")
HEADER = os.path.join(HERE, "..", "include", "fast.h")

STATUS = {0: "FAST_OK", 1: "FAST_EINVAL", 2: "FAST_ENOMEM", 3: "FAST_EBUDGET", 4: "FAST_EMAPFULL",
          5: "FAST_ETIMEOUT", 6: "FAST_EPENDING", 7: "FAST_ECUDA", 8: "FAST_EINTERNAL"}
FAST_OK, FAST_EINVAL, FAST_ENOMEM, FAST_EBUDGET, FAST_EMAPFULL, FAST_ETIMEOUT, FAST_EPENDING, FAST_ECUDA, \
    FAST_EINTERNAL = range(9)
FAST_MINHASH, FAST_MINMAX = 0, 1


class FastError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class fast_params(ctypes.Structure):
    _fields_ = [("D", ctypes.c_uint32), ("K", ctypes.c_uint32), ("b", ctypes.c_uint32), ("r", ctypes.c_uint32),
                ("kind", ctypes.c_uint32), ("seed", ctypes.c_uint64), ("v", ctypes.c_uint32),
                ("excl", ctypes.c_uint32), ("occ_num", ctypes.c_uint32), ("occ_den", ctypes.c_uint32),
                ("table_group", ctypes.c_uint32), ("query_part", ctypes.c_uint32)]


class fast_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_float) for n in ("ms_sig", "ms_sort", "ms_filter", "ms_enum", "ms_dense", "ms_sparse",
                                              "ms_output", "ms_total")] + \
               [(n, ctypes.c_uint64) for n in ("n_fingerprints", "n_dropped", "n_emissions", "n_dense_pairs",
                                               "n_groups", "n_detections", "map_slots", "n_launches", "n_long_rows", "n_huge_rows", "max_row")] + \
               [("query_parts", ctypes.c_uint32), ("sort_passes", ctypes.c_uint32)] + \
               [(n, ctypes.c_float) for n in ("ms_pair_count", "ms_pair_emit", "ms_vote", "ms_k_pairs", "ms_k_vote")] + \
               [("n_pairs_small", ctypes.c_uint64), ("peak_bytes", ctypes.c_uint64),
                ("n_overflow", ctypes.c_uint64), ("max_group", ctypes.c_uint64)] + \
               [(n, ctypes.c_float) for n in ("ms_k_medium", "ms_k_vote_block", "ms_k_count_small",
                                              "ms_k_count_medium")] + \
               [("dense_fallback", ctypes.c_uint32), ("large_min", ctypes.c_uint32),
                ("group_shift", ctypes.c_uint32), ("region_slots", ctypes.c_uint32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class fast_plan_choice(ctypes.Structure):
    _fields_ = [("vote_map", ctypes.c_uint32), ("large_min", ctypes.c_uint32), ("map_load", ctypes.c_float),
                ("ms", ctypes.c_float), ("group_pairs", ctypes.c_uint32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class fast_plan_info_t(ctypes.Structure):
    _fields_ = [("graph_nodes", ctypes.c_uint64), ("graph_kernels", ctypes.c_uint64), ("arena_bytes", ctypes.c_uint64),
                ("build_ms", ctypes.c_float), ("tuned", ctypes.c_uint32), ("n_tried", ctypes.c_uint32),
                ("best", fast_plan_choice), ("tried", fast_plan_choice * 8)]


_lib = None

# int fill(void *user, uint64_t row0, uint64_t n, uint32_t ld, uint16_t *h_rows)
FILL_ROWS = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32,
                             ctypes.c_void_p)


def load():
    """Loads libfast.so (built by ``__graft_entry__.build()``); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build the CUDA library first (__graft_entry__.build()); "
                          "there is no CPU fallback")
    lib = ctypes.CDLL(LIB_PATH)
    vp, u64, u32, st = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
    pp = ctypes.POINTER
    sigs = {
        "fast_create": (st, [pp(fast_params), u64, pp(vp)]),
        "fast_destroy": (None, [vp]),
        "fast_last_error": (ctypes.c_char_p, [vp]),
        "fast_sig": (st, [vp, vp, u64, u32, vp, vp]),
        "fast_sig_rows": (st, [vp, vp, u64, u32, vp, u64, u64, vp]),
        "fast_detect_chunked": (st, [vp, u64, u32, u64, FILL_ROWS, vp, pp(vp), vp]),
        "fast_build_tables": (st, [vp, vp, u64, pp(vp), vp]),
        "fast_tables_view": (st, [vp, pp(u64), pp(u32), pp(vp), pp(vp), pp(vp)]),
        "fast_tables_free": (None, [vp]),
        "fast_search": (st, [vp, vp, pp(vp), vp]),
        "fast_detect": (st, [vp, vp, u64, u32, pp(vp), vp]),
        "fast_detect_batch": (st, [vp, vp, vp, u32, u32, vp, vp]),
        "fast_detect_host": (st, [vp, vp, u64, u32, pp(u64), vp, vp, vp, u64, vp]),
        "fast_result_view": (st, [vp, pp(u64), pp(vp), pp(vp), pp(vp)]),
        "fast_result_free": (None, [vp]),
        "fast_get_stats": (st, [vp, pp(fast_stats)]),
        "fast_set_option": (st, [vp, ctypes.c_char_p, ctypes.c_double]),
        "fast_table_sort_static": (st, [vp, u64, vp, vp, vp]),
        "fast_server_create": (st, [pp(fast_params), u32, u64, u64, pp(vp)]),
        "fast_server_destroy": (None, [vp]),
        "fast_server_last_error": (ctypes.c_char_p, [vp]),
        "fast_server_load_history": (st, [vp, u32, vp, u64, u32]),
        "fast_stream_submit": (st, [vp, u32, vp, u32, u32, pp(u64)]),
        "fast_stream_poll": (st, [vp, u64, u64, pp(u64), pp(u64), pp(vp), pp(vp), pp(vp)]),
        "fast_stream_latency": (st, [vp, u64, pp(ctypes.c_double)]),
        "fast_stream_release": (st, [vp, u64]),
        "fast_server_inject_failure": (st, [vp, u64]),
        "fast_server_hold_budget": (st, [vp, u64]),
        "fast_query_only": (st, [vp, vp, u64, vp, vp, u64, u32, pp(vp), vp]),
        "fast_channel_merge": (st, [vp, u64, u32, vp, vp, vp, vp, u32, pp(vp), vp]),
        "fast_merged_view": (st, [vp, pp(u64), pp(vp), pp(vp), pp(vp)]),
        "fast_merged_free": (None, [vp]),
        "fast_station_clusters": (st, [vp, vp, vp, vp, u64, u32, u32, u32, pp(vp), vp]),
        "fast_clusters_view": (st, [vp, pp(u64), pp(vp)]),
        "fast_clusters_free": (None, [vp]),
        "fast_server_set_option": (st, [vp, ctypes.c_char_p, ctypes.c_double]),
        "fast_plan_create": (st, [vp, vp, vp, u32, u32, vp, pp(vp)]),
        "fast_plan_run": (st, [vp, vp, vp]),
        "fast_plan_info": (st, [vp, pp(fast_plan_info_t)]),
        "fast_plan_destroy": (None, [vp]),
    }
    for name, (res, args) in sigs.items():
        fn = getattr(lib, name)
        fn.restype, fn.argtypes = res, args
    _lib = lib
    return lib


def _check(ctx, status: int):
    if status != FAST_OK:
        msg = load().fast_last_error(ctx).decode() if ctx else ""
        raise FastError(status, msg)


def _stream(stream):
    import torch
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _dptr(t, dtype=None):
    import torch
    if t is None:
        return None
    assert isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous(), "expected a contiguous CUDA tensor"
    if dtype is not None:
        assert t.dtype == dtype, f"expected {dtype}, got {t.dtype}"
    return ctypes.c_void_p(t.data_ptr())


def _hptr(a):
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    assert a.flags["C_CONTIGUOUS"]
    return ctypes.c_void_p(a.ctypes.data)


class _DevArray:
    """Zero-copy view of library-owned device memory (__cuda_array_interface__)."""

    def __init__(self, ptr, n, typestr, owner):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr or 0, False),
                                         "version": 3, "strides": None}
        self._owner = owner


def _view(ptr, n, typestr, owner):
    import torch
    if n == 0:
        dt = {"<i4": torch.int32, "|u1": torch.uint8, "<i2": torch.int16, "<i8": torch.int64}[typestr]
        return torch.empty(0, dtype=dt, device="cuda")
    return torch.as_tensor(_DevArray(ptr, n, typestr, owner), device="cuda")


def params_struct(params: dict) -> fast_params:
    p = fast_params()
    for k, _ in fast_params._fields_:
        setattr(p, k, int(params.get(k, 0)))
    return p


# --------------------------------------------------------------- C names

def fast_create(params: dict, hbm_budget_bytes: int = 0) -> ctypes.c_void_p:
    lib = load()
    out = ctypes.c_void_p()
    _check(None, lib.fast_create(ctypes.byref(params_struct(params)), hbm_budget_bytes, ctypes.byref(out)))
    return out


def fast_destroy(ctx):
    load().fast_destroy(ctx)


def fast_sig(ctx, d_idx, N: int, ld: int, d_sig, stream=None):
    import torch
    _check(ctx, load().fast_sig(ctx, _dptr(d_idx), N, ld, _dptr(d_sig), _stream(stream)))


def fast_build_tables(ctx, d_sig, N: int, stream=None):
    out = ctypes.c_void_p()
    _check(ctx, load().fast_build_tables(ctx, _dptr(d_sig), N, ctypes.byref(out), _stream(stream)))
    return out


def fast_tables_view(tb, owner=None):
    """(skey [b*N] int32 view, sid [b*N] int32 view, drop [N] uint8 view)."""
    N, b = ctypes.c_uint64(), ctypes.c_uint32()
    k, s, d = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
    _check(None, load().fast_tables_view(tb, ctypes.byref(N), ctypes.byref(b), ctypes.byref(k), ctypes.byref(s),
                                         ctypes.byref(d)))
    n = N.value * b.value
    return (_view(k.value, n, "<i4", owner), _view(s.value, n, "<i4", owner), _view(d.value, N.value, "|u1", owner))


def fast_tables_free(tb):
    load().fast_tables_free(tb)


def fast_sig_rows(ctx, d_idx, n: int, ld: int, d_sig, N: int, col0: int, stream=None):
    _check(ctx, load().fast_sig_rows(ctx, _dptr(d_idx), n, ld, _dptr(d_sig), N, col0, _stream(stream)))


def fast_detect_chunked(ctx, N: int, ld: int, chunk_rows: int, fill, stream=None):
    """fill(row0, n, rows) writes windows row0 .. row0 + n - 1 into the
    [n, ld] uint16 numpy view `rows` of the library's pinned staging buffer."""
    import numpy as np
    err = []

    def cb(_user, row0, n, ld_, ptr):
        try:
            rows = np.ctypeslib.as_array(ctypes.cast(ptr, ctypes.POINTER(ctypes.c_uint16)), (n, ld_))
            fill(row0, n, rows)
            return 0
        except Exception as e:  # reported as the call's failure
            err.append(e)
            return 1

    fn = FILL_ROWS(cb)
    out = ctypes.c_void_p()
    st = load().fast_detect_chunked(ctx, N, ld, chunk_rows, fn, None, ctypes.byref(out), _stream(stream))
    if err:
        raise err[0]
    _check(ctx, st)
    return out


def fast_search(ctx, tb, stream=None):
    out = ctypes.c_void_p()
    _check(ctx, load().fast_search(ctx, tb, ctypes.byref(out), _stream(stream)))
    return out


def fast_detect(ctx, d_idx, N: int, ld: int, stream=None):
    out = ctypes.c_void_p()
    _check(ctx, load().fast_detect(ctx, _dptr(d_idx), N, ld, ctypes.byref(out), _stream(stream)))
    return out


def fast_detect_host(ctx, h_idx, N: int, ld: int, h_i, h_j, h_votes, cap: int, stream=None) -> int:
    M = ctypes.c_uint64()
    _check(ctx, load().fast_detect_host(ctx, _hptr(h_idx), N, ld, ctypes.byref(M),
                                        _hptr(h_i) if cap else None, _hptr(h_j) if cap else None,
                                        _hptr(h_votes) if cap else None, cap, _stream(stream)))
    return M.value


def fast_result_view(res, owner=None):
    """(M, i [M] int32 view, j [M] int32 view, votes [M] uint8 view)."""
    M = ctypes.c_uint64()
    i, j, v = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
    _check(None, load().fast_result_view(res, ctypes.byref(M), ctypes.byref(i), ctypes.byref(j), ctypes.byref(v)))
    m = M.value
    return m, _view(i.value, m, "<i4", owner), _view(j.value, m, "<i4", owner), _view(v.value, m, "|u1", owner)


def fast_result_free(res):
    load().fast_result_free(res)


def fast_query_only(ctx, d_hist, N0: int, d_hist_drop, d_batch, n: int, ld: int, stream=None):
    out = ctypes.c_void_p()
    _check(ctx, load().fast_query_only(ctx, _dptr(d_hist), N0, _dptr(d_hist_drop), _dptr(d_batch), n, ld,
                                       ctypes.byref(out), _stream(stream)))
    return out


def fast_channel_merge(ctx, N: int, lists, thr: int, stream=None):
    """lists: per channel (M, d_i, d_j, d_votes), device tensors (int32 views
    of uint32 ids, uint8 votes)."""
    nch = len(lists)
    arr = ctypes.c_void_p * max(1, nch)
    M = (ctypes.c_uint64 * max(1, nch))(*[int(m) for m, _, _, _ in lists])
    cols = [[(l[k + 1].data_ptr() if int(l[0]) else None) for l in lists] for k in range(3)]  # i, j, votes
    ptrs = [arr(*col) for col in cols]
    out = ctypes.c_void_p()
    _check(ctx, load().fast_channel_merge(ctx, N, nch, M, ctypes.cast(ptrs[0], ctypes.c_void_p),
                                          ctypes.cast(ptrs[1], ctypes.c_void_p), ctypes.cast(ptrs[2], ctypes.c_void_p),
                                          thr, ctypes.byref(out), _stream(stream)))
    return out


def fast_merged_view(res, owner=None):
    """(M, i [M] int32 view, j [M] int32 view, sim [M] int16 view of uint16)."""
    M = ctypes.c_uint64()
    i, j, v = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
    _check(None, load().fast_merged_view(res, ctypes.byref(M), ctypes.byref(i), ctypes.byref(j), ctypes.byref(v)))
    m = M.value
    return m, _view(i.value, m, "<i4", owner), _view(j.value, m, "<i4", owner), _view(v.value, m, "<i2", owner)


def fast_merged_free(res):
    load().fast_merged_free(res)


def fast_station_clusters(ctx, d_i, d_j, d_sim, n: int, gap: int, width: int, min_n: int, stream=None):
    out = ctypes.c_void_p()
    _check(ctx, load().fast_station_clusters(ctx, _dptr(d_i), _dptr(d_j), _dptr(d_sim), n, gap, width, min_n,
                                             ctypes.byref(out), _stream(stream)))
    return out


def fast_clusters_view(res, owner=None):
    """(n, boxes [n * 6] int64 view)."""
    n = ctypes.c_uint64()
    b = ctypes.c_void_p()
    _check(None, load().fast_clusters_view(res, ctypes.byref(n), ctypes.byref(b)))
    return n.value, _view(b.value, 6 * n.value, "<i8", owner)


def fast_clusters_free(res):
    load().fast_clusters_free(res)


def fast_get_stats(ctx) -> dict:
    s = fast_stats()
    _check(ctx, load().fast_get_stats(ctx, ctypes.byref(s)))
    return s.as_dict()


def fast_set_option(ctx, name: str, value: float):
    _check(ctx, load().fast_set_option(ctx, name.encode(), float(value)))


def header_functions() -> list[str]:
    """Names of the entry points declared in include/*.h."""
    import glob
    import re
    names = []
    for h in sorted(glob.glob(os.path.join(HERE, "..", "include", "*.h"))):
        src = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names += re.findall(r"^\s*(?:[A-Za-z_][\w\s\*]*?[\s\*])(fast_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def fast_last_error(ctx) -> str:
    return load().fast_last_error(ctx).decode()


def fast_table_sort_static(d_keys, n: int, d_skey, d_sid, stream=None):
    """Sorts one table's keys with the library's fixed scratch (no allocation)."""
    _check(None, load().fast_table_sort_static(_dptr(d_keys), n, _dptr(d_skey), _dptr(d_sid), _stream(stream)))


# ------------------------------------------------------------- serving

def _scheck(srv, status: int):
    if status != FAST_OK:
        raise FastError(status, load().fast_server_last_error(srv).decode() if srv else "")


def fast_server_create(params: dict, n_stations: int, max_stream_windows: int, hbm_budget_bytes: int = 0):
    out = ctypes.c_void_p()
    _scheck(None, load().fast_server_create(ctypes.byref(params_struct(params)), n_stations, max_stream_windows,
                                            hbm_budget_bytes, ctypes.byref(out)))
    return out


def fast_server_destroy(srv):
    load().fast_server_destroy(srv)


def fast_server_last_error(srv) -> str:
    return load().fast_server_last_error(srv).decode()


def fast_server_load_history(srv, station: int, h_idx):
    N, ld = h_idx.shape
    _scheck(srv, load().fast_server_load_history(srv, station, _hptr(h_idx), N, ld))


def fast_stream_submit(srv, station: int, h_idx) -> int:
    n, ld = h_idx.shape
    rid = ctypes.c_uint64()
    _scheck(srv, load().fast_stream_submit(srv, station, _hptr(h_idx), n, ld, ctypes.byref(rid)))
    return rid.value


def fast_stream_poll(srv, req_id: int, timeout_us: int = 0):
    """None while pending; else (first_id, i, j, votes) as numpy copies."""
    import numpy as np
    M, first = ctypes.c_uint64(), ctypes.c_uint64()
    pi, pj, pv = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
    st = load().fast_stream_poll(srv, req_id, timeout_us, ctypes.byref(M), ctypes.byref(first), ctypes.byref(pi),
                                 ctypes.byref(pj), ctypes.byref(pv))
    if st == FAST_EPENDING:
        return None
    _scheck(srv, st)
    m = M.value

    def arr(p, ct, dt):
        if not m:
            return np.empty(0, dt)
        return np.ctypeslib.as_array(ctypes.cast(p, ctypes.POINTER(ct)), (m,)).copy()

    return first.value, arr(pi, ctypes.c_uint32, np.uint32), arr(pj, ctypes.c_uint32, np.uint32), \
        arr(pv, ctypes.c_uint8, np.uint8)


def fast_stream_latency(srv, req_id: int) -> float:
    sec = ctypes.c_double()
    _scheck(srv, load().fast_stream_latency(srv, req_id, ctypes.byref(sec)))
    return sec.value


def fast_stream_release(srv, req_id: int):
    _scheck(srv, load().fast_stream_release(srv, req_id))


def fast_server_inject_failure(srv, req_id: int):
    _scheck(srv, load().fast_server_inject_failure(srv, req_id))


def fast_server_hold_budget(srv, nbytes: int):
    _scheck(srv, load().fast_server_hold_budget(srv, nbytes))


def fast_server_set_option(srv, name: str, value: float):
    _scheck(srv, load().fast_server_set_option(srv, name.encode(), float(value)))


def fast_detect_batch(ctx, d_idx, station_N, ld: int, stream=None):
    """One pass over several stations (rows concatenated in d_idx); one result per station."""
    n = len(station_N)
    arr = (ctypes.c_uint64 * n)(*[int(x) for x in station_N])
    out = (ctypes.c_void_p * n)()
    _check(ctx, load().fast_detect_batch(ctx, _dptr(d_idx), ctypes.cast(arr, ctypes.c_void_p), n, ld,
                                         ctypes.cast(out, ctypes.c_void_p), _stream(stream)))
    return [ctypes.c_void_p(out[k]) for k in range(n)]


# ------------------------------------------------------------- batch plans

def fast_plan_create(ctx, d_idx, station_N, ld: int, stream):
    """A batch plan over the rows of d_idx (read again on every run)."""
    n = len(station_N)
    arr = (ctypes.c_uint64 * n)(*[int(x) for x in station_N])
    out = ctypes.c_void_p()
    _check(ctx, load().fast_plan_create(ctx, _dptr(d_idx), ctypes.cast(arr, ctypes.c_void_p), n, ld, _stream(stream),
                                        ctypes.byref(out)))
    return out


def fast_plan_run(ctx, plan, n_st: int, stream):
    out = (ctypes.c_void_p * n_st)()
    _check(ctx, load().fast_plan_run(plan, ctypes.cast(out, ctypes.c_void_p), _stream(stream)))
    return [ctypes.c_void_p(out[k]) for k in range(n_st)]


def fast_plan_info(plan) -> dict:
    info = fast_plan_info_t()
    _check(None, load().fast_plan_info(plan, ctypes.byref(info)))
    return {"graph_nodes": info.graph_nodes, "graph_kernels": info.graph_kernels, "arena_bytes": info.arena_bytes,
            "build_ms": info.build_ms, "tuned": bool(info.tuned), "best": info.best.as_dict(),
            "tried": [info.tried[k].as_dict() for k in range(info.n_tried)]}


def fast_plan_destroy(plan):
    load().fast_plan_destroy(plan)
