"""CPU oracle of the LSH fingerprint search -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The
product path (``paper_1803_09835_gb300``) never does, and shares no code with
it.  See ``oracle.c`` for the readings of the paper it implements.

Every function takes a plain ``params`` dict with keys
``D, K, b, r, kind, seed, v, excl, occ_num, occ_den`` and numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")


class _Params(ctypes.Structure):
    _fields_ = [("D", ctypes.c_uint32), ("K", ctypes.c_uint32), ("b", ctypes.c_uint32),
                ("r", ctypes.c_uint32), ("kind", ctypes.c_uint32), ("seed", ctypes.c_uint64),
                ("v", ctypes.c_uint32), ("excl", ctypes.c_uint32), ("occ_num", ctypes.c_uint32),
                ("occ_den", ctypes.c_uint32)]


def build() -> str:
    """Compile oracle.c into liboracle.so (plain C, -O2, pthreads)."""
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-shared", "-fPIC", "-pthread",
                           _SRC, "-o", tmp])
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _L():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        build()
    lib = ctypes.CDLL(_LIB)
    P, u64, u32, i32, vp = ctypes.POINTER(_Params), ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, ctypes.c_void_p
    pp = ctypes.POINTER
    sig = {
        "orc_mix64": (u64, [u64]),
        "orc_sm64": (u64, [u64, u64]),
        "orc_nfuncs": (u32, [P]),
        "orc_hash_params": (None, [P, vp, vp]),
        "orc_h": (u32, [u64, u64, u32]),
        "orc_values": (None, [P, vp, u64, u32, vp, vp]),
        "orc_keys": (i32, [P, vp, u64, u32, vp, i32]),
        "orc_table": (None, [vp, u64, vp, vp]),
        "orc_drop": (i32, [P, vp, u64, vp, vp, i32]),
        "orc_search": (u64, [P, vp, vp, u64, pp(vp), pp(vp), pp(vp)]),
        "orc_search_brute": (u64, [P, vp, vp, u64, pp(vp), pp(vp), pp(vp)]),
        "orc_search_row": (u64, [P, vp, vp, u64, u64, pp(vp), pp(vp)]),
        "orc_pair_votes": (u32, [P, vp, u64, u64, u64]),
        "orc_stream_query": (u64, [P, vp, u64, u64, u64, vp, pp(vp), pp(vp), pp(vp)]),
        "orc_channel_merge": (u64, [u32, vp, vp, vp, vp, u32, vp, vp, vp, u64]),
        "orc_station_clusters": (u64, [vp, vp, vp, u64, u32, u32, u32, vp, u64]),
        "orc_free": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype, fn.argtypes = res, args
    _lib = lib
    return lib


def _p(params: dict) -> _Params:
    return _Params(**{k: int(params[k]) for k, _ in _Params._fields_})


def _ptr(a: np.ndarray | None):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


def mix64(z: int) -> int:
    return _L().orc_mix64(z)


def sm64(seed: int, n: int) -> int:
    return _L().orc_sm64(seed, n)


def nfuncs(params: dict) -> int:
    return _L().orc_nfuncs(ctypes.byref(_p(params)))


def hash_params(params: dict):
    F = nfuncs(params)
    a = np.empty(F, np.uint64)
    b = np.empty(F, np.uint64)
    _L().orc_hash_params(ctypes.byref(_p(params)), _ptr(a), _ptr(b))
    return a, b


def h(a: int, b: int, x: int) -> int:
    return _L().orc_h(a, b, x)


def values(params: dict, idx: np.ndarray):
    """Per-function (min, max) arrays of shape [N, F]; max is None for MinHash."""
    idx = np.ascontiguousarray(idx, dtype=np.uint16)
    N, ld = idx.shape
    F = nfuncs(params)
    mn = np.empty((N, F), np.uint32)
    mx = np.empty((N, F), np.uint32) if params["kind"] == 1 else None
    _L().orc_values(ctypes.byref(_p(params)), _ptr(idx), N, ld, _ptr(mn), _ptr(mx))
    return mn, mx


def keys(params: dict, idx: np.ndarray, threads: int = 0, return_threads: bool = False):
    """Bucket keys, table-major [b, N] uint32."""
    idx = np.ascontiguousarray(idx, dtype=np.uint16)
    N, ld = idx.shape
    out = np.empty((params["b"], N), np.uint32)
    used = _L().orc_keys(ctypes.byref(_p(params)), _ptr(idx), N, ld, _ptr(out), threads)
    return (out, used) if return_threads else out


def table(keys_t: np.ndarray):
    """Canonical listing of one table: (key, id) sorted by key then id."""
    keys_t = np.ascontiguousarray(keys_t, dtype=np.uint32)
    N = keys_t.shape[0]
    sk = np.empty(N, np.uint32)
    si = np.empty(N, np.uint32)
    _L().orc_table(_ptr(keys_t), N, _ptr(sk), _ptr(si))
    return sk, si


def drop(params: dict, keys_: np.ndarray, threads: int = 0, heavy_cnt: bool = False):
    """Occurrence-filter drop mask [N] uint8 (and the heavy-table counts)."""
    keys_ = np.ascontiguousarray(keys_, dtype=np.uint32)
    N = keys_.shape[1]
    d = np.empty(N, np.uint8)
    c = np.empty(N, np.uint32)
    _L().orc_drop(ctypes.byref(_p(params)), _ptr(keys_), N, _ptr(d), _ptr(c), threads)
    return (d, c) if heavy_cnt else d


def _take(n, pi, pj, pv):
    L = _L()
    i = np.ctypeslib.as_array(ctypes.cast(pi, ctypes.POINTER(ctypes.c_uint32)), (n,)).copy() if n else np.empty(0, np.uint32)
    j = np.ctypeslib.as_array(ctypes.cast(pj, ctypes.POINTER(ctypes.c_uint32)), (n,)).copy() if n else np.empty(0, np.uint32)
    v = np.ctypeslib.as_array(ctypes.cast(pv, ctypes.POINTER(ctypes.c_uint8)), (n,)).copy() if n else np.empty(0, np.uint8)
    for p in (pi, pj, pv):
        L.orc_free(p)
    return i, j, v


def search(params: dict, keys_: np.ndarray, drop_: np.ndarray | None = None, brute: bool = False):
    """Detections (i, j, votes) sorted by (i, j)."""
    keys_ = np.ascontiguousarray(keys_, dtype=np.uint32)
    N = keys_.shape[1]
    pi, pj, pv = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
    fn = _L().orc_search_brute if brute else _L().orc_search
    n = fn(ctypes.byref(_p(params)), _ptr(keys_), _ptr(drop_), N, ctypes.byref(pi), ctypes.byref(pj), ctypes.byref(pv))
    return _take(n, pi, pj, pv)


def search_row(params: dict, keys_: np.ndarray, drop_: np.ndarray | None, i: int):
    """Row i of the detection list: (j, votes) for every detected j > i."""
    keys_ = np.ascontiguousarray(keys_, dtype=np.uint32)
    N = keys_.shape[1]
    pj, pv = ctypes.c_void_p(), ctypes.c_void_p()
    n = _L().orc_search_row(ctypes.byref(_p(params)), _ptr(keys_), _ptr(drop_), N, i, ctypes.byref(pj), ctypes.byref(pv))
    L = _L()
    j = np.ctypeslib.as_array(ctypes.cast(pj, ctypes.POINTER(ctypes.c_uint32)), (n,)).copy() if n else np.empty(0, np.uint32)
    v = np.ctypeslib.as_array(ctypes.cast(pv, ctypes.POINTER(ctypes.c_uint8)), (n,)).copy() if n else np.empty(0, np.uint8)
    L.orc_free(pj)
    L.orc_free(pv)
    return j, v


def pair_votes(params: dict, keys_: np.ndarray, i: int, j: int) -> int:
    keys_ = np.ascontiguousarray(keys_, dtype=np.uint32)
    return _L().orc_pair_votes(ctypes.byref(_p(params)), _ptr(keys_), keys_.shape[1], i, j)


def run(params: dict, idx: np.ndarray, threads: int = 0, brute: bool = False):
    """The whole path on the CPU: keys -> filter -> detections."""
    k = keys(params, idx, threads)
    d = drop(params, k, threads)
    return search(params, k, d, brute=brute)


def stream_query(params: dict, keys_all: np.ndarray, n0: int, j0: int, hist_drop: np.ndarray | None):
    """One streamed request by definition: pairs (i, j) with j in [j0, N)."""
    keys_all = np.ascontiguousarray(keys_all, dtype=np.uint32)
    N = keys_all.shape[1]
    pi, pj, pv = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
    n = _L().orc_stream_query(ctypes.byref(_p(params)), _ptr(keys_all), N, n0, j0, _ptr(hist_drop),
                              ctypes.byref(pi), ctypes.byref(pj), ctypes.byref(pv))
    return _take(n, pi, pj, pv)


def channel_merge(lists, thr: int):
    """Channel level (§7.1, by the sort-merge-reduce of §7.2): the channels'
    (i, j, votes) lists summed per pair and thresholded at thr.  Returns
    (i, j, summed votes) as uint32 / uint32 / uint16 arrays in (dt, idx1) order,
    dt = j - i, idx1 = i."""
    lists = [tuple(np.ascontiguousarray(a, dtype=t) for a, t in zip(l, (np.uint32, np.uint32, np.uint8)))
             for l in lists]
    nch = len(lists)
    M = np.array([len(l[0]) for l in lists] or [0], dtype=np.uint64)
    ptrs = [(ctypes.c_void_p * max(1, nch))(*[l[k].ctypes.data if len(l[k]) else None for l in lists])
            for k in range(3)]
    total = int(M.sum()) if nch else 0
    oi = np.empty(max(1, total), np.uint32)
    oj = np.empty(max(1, total), np.uint32)
    os_ = np.empty(max(1, total), np.uint16)
    n = _L().orc_channel_merge(nch, _ptr(M), ctypes.cast(ptrs[0], ctypes.c_void_p),
                               ctypes.cast(ptrs[1], ctypes.c_void_p), ctypes.cast(ptrs[2], ctypes.c_void_p),
                               thr, _ptr(oi), _ptr(oj), _ptr(os_), total)
    return oi[:n].copy(), oj[:n].copy(), os_[:n].copy()


def station_clusters(i, j, sim, gap: int, width: int, min_n: int):
    """Station level (§7.1, §7.2): thin diagonal clusters of a (dt, idx1)-ordered
    list (i, j, sim) -- runs along each diagonal with gaps below `gap`, merged
    across adjacent diagonals up to `width` diagonals, pruned below `min_n`
    entries.  Returns an int64 array [clusters, 6]: dt_min, dt_max, idx1_min,
    idx1_max, entries, summed sim, in (dt_min, idx1_min) order."""
    if gap < 1 or width < 1:
        raise ValueError("gap and width must be >= 1")
    i = np.ascontiguousarray(i, dtype=np.uint32)
    j = np.ascontiguousarray(j, dtype=np.uint32)
    sim = np.ascontiguousarray(sim, dtype=np.uint16)
    n = len(i)
    # the runs are read off consecutive entries: the list must be in (dt, idx1)
    # order (the search's own (i, j) order would split every run)
    dt = j.astype(np.int64) - i.astype(np.int64)
    if n > 1:
        ddt, di = np.diff(dt), np.diff(i.astype(np.int64))
        if (ddt < 0).any() or ((ddt == 0) & (di <= 0)).any():
            raise ValueError("station_clusters needs its entries in strictly increasing (dt, idx1) order")
    out = np.empty((max(1, n), 6), np.uint64)
    nc = _L().orc_station_clusters(_ptr(i), _ptr(j), _ptr(sim), n, gap, width, min_n, _ptr(out), max(1, n))
    return out[:nc].astype(np.int64)
