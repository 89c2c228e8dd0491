"""GB300-native LSH similarity search over binary waveform fingerprints.

The hot path of FAST-style earthquake detection (Rong et al., §6): MinHash /
Min-Max signatures, banding into per-table bucket keys, device radix sort into
hash tables, the occurrence filter, pair enumeration with near-time exclusion
and vote counting, thresholded to a canonical (i, j, votes) detection list.

All of it runs in the hand-written sm_103a kernels of ``libfast.so`` behind the
C-ABI of ``include/fast.h``; ``_lib`` binds those entry points under their C
names, and :class:`Searcher` is a convenience wrapper over them.  PyTorch only
provides device memory and streams.
"""
from __future__ import annotations

import numpy as np

from . import _lib
from ._lib import (FAST_MINHASH, FAST_MINMAX, FastError, fast_build_tables, fast_create, fast_destroy, fast_detect,
                   fast_detect_host, fast_get_stats, fast_result_free, fast_result_view, fast_search,
                   fast_server_create, fast_server_destroy, fast_server_inject_failure, fast_server_load_history,
                   fast_set_option, fast_sig, fast_stream_latency, fast_stream_poll, fast_stream_release,
                   fast_stream_submit, fast_tables_free, fast_tables_view)

__all__ = ["Searcher", "Plan", "Result", "Merged", "Clusters", "Tables", "FastError", "FAST_MINHASH", "FAST_MINMAX", "fast_create", "fast_destroy",
           "fast_sig", "fast_build_tables", "fast_tables_view", "fast_tables_free", "fast_search", "fast_detect",
           "fast_detect_host", "fast_result_view", "fast_result_free", "fast_get_stats", "fast_set_option", "Server",
           "fast_server_create", "fast_server_destroy", "fast_server_load_history", "fast_stream_submit",
           "fast_stream_poll", "fast_stream_latency", "fast_stream_release", "fast_server_inject_failure"]


def _track(searcher, obj):
    """Registers a library object with the context that made it: closing the
    context frees it first (an object may not outlive its context)."""
    if searcher is not None:
        searcher._live.add(obj)


class Result:
    """A detection list held in device memory by the library."""

    def __init__(self, handle, searcher=None):
        self.handle = handle
        _track(searcher, self)
        self.M, self.i, self.j, self.votes = fast_result_view(handle, owner=self)

    def numpy(self):
        """(i, j, votes) as numpy uint32 / uint32 / uint8 arrays."""
        return (self.i.cpu().numpy().view(np.uint32), self.j.cpu().numpy().view(np.uint32),
                self.votes.cpu().numpy())

    def free(self):
        if self.handle:
            fast_result_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Merged:
    """A channel-merged list (i, j, summed votes) in (dt, idx1) order, in device memory."""

    def __init__(self, handle, searcher=None):
        self.handle = handle
        _track(searcher, self)
        self.M, self.i, self.j, self.sim = _lib.fast_merged_view(handle, owner=self)

    def numpy(self):
        """(i, j, sim) as numpy uint32 / uint32 / uint16 arrays."""
        return (self.i.cpu().numpy().view(np.uint32), self.j.cpu().numpy().view(np.uint32),
                self.sim.cpu().numpy().view(np.uint16))

    def free(self):
        if self.handle:
            _lib.fast_merged_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Clusters:
    """Station-level clusters: rows (dt_min, dt_max, idx1_min, idx1_max, entries, sim)."""

    def __init__(self, handle, searcher=None):
        self.handle = handle
        _track(searcher, self)
        self.n, self.box = _lib.fast_clusters_view(handle, owner=self)

    def numpy(self):
        return self.box.cpu().numpy().reshape(-1, 6)

    def free(self):
        if self.handle:
            _lib.fast_clusters_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Tables:
    """Per-table sorted (key, id) arrays and the drop mask, in device memory."""

    def __init__(self, handle, sig, searcher=None):
        self.handle = handle
        _track(searcher, self)
        self.sig = sig  # the keys must outlive the tables (fast_search reads them)
        self.skey, self.sid, self.drop = fast_tables_view(handle, owner=self)

    def free(self):
        if self.handle:
            fast_tables_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Searcher:
    """One search context: parameters, hash functions, device workspace."""

    def __init__(self, params: dict, hbm_budget_bytes: int = 0, **options):
        import torch
        if not torch.cuda.is_available():
            raise FastError(_lib.FAST_ECUDA, "no CUDA device: this library has no CPU fallback")
        import weakref
        self._live = weakref.WeakSet()  # results, tables, ... made by this context
        self.params = dict(params)
        self.ctx = fast_create(self.params, hbm_budget_bytes)
        for k, v in options.items():
            fast_set_option(self.ctx, k, v)

    def close(self):
        if getattr(self, "ctx", None):
            for obj in list(self._live):  # nothing may outlive the context
                obj.free()
            fast_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_option(self, name: str, value: float):
        fast_set_option(self.ctx, name, value)

    def sig(self, idx, out=None, stream=None):
        """Bucket keys [b, N] (int32 view of uint32) of the fingerprints idx [N, ld]."""
        import torch
        N, ld = idx.shape
        if out is None:
            out = torch.empty((self.params["b"], N), dtype=torch.int32, device=idx.device)
        fast_sig(self.ctx, idx, N, ld, out, stream)
        return out

    def sig_rows(self, idx, sig, col0: int, stream=None):
        """Keys of rows col0 .. col0 + n - 1 of a station into its [b, N] key array (chunked input)."""
        n, ld = idx.shape
        _lib.fast_sig_rows(self.ctx, idx, n, ld, sig, sig.shape[1], col0, stream)

    def build_tables(self, sig, stream=None) -> Tables:
        return Tables(fast_build_tables(self.ctx, sig, sig.shape[1], stream), sig, self)

    def search(self, tables: Tables, stream=None) -> Result:
        return Result(fast_search(self.ctx, tables.handle, stream), self)

    def detect(self, idx, stream=None) -> Result:
        N, ld = idx.shape
        return Result(fast_detect(self.ctx, idx, N, ld, stream), self)

    def detect_chunked(self, N: int, ld: int, fill, chunk_rows: int = 1 << 22, stream=None) -> Result:
        """Whole path over a station produced chunk by chunk: fill(row0, n, rows)
        writes windows row0 .. row0 + n - 1 into the [n, ld] uint16 array rows."""
        return Result(_lib.fast_detect_chunked(self.ctx, N, ld, chunk_rows, fill, stream), self)

    def detect_batch(self, idx, station_N, stream=None):
        """Several stations in one pass: idx holds their rows one after another."""
        return [Result(h, self) for h in _lib.fast_detect_batch(self.ctx, idx, list(station_N), idx.shape[1],
                                                                stream)]

    def plan(self, idx, station_N, stream) -> "Plan":
        """A batch plan over idx (refill it between runs); see :class:`Plan`."""
        return Plan(self, idx, station_N, stream)

    def detect_host(self, idx: np.ndarray, cap: int | None = None, stream=None):
        """Whole path from host memory: returns (M, i, j, votes) numpy arrays."""
        N, ld = idx.shape
        if cap is None:
            cap = 1 << 20
        i = np.empty(cap, np.uint32)
        j = np.empty(cap, np.uint32)
        v = np.empty(cap, np.uint8)
        M = fast_detect_host(self.ctx, idx, N, ld, i, j, v, cap, stream)
        m = min(M, cap)
        return M, i[:m], j[:m], v[:m]

    def stats(self) -> dict:
        return fast_get_stats(self.ctx)

    def query_only(self, hist, batch, hist_drop=None, stream=None) -> Result:
        """Query-only hashing: the batch's pairs against the history (ids continue
        after it) without building tables of the history."""
        return Result(_lib.fast_query_only(self.ctx, hist, hist.shape[0], hist_drop, batch, batch.shape[0],
                                           batch.shape[1], stream), self)

    def channel_merge(self, results, N: int, thr: int, stream=None) -> Merged:
        """Channel level: the channels' Results summed per pair, kept at >= thr."""
        lists = [(r.M, r.i, r.j, r.votes) for r in results]
        return Merged(_lib.fast_channel_merge(self.ctx, N, lists, thr, stream), self)

    def station_clusters(self, merged, gap: int, width: int, min_n: int, stream=None) -> Clusters:
        """Station level over a (dt, idx1)-ordered list (a Merged, or (i, j, sim) device tensors)."""
        i, j, sim = (merged.i, merged.j, merged.sim) if isinstance(merged, Merged) else merged
        return Clusters(_lib.fast_station_clusters(self.ctx, i, j, sim, i.shape[0], gap, width, min_n, stream),
                        self)


class Plan:
    """A fixed batch shape: the build replays as a CUDA graph, the search options are autotuned once."""

    def __init__(self, searcher: Searcher, idx, station_N, stream):
        self.searcher = searcher
        self.idx = idx  # the graph reads this buffer on every run
        self.n_st = len(station_N)
        self.stream = stream
        self.handle = _lib.fast_plan_create(searcher.ctx, idx, list(station_N), idx.shape[1], stream)
        _track(searcher, self)

    def run(self):
        return [Result(h, self.searcher) for h in _lib.fast_plan_run(self.searcher.ctx, self.handle, self.n_st,
                                                                     self.stream)]

    def info(self) -> dict:
        return _lib.fast_plan_info(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            _lib.fast_plan_destroy(self.handle)
            self.handle = None

    free = close

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Streaming search: resident station histories, batches answered as they arrive."""

    def __init__(self, params: dict, n_stations: int, max_stream_windows: int, hbm_budget_bytes: int = 0,
                 **options):
        import torch
        if not torch.cuda.is_available():
            raise FastError(_lib.FAST_ECUDA, "no CUDA device: this library has no CPU fallback")
        self.params = dict(params)
        self.srv = fast_server_create(self.params, n_stations, max_stream_windows, hbm_budget_bytes)
        for k, v in options.items():
            _lib.fast_server_set_option(self.srv, k, v)

    def load_history(self, station: int, idx: np.ndarray):
        fast_server_load_history(self.srv, station, np.ascontiguousarray(idx))

    def submit(self, station: int, idx: np.ndarray) -> int:
        return fast_stream_submit(self.srv, station, np.ascontiguousarray(idx))

    def poll(self, req_id: int, timeout_s: float = 0.0):
        return fast_stream_poll(self.srv, req_id, int(timeout_s * 1e6))

    def wait(self, req_id: int, timeout_s: float = 600.0):
        r = self.poll(req_id, timeout_s)
        if r is None:
            raise FastError(_lib.FAST_ETIMEOUT, f"request {req_id} still pending after {timeout_s} s")
        return r

    def latency(self, req_id: int) -> float:
        return fast_stream_latency(self.srv, req_id)

    def release(self, req_id: int):
        fast_stream_release(self.srv, req_id)

    def inject_failure(self, req_id: int):
        fast_server_inject_failure(self.srv, req_id)

    def hold_budget(self, nbytes: int):
        _lib.fast_server_hold_budget(self.srv, nbytes)

    def set_option(self, name: str, value: float):
        _lib.fast_server_set_option(self.srv, name, value)

    def close(self):
        if getattr(self, "srv", None):
            fast_server_destroy(self.srv)
            self.srv = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
