"""Seeded synthetic fingerprint workloads shaped like the paper's station data.

The paper's inputs (one year of 100 Hz GeoNet data per station, a decade of
NCEDC data, §8 "Dataset") are not available, so every input here is drawn by
``gen.c`` from a counter-based generator.  This module is the single input
source shared by the CUDA path and the oracle; it contains none of the search
method's arithmetic (no hashing, no tables, no votes).

Workloads (all ids are 0-based window indices, 1 window = 1 s lag):

* ``c0``  N=8,192, D=2048, K=100, MinHash b=16 x r=4, v=2, E=5, filter off;
          40 templates x U{5..20} repeats at 10 % re-draw, the rest uniform.
* ``c1``  N=7,776,000 (3 months), D=8192, K=400, Min-Max b=100 x r=4, v=4,
          E=10, occurrence filter 0.5 % in > b/2 tables; 2,000 templates x
          U{3..50} at 15 %; periodic noise every 60 s, 300 s and 3600 s at 5 %.
* ``c2``  12 stations of 1..12 months (N_s = s * 2,592,000), C1's density per
          station, templates shared across stations at offsets U{0..30}.
* ``c3``  streaming: C1-shaped history per station plus request batches of
          60..3600 windows (log-uniform), Poisson arrivals.
* ``c4``  N=157,680,000 (5 years); 20,000 templates x U{3..200} at 15 %;
          periodic sources every 30, 60, 90, 3600 and 86400 s at 5 %.

Any workload can draw imbalanced bits (``skew``: bit weights
(1 + rank)^-skew over a random ranking of the D bits) with co-occurring
pairs (``corr``: a drawn bit's rank neighbour is set with it at that
probability), the structure §6.3 blames for oversized buckets.

``scaled(name, n)`` keeps a workload's shape (densities per window, periods,
parameters) at a smaller N for tests.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field, replace

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB = os.path.join(_HERE, "libsynth.so")

# One hash seed per deployment, shared by stations, history and requests.
HASH_SEED = 0x1803098350
MONTH = 2_592_000  # windows in 30 days at 1 s lag


def gen_seed(cfg_index: int, station: int) -> int:
    return 1803098350 + 100 * cfg_index + station


@dataclass(frozen=True)
class Workload:
    """Search parameters plus the recipe of one station's synthetic windows."""

    name: str
    N: int
    D: int
    K: int
    b: int
    r: int
    kind: int  # 0 MinHash, 1 Min-Max
    v: int
    excl: int
    occ_num: int
    occ_den: int
    seed: int  # generator seed of this station
    hash_seed: int = HASH_SEED
    periods: tuple = ()
    per_redraw: float = 0.05
    n_templates: int = 0
    rep_lo: int = 1
    rep_hi: int = 1
    tpl_redraw: float = 0.15
    tpl_seed: int = 0
    place_range: int = 0
    tpl_offset_max: int = 0
    skew: float = 0.0  # bit weights (1 + rank)^-skew over a random ranking of the D bits (0 = uniform)
    corr: float = 0.0  # probability that a drawn bit's partner (neighbouring rank) is set with it
    extra: dict = field(default_factory=dict, compare=False)

    def params(self) -> dict:
        return dict(D=self.D, K=self.K, b=self.b, r=self.r, kind=self.kind, seed=self.hash_seed,
                    v=self.v, excl=self.excl, occ_num=self.occ_num, occ_den=self.occ_den)


def _c1(N=7_776_000, station=0, cfg_index=1, n_templates=2000):
    s = gen_seed(cfg_index, station)
    return Workload("c1", N, 8192, 400, 100, 4, 1, 4, 10, 5, 1000, s, periods=(60, 300, 3600),
                    per_redraw=0.05, n_templates=n_templates, rep_lo=3, rep_hi=50, tpl_redraw=0.15,
                    tpl_seed=s)


def workload(name: str, station: int = 0) -> Workload:
    if name == "c0":
        s = gen_seed(0, station)
        return Workload("c0", 8192, 2048, 100, 16, 4, 0, 2, 5, 0, 1000, s, n_templates=40,
                        rep_lo=5, rep_hi=20, tpl_redraw=0.10, tpl_seed=s)
    if name == "c1":
        return _c1(station=station)
    if name == "c2":
        # station s (0-based) covers s+1 months; templates shared network-wide
        months = station + 1
        N = months * MONTH
        w = _c1(N=N, station=station, cfg_index=2, n_templates=round(2000 * 12 / 3))
        return replace(w, name="c2", tpl_seed=gen_seed(2, 99), place_range=12 * MONTH, tpl_offset_max=30)
    if name == "c3":
        return replace(_c1(station=station, cfg_index=3), name="c3")
    if name == "c4":
        s = gen_seed(4, station)
        return Workload("c4", 157_680_000, 8192, 400, 100, 4, 1, 4, 10, 5, 1000, s,
                        periods=(30, 60, 90, 3600, 86400), per_redraw=0.05, n_templates=20_000,
                        rep_lo=3, rep_hi=200, tpl_redraw=0.15, tpl_seed=s)
    raise KeyError(name)


def scaled(name: str, n: int, station: int = 0, **over) -> Workload:
    """The workload's shape at N = n: template count scaled with N, periods kept."""
    w = workload(name, station)
    nt = max(1, round(w.n_templates * n / w.N)) if w.n_templates else 0
    pr = round(w.place_range * n / w.N) if w.place_range else 0
    return replace(w, name=f"{name}@{n}", N=n, n_templates=nt, place_range=pr, **over)


def _load():
    if not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        build()
    lib = ctypes.CDLL(_LIB)
    u64, u32, i32, dbl, vp = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
    lib.synth_generate.restype = i32
    lib.synth_generate.argtypes = [u64, u32, u32, vp, u32, u64, u32, vp, dbl, u32, u32, u32, dbl,
                                   u64, u64, u32, i32, vp]
    lib.synth_generate_rows.restype = i32
    lib.synth_generate_rows.argtypes = [u64, u64, u64, u32, u32, vp, u32, u64, u32, vp, dbl, u32, u32, u32, dbl,
                                        u64, u64, u32, i32, vp, dbl, dbl]
    lib.synth_generate_ids.restype = i32
    lib.synth_generate_ids.argtypes = [u64, vp, u64, u32, u32, vp, u32, u64, u32, vp, dbl, u32, u32, u32, dbl,
                                       u64, u64, u32, i32, vp, dbl, dbl]
    return lib


def build() -> str:
    """Compile gen.c into libsynth.so (plain C, no GPU)."""
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-shared", "-fPIC", "-pthread",
                           _SRC, "-o", tmp, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def owners(w: Workload, rows: tuple | None = None) -> np.ndarray:
    """Only the source codes of windows r0 .. r1 - 1 (no fingerprints drawn):
    0 random, OWNER_PERIODIC | p, OWNER_TEMPLATE | tau."""
    global _lib
    if _lib is None:
        _lib = _load()
    r0, r1 = rows if rows is not None else (0, w.N)
    if not 0 <= r0 <= r1 <= w.N:
        raise ValueError("rows outside the station")
    own = np.empty(max(1, r1 - r0), dtype=np.uint32)
    periods = (ctypes.c_uint64 * max(1, len(w.periods)))(*w.periods)
    rc = _lib.synth_generate_rows(w.N, r0, r1 - r0, w.D, w.K, None, w.K, w.seed, len(w.periods), periods,
                                  w.per_redraw, w.n_templates, w.rep_lo, w.rep_hi, w.tpl_redraw, w.tpl_seed or w.seed,
                                  w.place_range, w.tpl_offset_max, 0, own.ctypes.data, float(w.skew), float(w.corr))
    if rc < 0:
        raise ValueError("synth_generate_rows: bad arguments")
    return own[:r1 - r0]


def generate_ids(w: Workload, ids, ld: int | None = None) -> np.ndarray:
    """The windows ids (any order) of the station, [len(ids), ld] uint16: each
    exactly that row of the whole station."""
    global _lib
    if _lib is None:
        _lib = _load()
    ld = ld or w.K
    ids = np.ascontiguousarray(ids, dtype=np.uint64)
    out = np.empty((max(1, len(ids)), ld), dtype=np.uint16)
    periods = (ctypes.c_uint64 * max(1, len(w.periods)))(*w.periods)
    rc = _lib.synth_generate_ids(w.N, ids.ctypes.data, len(ids), w.D, w.K, out.ctypes.data, ld, w.seed,
                                 len(w.periods), periods, w.per_redraw, w.n_templates, w.rep_lo, w.rep_hi,
                                 w.tpl_redraw, w.tpl_seed or w.seed, w.place_range, w.tpl_offset_max, 0, None,
                                 float(w.skew), float(w.corr))
    if rc < 0:
        raise ValueError("synth_generate_ids: bad arguments")
    return out[:len(ids)]


def generate(w: Workload, ld: int | None = None, out=None, threads: int = 0, owner: bool = False,
             rows: tuple | None = None):
    """Draw the workload's fingerprints into a [N, ld] uint16 array.

    ``out`` may be any writable C-contiguous uint16 buffer exposing
    ``__array_interface__`` or a ``data_ptr()`` (e.g. a pinned torch tensor).
    ``rows = (r0, r1)`` draws only windows r0 .. r1 - 1 (exactly those rows
    of the whole station) into an [r1 - r0, ld] array.
    Returns ``out`` (or a new numpy array), plus the owner codes if asked.
    """
    global _lib
    if _lib is None:
        _lib = _load()
    ld = ld or w.K
    r0, r1 = rows if rows is not None else (0, w.N)
    if not 0 <= r0 <= r1 <= w.N:
        raise ValueError("rows outside the station")
    n = r1 - r0
    if out is None:
        out = np.empty((n, ld), dtype=np.uint16)
    ptr = out.data_ptr() if hasattr(out, "data_ptr") else out.__array_interface__["data"][0]
    own = np.empty(n, dtype=np.uint32) if owner else None
    periods = (ctypes.c_uint64 * max(1, len(w.periods)))(*w.periods)
    rc = _lib.synth_generate_rows(w.N, r0, n, w.D, w.K, ptr, ld, w.seed, len(w.periods), periods, w.per_redraw,
                                  w.n_templates, w.rep_lo, w.rep_hi, w.tpl_redraw, w.tpl_seed or w.seed,
                                  w.place_range, w.tpl_offset_max, threads,
                                  own.ctypes.data if owner else None, float(w.skew), float(w.corr))
    if rc < 0:
        raise ValueError("synth_generate: bad arguments")
    return (out, own) if owner else out


OWNER_PERIODIC = 1 << 30
OWNER_TEMPLATE = 2 << 30


def requests(n_req: int, rate_hz: float, lo: int = 60, hi: int = 3600, n_stations: int = 12,
             seed: int = gen_seed(3, 99)):
    """Open-loop request schedule for the streaming workload.

    Returns arrays (arrival_s, station, size): Poisson arrivals at ``rate_hz``,
    a uniform station and a log-uniform batch size in [lo, hi] windows.
    """
    rng = np.random.Generator(np.random.Philox(key=seed))
    gaps = rng.exponential(1.0 / rate_hz, n_req)
    st = rng.integers(0, n_stations, n_req)
    size = np.floor(np.exp(rng.uniform(np.log(lo), np.log(hi), n_req))).astype(np.int64)
    return np.cumsum(gaps), st, np.clip(size, lo, hi)
