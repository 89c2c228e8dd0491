"""Streaming server vs the oracle's serial replay (GPU).

Each request must equal the replay of its station's submission sequence,
whether requests run one at a time or all at once across stations.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

N0 = 4000
SIZES = [60, 75, 400, 130, 60, 250, 90, 333, 61, 120]  # windows per request


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1803_09835_gb300 import _build
    _build.build()
    assert torch.cuda.is_available()


def _station(s, **over):
    w = synth.scaled("c3", N0 + sum(SIZES), station=s, D=2048, K=100, b=30, **over)
    return w, synth.generate(w, ld=104)


def _replay(p, idx, K):
    keys = oracle.keys(p, np.ascontiguousarray(idx[:, :K]))
    hd = oracle.drop(p, np.ascontiguousarray(keys[:, :N0]))
    out, j0 = [], N0
    for n in SIZES:
        out.append(oracle.stream_query(p, np.ascontiguousarray(keys[:, :j0 + n]), N0, j0, hd))
        j0 += n
    return out


def _server(p, n_st, **kw):
    from paper_1803_09835_gb300 import Server
    return Server(p, n_st, max_stream_windows=sum(SIZES) + 16, **kw)


def _slices(idx):
    out, j0 = [], N0
    for n in SIZES:
        out.append(idx[j0:j0 + n])
        j0 += n
    return out


def _same(a, b):
    return all(np.array_equal(x, y) for x, y in zip(a, b))


def test_concurrent_stations_match_serial_replay_and_alone():
    stations = [_station(s) for s in range(3)]
    p = stations[0][0].params()
    want = [_replay(p, idx, w.K) for w, idx in stations]
    assert sum(len(r[0]) for st in want for r in st) > 0

    # all requests of all stations submitted at once
    srv = _server(p, 3)
    for s, (w, idx) in enumerate(stations):
        srv.load_history(s, idx[:N0])
    ids = [[srv.submit(s, sl) for sl in _slices(idx)] for s, (w, idx) in enumerate(stations)]
    mix = [[srv.wait(r) for r in row] for row in ids]
    srv.close()

    # the same sequences, one request at a time on a fresh server
    srv = _server(p, 3)
    for s, (w, idx) in enumerate(stations):
        srv.load_history(s, idx[:N0])
    alone = []
    for s, (w, idx) in enumerate(stations):
        alone.append([srv.wait(srv.submit(s, sl)) for sl in _slices(idx)])
    srv.close()

    for s in range(3):
        j0 = N0
        for q, n in enumerate(SIZES):
            first, i, j, v = mix[s][q]
            assert first == j0
            assert _same((i, j, v), want[s][q]), f"station {s} request {q}"
            assert _same(alone[s][q][1:], (i, j, v)) and alone[s][q][0] == first
            j0 += n


def test_failure_injection_poll_timeout_and_capacity():
    from paper_1803_09835_gb300 import FastError, _lib
    w, idx = _station(5)
    p = w.params()
    srv = _server(p, 1)
    srv.load_history(0, idx[:N0])
    sl = _slices(idx)
    r0 = srv.submit(0, sl[0])
    srv.inject_failure(r0 + 1)
    r1 = srv.submit(0, sl[1])
    r2 = srv.submit(0, sl[2])
    assert srv.wait(r0) is not None
    with pytest.raises(FastError) as e:
        srv.wait(r1)
    assert e.value.status == _lib.FAST_EINTERNAL
    assert srv.wait(r2) is not None
    # a request past the station's delta capacity fails cleanly
    big = np.tile(sl[0], (30, 1))  # 1800 windows: more than the delta has left
    with pytest.raises(FastError) as e:
        srv.wait(srv.submit(0, big))
    assert e.value.status == _lib.FAST_EBUDGET
    srv.close()


def test_budget_admission_serialises_but_stays_exact():
    from paper_1803_09835_gb300 import FastError
    w, idx = _station(7)
    p = w.params()
    want = _replay(p, idx, w.K)
    # room for the resident tables plus about one request's working-set estimate
    srv = _server(p, 2, hbm_budget_bytes=24 << 20)
    srv.load_history(0, idx[:N0])
    srv.load_history(1, idx[:N0])
    ids = [srv.submit(0, sl) for sl in _slices(idx)]
    got = [srv.wait(r) for r in ids]
    for q in range(len(SIZES)):
        assert _same(got[q][1:], want[q])
    srv.close()
    with pytest.raises(FastError):
        tiny = _server(p, 1, hbm_budget_bytes=1 << 20)


def test_dense_groups_in_requests_stay_exact():
    # With large_min small enough for the noise and template copies of the
    # history to form dense groups, request windows meeting them are compared
    # with the groups key by key; results must not change.
    stations = [_station(s) for s in (11, 12)]
    p = stations[0][0].params()
    want = [_replay(p, idx, w.K) for w, idx in stations]
    for lm in (6, 12):
        srv = _server(p, 2, large_min=lm)
        for s, (w, idx) in enumerate(stations):
            srv.load_history(s, idx[:N0])
        ids = [[srv.submit(s, sl) for sl in _slices(idx)] for s, (w, idx) in enumerate(stations)]
        got = [[srv.wait(r) for r in row] for row in ids]
        srv.close()
        for s in range(2):
            for q in range(len(SIZES)):
                assert _same(got[s][q][1:], want[s][q]), f"large_min {lm} station {s} request {q}"


def test_admission_wait_is_bounded_and_short_polls_pend():
    # A request whose working set can never be admitted (the whole budget is
    # held by the test hook, as if by a request that never ends) stays
    # pending, then fails with FAST_ETIMEOUT when the admission wait runs out;
    # all of it on the host, nothing on the GPU waits.  Released, the budget
    # admits the next request again.
    import time

    from paper_1803_09835_gb300 import FastError, _lib
    w, idx = _station(9)
    p = w.params()
    budget = 64 << 20
    srv = _server(p, 1, hbm_budget_bytes=budget)
    srv.load_history(0, idx[:N0])
    sl = _slices(idx)
    srv.set_option("admit_timeout_ms", 400)
    srv.hold_budget(budget)
    t0 = time.perf_counter()
    r0 = srv.submit(0, sl[0])
    assert srv.poll(r0, 0.0) is None            # FAST_EPENDING at once
    assert srv.poll(r0, 0.001) is None          # and after a 1 ms wait
    with pytest.raises(FastError) as e:
        srv.wait(r0, timeout_s=60.0)
    assert e.value.status == _lib.FAST_ETIMEOUT
    assert 0.35 < time.perf_counter() - t0 < 30.0
    srv.hold_budget(0)
    first, i, j, v = srv.wait(srv.submit(0, sl[1]), timeout_s=60.0)
    assert first == N0 + SIZES[0]               # ids continue the station timeline
    assert np.all(j >= first) and np.all(i < j)
    with pytest.raises(FastError):
        srv.set_option("admit_timeout_ms", -1)
    srv.close()


def test_c3_shape_requests_match_serial_replay():
    # the streaming configuration's own shape: D = 8192, K = 400, Min-Max
    # b = 100 x r = 4, v = 4, E = 10, 0.5 % filter frozen on the history;
    # each request element-wise equal to the replay, alone and in the mix
    from paper_1803_09835_gb300 import Server
    n0 = 20_000
    stations = []
    for st in range(2):
        w = synth.scaled("c3", n0 + sum(SIZES), station=st)
        stations.append((w, synth.generate(w, ld=400)))
    p = stations[0][0].params()
    want = []
    for w, idx in stations:
        keys = oracle.keys(p, idx)
        hd = oracle.drop(p, np.ascontiguousarray(keys[:, :n0]))
        rows, j0 = [], n0
        for n in SIZES:
            rows.append(oracle.stream_query(p, np.ascontiguousarray(keys[:, :j0 + n]), n0, j0, hd))
            j0 += n
        want.append(rows)
    assert sum(len(r[0]) for st in want for r in st) > 0

    def run(mixed):
        srv = Server(p, 2, max_stream_windows=sum(SIZES) + 16)
        for s, (w, idx) in enumerate(stations):
            srv.load_history(s, idx[:n0])
        out = [[None] * len(SIZES) for _ in stations]
        if mixed:
            ids = []
            for q in range(len(SIZES)):
                for s, (w, idx) in enumerate(stations):
                    j0 = n0 + sum(SIZES[:q])
                    ids.append((s, q, srv.submit(s, idx[j0:j0 + SIZES[q]])))
            for s, q, r in ids:
                out[s][q] = srv.wait(r)
        else:
            for s, (w, idx) in enumerate(stations):
                for q in range(len(SIZES)):
                    j0 = n0 + sum(SIZES[:q])
                    out[s][q] = srv.wait(srv.submit(s, idx[j0:j0 + SIZES[q]]))
        srv.close()
        return out

    for got in (run(False), run(True)):
        for s in range(2):
            for q in range(len(SIZES)):
                first, i, j, v = got[s][q]
                assert first == n0 + sum(SIZES[:q])
                assert _same((i, j, v), want[s][q]), f"station {s} request {q}"
