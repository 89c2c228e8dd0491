"""Query-only hashing on the GPU (§6.4 "Partition": hash only the queries,
check every other item against their buckets) vs the oracle's streamed
request, and vs the server running the same request with the history's
tables resident: one list, three ways."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1803_09835_gb300 import _build
    _build.build()
    assert torch.cuda.is_available()


def _case(n0, n, **over):
    w = synth.scaled("c3", n0 + n, **over)
    idx = synth.generate(w, ld=((w.K + 7) // 8) * 8)
    return w, idx


def _eq(a, b):
    assert len(a[0]) == len(b[0]), (len(a[0]), len(b[0]))
    assert all(np.array_equal(x, y) for x, y in zip(a, b))


def _oracle(p, idx, K, n0, filt=True):
    keys = oracle.keys(p, np.ascontiguousarray(idx[:, :K]))
    hd = oracle.drop(p, np.ascontiguousarray(keys[:, :n0])) if filt and n0 else None
    return oracle.stream_query(p, keys, n0, n0, hd)


@pytest.mark.parametrize("n0,n,over", [
    (20_000, 600, dict(D=2048, K=100, b=30, occ_num=0)),      # no filter
    (20_000, 600, dict(D=2048, K=100, b=30)),                 # filter: history flags + heavy test of the batch
    (60_000, 3_000, dict()),                                  # C3's own shape, D=8192, K=400, Min-Max 100 x 4
    (0, 2_000, dict(D=2048, K=100, b=30)),                    # no history: pairs inside the batch only
    (15_000, 20_000, dict(D=2048, K=100, b=20, v=3)),         # batch larger than the shared-memory staging
])
def test_query_only_matches_streamed_request(n0, n, over):
    from paper_1803_09835_gb300 import Searcher
    w, idx = _case(n0, n, **over)
    p = w.params()
    s = Searcher(p)
    d = torch.from_numpy(idx).cuda()
    hist, batch = d[:n0], d[n0:]
    drop = None
    if n0 and p["occ_num"]:
        sig = s.sig(hist)
        tb = s.build_tables(sig)
        drop = tb.drop.clone()
        tb.free()
    r = s.query_only(hist, batch, hist_drop=drop)
    got = r.numpy()
    r.free()
    want = _oracle(p, idx, w.K, n0)
    assert len(want[0]) > 0
    _eq(got, want)
    s.close()


def test_query_only_equals_the_server_with_resident_tables():
    from paper_1803_09835_gb300 import Searcher, Server
    n0, n = 30_000, 1_500
    w, idx = _case(n0, n, D=2048, K=100, b=30)
    p = w.params()
    srv = Server(p, 1, max_stream_windows=n + 16)
    srv.load_history(0, idx[:n0])
    first, si, sj, sv = srv.wait(srv.submit(0, idx[n0:]))
    srv.close()
    s = Searcher(p)
    d = torch.from_numpy(idx).cuda()
    tb = s.build_tables(s.sig(d[:n0]))
    r = s.query_only(d[:n0], d[n0:], hist_drop=tb.drop)
    assert first == n0
    _eq(r.numpy(), (si, sj, sv))
    r.free()
    tb.free()
    s.close()


def test_query_only_empty_batch_and_bad_arguments():
    from paper_1803_09835_gb300 import FastError, Searcher
    w, idx = _case(5_000, 10, D=2048, K=100, b=30)
    s = Searcher(w.params())
    d = torch.from_numpy(idx).cuda()
    r = s.query_only(d[:5_000], d[5_000:5_000])
    assert r.M == 0
    with pytest.raises(FastError):
        s.query_only(d[:5_000, :50].contiguous(), d[5_000:, :50].contiguous())  # ld < K
    s.close()
