"""Splitting one station's search over several GPUs by table group.

Each rank owns a contiguous group of the b tables (§6.4: tables, and the
work per table, are independent until the votes are summed).  The exchange
steps of that split live here, as host-side orchestration around
``torch.distributed`` (NCCL on GPUs, gloo on CPU ranks):

* the occurrence filter (§6.5) needs, per fingerprint, the number of tables
  whose bucket is heavy: every rank counts over its own tables, one
  all-reduce (sum) gives the totals, and the drop rule is applied to them;
* the votes of a pair are spread over the ranks: every rank holds its
  partial votes (pairs sharing a bucket in at least one of its tables, with
  the number of such tables); each pair is owned by one rank, chosen by a
  hash of (i, j); one all-to-all sends every partial entry to its owner,
  which sums, applies the threshold v and orders its pairs by (i, j).

The concatenation of the owners' lists, merged by (i, j), is the search
over all b tables (votes are sums over tables).  No step here looks at
fingerprints or keys: the per-rank partial votes and heavy counts come
from the search library (or any source of the same quantities).
"""
from __future__ import annotations

import numpy as np

_MIX = 0x9E3779B97F4A7C15


def table_range(b: int, rank: int, world: int) -> tuple[int, int]:
    """Tables [t0, t1) owned by `rank`: b split into `world` contiguous groups
    whose sizes differ by at most one."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    return b * rank // world, b * (rank + 1) // world


def owner(i: np.ndarray, j: np.ndarray, world: int) -> np.ndarray:
    """Rank owning each pair: a multiplicative hash of the packed (i, j)."""
    key = (i.astype(np.uint64) << np.uint64(32)) | j.astype(np.uint64)
    with np.errstate(over="ignore"):
        h = key * np.uint64(_MIX)
    return ((h >> np.uint64(32)) % np.uint64(world)).astype(np.int64)


def all_reduce_counts(dist, counts: np.ndarray) -> np.ndarray:
    """Sum of every rank's per-fingerprint counts (the heavy-table counts of
    the occurrence filter)."""
    import torch
    t = torch.from_numpy(np.ascontiguousarray(counts, dtype=np.int32))
    if dist.get_backend() == "nccl":
        t = t.cuda()
    dist.all_reduce(t)
    return t.cpu().numpy().astype(np.uint32)


def drop_from_heavy(heavy_total: np.ndarray, b: int) -> np.ndarray:
    """The static filter's rule on the summed counts: dropped iff heavy in
    strictly more than b/2 tables."""
    return (2 * heavy_total.astype(np.int64) > b).astype(np.uint8)


def exchange(dist, i: np.ndarray, j: np.ndarray, votes: np.ndarray):
    """Sends every partial (i, j, votes) entry to the rank owning its pair
    (one all-to-all of the entry counts, one of the packed entries); returns
    the entries this rank received, unordered."""
    import torch
    world = dist.get_world_size()
    dest = owner(i, j, world)
    order = np.argsort(dest, kind="stable")
    packed = ((i.astype(np.int64) << 36) | (j.astype(np.int64) << 8) | votes.astype(np.int64))[order]
    send = np.bincount(dest, minlength=world).astype(np.int64)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    send_t = torch.from_numpy(send).to(dev)
    recv_t = torch.empty_like(send_t)
    dist.all_to_all_single(recv_t, send_t)
    recv = recv_t.cpu().numpy()
    out = torch.empty(int(recv.sum()), dtype=torch.int64, device=dev)
    dist.all_to_all_single(out, torch.from_numpy(packed).to(dev), output_split_sizes=recv.tolist(),
                           input_split_sizes=send.tolist())
    got = out.cpu().numpy()
    return ((got >> 36) & 0xFFFFFFF).astype(np.uint32), ((got >> 8) & 0xFFFFFFF).astype(np.uint32), \
        (got & 0xFF).astype(np.uint32)


def reduce_owned(i: np.ndarray, j: np.ndarray, votes: np.ndarray, v: int):
    """Sums the received partial votes per pair, keeps sums >= v, in (i, j)
    order: this rank's share of the detection list."""
    key = (i.astype(np.uint64) << np.uint64(32)) | j.astype(np.uint64)
    uk, inv = np.unique(key, return_inverse=True)
    tot = np.bincount(inv, weights=votes, minlength=len(uk)).astype(np.int64)
    keep = tot >= v
    uk = uk[keep]
    return (uk >> np.uint64(32)).astype(np.uint32), (uk & np.uint64(0xFFFFFFFF)).astype(np.uint32), \
        tot[keep].astype(np.uint8)


def gather_sorted(dist, part, root: int = 0):
    """The owners' lists merged into one (i, j)-ordered list on `root`
    (None elsewhere)."""
    every = [None] * dist.get_world_size() if dist.get_rank() == root else None
    dist.gather_object(part, every, dst=root)
    if dist.get_rank() != root:
        return None
    i = np.concatenate([p[0] for p in every])
    j = np.concatenate([p[1] for p in every])
    v = np.concatenate([p[2] for p in every])
    o = np.lexsort((j, i))
    return i[o], j[o], v[o]
