"""The sharded encode's exchange and merge path on CPU: two gloo ranks on 127.0.0.1, two shards
per rank (four shards in all), through paper_2607_14513_gb300.shard.Exchange.

Checked: reductions (sum / minimum / maximum) and gathers in shard order; gathers of rows whose
counts differ between shards; the exclusive scan over shards; moving rows to the shards that want
them (all_to_all); combining buffers written in disjoint places; and the selection protocol of
the scales end to end. For the last, each shard's partial histograms are computed on the host by
the test (what gsc_shard_select_hist computes on the device), combined through the Exchange, and
the digit of each pass picked from the combined counts: the 16 scales of the whole scene come
out equal to the oracle's, bit for bit, although no rank ever holds the whole scene.
"""
import json
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _hist(sh, prefix, shift):
    """Per scale k (coefficients 3k..3k+2 of every Gaussian): counts of bits [shift, shift + 8) of
    |x| among the values whose higher bits equal prefix[k]'s."""
    u = sh.view(np.uint32).reshape(sh.shape[0], 16, 3) & np.uint32(0x7FFFFFFF)
    h = np.zeros((16, 256), np.int64)
    hs = shift + 8
    for k in range(16):
        v = u[:, k, :].ravel().astype(np.uint64)
        if hs < 32:
            v = v[(v >> hs) == (int(prefix[k]) >> hs)]
        np.add.at(h[k], ((v >> shift) & 255).astype(np.int64), 1)
    return h


def _rank_main(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    from paper_2607_14513_gb300 import shard
    from paper_2607_14513_gb300 import synthetic as S

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ex = shard.Exchange(2)
    res = {"n_shards": ex.n_shards, "first": ex.first}
    mine = [ex.first, ex.first + 1]
    # reductions and gathers: shard s contributes [s, -s, 10 s + 1]
    parts = [torch.tensor([s, -s, 10 * s + 1], dtype=torch.int64) for s in mine]
    res["sum"] = ex.reduce(parts, "sum").tolist()
    res["min"] = ex.reduce(parts, "min").tolist()
    res["max"] = ex.reduce(parts, "max").tolist()
    res["gather"] = ex.gather(parts).tolist()
    res["scan"] = ex.exclusive_scan(torch.tensor([5, 0, 7, 2], dtype=torch.int64)).tolist()
    # rows of different counts per shard (shard s: s + 1 rows valued 100 s + i)
    rows = [torch.tensor([[100 * s + i, s] for i in range(s + 1)], dtype=torch.int64) for s in mine]
    res["rows"] = ex.gather_rows(rows).tolist()
    # moving rows: the scene's input rows are split over the shards in input order; each shard
    # wants a seeded selection of input indices
    n = 1000
    in_bounds = [0, 170, 400, 401, 1000]
    pos = torch.arange(3 * n, dtype=torch.float32).view(n, 3)
    local = [pos[in_bounds[ex.first]:in_bounds[ex.first + 2]]]
    order = torch.from_numpy(np.random.default_rng(3).permutation(n).astype(np.int32))
    bounds = [0, 256, 512, 768, 1000]
    wanted = [order[bounds[s]:bounds[s + 1]] for s in mine]
    moved = ex.move_rows(local, in_bounds, wanted)
    res["moved_ok"] = all(torch.equal(m[0], pos[w.long()]) for m, w in zip(moved, wanted))
    # disjoint writes
    buf = torch.zeros(8, dtype=torch.uint8)
    buf[2 * rank:2 * rank + 2] = torch.tensor([rank + 1, 200 + rank], dtype=torch.uint8)
    res["disjoint"] = ex.combine_disjoint(buf).tolist()
    # the selection protocol of the scales over four shards of one scene
    sc = S.make_scene(n=6001, seed=91, clusters=4, heavy_frac=0.2)
    cuts = [0, 1000, 1001, 4000, 6001]
    sh_parts = [sc.sh[cuts[s]:cuts[s + 1]] for s in mine]
    ntot = 6001
    r = ((995 * 3 * ntot + 999) // 1000 - 1)
    prefix = np.zeros(16, np.uint64)
    rank_left = np.full(16, r, np.int64)
    for shift in (24, 16, 8, 0):
        hist = ex.reduce([torch.from_numpy(_hist(p, prefix, shift)) for p in sh_parts], "sum").numpy()
        for k in range(16):
            cum = np.concatenate([[0], np.cumsum(hist[k])])
            d = int(np.searchsorted(cum[1:], rank_left[k], side="right"))
            d = min(d, 255)
            prefix[k] |= np.uint64(d << shift)
            rank_left[k] -= cum[d]
    a = prefix.astype(np.uint32).view(np.float32)
    scales = np.where(a == 0, np.float32(1.0), np.float32(2.0) * a).astype(np.float32)
    res["scales"] = scales.view(np.uint32).tolist()
    with open(os.path.join(out_dir, "rank%d.json" % rank), "w") as f:
        json.dump(res, f)
    dist.destroy_process_group()


def test_exchange_two_ranks_two_shards_each(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.spawn(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    r = [json.load(open(tmp_path / ("rank%d.json" % i))) for i in range(2)]
    for x in r:
        assert x["n_shards"] == 4
        assert x["sum"] == [6, -6, 64] and x["min"] == [0, -3, 1] and x["max"] == [3, 0, 31]
        assert x["gather"] == [[s, -s, 10 * s + 1] for s in range(4)]
        assert x["scan"] == [0, 5, 5, 12]
        assert x["rows"] == [[100 * s + i, s] for s in range(4) for i in range(s + 1)]
        assert x["moved_ok"]
        assert x["disjoint"] == [1, 200, 2, 201, 0, 0, 0, 0]
    assert [x["first"] for x in r] == [0, 2]
    assert r[0]["scales"] == r[1]["scales"]
    sys.path.insert(0, ROOT)
    from oracle import oracle as O
    from paper_2607_14513_gb300 import synthetic as S
    O.lib()
    sc = S.make_scene(n=6001, seed=91, clusters=4, heavy_frac=0.2)
    assert r[0]["scales"] == O.scales(sc.sh).astype(np.float32).view(np.uint32).tolist()


def test_shard_bounds_are_chunk_aligned():
    sys.path.insert(0, ROOT)
    from paper_2607_14513_gb300 import gsc
    assert gsc.shard_bounds(262144, 2, 4096) == [0, 131072, 262144]
    assert gsc.shard_bounds(50001, 3, 256) == [0, 16640, 33280, 50001]
    assert gsc.shard_bounds(3001, 5, 1024) == [0, 0, 1024, 1024, 2048, 3001]
    assert gsc.shard_bounds(0, 2, 16) == [0, 0, 0]
    for n, S_, g in [(1000003, 7, 4096), (17, 4, 16), (4096, 3, 4096)]:
        b = gsc.shard_bounds(n, S_, g)
        assert b[0] == 0 and b[-1] == n and all(x <= y for x, y in zip(b, b[1:]))
        assert all(x % g == 0 for x in b[:-1])
    with pytest.raises(gsc.GscError):
        gsc.shard_bounds(10, 0, 16)
    with pytest.raises(gsc.GscError):
        gsc.shard_bounds(10, 2, 24)
