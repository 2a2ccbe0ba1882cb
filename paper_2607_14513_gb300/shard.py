"""One scene split over shards: the host side of the sharded encode.

Every step of the method runs in the library (the gsc_shard_* calls of include/gsc.h); this
module only moves partials between shards and combines them with collectives (minimum, maximum,
sum, gather, exclusive scan over the shards) and moves each shard's Gaussians to the shard that
owns them in the spatial order. Shards are held `k` to a process; with torch.distributed
initialised, rank r holds shards [r k, (r + 1) k) and the collectives span the ranks. The result
equals gsc_plan_reorder (sort, group_size > 0) followed by gsc_encode (rate format) on the
whole scene, byte for byte (Sec. V-A: scales of the whole scene; Sec. III-C: the reorder works
chunk by chunk in the spatial order; Sec. IV-B: one rate budget).
"""
from __future__ import annotations

import torch

from . import gsc


def _dist():
    import torch.distributed as dist
    return dist if dist.is_available() and dist.is_initialized() else None


class Exchange:
    """Collectives over all shards: the `k` shards of this process, and those of every other rank."""

    def __init__(self, k: int):
        self.k = k
        d = _dist()
        self.world = d.get_world_size() if d else 1
        self.rank = d.get_rank() if d else 0

    @property
    def n_shards(self):
        return self.world * self.k

    @property
    def first(self):
        return self.rank * self.k

    def reduce(self, parts, op="sum"):
        """Elementwise sum / min / max of the partials of every shard (the same tensor for each)."""
        t = parts[0].clone()
        for p in parts[1:]:
            t = {"sum": torch.add, "min": torch.minimum, "max": torch.maximum}[op](t, p)
        d = _dist()
        if d and self.world > 1:
            d.all_reduce(t, op={"sum": d.ReduceOp.SUM, "min": d.ReduceOp.MIN, "max": d.ReduceOp.MAX}[op])
        return t

    def gather(self, parts):
        """[n_shards, ...]: every shard's partial, in shard order."""
        t = torch.stack(parts)
        d = _dist()
        if d and self.world > 1:
            out = [torch.empty_like(t) for _ in range(self.world)]
            d.all_gather(out, t)
            t = torch.cat(out)
        return t

    def gather_rows(self, parts):
        """The rows of every process's `parts` (counts may differ), concatenated in rank order."""
        mine = torch.cat(parts) if len(parts) > 1 else parts[0]
        d = _dist()
        if not d or self.world == 1:
            return mine
        cnt = torch.tensor([mine.shape[0]], dtype=torch.int64, device=mine.device)
        cnts = [torch.empty_like(cnt) for _ in range(self.world)]
        d.all_gather(cnts, cnt)
        per_rank = [int(c.item()) for c in cnts]
        pad = torch.zeros((max(per_rank),) + tuple(mine.shape[1:]), dtype=mine.dtype, device=mine.device)
        pad[:mine.shape[0]] = mine
        out = [torch.empty_like(pad) for _ in range(self.world)]
        d.all_gather(out, pad)
        return torch.cat([o[:c] for o, c in zip(out, per_rank)])

    def exclusive_scan(self, values):
        """values [n_shards] -> for each shard, the sum of the values of the shards before it."""
        return torch.cumsum(values, 0) - values

    def move_rows(self, local_inputs, in_bounds, wanted):
        """Rows by input index. local_inputs: this process's input rows, one tensor per field,
        covering inputs [in_bounds[first], in_bounds[first + k]); wanted: for each of this
        process's shards, the input indices it needs, in its order. Returns, per shard, the
        fields' rows in that order."""
        lo, hi = in_bounds[self.first], in_bounds[self.first + self.k]
        d = _dist()
        if not d or self.world == 1:
            return [[f[w.long() - lo] for f in local_inputs] for w in wanted]
        dev = local_inputs[0].device
        mine = torch.cat(wanted).long() if wanted else torch.zeros(0, dtype=torch.long, device=dev)
        # what every rank wants, to know what to send it
        want_all = self.gather_rows([mine.to(torch.int64)])
        cnt = torch.tensor([mine.shape[0]], dtype=torch.int64, device=dev)
        cnts = [torch.empty_like(cnt) for _ in range(self.world)]
        d.all_gather(cnts, cnt)
        counts = [int(c.item()) for c in cnts]
        starts = [0]
        for c in counts:
            starts.append(starts[-1] + c)
        rank_bounds = torch.tensor([in_bounds[r * self.k] for r in range(self.world)] + [in_bounds[-1]],
                                   dtype=torch.int64, device=dev)
        send_idx, send_sizes = [], []
        for q in range(self.world):
            wq = want_all[starts[q]:starts[q + 1]]
            sel = wq[(wq >= lo) & (wq < hi)]
            send_idx.append(sel - lo)
            send_sizes.append(int(sel.shape[0]))
        src = torch.searchsorted(rank_bounds, mine, right=True) - 1
        recv_sizes = [int((src == p).sum()) for p in range(self.world)]
        arrival = torch.argsort(src, stable=True)   # received rows come grouped by source, in wanted order
        send_idx = torch.cat(send_idx)
        out_fields = []
        for f in local_inputs:
            buf = f[send_idx].contiguous()
            got = torch.empty((mine.shape[0],) + tuple(f.shape[1:]), dtype=f.dtype, device=dev)
            d.all_to_all_single(got, buf, recv_sizes, send_sizes)
            res = torch.empty_like(got)
            res[arrival] = got
            out_fields.append(res)
        res, o = [], 0
        for w in wanted:
            res.append([f[o:o + w.shape[0]] for f in out_fields])
            o += w.shape[0]
        return res

    def combine_disjoint(self, t):
        """Buffers that each rank wrote in disjoint places (zero elsewhere): the whole."""
        d = _dist()
        if d and self.world > 1:
            d.all_reduce(t, op=d.ReduceOp.SUM)
        return t


def encode_scene_sharded(ctx, pos_parts, sh_parts, target_x4, group_size=256, permille=995, ex=None, stream=None):
    """Rate-controlled encode of one scene held as shards (this process's shards: pos_parts[j]
    [m_j, 3], sh_parts[j] [m_j, 48], contiguous input ranges in shard order). Returns
    (scales, table, blocks, perm): the whole scene's, identical on every rank."""
    ex = ex or Exchange(len(pos_parts))
    dev = pos_parts[0].device
    sizes = ex.gather([torch.tensor([p.shape[0]], dtype=torch.int64, device=dev) for p in pos_parts]).view(-1)
    in_bounds = [0] + torch.cumsum(sizes, 0).tolist()
    n_total = in_bounds[-1]
    # 1-3: spatial order of the scene, and the chunk-aligned range each shard owns
    bbs = [gsc.gsc_shard_bbox(ctx, p, stream=stream) for p in pos_parts]
    lo, hi = ex.reduce(bbs, "min"), ex.reduce(bbs, "max")
    bb = torch.cat([lo[:3], hi[3:]])
    keys = ex.gather_rows([gsc.gsc_shard_morton(ctx, p, bb, stream=stream) for p in pos_parts])
    order = gsc.gsc_shard_order(ctx, keys, stream=stream)
    bounds = gsc.shard_bounds(n_total, ex.n_shards, group_size)
    mine = [ex.first + j for j in range(ex.k)]
    wanted = [order[bounds[s]:bounds[s + 1]] for s in mine]
    local_in = [torch.cat(pos_parts), torch.cat(sh_parts)] if ex.k > 1 else [pos_parts[0], sh_parts[0]]
    owned = ex.move_rows(local_in, in_bounds, wanted)
    # 4: scales of the whole scene
    states = [gsc.shard_select_state(ctx, dev) for _ in mine]
    for st in states:
        gsc.gsc_shard_select_begin(ctx, n_total, permille, st, stream=stream)
    for p in range(gsc.SHARD_SELECT_PASSES):
        hist = ex.reduce([gsc.gsc_shard_select_hist(ctx, sh, p, st, stream=stream)
                          for sh, st in zip(sh_parts, states)], "sum")
        for st in states:
            gsc.gsc_shard_select_pick(ctx, st, hist, p, stream=stream)
    scales = gsc.gsc_shard_select_scales(ctx, states[0], stream=stream)
    # 5: each shard's slot order
    perms = [gsc.gsc_shard_plan(ctx, o[1].contiguous(), scales, group_size, stream=stream) for o in owned]
    # 6-8: rate control over the whole scene
    rates = [gsc.ShardRate(ctx, o[0].shape[0], dev) for o in owned]
    mt = ex.reduce([r.begin(o[1].contiguous(), pm, scales, stream=stream) for r, o, pm in zip(rates, owned, perms)])
    for r in rates:
        r.search_begin(n_total, target_x4, mt, stream=stream)
    for p in range(gsc.SHARD_RATE_PASSES):
        tot = ex.reduce([r.count(p, stream=stream) for r in rates])
        for r in rates:
            r.narrow(p, tot, stream=stream)
    fills = ex.gather([r.fill(stream=stream) for r in rates])            # [S, 2]
    before = ex.exclusive_scan(fills[:, 1])
    total_star = fills[:, 0].sum()
    parts = ex.gather([r.apply(torch.stack([total_star, before[s]]), stream=stream) for r, s in zip(rates, mine)])
    ng = (n_total + 15) // 16
    blocks = torch.zeros(max(ng * 256, 16), dtype=torch.uint8, device=dev)
    perm = torch.zeros(ng * 16, dtype=torch.int32, device=dev)
    table = None
    for r, s, pm, w in zip(rates, mine, perms, wanted):
        table = r.assemble(pm, w, scales, parts, s, n_total, blocks, perm, stream=stream)
    ex.combine_disjoint(blocks)
    ex.combine_disjoint(perm)
    return scales, table, blocks[:table.total_bytes], perm
