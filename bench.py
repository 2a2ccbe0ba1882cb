#!/usr/bin/env python3
"""Benchmark of the SH block-texture codec on GB300 (one JSON line on rank 0).

Workload (default): scene-scale plain method, 3,000,000 synthetic Gaussians (64 clusters,
10% heavy-tailed bands 2-3), SH degree 3. One step runs every stage of the hot path once:
scales + quantisation + reorder plan; rate-controlled encode at 6 bits per texel, which
codes every block with both BC1 and BC7 (kept as the all-BC1 4 bpt and all-BC7 8 bpt
codings) and selects the fixed-rate streams; fused decode + SH evaluation for 8 camera
poses of each of the three codings; software decode and texture-unit decode of the BC1
and BC7 codings, compared bit for bit on the device.

`value` is whole-job throughput in millions of Gaussians per second through that step
(inputs resident in HBM). Multi-GPU runs are weak scaling: every rank codes its own scene.
The same line carries the batched form (64 scenes in one persistent encode launch and one
captured evaluation graph, against per-scene calls on the same data: `batched`) and the served
form (a Poisson request trace of `--serve-seconds` against the request loop with continuous
batching and against a one-slot queue: `served`); `--scene-only` leaves both out.
`--impl reference` times the plain CPU oracle on this host's cores on a bounded sample of
the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2607_14513_gb300 import synthetic as S  # noqa: E402

METRIC = "BC1/BC7 encode Mblocks/s; decode+SH-eval MGauss/s & GB/s; served p50/p99 ms"
UNIT = "MGauss/s"
RATE_TARGET_X4 = 24          # 6 bits per coefficient texel
N_CAMS = 8
# BC7 search: palette-distance evaluations per block (the candidate enumeration of the
# encoder: initial indices + every p-bit combination, per mode / partition / rotation /
# index selection), and integer operations per evaluation (3 differences, 3 squares
# accumulated, compare, select).
BC7_EVALS_PER_BLOCK = (16 * (16 * 8 + 4 * 16 * 8) + 64 * (16 * 8 + 2 * 16 * 8) + 64 * (16 * 4 + 16 * 4)
                       + 64 * (16 * 4 + 4 * 16 * 4) + (128 + 256 + 3 * 768) + (128 + 3 * 256)
                       + (16 * 16 + 4 * 16 * 16) + 64 * (16 * 4 + 4 * 16 * 4))
# integer operations of one palette evaluation as the search kernel computes it (best_key in
# csrc/bc7.cu): the byte dot product of texel and entry, the entry's key minus 32 x that product,
# and the running minimum; gsc_probe_op_rate kind 5 runs exactly this mix
OPS_PER_EVAL = 3
# per launch, measured with ncu for the kernels as they stand (to be reset to None when a kernel
# changes): DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) on the 3M-Gaussian workload,
# and the BC7 search's thread instructions per block (smsp__thread_inst_executed.sum / blocks)
MEASURED_TRAFFIC = {"scene3m": {"k_bc7": None, "k_eval2_bc7_slots": 324060000, "k_eval_tex_bc7": 388227328}}
MEASURED_BC7_THREAD_INSTR_PER_BLOCK = 582878   # 262,144-Gaussian scene (the search is exhaustive: size-independent)
ISSUE_LANES_PER_CLK_SM = 128   # 4 schedulers x 32 lanes, one warp instruction each per clock


def workload_cfg(name):
    return {"scene3m": S.SCENE, "medium262k": S.MEDIUM, "tiny4k": S.TINY, "layouts3m": S.SCENE,
            "render3m": S.SCENE}[name]


def scene_config(cfg, world):
    """The `config` of a plain-method scene workload (both arms print the same one)."""
    n = cfg["n"]
    return {"workload": "scene-scale plain method: %d Gaussians, SH degree 3, %d clusters, %d%% heavy "
                        "tail; rate 6 bpt + all-BC1 4 bpt + all-BC7 8 bpt; %d camera poses"
                        % (n, cfg["clusters"], int(cfg["heavy_frac"] * 100), N_CAMS),
            "n_gaussians": n, "parallelism": "weak, one scene per GPU" if world > 1 else "single GPU",
            "l2": ("inputs larger than L2 (SH 192 B/Gaussian)" if 192 * n > L2_BYTES
                   else "inputs fit in L2 (a parity-size case, not an HBM measurement)")}


# Table I's fixed codings of the other block layouts (Figs. SetupA / SetupB), and layout D's
# BC7-on-the-first-block mix: (name, layout, format, BC7 blocks per group, bytes per Gaussian that
# Table I prints; for layout D it prints one block per group more than the coded blocks)
LAYOUT_CODINGS = [("A_bc1", 1, 1, 0, 8.0), ("A_bc7", 1, 7, 16, 16.0), ("B_bc7_first", 2, 2, 4, 10.0),
                  ("D_bc7_first", 0, 2, 1, 9.0)]


L2_BYTES = 129e6  # GB300 L2
HBM_NOMINAL_GBS = 7900.0  # GB300 HBM3e nominal, reported beside the measured copy bandwidth


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = uuid
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--id=" + self.uuid, "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        loaded = [x for x in sm if mx and x > 0.5 * max(mx)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world, device):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------------------------------------
def run_gsc(args, world, rank, local):
    import torch
    from paper_2607_14513_gb300 import gsc

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    cfg = dict(workload_cfg(args.workload))
    cfg["seed"] = cfg["seed"] + 1000 * rank
    n = cfg["n"]
    ng = (n + 15) // 16
    ns = ng * 16
    sc = S.make_scene(**cfg)
    cams_np = S.make_cams(N_CAMS, 1100 + rank)
    ctx = gsc.Context(local)
    stream = torch.cuda.Stream(dev)
    pos = torch.from_numpy(sc.pos).to(dev)
    sh = torch.from_numpy(sc.sh).to(dev)
    cams = torch.from_numpy(cams_np).to(dev)
    ws = ctx.workspace(n, gsc.FMT_RATE, RATE_TARGET_X4)
    bc1 = torch.empty(ng * 128, dtype=torch.uint8, device=dev)
    bc7 = torch.empty(ng * 256, dtype=torch.uint8, device=dev)
    # the step's outputs in two sets, so that end to end a step can run while the previous one's
    # results are copied out
    rate_bufs = [torch.empty(ng * 256, dtype=torch.uint8, device=dev) for _ in range(2)]
    rate_perms = [torch.empty(ns, dtype=torch.int32, device=dev) for _ in range(2)]
    rgbs = [torch.empty((3, ns, N_CAMS, 3), dtype=torch.float32, device=dev) for _ in range(2)]
    rgb = rgbs[0]
    pos_slot = torch.empty((ns, 3), dtype=torch.float32, device=dev)
    pos_slot_r = torch.empty((ns, 3), dtype=torch.float32, device=dev)
    ok = torch.ones((), dtype=torch.bool, device=dev)

    last_perm = [None, None]

    def step(pos_d, sh_d, b=0):
        rate_buf, rate_perm, rgb = rate_bufs[b], rate_perms[b], rgbs[b]
        perm, scales = gsc.gsc_plan_reorder(ctx, pos_d, sh_d, ws=ws, stream=stream)
        last_perm[0], last_perm[1] = perm, scales
        gsc.gsc_positions_to_slots(ctx, pos_d, perm, out=pos_slot, stream=stream)
        rblk, rperm, rtab = gsc.gsc_encode(ctx, sh_d, perm, scales, gsc.FMT_RATE, RATE_TARGET_X4, ws=ws,
                                           out=rate_buf, perm_out=rate_perm, stream=stream, bc1_all=bc1, bc7_all=bc7)
        gsc.gsc_positions_to_slots(ctx, pos_d, rperm, out=pos_slot_r, stream=stream)
        t1, t7 = gsc.forced_table(rtab, gsc.FMT_BC1), gsc.forced_table(rtab, gsc.FMT_BC7)
        for i, (tab, blk, p, ps) in enumerate([(t7, bc7, perm, pos_slot), (t1, bc1, perm, pos_slot),
                                               (rtab, rblk, rperm, pos_slot_r)]):
            gsc.gsc_decode_eval_sh_slots(ctx, tab, blk, p, pos_slot=ps, cams=cams, out_order=gsc.OUT_SLOT_ROWS,
                                         out=rgb[i], stream=stream)
        with torch.cuda.stream(stream):
            for tab, blk in [(t7, bc7), (t1, bc1)]:
                sw = gsc.gsc_decode(ctx, tab, blk, perm, stream=stream)
                hw = gsc.gsc_decode_tex(ctx, tab, blk, perm, stream=stream)
                ok.logical_and_((sw == hw).all())
        return rtab, rblk, rperm

    # warm-up (also compiles nothing: the library is prebuilt)
    for _ in range(args.warmup):
        step(pos, sh)
    stream.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    uuid = str(torch.cuda.get_device_properties(dev).uuid)
    uuid = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    clocks = ClockSampler(uuid)
    clocks.start()
    gsc.set_timing(ctx, True)
    launches0 = gsc.launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        rtab, rblk, rperm = step(pos, sh)
    e1.record(stream)
    perm_last = last_perm[0]
    stream.synchronize()
    launches = gsc.launch_count() - launches0
    barrier(world)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms_total = e0.elapsed_time(e1)
    kt = {k: gsc.kernel_time(ctx, k) for k in ["plan", "bc1_encode", "bc7_encode", "rate_select", "decode",
                                               "decode_eval", "decode_tex"]}
    gsc.set_timing(ctx, False)
    ms_step = max_over_ranks(ms_total / args.steps, world, dev)
    value = world * n / (ms_step * 1e-3) / 1e6
    match = bool(ok.item())

    # dominant kernel: the BC7 search (integer ALU bound)
    bc7_ms = kt["bc7_encode"][0] / max(1, kt["bc7_encode"][1])
    roofline = bc7_roofline(ctx, gsc, stream, dev, clk, BC7_EVALS_PER_BLOCK * ns, bc7_ms,
                            "k_bc7 (BC7 candidate search, thread per block)", ns,
                            MEASURED_TRAFFIC.get(args.workload, {}).get("k_bc7"))
    # the fused decode + SH evaluation (HBM bound) of each coding, timed alone after the step, with
    # the centres resident in slot order (the step's own gsc_positions_to_slots output): algorithmic
    # bytes per launch = the coded blocks + 4 B slot entry + 12 B centre + 8 x 12 B output per Gaussian
    hbm, hbm_src = peaks()
    t1, t7 = gsc.forced_table(rtab, gsc.FMT_BC1), gsc.forced_table(rtab, gsc.FMT_BC7)
    codings = {"bc7": (t7, bc7, last_perm[0], pos_slot), "bc1": (t1, bc1, last_perm[0], pos_slot),
               "rate": (rtab, rblk, rperm, pos_slot_r)}

    def time_eval(name, order, out, slots=True):
        tab, blk, p, ps = codings[name]

        def call():
            if slots:
                gsc.gsc_decode_eval_sh_slots(ctx, tab, blk, p, pos_slot=ps, cams=cams, out_order=order, out=out,
                                             stream=stream)
            else:
                gsc.gsc_decode_eval_sh(ctx, tab, blk, p, pos=pos, cams=cams, out_order=order, out=out, stream=stream)
        for _ in range(3):
            call()
        stream.synchronize()
        gsc.set_timing(ctx, True)
        for _ in range(max(10, args.steps)):
            call()
        ms_, cnt_ = gsc.kernel_time(ctx, "decode_eval")
        gsc.set_timing(ctx, False)
        return ms_ / max(1, cnt_)

    def eval_bytes(name):
        return codings[name][0].total_bytes + (4 + 12 + N_CAMS * 12) * n

    ev_ms3 = kt["decode_eval"][0] / max(1, kt["decode_eval"][1])
    per_coding = {}
    for name in ("bc7", "bc1", "rate"):
        ms_c = time_eval(name, gsc.OUT_SLOT_ROWS, rgb[0])
        gbs_c = eval_bytes(name) / (ms_c * 1e-3) / 1e9
        ms_o = time_eval(name, gsc.OUT_GAUSS_MAJOR, rgb[0])
        gbs_o = eval_bytes(name) / (ms_o * 1e-3) / 1e9
        per_coding[name] = {"ms": round(ms_c, 4), "GB_s": round(gbs_c, 1), "frac": round(gbs_c / hbm, 4),
                            "bytes_per_gaussian": round(eval_bytes(name) / n, 2),
                            "original_order_ms": round(ms_o, 4), "original_order_frac": round(gbs_o / hbm, 4)}
    ev_ms = per_coding["bc7"]["ms"]
    ev_bytes = eval_bytes("bc7")
    ev_gbs = ev_bytes / (ev_ms * 1e-3) / 1e9
    roofline_eval = {"bound": "hbm", "achieved": round(ev_gbs, 1), "peak": hbm, "unit": "GB/s",
                     "frac": round(ev_gbs / hbm, 4), "peak_source": hbm_src,
                     "frac_of_nominal": round(ev_gbs / HBM_NOMINAL_GBS, 4),
                     "traffic": MEASURED_TRAFFIC.get(args.workload, {}).get("k_eval2_bc7_slots"),
                     "kernel": "k_eval2 (software BC7 decode + SH eval, all-BC7 coding, %d cameras, centres and "
                               "colour rows in slot order, the coded scene's own order; the same rows by original "
                               "index: codings.*.original_order_*)" % N_CAMS,
                     "algorithmic": "16 B block + 4 B slot entry + 12 B centre + %d x 12 B output per Gaussian"
                                    % N_CAMS,
                     "codings": per_coding}
    stages = {}
    for k, (ms, cnt) in kt.items():
        stages[k + "_ms"] = round(ms / max(1, cnt), 4)
    stages["bc1_encode_Mblocks_s"] = round(ns / (kt["bc1_encode"][0] / max(1, kt["bc1_encode"][1]) * 1e-3) / 1e6, 2)
    stages["bc7_encode_Mblocks_s"] = round(ns / (bc7_ms * 1e-3) / 1e6, 3)
    stages["decode_eval_bc7_ms"] = round(ev_ms, 4)
    stages["decode_eval_bc7_MGauss_s"] = round(n / (ev_ms * 1e-3) / 1e6, 1)
    stages["decode_eval_bc7_GB_s"] = round(ev_gbs, 1)
    stages["decode_eval_3codings_mean_ms"] = round(ev_ms3, 4)
    # the same call with the centres gathered through the slot order (gsc_decode_eval_sh)
    ms_g = time_eval("bc7", gsc.OUT_SLOT_ROWS, rgb[0], slots=False)
    stages["decode_eval_bc7_gather_ms"] = round(ms_g, 4)
    stages["decode_eval_bc7_gather_GB_s"] = round(ev_bytes / (ms_g * 1e-3) / 1e9, 1)
    stages["rate_bits_per_texel"] = round(rtab.used_bits / (16.0 * n), 4)

    # the same evaluation on resident texture scenes (blocks decoded by the texture unit)
    tex_stats = time_tex_eval(args, ctx, gsc, stream, dev, rtab, bc1, bc7, perm_last, pos, cams, n, ns)
    stages.update(tex_stats["stages"])
    # coalesced comparison: the all-BC7 coding evaluated into slot order (no scattered stores)
    rgb_slot = torch.empty((N_CAMS, ns, 3), dtype=torch.float32, device=dev)
    ms_slot = time_eval("bc7", gsc.OUT_SLOT_ORDER, rgb_slot)
    stages["decode_eval_bc7_slot_order_ms"] = round(ms_slot, 4)
    stages["decode_eval_bc7_slot_order_GB_s"] = round(ev_bytes / (ms_slot * 1e-3) / 1e9, 1)
    del rgb_slot

    # the BC7 search's thread mapping: mode 1 alone, thread per block against warp per block
    stages.update(time_bc7_mappings(ctx, gsc, stream, sh, last_perm[0], last_perm[1], n))

    # end to end through the public API with host buffers
    e2e = run_e2e(args, ctx, gsc, stream, dev, sc, step, world, rgbs)

    out = {"metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(ms_step, 3), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "u8 texels / int32 search / f32 SH eval",
           "data": "synthetic (seeded; stands in for the paper's trained scenes)",
           "config": dict(scene_config(cfg, world), texture_path_bit_exact=match),
           "roofline": roofline, "roofline_decode_eval": roofline_eval,
           "roofline_decode_eval_tex": tex_stats["roofline"], "stages": stages,
           "clocks": clk, "e2e": e2e, "gpu_launches": int(launches)}
    if world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args.workload, budget_s=args.cpu_seconds)
    ctx.close()
    return out


def bc7_roofline(ctx, gsc, stream, dev, clk, evals, ms, kernel, blocks, traffic):
    """The BC7 search against the measured rate of its own evaluation mix (gsc_probe_op_rate kind 5),
    and against the SM's issue ceiling (128 lanes per clock per SM at the sampled SM clock), with the
    per-instruction probe rates beside them."""
    import torch
    probes = {gsc.PROBE_KINDS[k]: gsc.op_rate(ctx, k, stream=stream) for k in sorted(gsc.PROBE_KINDS)}
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = clk.get("sm_mhz") or 2070.0
    per_clk = {k: round(v / (sms * mhz * 1e6), 2) for k, v in probes.items()}
    issue = sms * ISSUE_LANES_PER_CLK_SM * mhz * 1e6
    peak = probes["bc7_palette_eval"]
    ops = evals * OPS_PER_EVAL
    ach = ops / (ms * 1e-3)
    out = {"bound": "alu", "achieved": round(ach / 1e12, 3), "peak": round(peak / 1e12, 3), "unit": "Tops/s",
           "frac": round(ach / peak, 4), "traffic": traffic, "kernel": kernel,
           "peak_source": "measured on this GPU: gsc_probe_op_rate kind 5, the evaluation's own mix (dp4a, "
                          "scaled key, minimum) in independent chains at full occupancy",
           "algorithmic": "%d palette evaluations x %d int ops (dot, key, minimum), %d blocks"
                          % (evals // max(1, blocks), OPS_PER_EVAL, blocks),
           "issue_ceiling_Tops_s": round(issue / 1e12, 3), "frac_of_issue_ceiling": round(ach / issue, 4),
           "probes_Tops_s": {k: round(v / 1e12, 3) for k, v in probes.items()},
           "probes_ops_per_clk_per_sm": per_clk}
    if MEASURED_BC7_THREAD_INSTR_PER_BLOCK:
        ti = MEASURED_BC7_THREAD_INSTR_PER_BLOCK * blocks / (ms * 1e-3)
        out["instructions"] = {"thread_instr_per_block": MEASURED_BC7_THREAD_INSTR_PER_BLOCK,
                               "thread_instr_per_eval": round(MEASURED_BC7_THREAD_INSTR_PER_BLOCK * blocks / evals, 2),
                               "Tinstr_s": round(ti / 1e12, 3), "frac_of_issue_ceiling": round(ti / issue, 4)}
    return out


def time_bc7_mappings(ctx, gsc, stream, sh, perm, scales, n):
    """The mode-1 search (64 partitions) over the scene's staged BC7 texels, thread per block and
    warp per block (gsc_probe_bc7_mode1): launch times and whether the results agree."""
    import torch
    q = gsc.gsc_quantise(ctx, sh, scales, stream=stream)
    with torch.cuda.stream(stream):
        qp = torch.cat([q.reshape(n, 48), torch.full((1, 48), 128, dtype=torch.uint8, device=q.device)])
        idx = torch.where(perm < 0, torch.full_like(perm, n), perm).long()
        tex = qp[idx].view(-1, 16, 16, 3).permute(0, 2, 1, 3).reshape(-1, 16, 3).contiguous()
    res, out = {}, {}
    for name, warp in (("thread_per_block", False), ("warp_per_block", True)):
        gsc.bc7_mode1(ctx, tex, warp, stream=stream)
        times = []
        for _ in range(3):
            sse, part, ms = gsc.bc7_mode1(ctx, tex, warp, stream=stream)
            times.append(ms)
        out[name] = (sse, part)
        res["bc7_mode1_%s_ms" % name] = round(min(times), 3)
    a, b = out["thread_per_block"], out["warp_per_block"]
    res["bc7_mode1_mappings_equal"] = bool(torch.equal(a[0], b[0]) and torch.equal(a[1], b[1]))
    return res


def time_tex_eval(args, ctx, gsc, stream, dev, rtab, bc1, bc7, perm, pos, cams, n, ns):
    """Fused evaluation of the all-BC7 and all-BC1 codings kept resident as texture objects."""
    import torch
    out = torch.empty((n, N_CAMS, 3), dtype=torch.float32, device=dev)
    res = {"stages": {}}
    hbm, hbm_src = peaks()
    for name, fmt, blk, bpg in [("bc7", gsc.FMT_BC7, bc7, 16), ("bc1", gsc.FMT_BC1, bc1, 8)]:
        tab = gsc.forced_table(rtab, fmt)
        scene = gsc.TexScene(ctx, tab, blk, perm=perm, pos=pos, stream=stream)
        for _ in range(3):
            gsc.gsc_decode_eval_sh_tex(ctx, scene, perm, cams=cams, out_order=gsc.OUT_GAUSS_MAJOR, out=out,
                                       stream=stream)
        stream.synchronize()
        gsc.set_timing(ctx, True)
        for _ in range(max(5, args.steps)):
            gsc.gsc_decode_eval_sh_tex(ctx, scene, perm, cams=cams, out_order=gsc.OUT_GAUSS_MAJOR, out=out,
                                       stream=stream)
        ms, cnt = gsc.kernel_time(ctx, "decode_eval_tex")
        gsc.set_timing(ctx, False)
        scene.close()
        ms /= max(1, cnt)
        by = (bpg + 4 + 12 + N_CAMS * 12) * n
        gbs = by / (ms * 1e-3) / 1e9
        res["stages"]["decode_eval_tex_%s_ms" % name] = round(ms, 4)
        res["stages"]["decode_eval_tex_%s_GB_s" % name] = round(gbs, 1)
        res["stages"]["decode_eval_tex_%s_MGauss_s" % name] = round(n / (ms * 1e-3) / 1e6, 1)
        if name == "bc7":
            res["roofline"] = {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm, "unit": "GB/s",
                               "frac": round(gbs / hbm, 4), "peak_source": hbm_src,
                               "frac_of_nominal": round(gbs / HBM_NOMINAL_GBS, 4),
                               "traffic": MEASURED_TRAFFIC.get(args.workload, {}).get("k_eval_tex_bc7"),
                               "kernel": "k_eval_tex (texture-unit decode + SH eval, all-BC7, %d cameras, "
                                         "Gaussian-major output)" % N_CAMS,
                               "algorithmic": "16 B block + 4 B perm + 12 B position + %d x 12 B output per Gaussian"
                                              % N_CAMS}
    return res


def run_e2e(args, ctx, gsc, stream, dev, sc, step, world, rgbs):
    """The step end to end from pinned host memory, pipelined the way a streaming caller would run
    it: step i+1's inputs go up on a copy stream while step i computes, and step i's results (rate
    streams, slot order, the three codings' colours) come back on it while step i+1 computes. Two
    sets of device inputs and outputs alternate; events order every reuse."""
    import torch
    pos_h = torch.from_numpy(sc.pos).pin_memory()
    sh_h = torch.from_numpy(sc.sh).pin_memory()
    pos_d = [torch.empty_like(pos_h, device=dev) for _ in range(2)]
    sh_d = [torch.empty_like(sh_h, device=dev) for _ in range(2)]
    n = sc.pos.shape[0]
    ns = (n + 15) // 16 * 16
    out_blocks = torch.empty(ns * 16, dtype=torch.uint8).pin_memory()
    out_perm = torch.empty(ns, dtype=torch.int32).pin_memory()
    out_rgb = torch.empty(rgbs[0].shape, dtype=rgbs[0].dtype).pin_memory()
    copy = torch.cuda.Stream(dev)
    up = [torch.cuda.Event() for _ in range(2)]
    done = [torch.cuda.Event() for _ in range(2)]
    down = [torch.cuda.Event() for _ in range(2)]
    used = [False, False]
    bo = 0

    def upload(i):
        b = i % 2
        if used[b]:
            copy.wait_event(done[b])       # step i - 2 has finished reading this input set
        with torch.cuda.stream(copy):
            pos_d[b].copy_(pos_h, non_blocking=True)
            sh_d[b].copy_(sh_h, non_blocking=True)
        up[b].record(copy)

    def run(i):
        nonlocal bo
        b = i % 2
        stream.wait_event(up[b])
        if used[b]:
            stream.wait_event(down[b])     # step i - 2's results have left this output set
        rtab, rblk, rperm = step(pos_d[b], sh_d[b], b)
        done[b].record(stream)
        used[b] = True
        copy.wait_event(done[b])
        with torch.cuda.stream(copy):
            out_blocks[:rtab.total_bytes].copy_(rblk, non_blocking=True)
            out_perm.copy_(rperm, non_blocking=True)
            out_rgb.copy_(rgbs[b], non_blocking=True)
        down[b].record(copy)
        bo = rtab.total_bytes + 4 * ns + rgbs[b].numel() * rgbs[b].element_size()

    def steps(k):
        upload(0)
        for i in range(k):
            if i + 1 < k:
                upload(i + 1)
            run(i)
        stream.synchronize()
        copy.synchronize()

    steps(max(2, args.warmup // 2))
    barrier(world)
    # at least 10 steps, so that filling and draining the pipeline weighs little per step
    k = max(10, args.steps)
    t0 = time.perf_counter()
    steps(k)
    t = (time.perf_counter() - t0) / k
    t = max_over_ranks(t, world, dev)
    return {"value": round(world * n / t / 1e6, 3), "unit": UNIT, "h2d_bytes_per_step": int(n * (12 + 192)),
            "d2h_bytes_per_step": int(bo), "ms_per_step": round(t * 1e3, 3), "steps": k,
            "path": "pinned host pos+SH -> plan/encode/decode/eval/texture compare -> rate streams, perm and the "
                    "three codings' evaluated colours to pinned host memory; uploads and read-backs on a copy "
                    "stream overlapping the neighbouring steps' compute"}


# ------------------------------------------------------------------------------------------------
def run_layouts(args, world, rank, local):
    """One step: the reorder plan, then every coding of LAYOUT_CODINGS (encode, then fused decode +
    SH evaluation of 8 cameras into Gaussian-major rows) of the 3M-Gaussian scene."""
    import torch
    from paper_2607_14513_gb300 import gsc

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    cfg = dict(S.SCENE)
    cfg["seed"] = cfg["seed"] + 1000 * rank
    n = cfg["n"]
    ng = (n + 15) // 16
    ns = ng * 16
    sc = S.make_scene(**cfg)
    ctx = gsc.Context(local)
    stream = torch.cuda.Stream(dev)
    pos = torch.from_numpy(sc.pos).to(dev)
    sh = torch.from_numpy(sc.sh).to(dev)
    cams = torch.from_numpy(S.make_cams(N_CAMS, 1100 + rank)).to(dev)
    ws_bytes = max(int(ctx.lib.gsc_workspace_bytes(n, C_ref(gsc.EncodeParams(f, 0, None, None, lay, j))))
                   for _, lay, f, j, _ in LAYOUT_CODINGS)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
    bufs = {c[0]: torch.empty(ng * 256, dtype=torch.uint8, device=dev) for c in LAYOUT_CODINGS}
    perms = {c[0]: torch.empty(ns, dtype=torch.int32, device=dev) for c in LAYOUT_CODINGS}
    rgb = torch.empty((n, N_CAMS, 3), dtype=torch.float32, device=dev)
    ev = {c[0]: [torch.cuda.Event(enable_timing=True) for _ in range(3)] for c in LAYOUT_CODINGS}
    acc = {c[0]: [0.0, 0.0] for c in LAYOUT_CODINGS}
    tables = {}

    def step(pos_d, sh_d, record=False):
        perm, scales = gsc.gsc_plan_reorder(ctx, pos_d, sh_d, ws=ws, stream=stream)
        out = []
        for name, lay, fmt, j, _ in LAYOUT_CODINGS:
            e = ev[name]
            e[0].record(stream)
            blk, po, tab = gsc.gsc_encode(ctx, sh_d, perm, scales, fmt, ws=ws, out=bufs[name], perm_out=perms[name],
                                          stream=stream, layout=lay, bc7_blocks=j)
            e[1].record(stream)
            gsc.gsc_decode_eval_sh(ctx, tab, blk, po, pos=pos_d, cams=cams, out_order=gsc.OUT_GAUSS_MAJOR, out=rgb,
                                   stream=stream)
            e[2].record(stream)
            tables[name] = tab
            out.append((tab, blk, po))
        if record:
            stream.synchronize()
            for name in acc:
                acc[name][0] += ev[name][0].elapsed_time(ev[name][1])
                acc[name][1] += ev[name][1].elapsed_time(ev[name][2])
        return out

    for _ in range(args.warmup):
        step(pos, sh)
    stream.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    uuid = str(torch.cuda.get_device_properties(dev).uuid)
    uuid = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    clocks = ClockSampler(uuid)
    clocks.start()
    gsc.set_timing(ctx, True)
    launches0 = gsc.launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step(pos, sh)
    e1.record(stream)
    stream.synchronize()
    launches = gsc.launch_count() - launches0
    barrier(world)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms_total = e0.elapsed_time(e1)
    kt = {k: gsc.kernel_time(ctx, k) for k in ["plan", "bc1_encode", "bc7_encode", "decode_eval"]}
    gsc.set_timing(ctx, False)
    ms_step = max_over_ranks(ms_total / args.steps, world, dev)
    value = world * n / (ms_step * 1e-3) / 1e6
    # per-coding times (event pairs around each call; a separate pass so the timed loop has no extra syncs)
    for _ in range(args.steps):
        step(pos, sh, record=True)

    hbm, hbm_src = peaks()
    bc7_blocks_step = sum(ng * j for _, _, _, j, _ in LAYOUT_CODINGS)
    bc7_ms = kt["bc7_encode"][0] / max(1, args.steps)
    roofline = bc7_roofline(ctx, gsc, stream, dev, clk, BC7_EVALS_PER_BLOCK * bc7_blocks_step, bc7_ms,
                            "k_bc7 on staged texels (every BC7 block of the step's codings)", bc7_blocks_step, None)
    stages, rooflines = {}, {}
    for name, lay, fmt, j, bpg in LAYOUT_CODINGS:
        enc_ms, ev_ms = acc[name][0] / args.steps, acc[name][1] / args.steps
        tab = tables[name]
        by = (tab.total_bytes / n + 4 + 12 + N_CAMS * 12) * n
        gbs = by / (ev_ms * 1e-3) / 1e9
        stages[name] = {"bytes_per_gaussian": round(tab.total_bytes / n, 4), "table_one_bytes": bpg,
                        "encode_ms": round(enc_ms, 3), "encode_MGauss_s": round(n / (enc_ms * 1e-3) / 1e6, 2),
                        "decode_eval_ms": round(ev_ms, 4), "decode_eval_GB_s": round(gbs, 1),
                        "decode_eval_frac_hbm": round(gbs / hbm, 4)}
        if name == "A_bc7":
            rooflines = {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm, "unit": "GB/s",
                         "frac": round(gbs / hbm, 4), "peak_source": hbm_src,
                         "frac_of_nominal": round(gbs / HBM_NOMINAL_GBS, 4), "traffic": None,
                         "kernel": "k_eval2 layout A, all-BC7 (16 B block + 4 B perm + 12 B position + %d x 12 B "
                                   "output per Gaussian)" % N_CAMS}
    stages["plan_ms"] = round(kt["plan"][0] / max(1, args.steps), 4)

    # end to end: pinned host inputs in, every coding's blocks and slot order back to the host
    pos_h = torch.from_numpy(sc.pos).pin_memory()
    sh_h = torch.from_numpy(sc.sh).pin_memory()
    pos_d, sh_d = torch.empty_like(pos_h, device=dev), torch.empty_like(sh_h, device=dev)
    host_out = {c[0]: torch.empty(ng * 256, dtype=torch.uint8).pin_memory() for c in LAYOUT_CODINGS}
    host_perm = torch.empty(ns, dtype=torch.int32).pin_memory()
    bo = [0]

    def one():
        with torch.cuda.stream(stream):
            pos_d.copy_(pos_h, non_blocking=True)
            sh_d.copy_(sh_h, non_blocking=True)
        res = step(pos_d, sh_d)
        bo[0] = 4 * ns
        with torch.cuda.stream(stream):
            for (name, _, _, _, _), (tab, blk, po) in zip(LAYOUT_CODINGS, res):
                host_out[name][:tab.total_bytes].copy_(blk, non_blocking=True)
                bo[0] += tab.total_bytes
            host_perm.copy_(res[-1][2], non_blocking=True)

    one()
    stream.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        one()
    stream.synchronize()
    t = max_over_ranks((time.perf_counter() - t0) / args.steps, world, dev)
    e2e = {"value": round(world * n / t / 1e6, 3), "unit": UNIT, "h2d_bytes_per_step": int(n * (12 + 192)),
           "d2h_bytes_per_step": int(bo[0]), "ms_per_step": round(t * 1e3, 3),
           "path": "pinned host pos+SH -> plan, four codings, their decode + SH eval -> every coding's blocks "
                   "and the slot order to host"}
    out = {"metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": round(ms_step, 3), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "u8 texels / int32 search / f32 SH eval",
           "data": "synthetic (seeded; stands in for the paper's trained scenes)",
           "config": {"workload": "layouts: %d Gaussians; Table I codings of layout A (BC1, BC7), layout B (BC7 on "
                                  "the first block of each quad, BC1 on the rest) and layout D (BC7 on block 0); "
                                  "each decoded + SH-evaluated for %d camera poses" % (n, N_CAMS),
                      "n_gaussians": n, "parallelism": "weak, one scene per GPU" if world > 1 else "single GPU",
                      "l2": "inputs larger than L2 (SH 192 B/Gaussian)"},
           "roofline": roofline, "roofline_decode_eval": rooflines, "stages": stages, "clocks": clk, "e2e": e2e,
           "gpu_launches": int(launches)}
    if world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline("layouts3m", budget_s=args.cpu_seconds)
    ctx.close()
    return out


def run_render(args, world, rank, local):
    """One step: the 3M-Gaussian scene, coded all-BC7 (layout D), rendered for 4 cameras at
    1920 x 1080 (fused decode + SH colour, splat setup, tile sort, per-tile blending)."""
    import torch
    from paper_2607_14513_gb300 import gsc

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    cfg = dict(S.RENDER)
    n, W, H, V = cfg["n"], cfg["width"], cfg["height"], cfg["views"]
    sc = S.make_scene(n=n, seed=cfg["seed"] + 1000 * rank, clusters=cfg["clusters"], heavy_frac=cfg["heavy_frac"])
    geo = S.make_geometry(n, cfg["geom_seed"] + 1000 * rank, scale=cfg["scale"])
    cams = S.make_views(V, cfg["view_seed"] + rank, W, H)
    ctx = gsc.Context(local)
    stream = torch.cuda.Stream(dev)
    pos, sh = torch.from_numpy(sc.pos).to(dev), torch.from_numpy(sc.sh).to(dev)
    scale, rot = torch.from_numpy(geo.scale).to(dev), torch.from_numpy(geo.rot).to(dev)
    logit = torch.from_numpy(geo.logit).to(dev)
    perm, scales = gsc.gsc_plan_reorder(ctx, pos, sh, stream=stream)
    blk, po, tab = gsc.gsc_encode(ctx, sh, perm, scales, gsc.FMT_BC7, stream=stream)
    r = gsc.Renderer(ctx)
    imgs = torch.empty((V, H, W, 3), dtype=torch.float32, device=dev)
    pairs = [0] * V

    def step(blk_d, po_d, pos_d, scale_d, rot_d, logit_d):
        for v in range(V):
            _, _, pairs[v] = r.render(tab, blk_d, po_d, pos_d, scale_d, rot_d, logit_d, cams[v], image=imgs[v],
                                      stream=stream)

    for _ in range(max(3, args.warmup)):
        step(blk, po, pos, scale, rot, logit)
    stream.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    uuid = str(torch.cuda.get_device_properties(dev).uuid)
    uuid = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    clocks = ClockSampler(uuid)
    clocks.start()
    gsc.set_timing(ctx, True)
    launches0 = gsc.launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step(blk, po, pos, scale, rot, logit)
    e1.record(stream)
    stream.synchronize()
    launches = gsc.launch_count() - launches0
    barrier(world)
    torch.cuda.synchronize()
    clk = clocks.stop()
    kt = {k: gsc.kernel_time(ctx, k) for k in ["render", "render_blend"]}
    gsc.set_timing(ctx, False)
    ms_step = max_over_ranks(e0.elapsed_time(e1) / args.steps, world, dev)
    value = world * n * V / (ms_step * 1e-3) / 1e6
    frames = args.steps * V
    blend_ms = kt["render_blend"][0] / max(1, frames)
    call_ms = kt["render"][0] / max(1, frames)
    # the blending kernel: every pixel of a tile evaluates every splat of the tile's list
    # (20 FP32 flops per evaluation: offset 2, quadratic form 8, weight 1, colour 6, transmittance 3;
    # plus one exp2 on the special-function unit); peak = SMs x 128 FP32 lanes x 2 flops x SM clock
    evals = 256 * sum(pairs) / V
    sm = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = clk.get("sm_mhz") or 2070.0
    peak = sm * 128 * 2 * mhz * 1e6 / 1e12
    achieved = evals * 20 / (blend_ms * 1e-3) / 1e12
    roofline = {"bound": "alu", "achieved": round(achieved, 3), "peak": round(peak, 2), "unit": "TFLOP/s",
                "frac": round(achieved / peak, 4), "traffic": None,
                "kernel": "k_render (per-tile front-to-back blending, one thread per pixel)",
                "peak_source": "FP32 FMA peak from the SM count, 128 lanes/SM and the sampled SM clock",
                "algorithmic": "256 pixels x %d (Gaussian, tile) pairs per frame (mean) x 20 flops" % (sum(pairs) // V)}
    stages = {"frame_ms": round(ms_step / V, 3), "render_call_ms": round(call_ms, 3),
              "blend_kernel_ms": round(blend_ms, 3), "pairs_per_frame": int(sum(pairs) // V),
              "frames_per_s": round(V / (ms_step * 1e-3), 1)}

    # the fully coded scene: geometry streams (17 B per slot) and chunks of 4096 slots culled by the
    # view test; the same cameras, and a close view of one corner that keeps part of the scene
    chunk_slots = 4096
    perm2, scales2 = gsc.gsc_plan_reorder(ctx, pos, sh, group_size=chunk_slots, stream=stream)
    blk2, po2, tab2 = gsc.gsc_encode(ctx, sh, perm2, scales2, gsc.FMT_BC7, stream=stream)
    geom = gsc.gsc_geometry_encode(ctx, pos, scale, rot, logit, po2, chunk_slots, stream=stream)
    close = S.look_at([0.3, 0.3, 0.3], [0.9, 0.9, 0.6], W, H, fov_x_deg=50.0)

    def coded_ms(cam_list, reps):
        kept = 0
        for cam in cam_list:
            r.render_coded(tab2, blk2, po2, geom, chunk_slots, cam, image=imgs[0], stream=stream)
        stream.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            for cam in cam_list:
                _, _, _, kept = r.render_coded(tab2, blk2, po2, geom, chunk_slots, cam, image=imgs[0], stream=stream)
        b.record(stream)
        stream.synchronize()
        return a.elapsed_time(b) / (reps * len(cam_list)), kept

    def float_ms(cam_list, reps):
        for cam in cam_list:
            r.render(tab2, blk2, po2, pos, scale, rot, logit, cam, image=imgs[0], stream=stream)
        stream.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            for cam in cam_list:
                r.render(tab2, blk2, po2, pos, scale, rot, logit, cam, image=imgs[0], stream=stream)
        b.record(stream)
        stream.synchronize()
        return a.elapsed_time(b) / (reps * len(cam_list))

    n_chunks = (po2.shape[0] + chunk_slots - 1) // chunk_slots
    ms_c, kept_all = coded_ms(cams, max(2, args.steps))
    ms_cc, kept_close = coded_ms([close], max(2, args.steps))
    ms_fc = float_ms([close], max(2, args.steps))
    stages["coded"] = {"frame_ms": round(ms_c, 3), "geometry_bytes_per_gaussian": 17,
                       "colour_bytes_per_gaussian": 16, "chunks": int(n_chunks), "kept_chunks_last_view": int(kept_all),
                       "close_view_frame_ms": round(ms_cc, 3), "close_view_kept_chunks": int(kept_close),
                       "close_view_float_geometry_frame_ms": round(ms_fc, 3)}

    # end to end: the coded scene and the geometry from pinned host memory, the frames back to the host
    hosts = [t.cpu().pin_memory() for t in (blk, po, pos, scale, rot, logit)]
    devs = [torch.empty_like(h, device=dev) for h in hosts]
    out_h = torch.empty((V, H, W, 3), dtype=torch.float32).pin_memory()

    def one():
        with torch.cuda.stream(stream):
            for d_, h_ in zip(devs, hosts):
                d_.copy_(h_, non_blocking=True)
        step(*devs)
        with torch.cuda.stream(stream):
            out_h.copy_(imgs, non_blocking=True)

    one()
    stream.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        one()
    stream.synchronize()
    t = max_over_ranks((time.perf_counter() - t0) / args.steps, world, dev)
    e2e = {"value": round(world * n * V / t / 1e6, 3), "unit": UNIT,
           "h2d_bytes_per_step": int(sum(h.numel() * h.element_size() for h in hosts)),
           "d2h_bytes_per_step": int(out_h.numel() * 4), "ms_per_step": round(t * 1e3, 3),
           "path": "pinned host BC7 blocks + slot order + geometry -> %d frames -> frames to host" % V}
    out = {"metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": max(3, args.warmup), "ms_per_step": round(ms_step, 3), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "u8 texels / f32 splatting",
           "data": "synthetic (seeded; stands in for the paper's trained scenes)",
           "config": {"workload": "render: %d Gaussians coded all-BC7 (8 bpt), %d cameras at %d x %d, splat scale "
                                  "%.3f" % (n, V, W, H, cfg["scale"]),
                      "n_gaussians": n, "parallelism": "weak, one scene per GPU" if world > 1 else "single GPU",
                      "l2": "scene larger than L2 (BC7 blocks 48 MB, geometry 96 MB)"},
           "roofline": roofline, "stages": stages, "clocks": clk, "e2e": e2e, "gpu_launches": int(launches)}
    if world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline_render(budget_s=args.cpu_seconds)
    ctx.close()
    return out


def cpu_baseline_render(budget_s=20.0):
    """The oracle renderer on a bounded sample: a 20,000-Gaussian piece of the scene coded and
    rendered at 480 x 270 for one camera, charged per Gaussian per frame."""
    from oracle import oracle as O
    cfg = S.RENDER
    n = 20000
    sc = S.make_scene(n=n, seed=cfg["seed"], clusters=cfg["clusters"], heavy_frac=cfg["heavy_frac"])
    geo = S.make_geometry(n, cfg["geom_seed"], scale=cfg["scale"] * 4)
    cam = S.make_views(1, cfg["view_seed"], 480, 270)[0]
    osc = O.scales(sc.sh)
    q = O.quantise(sc.sh, osc)
    r = O.encode(q, np.arange(n, dtype=np.int32), osc, 1)      # coding is outside the timed frame
    t0 = time.perf_counter()
    tex = O.decode(r["table"], r["blocks"], r["perm"])
    colour = O.eval_sh(tex, osc, pos=sc.pos, cams=O.camera_centre(cam)[None, :])[0]
    O.render(sc.pos, geo.scale, geo.rot, geo.logit, colour, cam)
    t = time.perf_counter() - t0
    return {"value": round(n / t / 1e6, 6), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "decode + SH colour + splatting of %d Gaussians for one 480 x 270 frame (BC1-coded sample), "
                      "per Gaussian per frame" % n}


def C_ref(x):
    import ctypes
    return ctypes.byref(x)


# ------------------------------------------------------------------------------------------------
def run_batch(args, world, rank, local, cpu=True):
    """64 scenes of uneven sizes: one persistent encode launch + one captured evaluation graph,
    against per-scene plain calls (plan, encode, decode + SH eval per scene) on the same data."""
    import torch
    from paper_2607_14513_gb300 import gsc

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    mix = S.batch_mix(**dict(S.BATCH, seed=S.BATCH["seed"] + 1000 * rank))
    fmt_of = {"bc1": gsc.FMT_BC1, "bc7": gsc.FMT_BC7, "rate": gsc.FMT_RATE}
    ctx = gsc.Context(local)
    stream = torch.cuda.Stream(dev)
    cams = torch.from_numpy(S.make_cams(N_CAMS, 1100 + rank)).to(dev)
    scenes, host = [], []
    for n, seed, f, t4 in mix:
        sc = S.make_scene(n, seed, clusters=S.SCENE["clusters"], heavy_frac=S.SCENE["heavy_frac"])
        pos_h = torch.from_numpy(sc.pos).pin_memory()
        sh_h = torch.from_numpy(sc.sh).pin_memory()
        host.append((pos_h, sh_h))
        scenes.append((pos_h.to(dev), sh_h.to(dev), fmt_of[f], t4))
    total_n = sum(m[0] for m in mix)
    batch = gsc.Batch(ctx, scenes, group_size=4096)
    torch.cuda.synchronize()
    tuning, proxy_ms = batch.autotune(stream=stream)
    outs = [torch.empty((n, N_CAMS, 3), dtype=torch.float32, device=dev) for n, _, _, _ in mix]
    outs_plain = [torch.empty((n, N_CAMS, 3), dtype=torch.float32, device=dev) for n, _, _, _ in mix]
    batch.encode(tuning, stream=stream)
    graph = batch.eval_graph(cams, outs, stream=stream)

    def batched():
        batch.encode(tuning, stream=stream)
        graph.launch(stream=stream)

    n_max = max(m[0] for m in mix)
    ws = ctx.workspace(n_max, gsc.FMT_RATE, 32)
    ng_max = (n_max + 15) // 16
    blk = torch.empty(ng_max * 256, dtype=torch.uint8, device=dev)
    po = torch.empty(ng_max * 16, dtype=torch.int32, device=dev)

    def plain():
        for (pos, sh, fmt, t4), out in zip(scenes, outs_plain):
            perm, scales = gsc.gsc_plan_reorder(ctx, pos, sh, ws=ws, stream=stream)
            b, p, tab = gsc.gsc_encode(ctx, sh, perm, scales, fmt, t4, ws=ws, out=blk, perm_out=po, stream=stream)
            gsc.gsc_decode_eval_sh(ctx, tab, b, p, pos=pos, cams=cams, out_order=gsc.OUT_GAUSS_MAJOR, out=out,
                                   stream=stream)

    def timed(fn, steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        stream.synchronize()
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        stream.synchronize()
        return e0.elapsed_time(e1) / steps

    for _ in range(args.warmup):
        batched()
        plain()
    stream.synchronize()
    same = all(torch.equal(a, b) for a, b in zip(outs, outs_plain))
    barrier(world)
    torch.cuda.synchronize()
    uuid = str(torch.cuda.get_device_properties(dev).uuid)
    uuid = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    clocks = ClockSampler(uuid)
    clocks.start()
    gsc.set_timing(ctx, True)
    launches0 = gsc.launch_count()
    ms_batched = timed(batched, args.steps)
    launches = gsc.launch_count() - launches0
    kb_ms, kb_cnt = gsc.kernel_time(ctx, "batch_encode")
    gsc.set_timing(ctx, False)
    ms_plain = timed(plain, args.steps)
    clk = clocks.stop()
    ms_step = max_over_ranks(ms_batched, world, dev)
    ms_plain = max_over_ranks(ms_plain, world, dev)
    ms_graph = timed(lambda: graph.launch(stream=stream), max(5, args.steps))
    res_tabs = [batch.result(i) for i in range(len(mix))]

    def eval_per_scene():
        for i, (pos, _, _, _) in enumerate(scenes):
            _, _, b, p, tab = res_tabs[i]
            gsc.gsc_decode_eval_sh(ctx, tab, b, p, pos=pos, cams=cams, out_order=gsc.OUT_GAUSS_MAJOR, out=outs_plain[i],
                                   stream=stream)

    ms_eval_plain = timed(eval_per_scene, max(5, args.steps))

    # the persistent encode launch: BC7 candidate search of every BC7-searched block (BC1 work not counted)
    nb7 = sum(((m[0] + 15) // 16) * 16 for m in mix if m[2] != "bc1")
    kb_ms /= max(1, kb_cnt)
    roofline = bc7_roofline(ctx, gsc, stream, dev, clk, BC7_EVALS_PER_BLOCK * nb7, kb_ms,
                            "k_batch (persistent BC1/BC7 search over all scenes, schedule %d, %d CTAs/SM, BC1 "
                            "tiles of %d groups)" % (tuning.schedule, tuning.ctas_per_sm, tuning.bc1_tile_groups),
                            nb7, None)
    hbm, hbm_src = peaks()
    ev_bytes = 0
    for i, (n, _, f, _) in enumerate(mix):
        ns = (n + 15) // 16 * 16
        ev_bytes += batch.result(i)[4].total_bytes + 4 * ns + 12 * n + N_CAMS * 12 * n
    ev_gbs = ev_bytes / (ms_graph * 1e-3) / 1e9
    roofline_eval = {"bound": "hbm", "achieved": round(ev_gbs, 1), "peak": hbm, "unit": "GB/s",
                     "frac": round(ev_gbs / hbm, 4), "traffic": None, "peak_source": hbm_src,
                     "kernel": "captured graph of k_eval2 over 64 scenes (%d cameras, Gaussian-major)" % N_CAMS}

    # end to end: pinned host scenes in, every scene's blocks and slot order out
    blocks_h = [torch.empty(max(1, batch.result(i)[2].numel()), dtype=torch.uint8).pin_memory()
                for i in range(len(mix))]
    perm_h = [torch.empty(max(1, batch.result(i)[3].numel()), dtype=torch.int32).pin_memory()
              for i in range(len(mix))]

    def e2e_step():
        with torch.cuda.stream(stream):
            for (pos_h, sh_h), (pos, sh, _, _) in zip(host, scenes):
                pos.copy_(pos_h, non_blocking=True)
                sh.copy_(sh_h, non_blocking=True)
        batched()
        with torch.cuda.stream(stream):
            for i in range(len(mix)):
                _, _, b, p, _ = batch.result(i)
                blocks_h[i][:b.numel()].copy_(b, non_blocking=True)
                perm_h[i][:p.numel()].copy_(p, non_blocking=True)
        return sum(batch.result(i)[2].numel() + 4 * batch.result(i)[3].numel() for i in range(len(mix)))

    e2e_step()
    stream.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        bo = e2e_step()
    stream.synchronize()
    t_e2e = max_over_ranks((time.perf_counter() - t0) / args.steps, world, dev)

    out = {"metric": METRIC, "value": round(world * total_n / (ms_step * 1e-3) / 1e6, 3), "unit": UNIT,
           "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 3),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "u8 texels / int32 search / f32 SH eval", "data": "synthetic (seeded)",
           "config": {"workload": "batched form: %d scenes, %d..%d Gaussians log-uniform (%d total), formats "
                                  "cycling BC1 / BC7 / rate 3-4-6-8 bpt; one persistent encode launch + one "
                                  "captured evaluation graph (%d cameras)" % (len(mix), S.BATCH["lo"],
                                                                             S.BATCH["hi"], total_n, N_CAMS),
                      "n_gaussians": total_n, "parallelism": "weak, one batch per GPU" if world > 1 else "single GPU",
                      "l2": "inputs larger than L2", "bit_exact_vs_per_scene": same},
           "batched_vs_per_scene": {"batched_ms": round(ms_step, 3), "per_scene_ms": round(ms_plain, 3),
                                    "speedup": round(ms_plain / ms_step, 3),
                                    "per_scene_value": round(world * total_n / (ms_plain * 1e-3) / 1e6, 3),
                                    "tuning": {"schedule": tuning.schedule, "ctas_per_sm": tuning.ctas_per_sm,
                                               "bc1_tile_groups": tuning.bc1_tile_groups,
                                               "proxy_ms": round(proxy_ms, 3)}},
           "roofline": roofline, "roofline_decode_eval": roofline_eval,
           "stages": {"batch_encode_ms": round(kb_ms, 3), "eval_graph_ms": round(ms_graph, 3),
                      "eval_per_scene_ms": round(ms_eval_plain, 3)},
           "clocks": clk,
           "e2e": {"value": round(world * total_n / t_e2e / 1e6, 3), "unit": UNIT,
                   "h2d_bytes_per_step": int(total_n * (12 + 192)), "d2h_bytes_per_step": int(bo),
                   "ms_per_step": round(t_e2e * 1e3, 3)},
           "gpu_launches": int(launches)}
    if cpu and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline_mix(mix, budget_s=args.cpu_seconds)
    graph.close()
    ctx.close()
    return out


def run_serve(args, world, rank, local):
    """A Poisson stream of encode and evaluation requests against the request loop: continuous
    batching (4 slots, merged evaluations, high-priority evaluation streams) and, on the same
    trace, a plain queue (one slot, no merging). Latency is the server's submit-to-done time."""
    import queue
    import torch
    from paper_2607_14513_gb300 import gsc

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    cfg = dict(S.SERVE, seed=S.SERVE["seed"] + 1000 * rank)
    pool, reqs = S.serve_trace(**cfg, seconds=args.serve_seconds)
    fmt_of = {"bc1": gsc.FMT_BC1, "bc7": gsc.FMT_BC7}
    ctx = gsc.Context(local)
    host = []
    for n, seed, f in pool:
        sc = S.make_scene(n, seed, clusters=S.SCENE["clusters"], heavy_frac=S.SCENE["heavy_frac"])
        host.append((torch.from_numpy(sc.pos).pin_memory(), torch.from_numpy(sc.sh).pin_memory(), fmt_of[f]))
    cams = [torch.from_numpy(S.make_cams(V, cs)).to(dev) for _, _, _, V, cs in reqs]
    budget = 120 * (1 << 30)

    def play(n_slots, merge, priority):
        srv = gsc.Server(ctx, budget, n_slots=n_slots, merge=merge, priority=priority)
        ts = [srv.encode(i, h[0], h[1], h[2]) for i, h in enumerate(host)]
        for t in ts:
            assert srv.wait(t).status == 0
        done = []
        q = queue.Queue()

        def waiter():
            while True:
                item = q.get()
                if item is None:
                    return
                t, kind, n, V = item
                done.append((kind, srv.wait(t), n, V))

        th = threading.Thread(target=waiter)
        th.start()
        lag = 0.0
        t0 = time.perf_counter()
        for k, (ta, kind, i, V, _) in enumerate(reqs):
            dt = ta - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            lag = max(lag, time.perf_counter() - t0 - ta)
            n = pool[i][0]
            if kind == "encode":
                q.put((srv.encode(i, host[i][0], host[i][1], host[i][2]), kind, n, i))
            else:
                out = torch.empty((n, V, 3), dtype=torch.float32, device=dev)
                q.put((srv.eval(i, n, out, cams=cams[k]), kind, n, i))
        q.put(None)
        th.join()
        span = time.perf_counter() - t0
        st = srv.stats()
        srv.close()
        lat = {kd: np.array([r.t_done_ms - r.t_submit_ms for k2, r, _, _ in done if kd in (k2, "all")])
               for kd in ("all", "encode", "eval")}
        # evaluations that had to wait for an earlier re-encode of their scene (submission order)
        enc_spans = {}
        for k2, r, _, sc in done:
            if k2 == "encode":
                enc_spans.setdefault(sc, []).append((r.t_submit_ms, r.t_done_ms))
        free, dep = [], []
        for k2, r, _, sc in done:
            if k2 != "eval":
                continue
            waited = any(a < r.t_submit_ms < b for a, b in enc_spans.get(sc, []))
            (dep if waited else free).append(r.t_done_ms - r.t_submit_ms)
        lat["eval_no_pending_encode"] = np.array(free)
        lat["eval_behind_encode"] = np.array(dep)
        lat["queue_wait"] = np.array([r.t_admit_ms - r.t_submit_ms for _, r, _, _ in done])
        lat["service"] = np.array([r.t_done_ms - r.t_admit_ms for _, r, _, _ in done])
        bad = sum(r.status != 0 for _, r, _, _ in done)
        gauss = sum(n for _, r, n, _ in done)
        pct = {}
        for kd, a in lat.items():
            if a.size:
                pct[kd] = {"p50_ms": round(float(np.percentile(a, 50)), 3),
                           "p99_ms": round(float(np.percentile(a, 99)), 3), "count": int(a.size)}
        return {"latency": pct, "served_req_s": round(len(done) / span, 2), "MGauss_s": round(gauss / span / 1e6, 3),
                "span_s": round(span, 3), "failed": int(bad), "merged": int(st.merged), "evictions": int(st.evictions),
                "peak_bytes": int(st.peak_bytes), "max_submit_lag_ms": round(lag * 1e3, 3),
                "slots": n_slots, "merge": bool(merge), "priority": bool(priority)}

    barrier(world)
    uuid = str(torch.cuda.get_device_properties(dev).uuid)
    uuid = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    clocks = ClockSampler(uuid)
    clocks.start()
    launches0 = gsc.launch_count()
    cb = play(4, True, True)
    launches = gsc.launch_count() - launches0
    clk = clocks.stop()
    plain = play(1, False, False)
    value = max_over_ranks(-cb["MGauss_s"], world, dev) * -1 * world
    out = {"metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": 1, "warmup": 1,
           "ms_per_step": round(cb["span_s"] * 1e3, 3), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "u8 texels / int32 search / f32 SH eval", "data": "synthetic (seeded)",
           "config": {"workload": "served form: Poisson %.0f req/s for %.0f s, %.0f%% re-encodes of a pool of %d "
                                  "scenes (%d..%d Gaussians log-uniform, half BC1 / half BC7), the rest decode + SH "
                                  "eval of 1..32 camera centres; 120 GB HBM admission budget"
                                  % (cfg["rate_hz"], args.serve_seconds, 100 * cfg["encode_frac"], cfg["n_scenes"],
                                     cfg["lo"], cfg["hi"]),
                      "requests": len(reqs), "pool_gaussians": int(sum(p[0] for p in pool))},
           "serving": {"continuous_batching": cb, "plain_queue": plain},
           "clocks": clk, "gpu_launches": int(launches),
           "e2e": {"value": round(value, 3), "unit": UNIT, "h2d_bytes_per_step": None, "d2h_bytes_per_step": 0,
                   "note": "requests carry pinned host scenes (encode) and device outputs (eval)"}}
    ctx.close()
    return out


def cpu_baseline_mix(mix, budget_s=20.0):
    """The oracle's per-Gaussian stage times (scene-scale sample) charged to each scene of a
    batch by its format: plan + its coding(s) + one decode + SH evaluation."""
    b = cpu_baseline("scene3m", budget_s=budget_s)
    st = {k: v * 1e-6 for k, v in b["stage_us_per_gaussian"].items()}
    enc = {"bc1": st["bc1"], "bc7": st["bc7"], "rate": st["bc1"] + st["bc7"]}
    t = sum(n * (st["plan"] + enc[f] + st["decode_eval"]) for n, _, f, _ in mix)
    return {"value": round(sum(m[0] for m in mix) / t / 1e6, 6), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": b["sample"] + "; charged per scene by format"}


# ------------------------------------------------------------------------------------------------
def cpu_baseline(workload, budget_s=20.0):
    if workload == "layouts3m":
        return cpu_baseline_layouts(budget_s)
    if workload == "render3m":
        return cpu_baseline_render(budget_s)
    return cpu_baseline_d(workload, budget_s)


def cpu_baseline_layouts(budget_s=20.0):
    """The oracle's per-block coding times (scene-scale sample of layout D's blocks) charged per
    Gaussian to the layout codings of one step: BC7 / BC1 blocks per Gaussian of each coding, plus
    the plan and one decode + SH evaluation per coding."""
    b = cpu_baseline_d("scene3m", budget_s=budget_s)
    st = {k: v * 1e-6 for k, v in b["stage_us_per_gaussian"].items()}
    per_g = st["plan"] + sum((j / 16.0) * st["bc7"] + (1 - j / 16.0) * st["bc1"] + st["decode_eval"]
                             for _, _, _, j, _ in LAYOUT_CODINGS)
    return {"value": round(1.0 / per_g / 1e6, 6), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": b["sample"] + "; charged per Gaussian by each coding's BC7 / BC1 block counts"}


def cpu_baseline_d(workload, budget_s=20.0):
    """The oracle, as it stands, single-threaded on a bounded sample of the workload.

    Per stage it codes a sample and charges the per-Gaussian time; the stages are the
    step's: plan (scales, quantisation, reorder), BC1 and BC7 coding of every block plus
    the rate control, decode + SH evaluation of 8 cameras for three codings, and the
    software decode twice (the CPU has no texture unit: the second decode stands in)."""
    from oracle import oracle as O
    cfg = dict(workload_cfg(workload))
    n_plan = min(cfg["n"], 200_000)
    sc = S.make_scene(**dict(cfg, n=n_plan))
    cams = S.make_cams(N_CAMS, 1100)
    t0 = time.perf_counter()
    scl = O.scales(sc.sh)
    q = O.quantise(sc.sh, scl)
    perm = O.plan(sc.pos, q, 4096, 1)
    t_plan = (time.perf_counter() - t0) / n_plan
    st = O.stage(q, perm[: (min(n_plan, 4096) // 16) * 16])
    blocks = st.reshape(-1, 16, 3)
    nb7 = 256 if budget_s < 10 else 1024
    t0 = time.perf_counter()
    O.encode_blocks(blocks[:nb7], 7, threads=1)
    t_bc7 = (time.perf_counter() - t0) / nb7
    nb1 = min(blocks.shape[0], 8192)
    t0 = time.perf_counter()
    O.encode_blocks(blocks[:nb1], 1, threads=1)
    t_bc1 = (time.perf_counter() - t0) / nb1
    # the dominant stage again on every host core (the same scalar code, blocks split across threads)
    cores = os.cpu_count() or 1
    nb7_all = min(blocks.shape[0], nb7 * max(1, cores // 2))
    t0 = time.perf_counter()
    O.encode_blocks(blocks[:nb7_all], 7, threads=cores)
    t_bc7_all = (time.perf_counter() - t0) / nb7_all
    n_ev = 4096
    r = O.encode(q[:n_ev], np.arange(n_ev, dtype=np.int32), scl, 1)
    t0 = time.perf_counter()
    for _ in range(3):
        tex = O.decode(r["table"], r["blocks"], r["perm"])
        O.eval_sh(tex, scl, pos=sc.pos[:n_ev], cams=cams)
    t_eval = (time.perf_counter() - t0) / (3 * n_ev)
    t0 = time.perf_counter()
    for _ in range(4):
        O.decode(r["table"], r["blocks"], r["perm"])
    t_dec = (time.perf_counter() - t0) / n_ev
    # one block per Gaussian per coding (16 blocks per 16-Gaussian group)
    per_gauss = t_plan + t_bc7 + t_bc1 + t_eval + t_dec
    per_gauss_all = t_plan + t_bc7_all + t_bc1 + t_eval + t_dec
    return {"value": round(1.0 / per_gauss / 1e6, 6), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "plan on %d Gaussians; BC7 on %d and BC1 on %d staged blocks; decode + SH eval (8 cams, x3) "
                      "and 4 decodes on %d Gaussians; scaled per Gaussian" % (n_plan, nb7, nb1, n_ev),
            "stage_us_per_gaussian": {"plan": round(t_plan * 1e6, 3), "bc7": round(t_bc7 * 1e6, 1),
                                      "bc1": round(t_bc1 * 1e6, 2), "decode_eval": round(t_eval * 1e6, 2),
                                      "decode": round(t_dec * 1e6, 2)},
            "all_cores": {"value": round(1.0 / per_gauss_all / 1e6, 6), "cores": cores,
                          "bc7_us_per_block": round(t_bc7_all * 1e6, 2),
                          "sample": "BC7 (the dominant stage) on %d blocks over %d threads; other stages as "
                                    "single-threaded" % (nb7_all, cores)}}


def run_reference(args, world, rank):
    if rank != 0:
        return
    if args.workload == "serve":
        print(json.dumps({"impl": "reference", "unavailable": "the oracle has no request loop; the served "
                          "form's per-request work is the batch64 and scene3m reference arms' work"}), flush=True)
        return
    times = []
    base = None
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        if args.workload == "batch64":
            base = cpu_baseline_mix(S.batch_mix(**S.BATCH), budget_s=5.0)
        else:
            base = cpu_baseline(args.workload, budget_s=5.0)
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    v = base["value"]
    out = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": round(1e3 * statistics.median(times), 3), "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "u8 texels / int search / f64 SH eval", "impl": "reference",
           "data": "synthetic (seeded)",
           "config": (scene_config(workload_cfg(args.workload), world)
                      if args.workload in ("scene3m", "medium262k", "tiny4k") else {"workload": args.workload}),
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": base["cores"], "kind": "oracle",
                            "sample": base["sample"]},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gsc", choices=["gsc", "reference"])
    ap.add_argument("--workload", default="scene3m",
                    choices=["scene3m", "medium262k", "tiny4k", "layouts3m", "render3m", "batch64", "serve"])
    ap.add_argument("--serve-seconds", type=float, default=60.0)
    ap.add_argument("--scene-only", action="store_true", help="scene3m without the batched and served forms")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    import torch
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    run = {"batch64": run_batch, "serve": run_serve, "layouts3m": run_layouts, "render3m": run_render}
    out = run.get(args.workload, run_gsc)(args, world, rank, local)
    if args.workload == "scene3m" and not args.scene_only:
        # the batched and served forms, beside the scene step on the same GPU(s)
        torch.cuda.empty_cache()
        b = run_batch(args, world, rank, local, cpu=False)
        out["batched"] = {"value": b["value"], "unit": UNIT, "per_scene_value": b["batched_vs_per_scene"]["per_scene_value"],
                          "ratio": b["batched_vs_per_scene"]["speedup"],
                          "bit_identical": b["config"]["bit_exact_vs_per_scene"],
                          "batched_ms": b["batched_vs_per_scene"]["batched_ms"],
                          "per_scene_ms": b["batched_vs_per_scene"]["per_scene_ms"],
                          "workload": b["config"]["workload"], "clocks": b["clocks"],
                          "gpu_launches": b["gpu_launches"], "e2e": b["e2e"]}
        torch.cuda.empty_cache()
        v = run_serve(args, world, rank, local)
        srv = v["serving"]
        out["served"] = {kind: {"p50_ms": srv[kind]["latency"]["all"]["p50_ms"],
                                "p99_ms": srv[kind]["latency"]["all"]["p99_ms"],
                                "req_s": srv[kind]["served_req_s"], "MGauss_s": srv[kind]["MGauss_s"],
                                "span_s": srv[kind]["span_s"], "failed": srv[kind]["failed"],
                                "latency": srv[kind]["latency"]}
                         for kind in ("continuous_batching", "plain_queue")}
        out["served"]["trace"] = v["config"]["workload"]
        out["served"]["clocks"] = v["clocks"]
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
