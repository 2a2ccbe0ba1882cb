"""The bench's N > 1 path on CPU: one process per rank over gloo on 127.0.0.1.

Multi-GPU runs are weak scaling: every rank codes its own scene, and the only collectives are
the timing barrier and the max over ranks of the step time (no data-path exchange). These
tests run that path with world size 2: each rank times its own (oracle) plan of its own
scene, the barrier and the max-over-ranks reduction give every rank the slowest rank's time,
and the whole-job value counts every rank's Gaussians. The reference arm under two ranks
prints one line from rank 0 and nothing from rank 1.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import time

    import numpy as np
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench
    from oracle import oracle as O
    from paper_2607_14513_gb300 import synthetic as S

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    cfg = dict(S.TINY)
    cfg["seed"] = cfg["seed"] + 1000 * rank          # each rank its own scene, as bench.py does
    sc = S.make_scene(**cfg)
    O.lib()
    bench.barrier(world)
    t0 = time.perf_counter()
    q = O.quantise(sc.sh, O.scales(sc.sh))
    perm = O.plan(sc.pos, q, 4096, 1)
    own = (time.perf_counter() - t0) * 1e3 + 10.0 * rank   # make the ranks' times differ
    slowest = bench.max_over_ranks(own, world, "cpu")
    value = world * cfg["n"] / (slowest * 1e-3) / 1e6
    with open(os.path.join(out_dir, "rank%d.json" % rank), "w") as f:
        json.dump({"own": own, "slowest": slowest, "value": value, "perm_head": perm[:32].tolist(),
                   "checksum": int(np.asarray(perm, np.int64).sum())}, f)
    dist.destroy_process_group()


def test_weak_scaling_timing_path_two_ranks(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.spawn(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    r = [json.load(open(tmp_path / ("rank%d.json" % i))) for i in range(2)]
    slowest = max(x["own"] for x in r)
    assert all(x["slowest"] == pytest.approx(slowest) for x in r)       # every rank sees the max
    assert all(x["value"] == pytest.approx(2 * 4096 / (slowest * 1e-3) / 1e6) for x in r)
    assert r[0]["perm_head"] != r[1]["perm_head"]                       # independent scenes per rank
    # a rank's work does not depend on the other rank: rank 0 alone reproduces its plan
    sys.path.insert(0, ROOT)
    import numpy as np
    from oracle import oracle as O
    from paper_2607_14513_gb300 import synthetic as S
    O.lib()
    sc = S.make_scene(**S.TINY)
    perm = O.plan(sc.pos, O.quantise(sc.sh, O.scales(sc.sh)), 4096, 1)
    assert int(np.asarray(perm, np.int64).sum()) == r[0]["checksum"]


def test_reference_arm_prints_once_under_two_ranks():
    procs = []
    for rank in range(2):
        env = dict(os.environ, RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(_free_port()))
        procs.append(subprocess.Popen([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                                       "--gpus", "2", "--steps", "1", "--warmup", "0", "--workload", "tiny4k"],
                                      cwd=ROOT, env=env, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = [p.communicate(timeout=600) for p in procs]
    assert [p.returncode for p in procs] == [0, 0], [o[1][-2000:] for o in outs]
    lines0 = [ln for ln in outs[0][0].splitlines() if ln.strip()]
    assert len(lines0) == 1
    d = json.loads(lines0[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
    # the same workload config as the GPU arm prints for this workload
    import bench
    assert d["config"] == bench.scene_config(bench.workload_cfg("tiny4k"), 2)
    assert outs[1][0].strip() == ""
