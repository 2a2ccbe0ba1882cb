"""The checked build (libgsc_checked.so, GSC_CHECKED=1): slot-order entries outside [-1, n)
handed to the decoders are reported, never used.

Runs in a child process with GSC_CHECKED=1, which first makes sure the checked library is the
one loaded (the normal build trusts the slot order, so it must never see the corrupted one).
Every decode path (software decode, fused evaluation in three output orders, texture decode,
resident texture scene) reports GSC_ERR_DEVICE through gsc_ctx_sync, and the slots that were
not corrupted decode exactly as with the intact slot order.
"""
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import sys
import numpy as np
import torch
sys.path.insert(0, ROOT)
from paper_2607_14513_gb300 import gsc, synthetic as S
lib = gsc.load()
if lib.gsc_build_checked() != 1:
    sys.exit(3)                       # not the checked build: never hand it the corrupted order
ctx = gsc.Context(0)
n = 20000
sc = S.make_scene(n, 4500, clusters=4, heavy_frac=0.1)
pos, sh = torch.from_numpy(sc.pos).cuda(), torch.from_numpy(sc.sh).cuda()
perm, scales = gsc.gsc_plan_reorder(ctx, pos, sh)
blocks, perm_out, tab = gsc.gsc_encode(ctx, sh, perm, scales, gsc.FMT_RATE, 24)
ctx.sync()
bad = perm_out.clone()
bad_slots = [5, 777, 4321]
bad[5] = n + 1000
bad[777] = -9
bad[4321] = 2 ** 30
displaced = set(int(perm_out[s]) for s in bad_slots)
keep = np.array([o for o in range(n) if o not in displaced])

def expect_device_error(what):
    try:
        ctx.sync()
    except gsc.GscError as e:
        assert e.code == 7, (what, e.code)
        return
    raise AssertionError("no check failure reported: " + what)

good = gsc.gsc_decode(ctx, tab, blocks, perm_out)
ctx.sync()
got = gsc.gsc_decode(ctx, tab, blocks, bad)
expect_device_error("decode")
assert torch.equal(got[keep], good[keep])
cams = torch.from_numpy(S.make_cams(4, 9)).cuda()
for order in (0, 1, 2):
    gsc.gsc_decode_eval_sh(ctx, tab, blocks, bad, pos=pos, cams=cams, out_order=order)
    expect_device_error("eval %d" % order)
gsc.gsc_decode_tex(ctx, tab, blocks, bad)
expect_device_error("texture decode")
t7 = gsc.forced_table(tab, gsc.FMT_BC7)
blocks7, perm7, tab7 = gsc.gsc_encode(ctx, sh, perm, scales, gsc.FMT_BC7)
ctx.sync()
bad7 = perm7.clone()
bad7[9] = n
scene = gsc.TexScene(ctx, tab7, blocks7, perm=bad7, pos=pos)
expect_device_error("texture scene positions")
gsc.gsc_decode_eval_sh_tex(ctx, scene, bad7, cams=cams, out_order=gsc.OUT_GAUSS_MAJOR)
expect_device_error("texture evaluation")
scene.close()
# and an intact order afterwards reports nothing
gsc.gsc_decode(ctx, tab, blocks, perm_out)
ctx.sync()
print("ok")
'''


def test_checked_build_reports_bad_slot_entries():
    from paper_2607_14513_gb300 import gsc
    assert gsc.load().gsc_build_checked() == 0        # the normal build (this process)
    env = dict(os.environ, GSC_CHECKED="1")
    r = subprocess.run([sys.executable, "-c", "ROOT = %r\n" % ROOT + CHILD], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, (r.returncode, r.stdout[-2000:], r.stderr[-4000:])
    assert r.stdout.strip().endswith("ok")
