"""Checkpoint files of coded scenes (gsc_scene_write / gsc_scene_read) with host buffers, no GPU:
the bytes read back equal the bytes written, and a damaged, truncated, padded or foreign file, or
a buffer too small, is refused."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2607_14513_gb300 import gsc


def _scene(n=1000, fmt=7, seed=5):
    rng = np.random.default_rng(seed)
    ng = (n + 15) // 16
    t = gsc.StreamTable()
    t.n_streams, t.format, t.n, t.n_groups = 1, fmt, n, ng
    bpb = 16 if fmt == 7 else 8
    t.total_bytes = ng * 16 * bpb
    t.used_bits = t.total_bytes * 8
    t.scales[:] = list(rng.uniform(0.1, 2.0, 16).astype(np.float32))
    t.weights[:] = list(rng.integers(1, 65536, 16))
    t.s[0].bands, t.s[0].bc7_blocks, t.s[0].first_group, t.s[0].n_groups = 16, 16 if fmt == 7 else 0, 0, ng
    blocks = torch.from_numpy(rng.integers(0, 256, t.total_bytes, dtype=np.uint8))
    perm = torch.from_numpy(np.concatenate([rng.permutation(n), -np.ones(ng * 16 - n, np.int64)]).astype(np.int32))
    pos = torch.from_numpy(rng.uniform(0, 1, (n, 3)).astype(np.float32))
    return t, blocks, perm, pos


def _bytes(t):
    import ctypes
    return ctypes.string_at(ctypes.addressof(t), ctypes.sizeof(t))


@pytest.mark.parametrize("fmt,with_pos", [(7, True), (1, False)])
def test_round_trip(tmp_path, fmt, with_pos):
    t, blocks, perm, pos = _scene(fmt=fmt)
    p = tmp_path / "scene.gsc"
    gsc.scene_write(str(p), t, blocks, perm, pos if with_pos else None)
    t2, b2, p2, q2 = gsc.scene_read(str(p))
    assert _bytes(t2) == _bytes(t)
    assert torch.equal(b2, blocks) and torch.equal(p2, perm)
    if with_pos:
        assert torch.equal(q2, pos)
    else:
        assert q2 is None


def test_damaged_files_are_refused(tmp_path):
    t, blocks, perm, pos = _scene()
    p = tmp_path / "scene.gsc"
    gsc.scene_write(str(p), t, blocks, perm, pos)
    raw = bytearray(p.read_bytes())
    cases = {}
    flipped = bytearray(raw); flipped[-5] ^= 1; cases["payload bit"] = flipped
    cases["truncated"] = raw[:-7]
    cases["trailing"] = raw + b"x"
    magic = bytearray(raw); magic[0] ^= 0xFF; cases["magic"] = magic
    version = bytearray(raw); version[8] += 1; cases["version"] = version
    for name, data in cases.items():
        q = tmp_path / ("bad_%s.gsc" % name.replace(" ", "_"))
        q.write_bytes(bytes(data))
        with pytest.raises(gsc.GscError):
            gsc.scene_read(str(q))
    # a buffer that is too small
    small = torch.empty(10, dtype=torch.uint8)
    t2 = gsc.StreamTable()
    rc = gsc.load().gsc_scene_read(str(p).encode(), gsc.C.byref(t2), gsc._ptr(small), small.numel(), gsc._ptr(perm),
                                   4 * perm.numel(), None, 0)
    assert rc == 1
    with pytest.raises(gsc.GscError):
        gsc.scene_read(str(tmp_path / "missing.gsc"))
