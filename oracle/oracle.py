"""Python wrapper of the plain CPU oracle (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may
import this module. It builds ``liboracle.so`` from ``gsc_oracle.c`` with gcc
(``-O2 -ffp-contract=off``) and exposes numpy-level functions. Nothing here is
used by the CUDA product path, and nothing here imports the product package.

Every function mirrors one step of the paper's pipeline; the C source cites the
passage each follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "gsc_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")
SH = 16
MODES = 14

_lib = None
_lock = threading.Lock()
# A library to load instead of building liboracle.so (the pin tests' planted-mistake copies use it).
LIB_OVERRIDE = None


def build(force: bool = False) -> str:
    """Compile the oracle (plain C, one translation unit)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(
            os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "gsc_oracle.h"))):
        tmp = LIB + ".tmp.%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-pthread",
                               "-fPIC", "-shared", "-o", tmp, SRC, "-lm"])
        os.replace(tmp, LIB)
    return LIB


class Stream(C.Structure):
    _fields_ = [("bands", C.c_int32), ("bc7_blocks", C.c_int32), ("first_group", C.c_int64),
                ("n_groups", C.c_int64), ("byte_offset", C.c_int64)]


class Table(C.Structure):
    _fields_ = [("n_streams", C.c_int32), ("format", C.c_int32), ("n", C.c_int64), ("n_groups", C.c_int64),
                ("total_bytes", C.c_int64), ("budget_bits", C.c_uint64), ("used_bits", C.c_uint64),
                ("lambda_", C.c_uint64), ("scales", C.c_float * SH), ("weights", C.c_uint32 * SH),
                ("s", Stream * MODES), ("layout", C.c_int32)]

LAYOUT_D, LAYOUT_A, LAYOUT_B = 0, 1, 2


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(LIB_OVERRIDE or build())
            P = C.c_void_p
            i64, u64, i32, u32 = C.c_int64, C.c_uint64, C.c_int, C.c_uint32
            sig = {
                "or_scales": (i32, [P, i64, u32, P]),
                "or_quant1": (C.c_uint8, [C.c_float, C.c_float]),
                "or_quantise": (None, [P, i64, P, P]),
                "or_morton30": (u32, [u32, u32, u32]),
                "or_colour_key": (u32, [u32, u32, u32]),
                "or_plan": (i32, [P, P, i64, i64, i32, P]),
                "or_stage_group": (None, [P, P, i64, P]),
                "or_layout_map": (None, [i32, i32, i32, P, P]),
                "or_layout_ok": (i32, [i32, i32]),
                "or_layout_bc7": (i32, [i32, i32, i32]),
                "or_stage_layout": (None, [P, P, i32, i64, P]),
                "or_encode_layout": (i32, [P, i64, P, P, i32, i32, P, P]),
                "or_bc1_palette": (None, [C.c_uint16, C.c_uint16, P]),
                "or_bc1_decode": (None, [P, P]),
                "or_bc1_candidate_sse": (u64, [P, C.c_uint16, C.c_uint16]),
                "or_bc1_encode": (u64, [P, P]),
                "or_bc7_subset": (i32, [i32, i32, i32]),
                "or_bc7_anchor": (i32, [i32, i32, i32]),
                "or_bc7_decode": (None, [P, P]),
                "or_bc7_n_candidates": (i32, []),
                "or_bc7_candidate": (u64, [P, i32, P]),
                "or_bc7_encode": (u64, [P, P]),
                "or_encode_blocks": (None, [P, i64, i32, P, P]),
                "or_mode_table": (None, [P, P]),
                "or_weights": (None, [P, P]),
                "or_rate_choose": (i32, [P, i64, u64, P]),
                "or_rate_control": (i32, [P, i64, u64, P, P]),
                "or_encode": (i32, [P, i64, P, P, i32, u32, P, P, P, P]),
                "or_set_threads": (None, [i32]),
                "or_code_groups": (None, [P, i64, P, P, P, P, P]),
                "or_rate_assemble": (i32, [i64, P, P, u32, P, P, P, P, P, P]),
                "or_decode": (i32, [P, P, P, P]),
                "or_camera_centre": (None, [P, P]),
                "or_splat_setup": (i32, [P, P, P, P, P]),
                "or_render": (i32, [i64, P, P, P, P, P, P, P, i64, P, P, P]),
                "or_chunks": (i64, [i64, i64]),
                "or_chunk_table": (None, [P, P, P, i64, i64, P]),
                "or_geometry_encode": (None, [P, P, P, P, P, i64, i64, P, P, P, P, P]),
                "or_geometry_decode_slot": (None, [P, P, P, P, i64, i64, P, P, P, P, P]),
                "or_chunk_visible": (i32, [P, P]),
                "or_geometry_decode_all": (None, [P, P, P, P, i64, i64, P, P, P, P, P]),
                "or_sh_basis": (None, [C.c_double, C.c_double, C.c_double, P]),
                "or_eval_sh": (None, [P, i64, P, P, P, P, i32, P, P]),
            }
            for name, (res, args) in sig.items():
                f = getattr(_lib, name)
                f.restype = res
                f.argtypes = args
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# --- scales and quantisation (Sec. V-A) -------------------------------------------------
def scales(sh, permille=995):
    sh = _c(sh, np.float32)
    out = np.zeros(SH, np.float32)
    rc = lib().or_scales(_p(sh), sh.shape[0], permille, _p(out))
    if rc != 0:
        raise ValueError("or_scales failed: %d" % rc)
    return out


def quant1(x, s):
    return lib().or_quant1(float(np.float32(x)), float(np.float32(s)))


def quantise(sh, sc):
    sh = _c(sh, np.float32)
    sc = _c(sc, np.float32)
    q = np.zeros(sh.shape, np.uint8)
    lib().or_quantise(_p(sh), sh.shape[0], _p(sc), _p(q))
    return q


# --- reorder (Sec. III-C) -------------------------------------------------------------
def morton30(x, y, z):
    return lib().or_morton30(x, y, z)


def colour_key(r, g, b):
    return lib().or_colour_key(r, g, b)


def plan(pos, q, group_size=4096, sort=1):
    pos = _c(pos, np.float32)
    q = _c(q, np.uint8)
    n = pos.shape[0]
    ns = (n + 15) // 16 * 16
    perm = np.full(max(ns, 1), -1, np.int32)[:ns]
    rc = lib().or_plan(_p(pos), _p(q), n, group_size, sort, _p(perm))
    if rc != 0:
        raise ValueError("or_plan failed: %d" % rc)
    return perm


def stage(q, perm):
    """Layout-D texels of every group: [n_groups, 16 blocks, 16 texels, 3]."""
    q = _c(q, np.uint8)
    perm = _c(perm, np.int32)
    ng = perm.shape[0] // 16
    out = np.zeros((ng, 16, 16, 3), np.uint8)
    for g in range(ng):
        lib().or_stage_group(_p(q), _p(perm), g, _p(out[g]))
    return out


# --- BC1 / BC7 (Sec. III-A/B; the BC1 and BC7 format definitions) -------------------------
def bc1_palette(c0, c1):
    pal = np.zeros((4, 4), np.uint8)
    lib().or_bc1_palette(c0, c1, _p(pal))
    return pal


def bc1_decode(blk):
    blk = _c(blk, np.uint8)
    out = np.zeros((16, 4), np.uint8)
    lib().or_bc1_decode(_p(blk), _p(out))
    return out


def bc1_candidate_sse(tex, c0, c1):
    tex = _c(tex, np.uint8)
    return lib().or_bc1_candidate_sse(_p(tex), c0, c1)


def bc7_decode(blk):
    blk = _c(blk, np.uint8)
    out = np.zeros((16, 4), np.uint8)
    lib().or_bc7_decode(_p(blk), _p(out))
    return out


def bc7_subset(ns, part, t):
    return lib().or_bc7_subset(ns, part, t)


def bc7_anchor(ns, part, s):
    return lib().or_bc7_anchor(ns, part, s)


def bc7_n_candidates():
    return lib().or_bc7_n_candidates()


def bc7_candidate(tex, e):
    tex = _c(tex, np.uint8)
    out = np.zeros(16, np.uint8)
    s = lib().or_bc7_candidate(_p(tex), e, _p(out))
    return s, out


def encode_blocks(tex, fmt, threads=None):
    """Encode independent blocks tex [nblk, 16, 3] -> (blocks [nblk, 8|16], sse [nblk])."""
    tex = _c(tex, np.uint8).reshape(-1, 16, 3)
    nb = tex.shape[0]
    bpb = 16 if fmt == 7 else 8
    out = np.zeros((nb, bpb), np.uint8)
    sse = np.zeros(nb, np.uint64)
    threads = threads or min(32, os.cpu_count() or 1)
    L = lib()

    def run(lo, hi):
        L.or_encode_blocks(_p(tex[lo:hi]), hi - lo, fmt, _p(out[lo:hi]), _p(sse[lo:hi]))

    chunk = max(1, (nb + threads * 4 - 1) // (threads * 4))
    if threads <= 1 or nb <= chunk:
        run(0, nb)
    else:
        with ThreadPoolExecutor(threads) as ex:
            list(ex.map(lambda lo: run(lo, min(nb, lo + chunk)), range(0, nb, chunk)))
    return out, sse


def decode_blocks(blocks, fmt):
    blocks = _c(blocks, np.uint8)
    bpb = 16 if fmt == 7 else 8
    blocks = blocks.reshape(-1, bpb)
    out = np.zeros((blocks.shape[0], 16, 4), np.uint8)
    f = bc7_decode if fmt == 7 else bc1_decode
    for i in range(blocks.shape[0]):
        out[i] = f(blocks[i])
    return out


# --- rate control (Sec. IV-B) -------------------------------------------------------------
def mode_table():
    b = np.zeros(MODES, np.int32)
    j = np.zeros(MODES, np.int32)
    lib().or_mode_table(_p(b), _p(j))
    return b, j


def weights(sc):
    sc = _c(sc, np.float32)
    w = np.zeros(SH, np.uint32)
    lib().or_weights(_p(sc), _p(w))
    return w


def rate_choose(D, lam):
    D = _c(D, np.uint64)
    mode = np.zeros(D.shape[0], np.uint8)
    lib().or_rate_choose(_p(D), D.shape[0], lam, _p(mode))
    return mode


def rate_control(D, budget):
    D = _c(D, np.uint64)
    mode = np.zeros(max(D.shape[0], 1), np.uint8)[:D.shape[0]]
    lam = C.c_uint64(0)
    rc = lib().or_rate_control(_p(D), D.shape[0], budget, _p(mode), C.byref(lam))
    return rc, mode, lam.value


# --- block layouts (Sec. IV-B, Figs. SetupA / SetupB / SetupD; Table I) ---------------------
def layout_map(layout, k, t):
    """(slot in group, coefficient) held by texel t of block k (Sec. IV-B, Figs. SetupA/B/D)."""
    u, c = C.c_int(0), C.c_int(0)
    lib().or_layout_map(layout, k, t, C.byref(u), C.byref(c))
    return u.value, c.value


def layout_ok(layout, bc7_blocks):
    return bool(lib().or_layout_ok(layout, bc7_blocks))


def layout_bc7(layout, bc7_blocks, k):
    return bool(lib().or_layout_bc7(layout, bc7_blocks, k))


def stage_layout(q, perm, layout):
    """Texels of every group in a layout: [n_groups, 16 blocks, 16 texels, 3]."""
    q = _c(q, np.uint8)
    perm = _c(perm, np.int32)
    ng = perm.shape[0] // 16
    out = np.zeros((ng, 16, 16, 3), np.uint8)
    for g in range(ng):
        lib().or_stage_layout(_p(q), _p(perm), layout, g, _p(out[g]))
    return out


def encode_layout(q, perm, sc, layout, bc7_blocks):
    """Fixed coding of a layout: bc7_blocks BC7 blocks per group, the rest BC1 (one stream)."""
    q = _c(q, np.uint8)
    perm = _c(perm, np.int32)
    sc = _c(sc, np.float32)
    n = q.shape[0]
    ng = (n + 15) // 16
    blocks = np.zeros(max(ng * 256, 1), np.uint8)
    t = Table()
    rc = lib().or_encode_layout(_p(q), n, _p(perm), _p(sc), layout, bc7_blocks, _p(blocks), C.byref(t))
    if rc != 0:
        raise ValueError("or_encode_layout failed: %d" % rc)
    return dict(blocks=blocks[:t.total_bytes], perm=perm[:ng * 16].copy(), table=t)


# --- stream encode and decode of a scene (Sec. IV-B streams; Sec. I and III decode) --------
def table_dict(t: Table):
    return dict(n_streams=t.n_streams, format=t.format, n=t.n, n_groups=t.n_groups, total_bytes=t.total_bytes,
                layout=t.layout,
                budget_bits=t.budget_bits, used_bits=t.used_bits, lambda_=t.lambda_,
                scales=np.array(t.scales[:], np.float32), weights=np.array(t.weights[:], np.uint32),
                streams=[dict(bands=t.s[i].bands, bc7_blocks=t.s[i].bc7_blocks, first_group=t.s[i].first_group,
                              n_groups=t.s[i].n_groups, byte_offset=t.s[i].byte_offset) for i in range(t.n_streams)])


def encode(q, perm, sc, fmt, target_x4=0, want_dtab=False):
    """Layout-D encode; fmt 1 / 7 forced, 0 = rate control at target_x4 / 4 bits per texel."""
    q = _c(q, np.uint8)
    perm = _c(perm, np.int32)
    sc = _c(sc, np.float32)
    n = q.shape[0]
    ng = (n + 15) // 16
    blocks = np.zeros(max(ng * 256, 1), np.uint8)
    perm_out = np.full(max(ng * 16, 1), -1, np.int32)
    t = Table()
    dtab = np.zeros((max(ng, 1), MODES), np.uint64) if want_dtab else None
    rc = lib().or_encode(_p(q), n, _p(perm), _p(sc), fmt, target_x4, _p(blocks), _p(perm_out), C.byref(t), _p(dtab))
    if rc != 0:
        raise ValueError("or_encode failed: %d" % rc)
    res = dict(blocks=blocks[:t.total_bytes], perm=perm_out[:ng * 16], table=t)
    if want_dtab:
        res["dtab"] = dtab[:ng]
    return res


def encode_rates(q, perm, sc, targets_x4, threads=1):
    """Rate-controlled encode at several targets from one coding pass (the coding step split
    over `threads`; results equal encode(q, perm, sc, 0, t) for each target t)."""
    q = _c(q, np.uint8)
    perm = _c(perm, np.int32)
    sc = _c(sc, np.float32)
    n = q.shape[0]
    ng = (n + 15) // 16
    b1 = np.zeros(max(ng * 128, 1), np.uint8)
    b7 = np.zeros(max(ng * 256, 1), np.uint8)
    D = np.zeros((max(ng, 1), MODES), np.uint64)
    lib().or_set_threads(int(threads))
    try:
        lib().or_code_groups(_p(q), n, _p(perm), _p(sc), _p(b1), _p(b7), _p(D))
    finally:
        lib().or_set_threads(1)
    out = []
    for t4 in targets_x4:
        blocks = np.zeros(max(ng * 256, 1), np.uint8)
        perm_out = np.full(max(ng * 16, 1), -1, np.int32)
        t = Table()
        rc = lib().or_rate_assemble(n, _p(perm), _p(sc), int(t4), _p(b1), _p(b7), _p(D), _p(blocks), _p(perm_out),
                                    C.byref(t))
        if rc != 0:
            raise ValueError("or_rate_assemble failed: %d" % rc)
        out.append(dict(blocks=blocks[:t.total_bytes], perm=perm_out[:ng * 16], table=t))
    return out


def decode(table: Table, blocks, perm):
    blocks = _c(blocks, np.uint8)
    perm = _c(perm, np.int32)
    tex = np.zeros((table.n, SH, 3), np.uint8)
    buf = blocks if blocks.size else np.zeros(1, np.uint8)
    lib().or_decode(C.byref(table), _p(buf), _p(perm), _p(tex))
    return tex


# --- splatting renderer (Sec. II, Eqs. sigmoid / covar / opac / preblend) -----------------
class Camera(C.Structure):
    _fields_ = [("R", C.c_float * 9), ("t", C.c_float * 3), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("width", C.c_int32), ("height", C.c_int32),
                ("near_z", C.c_float)]


class Splat(C.Structure):
    _fields_ = [("u", C.c_float), ("v", C.c_float), ("depth", C.c_float), ("a", C.c_float), ("b", C.c_float),
                ("c", C.c_float), ("x0", C.c_int32), ("y0", C.c_int32), ("x1", C.c_int32), ("y1", C.c_int32),
                ("visible", C.c_int32)]


def camera(d):
    cam = Camera()
    cam.R[:] = [float(x) for x in d["R"]]
    cam.t[:] = [float(x) for x in d["t"]]
    cam.fx, cam.fy, cam.cx, cam.cy = float(d["fx"]), float(d["fy"]), float(d["cx"]), float(d["cy"])
    cam.width, cam.height, cam.near_z = int(d["width"]), int(d["height"]), float(d["near_z"])
    return cam


def camera_centre(d):
    f = np.zeros(3, np.float32)
    lib().or_camera_centre(C.byref(camera(d)), _p(f))
    return f


def splat_setup(p, s, q, d):
    sp = Splat()
    lib().or_splat_setup(_p(_c(p, np.float32)), _p(_c(s, np.float32)), _p(_c(q, np.float32)), C.byref(camera(d)),
                         C.byref(sp))
    return sp


def render(pos, scale, rot, logit, colour, cam, tiles=None, want_abs=False):
    """Eq. preblend image [H, W, 3] (float64), final transmittance [H, W] and optionally the sum of
    absolute terms; tiles: tile ids to render (others stay 0)."""
    pos, scale, rot = _c(pos, np.float32), _c(scale, np.float32), _c(rot, np.float32)
    logit, colour = _c(logit, np.float32), _c(colour, np.float64)
    c = camera(cam)
    img = np.zeros((c.height, c.width, 3), np.float64)
    tr = np.zeros((c.height, c.width), np.float64)
    ab = np.zeros((c.height, c.width, 3), np.float64) if want_abs else None
    tl = _c(tiles, np.int32) if tiles is not None else None
    rc = lib().or_render(pos.shape[0], _p(pos), _p(scale), _p(rot), _p(logit), _p(colour), C.byref(c), _p(tl),
                         0 if tl is None else tl.shape[0], _p(img), _p(tr), _p(ab))
    if rc != 0:
        raise ValueError("or_render failed: %d" % rc)
    return (img, tr, ab) if want_abs else (img, tr)


# --- geometry streams and chunk hierarchy (Sec. IV-A) ---------------------------------------
def geometry_encode(pos, scale, rot, logit, perm, chunk_slots=4096):
    """Fixed-rate geometry codes in slot order and the chunk table."""
    pos, scale, rot = _c(pos, np.float32), _c(scale, np.float32), _c(rot, np.float32)
    logit, perm = _c(logit, np.float32), _c(perm, np.int32)
    ns = perm.shape[0]
    nc = lib().or_chunks(ns, chunk_slots)
    chunk = np.zeros((nc, 8), np.float32)
    lib().or_chunk_table(_p(pos), _p(scale), _p(perm), ns, chunk_slots, _p(chunk))
    qpos = np.zeros((ns, 3), np.uint16)
    qscale = np.zeros((ns, 3), np.uint16)
    qrot = np.zeros(ns, np.uint32)
    qlogit = np.zeros(ns, np.uint8)
    lib().or_geometry_encode(_p(pos), _p(scale), _p(rot), _p(logit), _p(perm), ns, chunk_slots, _p(chunk), _p(qpos),
                             _p(qscale), _p(qrot), _p(qlogit))
    return dict(qpos=qpos, qscale=qscale, qrot=qrot, qlogit=qlogit, chunk=chunk, chunk_slots=chunk_slots)


def geometry_decode(g):
    """Decoded (position, scale, quaternion, logit) of every slot, in slot order (float32)."""
    ns = g["qrot"].shape[0]
    P_, S_, Q_, T_ = (np.zeros((ns, 3), np.float32), np.zeros((ns, 3), np.float32), np.zeros((ns, 4), np.float32),
                      np.zeros(ns, np.float32))
    q = [_c(g[k], t) for k, t in (("qpos", np.uint16), ("qscale", np.uint16), ("qrot", np.uint32),
                                   ("qlogit", np.uint8))]
    lib().or_geometry_decode_all(_p(q[0]), _p(q[1]), _p(q[2]), _p(q[3]), ns, g["chunk_slots"],
                                 _p(_c(g["chunk"], np.float32)), _p(P_), _p(S_), _p(Q_), _p(T_))
    return P_, S_, Q_, T_


def chunk_visible(entry, cam):
    return bool(lib().or_chunk_visible(_p(_c(entry, np.float32)), C.byref(camera(cam))))


# --- SH evaluation (Sec. II) --------------------------------------------------------------
def sh_basis(x, y, z):
    Y = np.zeros(SH, np.float64)
    lib().or_sh_basis(x, y, z, _p(Y))
    return Y


def eval_sh(texels, sc, pos=None, dirs=None, cams=None, want_abs=False):
    texels = _c(texels, np.uint8)
    sc = _c(sc, np.float32)
    n = texels.shape[0]
    src = dirs if dirs is not None else cams
    V = src.shape[0]
    out = np.zeros((V, n, 3), np.float64)
    ab = np.zeros((V, n, 3), np.float64) if want_abs else None
    pos_c = _c(pos, np.float32) if pos is not None else None
    lib().or_eval_sh(_p(texels), n, _p(sc), _p(pos_c), _p(_c(dirs, np.float32) if dirs is not None else None),
                     _p(_c(cams, np.float32) if cams is not None else None), V, _p(out), _p(ab))
    return (out, ab) if want_abs else out


def full_encode(pos, sh, fmt, target_x4=0, group_size=4096, sort=1, permille=995):
    """Scales -> quantise -> plan -> encode, the whole encode side of the oracle."""
    sc = scales(sh, permille)
    q = quantise(sh, sc)
    perm = plan(pos, q, group_size, sort)
    res = encode(q, perm, sc, fmt, target_x4)
    res["scales"] = sc
    res["q"] = q
    res["perm_plan"] = perm
    return res
