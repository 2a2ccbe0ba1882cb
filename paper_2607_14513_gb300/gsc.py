"""Thin Python binding of libgsc.so (include/gsc.h): argument marshalling only.

Every step of the codec runs in the CUDA library; PyTorch supplies device memory
and streams. There is no CPU fallback: if the library cannot be loaded, or no
sm_103 GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
import re
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "lib", "libgsc.so")
LIB_CHECKED_PATH = os.path.join(PKG, "lib", "libgsc_checked.so")  # GSC_CHECKED=1 selects it
HEADER = os.path.join(PKG, "..", "include", "gsc.h")

GSC_OK = 0
STATUS = {0: "GSC_OK", 1: "GSC_ERR_INVALID_ARG", 2: "GSC_ERR_CUDA", 3: "GSC_ERR_OOM", 4: "GSC_ERR_BUDGET",
          5: "GSC_ERR_TIMEOUT", 6: "GSC_ERR_UNSUPPORTED", 7: "GSC_ERR_DEVICE", 8: "GSC_ERR_CANCELLED"}
FMT_RATE, FMT_BC1, FMT_MIXED, FMT_BC7 = 0, 1, 2, 7
LAYOUT_D, LAYOUT_A, LAYOUT_B = 0, 1, 2
OUT_VIEW_MAJOR, OUT_SLOT_ORDER, OUT_GAUSS_MAJOR, OUT_SLOT_ROWS = 0, 1, 2, 3


class GscError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__("%s failed: %s (%d)" % (where, STATUS.get(code, "?"), code))


class PlanParams(C.Structure):
    _fields_ = [("n", C.c_int64), ("group_size", C.c_int64), ("sort", C.c_int32), ("quantile_permille", C.c_uint32)]


class EncodeParams(C.Structure):
    _fields_ = [("format", C.c_int32), ("target_bpt_x4", C.c_uint32), ("d_bc1_blocks", C.c_void_p),
                ("d_bc7_blocks", C.c_void_p), ("layout", C.c_int32), ("bc7_blocks", C.c_int32)]


class Stream(C.Structure):
    _fields_ = [("bands", C.c_int32), ("bc7_blocks", C.c_int32), ("first_group", C.c_int64),
                ("n_groups", C.c_int64), ("byte_offset", C.c_int64)]


class StreamTable(C.Structure):
    _fields_ = [("n_streams", C.c_int32), ("format", C.c_int32), ("n", C.c_int64), ("n_groups", C.c_int64),
                ("total_bytes", C.c_int64), ("budget_bits", C.c_uint64), ("used_bits", C.c_uint64),
                ("lambda_", C.c_uint64), ("scales", C.c_float * 16), ("weights", C.c_uint32 * 16),
                ("s", Stream * 14), ("layout", C.c_int32)]

    def streams(self):
        return [dict(bands=self.s[i].bands, bc7_blocks=self.s[i].bc7_blocks, first_group=self.s[i].first_group,
                     n_groups=self.s[i].n_groups, byte_offset=self.s[i].byte_offset) for i in range(self.n_streams)]


class Camera(C.Structure):
    _fields_ = [("R", C.c_float * 9), ("t", C.c_float * 3), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("width", C.c_int32), ("height", C.c_int32),
                ("near_z", C.c_float)]


def camera(d):
    """gsc_camera from a dict with R (9), t (3), fx, fy, cx, cy, width, height, near_z."""
    cam = Camera()
    cam.R[:] = [float(x) for x in d["R"]]
    cam.t[:] = [float(x) for x in d["t"]]
    cam.fx, cam.fy, cam.cx, cam.cy = float(d["fx"]), float(d["fy"]), float(d["cx"]), float(d["cy"])
    cam.width, cam.height, cam.near_z = int(d["width"]), int(d["height"]), float(d["near_z"])
    return cam


class BatchScene(C.Structure):
    _fields_ = [("d_pos", C.c_void_p), ("d_sh", C.c_void_p), ("n", C.c_int64), ("group_size", C.c_int64),
                ("sort", C.c_int32), ("format", C.c_int32), ("target_bpt_x4", C.c_uint32), ("d_perm", C.c_void_p),
                ("d_scales", C.c_void_p), ("d_blocks", C.c_void_p), ("d_perm_out", C.c_void_p),
                ("table", StreamTable)]


class BatchTuning(C.Structure):
    _fields_ = [("schedule", C.c_int32), ("ctas_per_sm", C.c_int32), ("bc1_tile_groups", C.c_int32)]


REQ_ENCODE, REQ_EVAL, REQ_LOAD = 0, 1, 2


class ServerParams(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_uint64), ("n_slots", C.c_int32), ("merge", C.c_int32),
                ("max_views", C.c_int32), ("priority", C.c_int32), ("encode_slots", C.c_int32), ("hold_us", C.c_int64)]


class Request(C.Structure):
    _fields_ = [("kind", C.c_int32), ("scene", C.c_int32), ("pos", C.c_void_p), ("sh", C.c_void_p),
                ("n", C.c_int64), ("format", C.c_int32), ("target_bpt_x4", C.c_uint32), ("group_size", C.c_int64),
                ("sort", C.c_int32), ("V", C.c_int32), ("dirs", C.c_void_p), ("cams", C.c_void_p),
                ("out_order", C.c_int32), ("out", C.c_void_p), ("path", C.c_char_p)]


class RequestResult(C.Structure):
    _fields_ = [("status", C.c_int32), ("kind", C.c_int32), ("scene", C.c_int32), ("merged", C.c_int32),
                ("n", C.c_int64), ("t_submit_ms", C.c_double), ("t_admit_ms", C.c_double), ("t_done_ms", C.c_double)]


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("done", C.c_uint64), ("failed", C.c_uint64), ("merged", C.c_uint64),
                ("evictions", C.c_uint64), ("resident_bytes", C.c_uint64), ("used_bytes", C.c_uint64),
                ("peak_bytes", C.c_uint64), ("queued", C.c_int32), ("resident_versions", C.c_int32)]


class SimRequest(C.Structure):
    _fields_ = [("kind", C.c_int32), ("scene", C.c_int32), ("n", C.c_int64), ("format", C.c_int32),
                ("target_bpt_x4", C.c_uint32), ("V", C.c_int32), ("out_order", C.c_int32), ("cams", C.c_int32),
                ("out_device", C.c_int32), ("host_input", C.c_int32), ("t_arrival_ms", C.c_double),
                ("service_ms", C.c_double)]


class SimResult(C.Structure):
    _fields_ = [("status", C.c_int32), ("merged", C.c_int32), ("evictions", C.c_int32), ("pad", C.c_int32),
                ("t_admit_ms", C.c_double), ("t_done_ms", C.c_double), ("used_bytes_at_admit", C.c_uint64)]


_lib = None
_lock = threading.Lock()

_P = C.c_void_p
_SIGS = {
    "gsc_ctx_create": [C.POINTER(C.c_void_p), C.c_int],
    "gsc_ctx_destroy": [_P],
    "gsc_ctx_sync": [_P, _P],
    "gsc_status_string": [C.c_int],
    "gsc_workspace_bytes": [C.c_int64, C.POINTER(EncodeParams)],
    "gsc_plan_reorder": [_P, _P, _P, C.POINTER(PlanParams), _P, _P, _P, C.c_size_t, _P],
    "gsc_plan_reorder_static": [_P, _P, _P, C.POINTER(PlanParams), _P, _P, _P],
    "gsc_quantise": [_P, _P, C.c_int64, _P, _P, _P],
    "gsc_encode": [_P, _P, C.c_int64, _P, _P, C.POINTER(EncodeParams), _P, _P, C.POINTER(StreamTable), _P,
                   C.c_size_t, _P],
    "gsc_decode": [_P, C.POINTER(StreamTable), _P, _P, _P, _P],
    "gsc_decode_eval_sh": [_P, C.POINTER(StreamTable), _P, _P, _P, _P, _P, C.c_int32, C.c_int32, _P, _P],
    "gsc_decode_eval_sh_slots": [_P, C.POINTER(StreamTable), _P, _P, _P, _P, _P, C.c_int32, C.c_int32, _P, _P],
    "gsc_positions_to_slots": [_P, _P, C.c_int64, _P, C.c_int64, _P, _P],
    "gsc_decode_tex": [_P, C.POINTER(StreamTable), _P, _P, _P, _P],
    "gsc_tex_scene_create": [_P, C.POINTER(StreamTable), _P, _P, _P, C.POINTER(C.c_void_p), _P],
    "gsc_tex_scene_destroy": [_P],
    "gsc_decode_eval_sh_tex": [_P, _P, _P, _P, _P, _P, C.c_int32, C.c_int32, _P, _P],
    "gsc_render_workspace_bytes": [C.c_int64, C.POINTER(Camera), C.c_int64],
    "gsc_geometry_bytes": [C.c_int64, C.c_int64],
    "gsc_geometry_layout": [C.c_int64, C.c_int64, C.POINTER(C.c_size_t)],
    "gsc_forced_table": [C.POINTER(StreamTable), C.c_int32, C.POINTER(StreamTable)],
    "gsc_geometry_encode": [_P, _P, _P, _P, _P, _P, C.c_int64, C.c_int64, _P, _P],
    "gsc_render_coded": [_P, C.POINTER(StreamTable), _P, _P, _P, C.c_int64, C.POINTER(Camera), _P, _P,
                         C.POINTER(C.c_int64), C.POINTER(C.c_int64), _P, C.c_size_t, _P],
    "gsc_render": [_P, C.POINTER(StreamTable), _P, _P, _P, _P, _P, _P, C.POINTER(Camera), _P, _P,
                   C.POINTER(C.c_int64), _P, C.c_size_t, _P],
    "gsc_encode_blocks": [_P, _P, C.c_int64, C.c_int32, _P, _P, _P],
    "gsc_decode_blocks": [_P, _P, C.c_int64, C.c_int32, _P, _P],
    "gsc_decode_blocks_tex": [_P, _P, C.c_int64, C.c_int32, _P, _P],
    "gsc_batch_workspace_bytes": [C.POINTER(BatchScene), C.c_int32],
    "gsc_batch_encode": [_P, C.POINTER(BatchScene), C.c_int32, C.POINTER(BatchTuning), _P, C.c_size_t, _P],
    "gsc_batch_autotune": [_P, C.POINTER(BatchScene), C.c_int32, C.POINTER(BatchTuning), C.POINTER(C.c_double), _P,
                           C.c_size_t, _P],
    "gsc_batch_eval_graph": [_P, C.POINTER(BatchScene), C.c_int32, _P, C.c_int32, C.c_int32, C.POINTER(C.c_void_p),
                             C.POINTER(C.c_void_p), _P],
    "gsc_graph_launch": [_P, _P],
    "gsc_graph_destroy": [_P],
    "gsc_server_create": [_P, C.POINTER(ServerParams), C.POINTER(C.c_void_p)],
    "gsc_server_submit": [_P, C.POINTER(Request), C.POINTER(C.c_uint64)],
    "gsc_server_wait": [_P, C.c_uint64, C.c_int64, C.POINTER(RequestResult)],
    "gsc_server_drain": [_P, C.c_int64],
    "gsc_server_read_scene": [_P, C.c_int32, C.POINTER(StreamTable), _P, C.c_size_t, _P, C.c_size_t],
    "gsc_server_evict": [_P, C.c_int32],
    "gsc_server_save_scene": [_P, C.c_int32, C.c_char_p],
    "gsc_server_cancel": [_P, C.c_uint64],
    "gsc_scene_write": [C.c_char_p, C.POINTER(StreamTable), _P, _P, _P],
    "gsc_scene_read_info": [C.c_char_p, C.POINTER(StreamTable), C.POINTER(C.c_int32)],
    "gsc_scene_read": [C.c_char_p, C.POINTER(StreamTable), _P, C.c_size_t, _P, C.c_size_t, _P, C.c_size_t],
    "gsc_server_get_stats": [_P, C.POINTER(ServerStats)],
    "gsc_server_destroy": [_P],
    "gsc_server_simulate": [C.POINTER(ServerParams), C.POINTER(SimRequest), C.c_int32, C.POINTER(SimResult),
                            C.POINTER(C.c_uint64)],
    "gsc_shard_bounds": [C.c_int64, C.c_int32, C.c_int64, C.POINTER(C.c_int64)],
    "gsc_shard_bbox": [_P, _P, C.c_int64, _P, _P],
    "gsc_shard_morton": [_P, _P, C.c_int64, _P, _P, _P],
    "gsc_shard_order_ws_bytes": [C.c_int64],
    "gsc_shard_order": [_P, _P, C.c_int64, _P, _P, C.c_size_t, _P],
    "gsc_shard_select_state_bytes": [],
    "gsc_shard_select_begin": [_P, C.c_int64, C.c_uint32, _P, _P],
    "gsc_shard_select_hist": [_P, _P, C.c_int64, C.c_int32, _P, _P, _P],
    "gsc_shard_select_pick": [_P, _P, _P, C.c_int32, _P],
    "gsc_shard_select_scales": [_P, _P, _P, _P],
    "gsc_shard_plan_ws_bytes": [C.c_int64],
    "gsc_shard_plan": [_P, _P, C.c_int64, _P, C.c_int64, _P, _P, C.c_size_t, _P],
    "gsc_shard_rate_ws_bytes": [C.c_int64],
    "gsc_shard_rate_begin": [_P, _P, C.c_int64, _P, _P, _P, _P, _P, C.c_size_t, _P, _P],
    "gsc_shard_rate_search_begin": [_P, C.c_int64, _P, C.c_int64, C.c_uint32, _P, _P],
    "gsc_shard_rate_count": [_P, C.c_int64, _P, C.c_int32, _P, _P],
    "gsc_shard_rate_narrow": [_P, C.c_int64, _P, C.c_int32, _P, _P],
    "gsc_shard_rate_fill": [_P, C.c_int64, _P, _P, _P],
    "gsc_shard_rate_apply": [_P, C.c_int64, _P, _P, _P, _P],
    "gsc_shard_rate_assemble": [_P, C.c_int64, _P, _P, _P, _P, _P, _P, _P, C.c_int32, C.c_int32, C.c_int64, _P, _P,
                                C.POINTER(StreamTable), _P],
    "gsc_build_checked": [],
    "gsc_launch_count": [],
    "gsc_probe_int_peak": [_P, C.POINTER(C.c_double), _P],
    "gsc_probe_op_rate": [_P, C.c_int32, C.POINTER(C.c_double), _P],
    "gsc_probe_bc7_mode1": [_P, _P, C.c_int64, C.c_int32, _P, _P, C.POINTER(C.c_double), _P],
    "gsc_ctx_set_timing": [_P, C.c_int],
    "gsc_kernel_time": [_P, C.c_char_p, C.POINTER(C.c_double), C.POINTER(C.c_int64)],
}


def header_symbols():
    """Names of the functions include/gsc.h declares."""
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(gsc_[a-z0-9_]+)\s*\(", txt)))


def load(path: str | None = None):
    """Load libgsc.so (raises if it is missing: there is no fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or (LIB_CHECKED_PATH if os.environ.get("GSC_CHECKED") == "1" else LIB_PATH)
            if not os.path.exists(p):
                raise RuntimeError("libgsc.so not built (%s); run __graft_entry__.build()" % p)
            lib = C.CDLL(p)
            for name, args in _SIGS.items():
                f = getattr(lib, name)
                f.argtypes = args
                f.restype = C.c_int
            lib.gsc_status_string.restype = C.c_char_p
            lib.gsc_workspace_bytes.restype = C.c_size_t
            lib.gsc_launch_count.restype = C.c_uint64
            lib.gsc_batch_workspace_bytes.restype = C.c_size_t
            lib.gsc_render_workspace_bytes.restype = C.c_size_t
            lib.gsc_geometry_bytes.restype = C.c_size_t
            lib.gsc_geometry_layout.restype = C.c_size_t
            for name in ("gsc_shard_order_ws_bytes", "gsc_shard_select_state_bytes", "gsc_shard_plan_ws_bytes",
                         "gsc_shard_rate_ws_bytes"):
                getattr(lib, name).restype = C.c_size_t
            _lib = lib
    return _lib


def _check(code, where):
    if code != GSC_OK:
        raise GscError(code, where)


def _ptr(t):
    if t is None:
        return None
    return C.c_void_p(t.data_ptr())


def _addr(t):
    return None if t is None else t.data_ptr()


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


class Context:
    """A gsc_ctx on one CUDA device."""

    def __init__(self, device: int = 0):
        self.lib = load()
        self.device = device
        h = C.c_void_p()
        _check(self.lib.gsc_ctx_create(C.byref(h), device), "gsc_ctx_create")
        self.h = h

    def close(self):
        if self.h:
            self.lib.gsc_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sync(self, stream=None):
        _check(self.lib.gsc_ctx_sync(self.h, _stream(stream)), "gsc_ctx_sync")

    def workspace(self, n, fmt=FMT_BC1, target_x4=0, layout=LAYOUT_D, bc7_blocks=0):
        import torch
        ep = EncodeParams(fmt, target_x4, None, None, layout, bc7_blocks)
        nb = self.lib.gsc_workspace_bytes(n, C.byref(ep))
        return torch.empty(max(int(nb), 256), dtype=torch.uint8, device="cuda:%d" % self.device)


def gsc_plan_reorder(ctx, pos, sh, group_size=4096, sort=1, permille=995, ws=None, stream=None):
    """-> (perm int32 [n_groups*16], scales float32 [16])."""
    import torch
    n = sh.shape[0]
    dev = sh.device
    ns = (n + 15) // 16 * 16
    perm = torch.empty(max(ns, 1), dtype=torch.int32, device=dev)[:ns]
    scales = torch.empty(16, dtype=torch.float32, device=dev)
    ws = ws if ws is not None else ctx.workspace(n)
    pp = PlanParams(n, group_size, sort, permille)
    _check(ctx.lib.gsc_plan_reorder(ctx.h, _ptr(pos), _ptr(sh), C.byref(pp), _ptr(perm), _ptr(scales), _ptr(ws),
                                    ws.numel(), _stream(stream)), "gsc_plan_reorder")
    return perm, scales


def gsc_quantise(ctx, sh, scales, stream=None):
    import torch
    q = torch.empty(sh.shape, dtype=torch.uint8, device=sh.device)
    _check(ctx.lib.gsc_quantise(ctx.h, _ptr(sh), sh.shape[0], _ptr(scales), _ptr(q), _stream(stream)), "gsc_quantise")
    return q


def gsc_encode(ctx, sh, perm, scales, fmt, target_x4=0, ws=None, out=None, perm_out=None, stream=None,
               bc1_all=None, bc7_all=None, layout=LAYOUT_D, bc7_blocks=0):
    """-> (blocks uint8 [total_bytes], perm_out int32, StreamTable).

    In rate mode, bc1_all / bc7_all (optional uint8 device tensors of n_groups*128 and
    n_groups*256 bytes) receive the all-BC1 and all-BC7 codings of the planned order.
    layout: LAYOUT_D / _A / _B; FMT_MIXED codes bc7_blocks blocks of every group BC7."""
    import torch
    n = sh.shape[0]
    ng = (n + 15) // 16
    dev = sh.device
    blocks = out if out is not None else torch.empty(max(ng * 256, 16), dtype=torch.uint8, device=dev)
    po = perm_out if perm_out is not None else torch.empty(max(ng * 16, 1), dtype=torch.int32, device=dev)
    ws = ws if ws is not None else ctx.workspace(n, fmt, target_x4, layout, bc7_blocks)
    ep = EncodeParams(fmt, target_x4, _ptr(bc1_all), _ptr(bc7_all), layout, bc7_blocks)
    tab = StreamTable()
    _check(ctx.lib.gsc_encode(ctx.h, _ptr(sh), n, _ptr(perm), _ptr(scales), C.byref(ep), _ptr(blocks), _ptr(po),
                              C.byref(tab), _ptr(ws), ws.numel(), _stream(stream)), "gsc_encode")
    return blocks[:tab.total_bytes], po[:ng * 16], tab


def forced_table(table, fmt):
    """Stream table of the all-BC1 / all-BC7 coding that shares `table`'s scene, scales and layout
    (gsc_forced_table)."""
    t = StreamTable()
    _check(load().gsc_forced_table(C.byref(table), fmt, C.byref(t)), "gsc_forced_table")
    return t


def int_peak(ctx, stream=None):
    v = C.c_double(0.0)
    _check(ctx.lib.gsc_probe_int_peak(ctx.h, C.byref(v), _stream(stream)), "gsc_probe_int_peak")
    return v.value


PROBE_KINDS = {1: "iadd3", 2: "lop3", 3: "imad", 4: "dp4a", 5: "bc7_palette_eval"}


def op_rate(ctx, kind, stream=None):
    """Operations per second of one instruction kind (gsc_probe_op_rate; kinds in PROBE_KINDS)."""
    v = C.c_double(0.0)
    _check(ctx.lib.gsc_probe_op_rate(ctx.h, kind, C.byref(v), _stream(stream)), "gsc_probe_op_rate")
    return v.value


def bc7_mode1(ctx, tex, warp_per_block, stream=None):
    """The mode-1 search alone (gsc_probe_bc7_mode1): -> (sse uint32 [n], partition int32 [n], ms)."""
    import torch
    n = tex.shape[0]
    sse = torch.empty(n, dtype=torch.int32, device=tex.device)
    part = torch.empty(n, dtype=torch.int32, device=tex.device)
    ms = C.c_double(0.0)
    _check(ctx.lib.gsc_probe_bc7_mode1(ctx.h, _ptr(tex), n, 1 if warp_per_block else 0, _ptr(sse), _ptr(part),
                                       C.byref(ms), _stream(stream)), "gsc_probe_bc7_mode1")
    return sse, part, ms.value


def set_timing(ctx, enable=True):
    _check(ctx.lib.gsc_ctx_set_timing(ctx.h, 1 if enable else 0), "gsc_ctx_set_timing")


def kernel_time(ctx, name):
    """-> (total ms, launches) of one kernel since timing was enabled."""
    ms, n = C.c_double(0.0), C.c_int64(0)
    _check(ctx.lib.gsc_kernel_time(ctx.h, name.encode(), C.byref(ms), C.byref(n)), "gsc_kernel_time")
    return ms.value, n.value


def launch_count():
    return int(load().gsc_launch_count())


def gsc_decode(ctx, table, blocks, perm, stream=None):
    import torch
    tex = torch.empty((max(table.n, 1), 16, 3), dtype=torch.uint8, device=blocks.device)[:table.n]
    _check(ctx.lib.gsc_decode(ctx.h, C.byref(table), _ptr(blocks), _ptr(perm), _ptr(tex), _stream(stream)),
           "gsc_decode")
    return tex


def gsc_decode_eval_sh(ctx, table, blocks, perm, dirs=None, pos=None, cams=None, out_order=OUT_VIEW_MAJOR,
                       out=None, stream=None):
    import torch
    src = dirs if dirs is not None else cams
    V = src.shape[0]
    n, ns = table.n, table.n_groups * 16
    shape = {OUT_VIEW_MAJOR: (V, n, 3), OUT_SLOT_ORDER: (V, ns, 3), OUT_GAUSS_MAJOR: (n, V, 3),
             OUT_SLOT_ROWS: (ns, V, 3)}[out_order]
    rgb = out if out is not None else torch.empty(shape, dtype=torch.float32, device=blocks.device)
    _check(ctx.lib.gsc_decode_eval_sh(ctx.h, C.byref(table), _ptr(blocks), _ptr(perm), _ptr(dirs), _ptr(pos),
                                      _ptr(cams), V, out_order, _ptr(rgb), _stream(stream)), "gsc_decode_eval_sh")
    return rgb


def gsc_decode_eval_sh_slots(ctx, table, blocks, perm, dirs=None, pos_slot=None, cams=None,
                             out_order=OUT_VIEW_MAJOR, out=None, stream=None):
    """gsc_decode_eval_sh with centres in slot order (pos_slot [n_groups * 16, 3])."""
    import torch
    src = dirs if dirs is not None else cams
    V = src.shape[0]
    n, ns = table.n, table.n_groups * 16
    shape = {OUT_VIEW_MAJOR: (V, n, 3), OUT_SLOT_ORDER: (V, ns, 3), OUT_GAUSS_MAJOR: (n, V, 3),
             OUT_SLOT_ROWS: (ns, V, 3)}[out_order]
    rgb = out if out is not None else torch.empty(shape, dtype=torch.float32, device=blocks.device)
    _check(ctx.lib.gsc_decode_eval_sh_slots(ctx.h, C.byref(table), _ptr(blocks), _ptr(perm), _ptr(dirs),
                                            _ptr(pos_slot), _ptr(cams), V, out_order, _ptr(rgb), _stream(stream)),
           "gsc_decode_eval_sh_slots")
    return rgb


def gsc_positions_to_slots(ctx, pos, perm, out=None, stream=None):
    """Centres in slot order: out[s] = pos[perm[s]] (zeros for padding slots)."""
    import torch
    n, ns = pos.shape[0], perm.shape[0]
    res = out if out is not None else torch.empty((ns, 3), dtype=torch.float32, device=pos.device)
    _check(ctx.lib.gsc_positions_to_slots(ctx.h, _ptr(pos), n, _ptr(perm), ns, _ptr(res), _stream(stream)),
           "gsc_positions_to_slots")
    return res


def gsc_decode_tex(ctx, table, blocks, perm, stream=None):
    import torch
    tex = torch.zeros((max(table.n, 1), 16, 3), dtype=torch.uint8, device=blocks.device)[:table.n]
    _check(ctx.lib.gsc_decode_tex(ctx.h, C.byref(table), _ptr(blocks), _ptr(perm), _ptr(tex), _stream(stream)),
           "gsc_decode_tex")
    return tex


class TexScene:
    """A coded scene resident as BC1/BC7 texture objects (gsc_tex_scene)."""

    def __init__(self, ctx, table, blocks, perm=None, pos=None, stream=None):
        self.ctx = ctx
        self.table = table
        h = C.c_void_p()
        _check(ctx.lib.gsc_tex_scene_create(ctx.h, C.byref(table), _ptr(blocks), _ptr(perm), _ptr(pos), C.byref(h),
                                            _stream(stream)), "gsc_tex_scene_create")
        self.h = h

    def close(self):
        if self.h:
            self.ctx.lib.gsc_tex_scene_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gsc_decode_eval_sh_tex(ctx, scene, perm, dirs=None, pos=None, cams=None, out_order=OUT_VIEW_MAJOR, out=None,
                           stream=None):
    import torch
    src = dirs if dirs is not None else cams
    V = src.shape[0]
    table = scene.table
    n, ns = table.n, table.n_groups * 16
    shape = {OUT_VIEW_MAJOR: (V, n, 3), OUT_SLOT_ORDER: (V, ns, 3), OUT_GAUSS_MAJOR: (n, V, 3),
             OUT_SLOT_ROWS: (ns, V, 3)}[out_order]
    rgb = out if out is not None else torch.empty(shape, dtype=torch.float32, device=perm.device)
    _check(ctx.lib.gsc_decode_eval_sh_tex(ctx.h, scene.h, _ptr(perm), _ptr(dirs), _ptr(pos), _ptr(cams), V,
                                          out_order, _ptr(rgb), _stream(stream)), "gsc_decode_eval_sh_tex")
    return rgb


def geometry_layout(n_slots, chunk_slots):
    """Byte offsets of (qpos, qscale, qrot, qlogit, chunks) in a geometry buffer and its size
    (gsc_geometry_layout)."""
    off = (C.c_size_t * 5)()
    size = load().gsc_geometry_layout(n_slots, chunk_slots, off)
    if size == 0:
        raise GscError(1, "gsc_geometry_layout")  # GSC_ERR_INVALID_ARG
    return list(off), int(size)


def gsc_geometry_encode(ctx, pos, scale, rot, logit, perm, chunk_slots=4096, out=None, stream=None):
    """-> uint8 device buffer with the geometry streams of the planned slot order `perm`."""
    import torch
    ns = perm.shape[0]
    nb = ctx.lib.gsc_geometry_bytes(ns, chunk_slots)
    geom = out if out is not None else torch.empty(max(nb, 256), dtype=torch.uint8, device=perm.device)
    _check(ctx.lib.gsc_geometry_encode(ctx.h, _ptr(pos), _ptr(scale), _ptr(rot), _ptr(logit), _ptr(perm), ns,
                                       chunk_slots, _ptr(geom), _stream(stream)), "gsc_geometry_encode")
    return geom


class Renderer:
    """gsc_render with a workspace that grows to the (Gaussian, tile) overlap count it needs."""

    def __init__(self, ctx):
        self.ctx = ctx
        self.ws = None

    def render(self, table, blocks, perm, pos, scale, rot, logit, cam, image=None, trans=None, stream=None):
        """-> (image float32 [H, W, 3], transmittance [H, W] or None, overlap count)."""
        import torch
        c = camera(cam)
        dev = perm.device
        img = image if image is not None else torch.empty((c.height, c.width, 3), dtype=torch.float32, device=dev)
        pairs = C.c_int64(0)
        n = table.n
        for _ in range(2):
            if self.ws is None:
                nb = self.ctx.lib.gsc_render_workspace_bytes(n, C.byref(c), max(16 * n, 1 << 16))
                self.ws = torch.empty(nb, dtype=torch.uint8, device=dev)
            code = self.ctx.lib.gsc_render(self.ctx.h, C.byref(table), _ptr(blocks), _ptr(perm), _ptr(pos),
                                           _ptr(scale), _ptr(rot), _ptr(logit), C.byref(c), _ptr(img), _ptr(trans),
                                           C.byref(pairs), _ptr(self.ws), self.ws.numel(), _stream(stream))
            if code == 3 and pairs.value > 0:        # GSC_ERR_OOM: grow to the overlap count, once
                nb = self.ctx.lib.gsc_render_workspace_bytes(n, C.byref(c), int(pairs.value * 5 // 4))
                self.ws = torch.empty(nb, dtype=torch.uint8, device=dev)
                continue
            _check(code, "gsc_render")
            return img, trans, pairs.value
        raise GscError(3, "gsc_render")

    def render_coded(self, table, blocks, perm, geom, chunk_slots, cam, image=None, trans=None, stream=None):
        """gsc_render_coded -> (image, transmittance or None, overlap count, kept chunks)."""
        import torch
        c = camera(cam)
        dev = perm.device
        img = image if image is not None else torch.empty((c.height, c.width, 3), dtype=torch.float32, device=dev)
        pairs, chunks = C.c_int64(0), C.c_int64(0)
        n = table.n
        for _ in range(2):
            if self.ws is None:
                nb = self.ctx.lib.gsc_render_workspace_bytes(n, C.byref(c), max(16 * n, 1 << 16))
                self.ws = torch.empty(nb, dtype=torch.uint8, device=dev)
            code = self.ctx.lib.gsc_render_coded(self.ctx.h, C.byref(table), _ptr(blocks), _ptr(perm), _ptr(geom),
                                                 chunk_slots, C.byref(c), _ptr(img), _ptr(trans), C.byref(pairs),
                                                 C.byref(chunks), _ptr(self.ws), self.ws.numel(), _stream(stream))
            if code == 3 and pairs.value > 0:
                nb = self.ctx.lib.gsc_render_workspace_bytes(n, C.byref(c), int(pairs.value * 5 // 4))
                self.ws = torch.empty(nb, dtype=torch.uint8, device=dev)
                continue
            _check(code, "gsc_render_coded")
            return img, trans, pairs.value, chunks.value
        raise GscError(3, "gsc_render_coded")


def gsc_encode_blocks(ctx, tex, fmt, stream=None):
    """tex uint8 [nblk, 16, 3] -> (blocks [nblk, 8|16], sse uint64 [nblk])."""
    import torch
    nb = tex.shape[0]
    bpb = 16 if fmt == FMT_BC7 else 8
    out = torch.empty((max(nb, 1), bpb), dtype=torch.uint8, device=tex.device)[:nb]
    sse = torch.empty(max(nb, 1), dtype=torch.int64, device=tex.device)[:nb]
    _check(ctx.lib.gsc_encode_blocks(ctx.h, _ptr(tex.contiguous()), nb, fmt, _ptr(out), _ptr(sse), _stream(stream)),
           "gsc_encode_blocks")
    return out, sse


def gsc_decode_blocks(ctx, blocks, fmt, stream=None):
    import torch
    nb = blocks.shape[0]
    rgba = torch.empty((max(nb, 1), 16, 4), dtype=torch.uint8, device=blocks.device)[:nb]
    _check(ctx.lib.gsc_decode_blocks(ctx.h, _ptr(blocks.contiguous()), nb, fmt, _ptr(rgba), _stream(stream)),
           "gsc_decode_blocks")
    return rgba


def gsc_decode_blocks_tex(ctx, blocks, fmt, stream=None):
    import torch
    nb = blocks.shape[0]
    rgba = torch.empty((max(nb, 1), 16, 4), dtype=torch.uint8, device=blocks.device)[:nb]
    _check(ctx.lib.gsc_decode_blocks_tex(ctx.h, _ptr(blocks.contiguous()), nb, fmt, _ptr(rgba), _stream(stream)),
           "gsc_decode_blocks_tex")
    return rgba


class Batch:
    """Many scenes coded through one persistent launch (gsc_batch_*). Holds the device
    buffers of every scene; `scenes` are (pos, sh, format, target_x4) device tensors."""

    def __init__(self, ctx, scenes, group_size=4096, sort=1):
        import torch
        self.ctx = ctx
        n = len(scenes)
        self.arr = (BatchScene * n)()
        self.keep = []
        for i, (pos, sh, fmt, t4) in enumerate(scenes):
            m = sh.shape[0]
            ng = (m + 15) // 16
            perm = torch.empty(max(ng * 16, 1), dtype=torch.int32, device=sh.device)
            scales = torch.empty(16, dtype=torch.float32, device=sh.device)
            blocks = torch.empty(max(ng * 256, 16), dtype=torch.uint8, device=sh.device)
            perm_out = torch.empty(max(ng * 16, 1), dtype=torch.int32, device=sh.device)
            self.keep.append((pos, sh, perm, scales, blocks, perm_out))
            self.arr[i] = BatchScene(_ptr(pos), _ptr(sh), m, group_size, sort, fmt, t4, _ptr(perm), _ptr(scales),
                                     _ptr(blocks), _ptr(perm_out), StreamTable())
        nb = ctx.lib.gsc_batch_workspace_bytes(self.arr, n)
        if nb == 0:
            raise GscError(1, "gsc_batch_workspace_bytes")
        self.ws = torch.empty(int(nb), dtype=torch.uint8, device="cuda:%d" % ctx.device)
        self.n = n

    def autotune(self, stream=None):
        t = BatchTuning()
        ms = C.c_double(0.0)
        _check(self.ctx.lib.gsc_batch_autotune(self.ctx.h, self.arr, self.n, C.byref(t), C.byref(ms), _ptr(self.ws),
                                               self.ws.numel(), _stream(stream)), "gsc_batch_autotune")
        return t, ms.value

    def encode(self, tuning, stream=None):
        _check(self.ctx.lib.gsc_batch_encode(self.ctx.h, self.arr, self.n, C.byref(tuning), _ptr(self.ws),
                                             self.ws.numel(), _stream(stream)), "gsc_batch_encode")

    def result(self, i):
        """(perm, scales, blocks, perm_out, table) of scene i."""
        pos, sh, perm, scales, blocks, perm_out = self.keep[i]
        t = self.arr[i].table
        return perm, scales, blocks[:t.total_bytes], perm_out[:t.n_groups * 16], t

    def eval_graph(self, cams, outs, out_order=OUT_GAUSS_MAJOR, stream=None):
        ptrs = (C.c_void_p * self.n)(*[o.data_ptr() for o in outs])
        g = C.c_void_p()
        _check(self.ctx.lib.gsc_batch_eval_graph(self.ctx.h, self.arr, self.n, _ptr(cams), cams.shape[0], out_order,
                                                 ptrs, C.byref(g), _stream(stream)), "gsc_batch_eval_graph")
        return Graph(self.ctx, g)


class Graph:
    def __init__(self, ctx, h):
        self.ctx = ctx
        self.h = h

    def launch(self, stream=None):
        _check(self.ctx.lib.gsc_graph_launch(self.h, _stream(stream)), "gsc_graph_launch")

    def close(self):
        if self.h:
            self.ctx.lib.gsc_graph_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def simulate(params, reqs):
    """Runs the request loop's admission policy on the host over a trace of SimRequest."""
    lib = load()
    n = len(reqs)
    arr = (SimRequest * max(n, 1))(*reqs)
    res = (SimResult * max(n, 1))()
    peak = C.c_uint64(0)
    _check(lib.gsc_server_simulate(C.byref(params), arr, n, res, C.byref(peak)), "gsc_server_simulate")
    return list(res)[:n], peak.value


class Server:
    """The request loop (gsc_server_*). Tensors passed to submit() must stay alive until the
    request completes; the object keeps a reference to them until wait() returns."""

    def __init__(self, ctx, budget_bytes, n_slots=4, merge=True, max_views=64, priority=True, hold_us=200_000,
                 encode_slots=0):
        self.ctx = ctx
        self.lib = ctx.lib
        self.params = ServerParams(int(budget_bytes), n_slots, int(merge), max_views, int(priority), encode_slots,
                                   hold_us)
        h = C.c_void_p()
        _check(self.lib.gsc_server_create(ctx.h, C.byref(self.params), C.byref(h)), "gsc_server_create")
        self.h = h
        self.keep = {}

    def encode(self, scene, pos, sh, fmt, target_x4=0, group_size=4096, sort=1):
        r = Request(REQ_ENCODE, scene, _addr(pos), _addr(sh), sh.shape[0], fmt, target_x4, group_size, sort, 0,
                    None, None, 0, None)
        return self._submit(r, (pos, sh))

    def load(self, scene, path, n):
        """Install a checkpoint file (written with positions) as the scene's next version."""
        r = Request(REQ_LOAD, scene, None, None, n, 0, 0, 0, 0, 0, None, None, 0, None, os.fsencode(path))
        return self._submit(r, ())

    def save(self, scene, path):
        _check(self.lib.gsc_server_save_scene(self.h, scene, os.fsencode(path)), "gsc_server_save_scene")

    def eval(self, scene, n, out, dirs=None, cams=None, out_order=OUT_GAUSS_MAJOR):
        src = dirs if dirs is not None else cams
        r = Request(REQ_EVAL, scene, None, None, n, 0, 0, 0, 0, src.shape[0], _addr(dirs), _addr(cams), out_order,
                    _addr(out))
        return self._submit(r, (src, out))

    def _submit(self, r, refs):
        t = C.c_uint64(0)
        _check(self.lib.gsc_server_submit(self.h, C.byref(r), C.byref(t)), "gsc_server_submit")
        self.keep[t.value] = refs
        return t.value

    def wait(self, ticket, timeout_ms=-1):
        res = RequestResult()
        _check(self.lib.gsc_server_wait(self.h, ticket, timeout_ms, C.byref(res)), "gsc_server_wait")
        self.keep.pop(ticket, None)
        return res

    def cancel(self, ticket):
        _check(self.lib.gsc_server_cancel(self.h, ticket), "gsc_server_cancel")

    def drain(self, timeout_ms=-1):
        _check(self.lib.gsc_server_drain(self.h, timeout_ms), "gsc_server_drain")

    def read_scene(self, scene):
        """(table, blocks uint8, perm int32) of a resident scene, as host tensors."""
        import torch
        t = StreamTable()
        _check(self.lib.gsc_server_read_scene(self.h, scene, C.byref(t), None, 0, None, 0), "gsc_server_read_scene")
        blocks = torch.empty(max(t.total_bytes, 1), dtype=torch.uint8)
        perm = torch.empty(max(t.n_groups * 16, 1), dtype=torch.int32)
        _check(self.lib.gsc_server_read_scene(self.h, scene, C.byref(t), _ptr(blocks), blocks.numel(), _ptr(perm),
                                              4 * perm.numel()), "gsc_server_read_scene")
        return t, blocks[:t.total_bytes], perm[:t.n_groups * 16]

    def evict(self, scene):
        _check(self.lib.gsc_server_evict(self.h, scene), "gsc_server_evict")

    def stats(self):
        st = ServerStats()
        _check(self.lib.gsc_server_get_stats(self.h, C.byref(st)), "gsc_server_get_stats")
        return st

    def close(self):
        if self.h:
            self.lib.gsc_server_destroy(self.h)
            self.h = None
            self.keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def scene_write(path, table, blocks, perm, pos=None):
    """Checkpoint file of a coded scene (host or device tensors)."""
    _check(load().gsc_scene_write(os.fsencode(path), C.byref(table), _ptr(blocks), _ptr(perm), _ptr(pos)),
           "gsc_scene_write")


def scene_read(path, device=None):
    """(table, blocks, perm, pos or None) read back from a checkpoint file, as tensors on `device`
    (host when None)."""
    import torch
    lib = load()
    t = StreamTable()
    has = C.c_int32(0)
    _check(lib.gsc_scene_read_info(os.fsencode(path), C.byref(t), C.byref(has)), "gsc_scene_read_info")
    dev = device if device is not None else "cpu"
    blocks = torch.empty(max(t.total_bytes, 1), dtype=torch.uint8, device=dev)
    perm = torch.empty(max(t.n_groups * 16, 1), dtype=torch.int32, device=dev)
    pos = torch.empty((max(t.n, 1), 3), dtype=torch.float32, device=dev) if has.value else None
    _check(lib.gsc_scene_read(os.fsencode(path), C.byref(t), _ptr(blocks), blocks.numel(), _ptr(perm),
                              4 * perm.numel(), _ptr(pos), 0 if pos is None else 4 * pos.numel()), "gsc_scene_read")
    return t, blocks[:t.total_bytes], perm[:t.n_groups * 16], (pos[:t.n] if pos is not None else None)


# ---- one scene split over shards (argument marshalling only; the driver is shard.py) ---------
SHARD_SELECT_PASSES = 4
SHARD_RATE_PASSES = 13
SHARD_RATE_PART = 15


def shard_bounds(n_total, n_shards, group_size):
    b = (C.c_int64 * (n_shards + 1))()
    _check(load().gsc_shard_bounds(n_total, n_shards, group_size, b), "gsc_shard_bounds")
    return [int(x) for x in b]


def _i64(n, device):
    import torch
    return torch.zeros(n, dtype=torch.int64, device=device)


def gsc_shard_bbox(ctx, pos, stream=None):
    bb = _i64(6, pos.device)
    _check(ctx.lib.gsc_shard_bbox(ctx.h, _ptr(pos), pos.shape[0], _ptr(bb), _stream(stream)), "gsc_shard_bbox")
    return bb


def gsc_shard_morton(ctx, pos, bb, stream=None):
    import torch
    keys = torch.empty(pos.shape[0], dtype=torch.int64, device=pos.device)
    _check(ctx.lib.gsc_shard_morton(ctx.h, _ptr(pos), pos.shape[0], _ptr(bb), _ptr(keys), _stream(stream)),
           "gsc_shard_morton")
    return keys


def gsc_shard_order(ctx, keys, stream=None):
    """Input indices in spatial order; `keys` (all shards' Morton codes in input order) is clobbered."""
    import torch
    n = keys.shape[0]
    order = torch.empty(n, dtype=torch.int32, device=keys.device)
    wsb = ctx.lib.gsc_shard_order_ws_bytes(n)
    ws = torch.empty(max(wsb, 256), dtype=torch.uint8, device=keys.device)
    _check(ctx.lib.gsc_shard_order(ctx.h, _ptr(keys), n, _ptr(order), _ptr(ws), wsb, _stream(stream)),
           "gsc_shard_order")
    return order


def shard_select_state(ctx, device):
    import torch
    return torch.zeros(ctx.lib.gsc_shard_select_state_bytes(), dtype=torch.uint8, device=device)


def gsc_shard_select_begin(ctx, n_total, permille, state, stream=None):
    _check(ctx.lib.gsc_shard_select_begin(ctx.h, n_total, permille, _ptr(state), _stream(stream)),
           "gsc_shard_select_begin")


def gsc_shard_select_hist(ctx, sh, p, state, stream=None):
    hist = _i64(16 * 256, state.device)
    _check(ctx.lib.gsc_shard_select_hist(ctx.h, _ptr(sh), sh.shape[0], p, _ptr(state), _ptr(hist), _stream(stream)),
           "gsc_shard_select_hist")
    return hist


def gsc_shard_select_pick(ctx, state, hist, p, stream=None):
    _check(ctx.lib.gsc_shard_select_pick(ctx.h, _ptr(state), _ptr(hist), p, _stream(stream)), "gsc_shard_select_pick")


def gsc_shard_select_scales(ctx, state, stream=None):
    import torch
    scales = torch.empty(16, dtype=torch.float32, device=state.device)
    _check(ctx.lib.gsc_shard_select_scales(ctx.h, _ptr(state), _ptr(scales), _stream(stream)),
           "gsc_shard_select_scales")
    return scales


def gsc_shard_plan(ctx, sh, scales, group_size, stream=None):
    import torch
    n = sh.shape[0]
    perm = torch.empty((n + 15) // 16 * 16, dtype=torch.int32, device=sh.device)
    wsb = ctx.lib.gsc_shard_plan_ws_bytes(n)
    ws = torch.empty(max(wsb, 256), dtype=torch.uint8, device=sh.device)
    _check(ctx.lib.gsc_shard_plan(ctx.h, _ptr(sh), n, _ptr(scales), group_size, _ptr(perm), _ptr(ws), wsb,
                                  _stream(stream)), "gsc_shard_plan")
    return perm


class ShardRate:
    """One shard's rate-control state (workspace and its BC1 / BC7 codings) across the phases."""

    def __init__(self, ctx, n, device):
        import torch
        self.ctx, self.n = ctx, n
        ng = (n + 15) // 16
        self.wsb = ctx.lib.gsc_shard_rate_ws_bytes(n)
        self.ws = torch.empty(self.wsb, dtype=torch.uint8, device=device)
        self.bc1 = torch.empty(max(ng * 128, 16), dtype=torch.uint8, device=device)
        self.bc7 = torch.empty(max(ng * 256, 16), dtype=torch.uint8, device=device)
        self.device = device

    def begin(self, sh, perm, scales, stream=None):
        part = _i64(1, self.device)
        _check(self.ctx.lib.gsc_shard_rate_begin(self.ctx.h, _ptr(sh), self.n, _ptr(perm), _ptr(scales),
                                                 _ptr(self.bc1), _ptr(self.bc7), _ptr(self.ws), self.wsb, _ptr(part),
                                                 _stream(stream)), "gsc_shard_rate_begin")
        return part

    def search_begin(self, n_total, target_x4, min_total, stream=None):
        _check(self.ctx.lib.gsc_shard_rate_search_begin(self.ctx.h, self.n, _ptr(self.ws), n_total, target_x4,
                                                        _ptr(min_total), _stream(stream)), "gsc_shard_rate_search_begin")

    def count(self, p, stream=None):
        part = _i64(64, self.device)
        _check(self.ctx.lib.gsc_shard_rate_count(self.ctx.h, self.n, _ptr(self.ws), p, _ptr(part), _stream(stream)),
               "gsc_shard_rate_count")
        return part

    def narrow(self, p, total, stream=None):
        _check(self.ctx.lib.gsc_shard_rate_narrow(self.ctx.h, self.n, _ptr(self.ws), p, _ptr(total), _stream(stream)),
               "gsc_shard_rate_narrow")

    def fill(self, stream=None):
        part = _i64(2, self.device)
        _check(self.ctx.lib.gsc_shard_rate_fill(self.ctx.h, self.n, _ptr(self.ws), _ptr(part), _stream(stream)),
               "gsc_shard_rate_fill")
        return part

    def apply(self, inp, stream=None):
        part = _i64(SHARD_RATE_PART, self.device)
        _check(self.ctx.lib.gsc_shard_rate_apply(self.ctx.h, self.n, _ptr(self.ws), _ptr(inp), _ptr(part),
                                                 _stream(stream)), "gsc_shard_rate_apply")
        return part

    def assemble(self, perm, index_map, scales, parts_all, shard, n_total, blocks, perm_out, stream=None):
        t = StreamTable()
        _check(self.ctx.lib.gsc_shard_rate_assemble(self.ctx.h, self.n, _ptr(self.ws), _ptr(self.bc1), _ptr(self.bc7),
                                                    _ptr(perm), _ptr(index_map), _ptr(scales), _ptr(parts_all),
                                                    parts_all.shape[0], shard, n_total, _ptr(blocks), _ptr(perm_out),
                                                    C.byref(t), _stream(stream)), "gsc_shard_rate_assemble")
        return t
