"""The C ABI library loads and exports every entry point include/gsc.h declares
(no GPU needed: nothing is called that touches a device)."""
import ctypes
import os

import pytest


def test_header_declares_the_boundary():
    from paper_2607_14513_gb300 import gsc
    names = gsc.header_symbols()
    for required in ["gsc_plan_reorder", "gsc_encode", "gsc_decode", "gsc_decode_eval_sh", "gsc_ctx_create",
                     "gsc_workspace_bytes", "gsc_decode_tex"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2607_14513_gb300 import build as B
    from paper_2607_14513_gb300 import gsc
    B.build()
    lib = ctypes.CDLL(gsc.LIB_PATH)
    for name in gsc.header_symbols():
        assert hasattr(lib, name), name
    # the binding knows the same set
    assert set(gsc.header_symbols()) == set(gsc._SIGS)


def test_no_gpu_is_reported_not_faked():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2607_14513_gb300 import gsc
    with pytest.raises(gsc.GscError) as e:
        gsc.Context(0)
    assert e.value.code == 6          # GSC_ERR_UNSUPPORTED


def test_host_side_sizes_and_strings():
    from paper_2607_14513_gb300 import gsc
    lib = gsc.load()
    ep = gsc.EncodeParams(gsc.FMT_RATE, 16)
    assert lib.gsc_workspace_bytes(3_000_000, ctypes.byref(ep)) > 3_000_000 * 16
    assert lib.gsc_workspace_bytes(-1, ctypes.byref(ep)) == 0
    assert lib.gsc_status_string(4) == b"rate target below the cheapest coding of the scene"


def test_struct_layouts_match_the_header(tmp_path):
    # every ctypes structure of the binding against the C compiler's view of include/gsc.h: the
    # size and the offset of every field
    import shutil
    import subprocess
    from paper_2607_14513_gb300 import gsc
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    pairs = [(gsc.PlanParams, "gsc_plan_params"), (gsc.EncodeParams, "gsc_encode_params"),
             (gsc.Stream, "gsc_stream"), (gsc.StreamTable, "gsc_stream_table"), (gsc.Camera, "gsc_camera"),
             (gsc.BatchScene, "gsc_batch_scene"), (gsc.BatchTuning, "gsc_batch_tuning"),
             (gsc.ServerParams, "gsc_server_params"), (gsc.Request, "gsc_request"),
             (gsc.RequestResult, "gsc_request_result"), (gsc.ServerStats, "gsc_server_stats"),
             (gsc.SimRequest, "gsc_sim_request"), (gsc.SimResult, "gsc_sim_result")]
    rename = {"lambda_": "lambda"}
    lines, want = [], []
    for py, c in pairs:
        lines.append('  printf("%%zu\\n", sizeof(%s));' % c)
        want.append(ctypes.sizeof(py))
        for name, _ in py._fields_:
            lines.append('  printf("%%zu\\n", offsetof(%s, %s));' % (c, rename.get(name, name)))
            want.append(getattr(py, name).offset)
    # the chunk table entry is read as eight floats per chunk (box low, box high, largest scale, pad)
    lines.append('  printf("%zu\\n", sizeof(gsc_chunk));')
    want.append(32)
    src = tmp_path / "abi.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "gsc.h"\nint main(void) {\n'
                   + "\n".join(lines) + "\n  return 0;\n}\n")
    exe = tmp_path / "abi"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.check_call([cc, "-I", inc, str(src), "-o", str(exe)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    assert got == want


def test_layout_workspace_sizes():
    from paper_2607_14513_gb300 import gsc
    lib = gsc.load()
    n = 1_000_000
    ng = (n + 15) // 16
    # layout B with BC7 on the first block of every quad stages 48 B texels per block and the two
    # coded arrays before the interleave
    ep = gsc.EncodeParams(gsc.FMT_MIXED, 0, None, None, gsc.LAYOUT_B, 4)
    assert lib.gsc_workspace_bytes(n, ctypes.byref(ep)) >= ng * 16 * 48 + ng * (4 * 16 + 12 * 8)
    ep = gsc.EncodeParams(gsc.FMT_BC7, 0, None, None, gsc.LAYOUT_A, 0)
    assert lib.gsc_workspace_bytes(n, ctypes.byref(ep)) >= ng * 16 * 48


def test_constants_match_the_header(tmp_path):
    # the binding's enum values against the header's, through the C compiler
    import shutil
    import subprocess
    from paper_2607_14513_gb300 import gsc
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    names = {"GSC_FMT_RATE": gsc.FMT_RATE, "GSC_FMT_BC1": gsc.FMT_BC1, "GSC_FMT_MIXED": gsc.FMT_MIXED,
             "GSC_FMT_BC7": gsc.FMT_BC7, "GSC_LAYOUT_D": gsc.LAYOUT_D, "GSC_LAYOUT_A": gsc.LAYOUT_A,
             "GSC_LAYOUT_B": gsc.LAYOUT_B, "GSC_OUT_VIEW_MAJOR": gsc.OUT_VIEW_MAJOR,
             "GSC_OUT_SLOT_ORDER": gsc.OUT_SLOT_ORDER, "GSC_OUT_GAUSS_MAJOR": gsc.OUT_GAUSS_MAJOR,
             "GSC_REQ_ENCODE": gsc.REQ_ENCODE, "GSC_REQ_EVAL": gsc.REQ_EVAL, "GSC_REQ_LOAD": gsc.REQ_LOAD}
    names.update({v: k for k, v in gsc.STATUS.items()})
    src = tmp_path / "enums.c"
    src.write_text('#include <stdio.h>\n#include "gsc.h"\nint main(void) {\n'
                   + "\n".join('  printf("%%d\\n", (int)%s);' % k for k in names) + "\n  return 0;\n}\n")
    exe = tmp_path / "enums"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.check_call([cc, "-I", inc, str(src), "-o", str(exe)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    assert got == list(names.values())


def _prototypes():
    """(name, return type, [parameter type]) of every function include/gsc.h declares."""
    import re
    from paper_2607_14513_gb300 import gsc
    txt = re.sub(r"/\*.*?\*/", "", open(gsc.HEADER).read(), flags=re.S)
    txt = re.sub(r"#[^\n]*", "", txt)
    out = []
    for m in re.finditer(r"([A-Za-z_][A-Za-z0-9_ ]*[ *]+)\b(gsc_[a-z0-9_]+)\s*\(([^()]*)\)\s*;", txt):
        ret = m.group(1).strip()
        ret = ret.split(";")[-1].split("}")[-1].strip()
        params = [p.strip() for p in m.group(3).split(",") if p.strip()]
        if params == ["void"]:
            params = []
        types = []
        for p in params:
            t = re.sub(r"\b[A-Za-z_][A-Za-z0-9_]*\s*$", "", p).strip()   # drop the parameter's name
            types.append(t if t else p)
        out.append((m.group(2), ret, types))
    return out


def test_binding_argument_widths_match_the_prototypes(tmp_path):
    # every argument's size as ctypes passes it against the C type's size (a 32/64-bit mismatch
    # shifts the arguments after it once they go on the stack), the argument counts, and the size of
    # the return value the binding reads
    import shutil
    import subprocess
    from paper_2607_14513_gb300 import gsc
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    protos = _prototypes()
    assert {n for n, _, _ in protos} == set(gsc._SIGS)
    lib = gsc.load()
    lines, want, where = [], [], []
    for name, ret, types in protos:
        assert len(types) == len(gsc._SIGS[name]), name
        lines.append('  printf("%%zu\\n", sizeof(%s));' % ret)
        want.append(ctypes.sizeof(getattr(lib, name).restype))
        where.append((name, "return", ret))
        for i, (t, a) in enumerate(zip(types, gsc._SIGS[name])):
            lines.append('  printf("%%zu\\n", sizeof(%s));' % t)
            want.append(ctypes.sizeof(a))
            where.append((name, i, t))
    src = tmp_path / "args.c"
    src.write_text('#include <stdio.h>\n#include "gsc.h"\nint main(void) {\n' + "\n".join(lines)
                   + "\n  return 0;\n}\n")
    exe = tmp_path / "args"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.check_call([cc, "-I", inc, str(src), "-o", str(exe)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    bad = [w for w, g, e in zip(where, got, want) if g != e]
    assert not bad, bad


def test_host_size_queries():
    # pure host functions: the geometry buffer size equals the binding's offsets, the render
    # workspace grows with the scene and the overlap count, and invalid arguments give 0
    from paper_2607_14513_gb300 import gsc
    from paper_2607_14513_gb300 import synthetic as S
    lib = gsc.load()
    # the geometry buffer as the header lays it out: five sections (6, 6, 4 and 1 bytes per slot,
    # 32 bytes per chunk), each starting 256-byte aligned
    al = lambda v: (v + 255) // 256 * 256
    for ns in (0, 16, 4096, 4112, 3_000_016):
        for cs in (16, 128, 4096):
            nc = (ns + cs - 1) // cs
            want, b = [], 0
            for size in (6 * ns, 6 * ns, 4 * ns, ns, 32 * max(nc, 1)):
                want.append(b)
                b = al(b + size)
            off, size = gsc.geometry_layout(ns, cs)
            assert (off, size) == (want, b), (ns, cs)
            assert lib.gsc_geometry_bytes(ns, cs) == b, (ns, cs)
    for ns, cs in ((-16, 16), (16, 0), (16, 8), (16, 24), (16, -16)):
        assert lib.gsc_geometry_bytes(ns, cs) == 0, (ns, cs)
        with pytest.raises(gsc.GscError):
            gsc.geometry_layout(ns, cs)
    cam = gsc.camera(S.look_at([0.5, 0.5, -1.5], [0.5, 0.5, 0.5], 1920, 1080))
    sizes = [lib.gsc_render_workspace_bytes(n, ctypes.byref(cam), p)
             for n, p in ((0, 0), (1000, 0), (1000, 10**6), (10**6, 10**6), (3 * 10**6, 3 * 10**7))]
    assert all(a < b for a, b in zip(sizes, sizes[1:])) and sizes[0] > 0
    assert lib.gsc_render_workspace_bytes(-1, ctypes.byref(cam), 0) == 0
    assert lib.gsc_render_workspace_bytes(10, ctypes.byref(cam), -1) == 0
    assert lib.gsc_render_workspace_bytes(10, None, 0) == 0
    bad = gsc.camera(S.look_at([0.5, 0.5, -1.5], [0.5, 0.5, 0.5], 0, 1080))
    assert lib.gsc_render_workspace_bytes(10, ctypes.byref(bad), 0) == 0


def test_missing_library_fails_loudly(tmp_path):
    # no fallback: without the built library the binding raises instead of computing anything
    from paper_2607_14513_gb300 import gsc
    saved = gsc._lib
    try:
        gsc._lib = None
        with pytest.raises(RuntimeError):
            gsc.load(str(tmp_path / "libgsc.so"))
    finally:
        gsc._lib = saved


def test_forced_table():
    # host only: the all-BC1 / all-BC7 table of a scene from any valid stream table of it
    from paper_2607_14513_gb300 import gsc
    lib = gsc.load()
    n, ng = 1000, 63
    t = gsc.StreamTable()
    t.n_streams, t.format, t.n, t.n_groups, t.layout = 2, gsc.FMT_RATE, n, ng, gsc.LAYOUT_D
    t.s[0].bands, t.s[0].bc7_blocks, t.s[0].first_group, t.s[0].n_groups, t.s[0].byte_offset = 16, 1, 0, 40, 0
    t.s[1].bands, t.s[1].bc7_blocks, t.s[1].first_group, t.s[1].n_groups = 4, 0, 40, 23
    t.s[1].byte_offset = 40 * (16 + 15 * 8)
    t.total_bytes = t.s[1].byte_offset + 23 * 4 * 8
    for k in range(16):
        t.scales[k], t.weights[k] = 0.25 + k, 1000 + k
    for fmt, bpb, j in ((gsc.FMT_BC1, 8, 0), (gsc.FMT_BC7, 16, 16)):
        f = gsc.forced_table(t, fmt)
        assert (f.n_streams, f.format, f.n, f.n_groups, f.layout) == (1, fmt, n, ng, gsc.LAYOUT_D)
        assert (f.s[0].bands, f.s[0].bc7_blocks, f.s[0].first_group, f.s[0].n_groups, f.s[0].byte_offset) == \
            (16, j, 0, ng, 0)
        assert f.total_bytes == ng * 16 * bpb and f.used_bits == 8 * f.total_bytes
        assert (f.budget_bits, f.lambda_) == (0, 0)
        assert list(f.scales) == list(t.scales) and list(f.weights) == list(t.weights)
    out = gsc.StreamTable()
    assert lib.gsc_forced_table(ctypes.byref(t), gsc.FMT_RATE, ctypes.byref(out)) == 1
    assert lib.gsc_forced_table(ctypes.byref(t), gsc.FMT_MIXED, ctypes.byref(out)) == 1
    t.total_bytes += 8  # no longer the sum of its streams
    assert lib.gsc_forced_table(ctypes.byref(t), gsc.FMT_BC7, ctypes.byref(out)) == 1
