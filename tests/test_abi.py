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
