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
