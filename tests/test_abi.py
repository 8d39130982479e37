"""The C-ABI library builds, loads without a GPU and exports every function that
include/vlasov.h declares; host-only argument checks answer with status codes."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def declared_functions():
    names = []
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+(vl_[A-Za-z0-9_]+)\s*\(",
                            text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2504_21450_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("vl_grid_create", "vl_grid_destroy", "vl_set_blocks", "vl_get_blocks",
                 "vl_translate", "vl_moments", "vl_mass", "vl_stats", "vl_status_str",
                 "vl_last_error", "vl_get_blocks_window"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_side_argument_checks(lib):
    from paper_2504_21450_gb300 import vlasov
    L = vlasov.load()
    assert vlasov.status_str(vlasov.VL_ECFL) == "VL_ECFL"
    o = vlasov.vl_translate_opts_default()
    assert o.form == vlasov.VL_FORM_FUSED and o.limiter == 1 and o.ghost == 3
    space = vlasov.vl_space_desc((ctypes.c_int * 3)(4, 4, 4), (ctypes.c_double * 3)(1, 1, 1),
                                 (ctypes.c_double * 3)(0, 0, 0))
    bad = vlasov.vl_vmesh_desc((ctypes.c_int * 3)(8, 8, 8), (ctypes.c_double * 3)(-4, -4, -4),
                               (ctypes.c_double * 3)(1, 1, 1), (ctypes.c_int * 3)(2, 4, 4))
    g = ctypes.c_void_p()
    st = L.vl_grid_create(ctypes.byref(space), ctypes.byref(bad), 0.0, 0, None, ctypes.byref(g))
    assert st == vlasov.VL_EINVAL and not g.value
    assert b"4x4x4" in L.vl_last_error(None)
    assert L.vl_grid_create(None, None, 0.0, 0, None, ctypes.byref(g)) == vlasov.VL_EINVAL
    assert L.vl_translate(None, 0.1, b"xyz", 1, None) == vlasov.VL_EINVAL
    assert L.vl_grid_destroy(None) == vlasov.VL_OK


def test_cost_model_host_side_checks(lib):
    """Argument checks and sizes of the cost-model entry points (no device work)."""
    from paper_2504_21450_gb300 import vlasov
    L = vlasov.load()
    space = vlasov.vl_space_desc((ctypes.c_int * 3)(19, 13, 10), (ctypes.c_double * 3)(1, 1, 1),
                                 (ctypes.c_double * 3)(0, 0, 0))
    assert vlasov.vl_tile_count(space, 8) == 3 * 2 * 2
    assert vlasov.vl_tile_count(space, 0) == -1
    assert vlasov.VL_MLP_NPARAM == 4801
    assert vlasov.vl_mlp_workspace_bytes(1000) >= 1000 * (4 * 64 * 4 + 8) + 4801 * 4
    assert L.vl_mlp_forward(None, None, 5, None, None) == vlasov.VL_EINVAL
    assert L.vl_mlp_forward(ctypes.c_void_p(256), None, 0, None, None) == vlasov.VL_OK  # nothing to do
    assert L.vl_cost_targets(ctypes.c_void_p(256), 3, 10, 4, ctypes.c_void_p(512), None) == vlasov.VL_EINVAL
    ws = ctypes.c_void_p(1 << 20)
    assert L.vl_mlp_train_step(ws, ws, ws, ws, ws, 10, 0, 1e-3, ws, 1 << 20, None, None) == vlasov.VL_EINVAL
    assert L.vl_mlp_train_step(ws, ws, ws, ws, ws, 10, 1, 1e-3, ctypes.c_void_p((1 << 20) + 8), 1 << 20,
                               None, None) == vlasov.VL_EINVAL  # misaligned workspace
    out = ctypes.c_int64()
    assert L.vl_mlp_capacity(ws, ws, 10, -1.0, ws, 1 << 20, ctypes.byref(out), None) == vlasov.VL_EINVAL
    assert L.vl_tile_features(None, 8, None, None) == vlasov.VL_EINVAL
