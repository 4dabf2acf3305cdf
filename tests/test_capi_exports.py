"""The C-ABI library loads without a GPU and exports every entry point that
include/gs.h declares (no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gs.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gs_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    import torch  # noqa: F401  (makes the CUDA runtime resolvable)
    from paper_2501_08672_b300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_path():
    names = declared_functions()
    for required in ("gs_project", "gs_bin", "gs_render_fwd", "gs_render_bwd", "gs_adam_step", "gs_pose_grad",
                     "gs_l1_loss", "gs_context_create", "gs_context_destroy", "gs_last_error",
                     "gs_workspace_query", "gs_sync_status"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_every_export():
    from paper_2501_08672_b300 import binding
    assert set(declared_functions()) <= set(binding.EXPORTED) | {"gs_config_default", "gs_version"}


def test_host_only_calls_work_without_a_gpu(lib):
    from paper_2501_08672_b300 import binding as B
    c = B.Config()
    lib.gs_config_default(ctypes.byref(c))
    assert c.tile_size == 16 and abs(c.alpha_min - 1 / 255) < 1e-9 and abs(c.alpha_max - 0.99) < 1e-7
    lib.gs_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.gs_version()
    # NULL context / output pointers are rejected on the host
    assert lib.gs_context_create(None, 0, None) == B.GS_ERR_INVALID_ARG
    lib.gs_last_error.restype = ctypes.c_char_p
    assert lib.gs_last_error(None) == b"context is NULL"
    assert lib.gs_project(None, None, None, 0, None, None) == B.GS_ERR_INVALID_ARG


@pytest.mark.parametrize("ts,bin_ts,ok", [(8, 0, True), (8, 8, True), (8, 16, True), (8, 32, True), (16, 32, True),
                                          (32, 32, True), (8, 24, False), (16, 8, False), (16, 64, False),
                                          (32, 64, False), (8, 12, False)])
def test_bin_tile_size_is_checked_on_the_host(lib, ts, bin_ts, ok):
    """gs_config.bin_tile_size must be 0 or 1, 2 or 4 times the tile size, at
    most 32; the check runs before any device call (a valid config then
    fails only for want of a GPU here)."""
    from paper_2501_08672_b300 import binding as B
    c = B.Config()
    lib.gs_config_default(ctypes.byref(c))
    assert c.bin_tile_size == 0
    c.tile_size = ts
    c.pixels_per_thread = 4 if ts == 32 else 2
    c.bin_tile_size = bin_ts
    h = ctypes.c_void_p()
    rc = lib.gs_context_create(ctypes.byref(h), 0, ctypes.byref(c))
    if rc == B.GS_OK:
        lib.gs_context_destroy(h)
    assert (rc != B.GS_ERR_INVALID_ARG) == ok


def header_struct_fields(name):
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    m = re.search(r"typedef struct %s \{(.*?)\} %s;" % (name, name), text, flags=re.S)
    assert m, name
    fields = []
    for decl in m.group(1).split(";"):
        decl = decl.strip()
        if not decl:
            continue
        decl = re.sub(r"\[[^\]]*\]", "", decl)
        for part in decl.split(","):
            fields.append(re.findall(r"\w+", part)[-1])
    return fields


@pytest.mark.parametrize("cname,pyname", [("gs_config", "Config"), ("gs_view", "View"),
                                          ("gs_gaussians", "Gaussians"), ("gs_grads", "Grads"),
                                          ("gs_workspace", "Workspace"), ("gs_ws_layout", "WsLayout"),
                                          ("gs_profile_entry", "ProfileEntry"),
                                          ("gs_lowp_segment", "LowpSegment"),
                                          ("gs_window_column", "WindowColumn")])
def test_binding_structs_match_header(cname, pyname):
    """Every ctypes mirror lists the header struct's fields in the same order."""
    from paper_2501_08672_b300 import binding
    py = [f[0] for f in getattr(binding, pyname)._fields_]
    assert py == header_struct_fields(cname)
