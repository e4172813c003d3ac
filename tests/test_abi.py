"""The C-ABI library builds, loads and exports every symbol include/dd.h
declares; host-side argument validation works without a GPU (no compute)."""
import ctypes
import os
import re

import pytest

import paper_1710_07041_gb300 as dd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "dd.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(dd_[A-Za-z0-9_]+)\s*\(", txt)))


def test_header_and_binding_agree():
    names = declared_functions()
    assert len(names) >= 19
    assert set(names) == set(dd.EXPORTS), set(names) ^ set(dd.EXPORTS)


def test_library_exports_every_declared_symbol():
    L = dd.lib()
    for name in declared_functions():
        assert hasattr(L, name), name
    assert "sm_103a" in dd.version()


def test_lattice_validation_on_host():
    L = dd.lib()
    h = ctypes.c_void_p()
    bad = [((4, 4, 4, 4), (3, 2, 2, 2)),   # not a power of two
           ((4, 4, 4, 6), (2, 2, 2, 2)),   # odd number of blocks in x
           ((4, 4, 4, 4), (4, 2, 2, 2))]   # one block in t: no red-black colouring
    for dims, blk in bad:
        rc = L.dd_create_lattice((ctypes.c_int * 4)(*dims), (ctypes.c_int * 4)(*blk), 1, ctypes.byref(h))
        assert rc == -1 and L.dd_last_error()
    lat = dd.Lattice((8, 4, 4, 12), (2, 2, 2, 2))
    assert lat.V == 8 * 4 * 4 * 12
    assert lat.field_bytes(dd.F64) == lat.V * 24 * 8
    assert lat.field_bytes(dd.F32) == lat.V * 24 * 4
    assert lat.field_bytes(dd.F16) == lat.field_bytes(dd.BF16) == lat.V * 24 * 2
    # 16-bit fixed point with one FP32 scale per site
    assert lat.field_bytes(dd.F16N) == lat.V * (24 * 2 + 4)
    assert L.dd_field_bytes(lat.handle, 7) == 0
    assert L.dd_field_bytes(lat.handle, dd.F64_DF) == 0   # not a storage format
    lat.close()


def test_null_arguments_are_rejected():
    L = dd.lib()
    assert L.dd_create_gauge(None, None, None) == -1
    assert L.dd_apply_D(None, 1, None, None, 1, None) == -1
    assert L.dd_sap_smooth(None, None, None, None, 1, None) == -1
    assert L.dd_solve(None, None, None, None, 1, None, None) == -1
    L.dd_destroy(None)


def test_release_workspace_with_nothing_cached():
    """dd_release_workspace on a process that has not solved anything (here,
    no GPU at all): nothing to free, DD_OK."""
    assert dd.lib().dd_release_workspace() == 0


def test_every_entry_point_rejects_missing_handles():
    """Each compute, server and two-level entry point returns DD_EINVAL (with
    a message) for a missing handle or out-of-range parameters, before any
    CUDA call; size queries return 0."""
    L = dd.lib()
    st = ctypes.c_int()
    t = ctypes.c_uint64()
    calls = {
        "dd_create_op": lambda: L.dd_create_op(None, 1.0, 0.0, dd.F32, None),
        "dd_create_op_clover": lambda: L.dd_create_op_clover(None, None, dd.F32, None),
        "dd_op_get_clover": lambda: L.dd_op_get_clover(None, None),
        "dd_pack": lambda: L.dd_pack(None, dd.F32, None, None, 1, 1.0, None),
        "dd_unpack": lambda: L.dd_unpack(None, dd.F32, None, None, 1, 1.0, None),
        "dd_sap_smooth_multi": lambda: L.dd_sap_smooth_multi(0, None, None, None, None, None, None),
        "dd_solve_noalloc": lambda: L.dd_solve_noalloc(None, None, None, None, None, None),
        "dd_create_mg": lambda: L.dd_create_mg(None, None, None, None),
        "dd_mg_restrict": lambda: L.dd_mg_restrict(None, None, None, None),
        "dd_mg_prolong": lambda: L.dd_mg_prolong(None, None, None, None),
        "dd_mg_coarse_apply": lambda: L.dd_mg_coarse_apply(None, None, None, None),
        "dd_mg_precondition": lambda: L.dd_mg_precondition(None, None, None, None),
        "dd_server_create": lambda: L.dd_server_create(ctypes.byref(dd.ServerParams(0, 0, 1)), None),
        "dd_submit": lambda: L.dd_submit(None, None, ctypes.byref(t)),
        "dd_poll": lambda: L.dd_poll(None, 1, ctypes.byref(st), None, None),
        "dd_cancel": lambda: L.dd_cancel(None, 1),
        "dd_server_get_stats": lambda: L.dd_server_get_stats(None, None),
        "dd_bench_link_product": lambda: L.dd_bench_link_product(-1, 1, 1, None, None),
    }
    for name, call in calls.items():
        assert call() == -1, name
        assert L.dd_last_error(), name
    # server parameters out of range (no thread is started)
    for p in (dd.ServerParams(0, 65, 1), dd.ServerParams(0, 1, 0), dd.ServerParams(0, 1, 1 << 20)):
        h = ctypes.c_void_p()
        assert L.dd_server_create(ctypes.byref(p), ctypes.byref(h)) == -1 and not h.value
    assert L.dd_mg_coarse_length(None) == 0
    assert L.dd_lattice_volume(None) == -1
    assert L.dd_field_bytes(None, dd.F32) == 0
