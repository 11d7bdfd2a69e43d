"""The C-ABI library loads and exports what include/bto.h declares (no GPU).

Only calls that fail argument validation before touching CUDA are made here.
"""
import ctypes
import os

import pytest

import __graft_entry__
from paper_2004_02003_gb300 import bto


@pytest.fixture(scope="module")
def lib():
    from paper_2004_02003_gb300 import build
    build.build()
    return bto.load()


def test_every_declared_function_is_exported(lib):
    names = bto.header_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), f"{name} declared in include/bto.h but not exported"


def test_no_undeclared_bto_exports(lib):
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", bto.LIB_PATH], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    ours = {s for s in exported if s.startswith("bto_")}
    assert ours == set(bto.header_functions())


def test_status_strings(lib):
    for s in range(7):
        assert bto.bto_status_string(s)
    assert bto.bto_status_string(99) == "unknown status"


def test_argument_checks_before_cuda(lib):
    def create(ext, org, spc, s, L):
        out = ctypes.c_void_p()
        return lib.bto_create((ctypes.c_int32 * 3)(*ext), (ctypes.c_float * 3)(*org),
                              (ctypes.c_float * 3)(*spc), s, L, ctypes.byref(out)), out.value

    for args in [((0, 4, 4), (0, 0, 0), (1, 1, 1), 1, 1),
                 ((4, 4, 4), (0, 0, 0), (1, 0, 1), 1, 1),
                 ((4, 4, 4), (0, 0, 0), (1, -1, 1), 1, 1),
                 ((4, 4, 4), (0, float("nan"), 0), (1, 1, 1), 1, 1),
                 ((4, 4, 4), (0, 0, 0), (1, float("inf"), 1), 1, 1),
                 ((4, 4, 4), (0, 0, 0), (1, 1, 1), 0, 1),
                 ((4, 4, 4), (0, 0, 0), (1, 1, 1), 1, 0),
                 ((1024, 1024, 1024), (0, 0, 0), (1, 1, 1), 1, 1)]:
        st, h = create(*args)
        assert st == bto.BTO_ERR_INVALID_ARG and h is None, args
    assert lib.bto_create(None, None, None, 1, 1, None) == bto.BTO_ERR_INVALID_ARG


def test_null_context_calls(lib):
    assert lib.bto_num_seeds(None) == -1
    assert lib.bto_num_blocks(None) == -1
    assert lib.bto_advect_cycle(None, None, 0.1, None) == bto.BTO_ERR_INVALID_ARG
    assert lib.bto_end_interval(None, None, None, None, None, None) == bto.BTO_ERR_INVALID_ARG
    assert lib.bto_set_field_layout(None, 0) == bto.BTO_ERR_INVALID_ARG
    assert lib.bto_last_error(None) == bto.BTO_ERR_INVALID_ARG
    cells = (ctypes.c_int32 * 3)(8, 8, 8)
    assert lib.bto_set_tiling(None, cells, 256) == bto.BTO_ERR_INVALID_ARG
    assert lib.bto_get_tiling(None, (ctypes.c_int32 * 8)()) == bto.BTO_ERR_INVALID_ARG
    assert lib.bto_test_wait_timeout(None, 1) == bto.BTO_ERR_INVALID_ARG
    assert lib.bto_set_launch(None, 128, 2, 0, 0) == bto.BTO_ERR_INVALID_ARG
    assert lib.bto_get_launch(None, (ctypes.c_int32 * 5)()) == bto.BTO_ERR_INVALID_ARG
    assert lib.bto_copy_active(None, None, None, None) == bto.BTO_ERR_INVALID_ARG
    assert lib.bto_tape_backward(None, None, None, None, None) == bto.BTO_ERR_INVALID_ARG
    lib.bto_destroy(None)
    lib.bto_tape_destroy(None)


def test_stitch_argument_checks(lib):
    lat = (ctypes.c_int32 * 3)(4, 4, 4)
    org = (ctypes.c_float * 3)(0, 0, 0)
    spc = (ctypes.c_float * 3)(1, 1, 1)
    fake = ctypes.c_void_p(4096)        # never dereferenced: the checks fail first
    for scheme in (-1, 2, 7):
        assert lib.bto_stitch_pathlines_ex(lat, org, spc, 1, fake, 1, fake, fake, scheme,
                                           None) == bto.BTO_ERR_INVALID_ARG
    assert lib.bto_stitch_pathlines_ex(lat, org, spc, 0, fake, 1, fake, fake, bto.BTO_STITCH_BARYCENTRIC,
                                       None) == bto.BTO_ERR_INVALID_ARG
    assert lib.bto_stitch_pathlines(None, org, spc, 1, fake, 1, fake, fake, None) == bto.BTO_ERR_INVALID_ARG


def test_batch_argument_checks(lib):
    out = ctypes.c_void_p()
    ext = (ctypes.c_int32 * 6)(4, 4, 4, 4, -1, 4)
    org = (ctypes.c_float * 6)(0, 0, 0, 0, 0, 0)
    spc = (ctypes.c_float * 6)(1, 1, 1, 1, 1, 1)
    strides = (ctypes.c_int32 * 2)(1, 1)
    assert lib.bto_batch_create(2, ext, org, spc, strides, 4, ctypes.byref(out)) == bto.BTO_ERR_INVALID_ARG
    assert lib.bto_batch_create(0, ext, org, spc, strides, 4, ctypes.byref(out)) == bto.BTO_ERR_INVALID_ARG


def test_build_entry_point_builds_everything():
    __graft_entry__.build()
    assert os.path.exists(bto.LIB_PATH)
