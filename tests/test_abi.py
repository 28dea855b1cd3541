"""The C-ABI library loads and exports every entry point include/cc.h declares
(no compute calls: runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"^\s*(?:const\s+)?[\w\*\s]+?\b(cc_\w+)\s*\(", src, flags=re.M))
    return names


@pytest.fixture(scope="module")
def libpath():
    import paper_2510_12053_gb300 as cc
    if not os.path.exists(cc.LIB_PATH):
        from paper_2510_12053_gb300 import build
        build.build()
    return cc.LIB_PATH


def test_header_declares_the_boundary():
    names = _declared()
    for required in ["cc_build_mesh", "cc_color", "cc_build_subspace", "cc_sweep", "cc_energy_grad",
                     "cc_solve_step", "cc_destroy_mesh", "cc_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    h = ctypes.CDLL(libpath)
    missing = [n for n in sorted(_declared()) if not hasattr(h, n)]
    assert not missing, missing


def test_binding_signatures_cover_the_header(libpath):
    import paper_2510_12053_gb300 as cc
    assert set(cc._SIGS) <= _declared()
    cc.lib()  # loads and binds every signature


def test_version_string(libpath):
    import paper_2510_12053_gb300 as cc
    assert "sm_103a" in cc.version()


def test_concurrent_solve_checks_its_arguments_before_any_cuda_call(libpath):
    import paper_2510_12053_gb300 as cc
    lib = cc.lib()
    opts = (cc.StepOpts * 2)()
    assert lib.cc_solve_concurrent(0, None, None, None, None, None, None) == cc.OK
    assert lib.cc_solve_concurrent(-1, None, None, None, opts, None, None) == cc.ERR_INVALID_ARG
    assert "negative" in lib.cc_last_error().decode()
    assert lib.cc_solve_concurrent(2, None, None, None, opts, None, None) == cc.ERR_INVALID_ARG
    null2 = (ctypes.c_void_p * 2)()
    assert lib.cc_solve_concurrent(2, null2, null2, None, opts, None, None) == cc.ERR_INVALID_ARG
    assert "NULL mesh" in lib.cc_last_error().decode()


def test_concurrent_solve_binding_checks_one_x_per_mesh():
    import paper_2510_12053_gb300 as cc
    with pytest.raises(cc.CCError) as ei:
        cc.solve_concurrent([object(), object()], [None])
    assert ei.value.status == cc.ERR_INVALID_ARG
