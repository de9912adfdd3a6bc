"""Host-side checks of the C-ABI library (no GPU needed, no compute calls).

The library builds for sm_103a, loads, exports every function that
include/ptycho.h declares, and rejects bad parameters before touching the
device.
"""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2205_06327_gb300 import _lib
    return _lib.load()


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "ptycho.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ptycho_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("ptycho_forward", "ptycho_loss_grad", "ptycho_step", "ptycho_plan_create",
                     "ptycho_plan_destroy", "ptycho_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2205_06327_gb300 import _lib
    names = _declared_functions()
    assert sorted(_lib.EXPORTED) == sorted(names)
    for n in names:
        assert hasattr(lib, n), n
    out = os.popen(f"nm -D --defined-only {_lib.LIB_PATH}").read()
    exported = set(re.findall(r"\bT (ptycho_[a-z0-9_]+)", out))
    assert set(names) <= exported
    # nothing else leaks from the library's C++ internals
    assert not [s for s in re.findall(r"\bT (\S+)", out) if "ptycho" in s and not s.startswith("ptycho_")]


def test_version_and_parameter_validation(lib):
    from paper_2205_06327_gb300._lib import (PTYCHO_ERR_ARG, PTYCHO_ERR_UNSUPPORTED, PtychoParams)
    assert b"sm_103a" in lib.ptycho_version()
    h = C.c_void_p(1234)
    p = PtychoParams(M=100, S=2, H=256, W=256, N=4, lambda_A=0.0251, dz_A=2.0, pixel_A=0.1)
    assert lib.ptycho_plan_create(C.byref(h), C.byref(p)) == PTYCHO_ERR_UNSUPPORTED
    assert h.value is None
    assert b"64 or 128" in lib.ptycho_last_error()
    p.M, p.S = 64, 0
    assert lib.ptycho_plan_create(C.byref(h), C.byref(p)) == PTYCHO_ERR_ARG
    p.S, p.H = 2, 32
    assert lib.ptycho_plan_create(C.byref(h), C.byref(p)) == PTYCHO_ERR_ARG
    p.H, p.tile_h, p.tile_w = 256, 128, 128
    assert lib.ptycho_plan_create(C.byref(h), C.byref(p)) == PTYCHO_ERR_ARG
    assert lib.ptycho_plan_create(None, C.byref(p)) == PTYCHO_ERR_ARG
    assert lib.ptycho_loss_grad(None, None, None, None, None, None, None, None, None) == PTYCHO_ERR_ARG
    assert lib.ptycho_loss_grad_host(None, None, None, None, None, None, None, None, None) == PTYCHO_ERR_ARG
    assert b"plan is NULL" in lib.ptycho_last_error()
    assert lib.ptycho_multi_loss_grad(None, -1, None) == PTYCHO_ERR_ARG
    assert lib.ptycho_multi_step(None, 0, float("nan"), 0.0, None) == PTYCHO_ERR_ARG
    assert b"finite" in lib.ptycho_last_error()
    assert lib.ptycho_step_accumulate(None, None, None, None, None, 1e-3, 0.0, None, 1, None, None) == PTYCHO_ERR_ARG
    assert b"plan is NULL" in lib.ptycho_last_error()
    assert lib.ptycho_plan_destroy(None) == PTYCHO_ERR_ARG


def test_product_path_has_no_cpu_fallback():
    """The package never imports the oracle; the API refuses to run without CUDA."""
    pkg = os.path.join(ROOT, "paper_2205_06327_gb300")
    for name in os.listdir(pkg):
        if name.endswith(".py"):
            src = open(os.path.join(pkg, name)).read()
            assert "oracle" not in re.sub(r"#.*", "", src).split("\n", 1)[-1] or name == "synth.py", name
    import torch
    if not torch.cuda.is_available():
        from paper_2205_06327_gb300 import api
        with pytest.raises(RuntimeError):
            api.Plan(api.Geometry(64, 1, 64, 64, 1))
