"""The C-ABI library builds for sm_103a, loads, and exports every entry point that
include/mg.h declares (no compute calls: these run without a GPU)."""
import ctypes
import os
import re

import paper_0707_4018_gb300 as mgpkg
from paper_0707_4018_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "mg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mg_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("mg_setup", "mg_solve", "mg_dslash", "mg_destroy", "mg_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = binding.load()
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert isinstance(getattr(lib, name), ctypes._CFuncPtr)


def test_binding_covers_every_declared_symbol():
    assert sorted(binding.exported_symbols()) == declared_functions()


def test_default_params_and_argument_errors_without_gpu():
    p = mgpkg.mg_default_params()
    assert p.levels == 2 and p.Nv[0] == 8 and p.nu_pre == 4 and abs(p.omega - 0.8) < 1e-15
    lib = binding.load()
    # argument validation happens before any device work
    g = binding.make_geom((64, 64))
    ctx = ctypes.c_void_p()
    bad = mgpkg.mg_default_params(blocks=[(5, 4)])
    code = lib.mg_setup(ctypes.byref(ctx), ctypes.byref(g), ctypes.c_void_p(1), 0.1, ctypes.byref(bad), None)
    assert code == 1 and b"divisible" in lib.mg_last_error()
    assert ctx.value is None
    code = lib.mg_solve(None, None, None, 1e-10, None)
    assert code == 1


def test_library_is_built_for_sm_103a():
    # the fatbin's architecture is recorded by the build flags; check the build recipe itself
    from paper_0707_4018_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)
    assert os.path.exists(build.LIB)
