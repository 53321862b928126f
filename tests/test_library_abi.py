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
    code = lib.mg_solve(None, None, None, 1, 1e-10, None)
    assert code == 1
    code = lib.mg_solve(None, None, None, 0, 1e-10, None)
    assert code == 1 and b"nrhs" in lib.mg_last_error()


def test_new_boundary_calls_reject_bad_arguments_without_gpu(tmp_path):
    lib = binding.load()
    ctx = ctypes.c_void_p()
    # a missing or foreign file is rejected before any device work
    code = lib.mg_load_setup(ctypes.byref(ctx), str(tmp_path / "missing.mgs").encode(), ctypes.c_void_p(1), None)
    assert code == 1 and ctx.value is None
    junk = tmp_path / "junk.mgs"
    junk.write_bytes(b"not a saved setup" * 100)
    code = lib.mg_load_setup(ctypes.byref(ctx), str(junk).encode(), ctypes.c_void_p(1), None)
    assert code == 1 and b"saved setup" in lib.mg_last_error()
    assert lib.mg_save_setup(None, b"x") == 1
    assert lib.mg_context_info(None, None, None, None) == 1
    # setup batches: count and null arrays are checked first
    assert lib.mg_setup_batch(0, None, None, None, None, None, None) == 1
    hs = (ctypes.c_void_p * 1)()
    assert lib.mg_setup_batch(1, hs, None, None, None, None, None) == 1


def test_stats_struct_matches_header():
    # mg_stats gained setup_s, solve_s and fine_D_apps at its end: the ctypes layout must follow
    names = [f[0] for f in binding.mg_stats._fields_]
    assert names[-3:] == ["setup_s", "solve_s", "fine_D_apps"]
    text = open(os.path.join(ROOT, "include", "mg.h")).read()
    body = text[text.index("typedef struct {\n  int iters;"):text.index("} mg_stats;")]
    for n in names:
        assert re.search(r"\b" + n + r"\b", body), n


def test_library_is_built_for_sm_103a():
    # the fatbin's architecture is recorded by the build flags; check the build recipe itself
    from paper_0707_4018_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)
    assert os.path.exists(build.LIB)
