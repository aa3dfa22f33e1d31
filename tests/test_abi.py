"""The C-ABI library builds, loads and exports every entry point that include/fmm.h declares
(no GPU needed: nothing here launches device work)."""
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fmm.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^[a-z][a-z_0-9 ]*[\s*]+(fmm_[a-z_0-9]+)\s*\(", src, re.M)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2604_19243_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("fmm_create", "fmm_build_tree", "fmm_precompute", "fmm_evaluate", "fmm_adjoint",
                 "fmm_destroy", "fmm_last_error"):
        assert must in names


@pytest.mark.parametrize("name", ["libfmm.so", "libfmm_debug.so"])
def test_library_exports_every_declared_symbol(libpath, name):
    # libfmm_debug.so: the same sources built with FMM_DEBUG (in-kernel bounds checks)
    path = os.path.join(os.path.dirname(libpath), name)
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT\s+(fmm_[a-z_0-9]+)$", out, re.M))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing


def test_binding_loads_all_entry_points(libpath):
    import paper_2604_19243_gb300 as pkg
    lib = pkg.lib()
    for name in declared_functions():
        assert hasattr(lib, name)
    assert set(pkg.ENTRY_POINTS) == set(declared_functions())


def test_default_options_and_validation_without_gpu(libpath):
    import ctypes
    import paper_2604_19243_gb300 as pkg
    lib = pkg.lib()
    opt = pkg.Options()
    assert lib.fmm_default_options(ctypes.byref(opt)) == 0
    assert (opt.order_p, opt.depth, opt.precision) == (6, 4, 0)
    assert opt.svd_rtol == 1e-6 and opt.pinv_rtol == 1e-7
    ctx = ctypes.c_void_p()
    # option checks run before any CUDA call
    for field, bad in (("order_p", 1), ("order_p", 11), ("depth", -1), ("depth", 11),
                       ("precision", 7), ("svd_rtol", 0.0), ("pinv_rtol", 2.0)):
        o = pkg.Options()
        lib.fmm_default_options(ctypes.byref(o))
        setattr(o, field, bad)
        assert lib.fmm_create(ctypes.byref(o), None, ctypes.byref(ctx)) == 1
    o = pkg.Options()
    lib.fmm_default_options(ctypes.byref(o))
    o.has_domain, o.side = 1, -1.0
    assert lib.fmm_create(ctypes.byref(o), None, ctypes.byref(ctx)) == 1
    # the modified Helmholtz kernel: kappa finite and > 0, a domain, no mean_free
    for kernel, kappa, has_domain, mean_free, want in ((3, 1.0, 1, 0, 1), (1, 0.0, 1, 0, 1),
                                                       (2, 0.0, 1, 0, 1), (2, 1.0, 0, 0, 6), (2, 1.0, 1, 1, 6),
                                                       (1, -1.0, 1, 0, 1), (1, float("nan"), 1, 0, 1),
                                                       (1, float("inf"), 1, 0, 1), (1, 1.0, 0, 0, 6),
                                                       (1, 1.0, 1, 1, 6)):
        o = pkg.Options()
        lib.fmm_default_options(ctypes.byref(o))
        assert o.kernel == 0 and o.kappa == 0.0
        o.kernel, o.kappa, o.has_domain, o.side, o.mean_free = kernel, kappa, has_domain, 1.0, mean_free
        assert lib.fmm_create(ctypes.byref(o), None, ctypes.byref(ctx)) == want, (kernel, kappa, has_domain)
    # null contexts are refused before any CUDA call
    ainfo = pkg.AdaptiveTreeInfo()
    assert lib.fmm_adaptive_setup(None, 8) == 1
    assert lib.fmm_adaptive_info(None, ctypes.byref(ainfo)) == 1
    assert lib.fmm_adaptive_export(None, pkg.ADAPTIVE_U, None, None, None) == 1
    assert lib.fmm_adaptive_evaluate(None, None, None, None, pkg.PART_ALL) == 1
    assert lib.fmm_partition_setup(None, 2, 4) == 1
    flags, ink = ctypes.c_uint32(7), ctypes.c_int32(7)
    assert lib.fmm_debug_check(None, ctypes.byref(flags), ctypes.byref(ink)) == 1
    assert lib.fmm_last_error(None) == b"null context"
    lib.fmm_destroy(None)


def test_product_path_does_not_import_the_oracle():
    pkg_dir = os.path.join(ROOT, "paper_2604_19243_gb300")
    for dirpath, _, files in os.walk(pkg_dir):
        for f in files:
            if f.endswith((".py", ".cu", ".cpp", ".h", ".cuh")):
                text = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in re.sub(r"#.*|//.*", "", text), f


def test_library_selection_loads_the_bounds_checked_build(libpath):
    # FMM_LIBRARY picks a build within _build/ by file name; the child loads it and reports the
    # path and the outcome of a null-context call (no CUDA call is made)
    code = ("import ctypes, paper_2604_19243_gb300 as pkg; L = pkg.lib(); "
            "f = ctypes.c_uint32(); print(pkg.LIB_PATH, L.fmm_debug_check(None, ctypes.byref(f), None))")
    for name in ("libfmm.so", "libfmm_debug.so", "../../../libfmm_debug.so"):
        env = dict(os.environ, FMM_LIBRARY=name)
        out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                             check=True).stdout.split()
        assert out[0] == os.path.join(os.path.dirname(libpath), os.path.basename(name)) and out[1] == "1"
