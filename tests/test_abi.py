"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/fe2.h declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(fe2_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2312_12771_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["fe2_create", "fe2_destroy", "fe2_rve_register", "fe2_micro_assemble",
                     "fe2_nullspace_reduce", "fe2_condense", "fe2_macro_step", "fe2_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2312_12771_gb300 import fe2
    assert set(declared_functions()) <= set(fe2.exported_symbols())


def test_binding_refuses_without_library(tmp_path):
    from paper_2312_12771_gb300 import fe2
    with pytest.raises(RuntimeError):
        fe2.load.__wrapped__(str(tmp_path / "missing.so")) if hasattr(fe2.load, "__wrapped__") else \
            _load_fresh(str(tmp_path / "missing.so"))


def _load_fresh(path):
    from paper_2312_12771_gb300 import fe2
    saved = fe2._lib
    fe2._lib = None
    try:
        return fe2.load(path)
    finally:
        fe2._lib = saved


def test_noalloc_argument_errors_return_before_any_device_work(lib):
    """fe2_rve_solve_noalloc refuses bad sizes, NULL pointers and requests
    beyond its fixed scratch array before it touches the device (so this runs
    without a GPU), each with a reason in fe2_noalloc_last_error."""
    from paper_2312_12771_gb300 import fe2
    f = fe2.load()
    P = ctypes.c_void_p
    dummy = P(256)                      # never dereferenced: every case returns first

    def call(N, n, nphase, ptr=dummy):
        return f.fe2_rve_solve_noalloc(N, n, nphase, ptr, ptr, ptr, ptr, ptr, ptr, None, None)

    cases = [(call(2, 4, 2), fe2.FE2_ERR_ARG),          # N < 3
             (call(8, 0, 2), fe2.FE2_ERR_ARG),          # no RVEs
             (call(8, 4, 9), fe2.FE2_ERR_ARG),          # nphase > 8
             (call(8, 4, 0), fe2.FE2_ERR_ARG),          # nphase < 1
             (call(8, 4, 2, P(0)), fe2.FE2_ERR_ARG),    # NULL inputs / outputs
             (call(32, 40, 2), fe2.FE2_ERR_BUDGET),     # 40 RVEs of 32^2 exceed 64 MiB (39 fit)
             (call(16, 231, 2), fe2.FE2_ERR_BUDGET)]    # 231 RVEs of 16^2 too (230 fit)
    for got, want in cases:
        assert got == want
        assert f.fe2_noalloc_last_error().decode() != ""
