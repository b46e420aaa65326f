"""Host-side checks that need no GPU: the library builds, loads without a driver,
and exports every entry point include/mm.h declares; the binding declares the
same set; the slice-count rule and the fixed-point shift behave as documented."""
import ctypes
import math
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "mm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mm_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2408_15384_gb300 import build, _lib
    build.build()
    return _lib.load()


def test_header_declares_the_boundary_calls():
    fns = header_functions()
    for f in ("mm_create", "mm_gemm", "mm_gemm_grouped", "mm_serve_submit", "mm_serve_poll", "mm_destroy"):
        assert f in fns


def test_library_exports_every_declared_symbol(lib):
    for f in header_functions():
        assert hasattr(lib, f), f


def test_binding_covers_header(lib):
    from paper_2408_15384_gb300 import _lib
    assert sorted(_lib.SIGNATURES) == header_functions()


def test_status_strings(lib):
    assert lib.mm_status_string(0) == b"ok"
    assert lib.mm_status_string(2) == b"invalid argument"
    assert lib.mm_status_string(999) == b"unknown status"


def test_slice_count_rule_matches_the_oracle(lib):
    """The library's decision function (the one the kernels run) against the
    oracle's, on a grid of k and spreads given as float32 values, decision for
    decision."""
    import numpy as np
    from oracle import emulation as em
    spreads = np.float32([0.5, 0.3, 0.25, 0.1, 0.05, 0.02, 1e-3, 1e-5, 0.0, np.inf])
    for k in [1, 5, 7, 64, 96, 700, 1000, 2048, 4096, 8192, 12288, 65536, 1 << 22]:
        for a in spreads:
            for b in spreads:
                assert lib.mm_slice_count_rule(k, float(a), float(b)) == \
                    em.slice_count_from_spread(k, float(a), float(b)), (k, a, b)
    assert lib.mm_slice_count_rule(0, 0.25, 0.25) == -1


def test_crt_rule_matches_the_oracle(lib):
    """The library's modular-form parameters (the function the decision kernel
    runs) against the oracle's, on a grid of k and float32 spreads."""
    import numpy as np
    from oracle import emulation as em
    spreads = np.float32([0.5, 0.3, 0.25, 0.1, 0.05, 0.02, 1e-3, 1e-5, 0.0, np.inf])
    b = ctypes.c_int(0)
    for k in [1, 5, 7, 64, 96, 700, 1000, 2048, 4096, 8192, 12288, 65536, 1 << 22]:
        for a in spreads:
            for c in spreads:
                N = lib.mm_crt_rule(k, float(a), float(c), ctypes.byref(b))
                want = em.crt_params_from_spread(k, float(a), float(c))
                assert (N, b.value) == ((want[1], want[0]) if want else (0, 0)), (k, a, c)
    assert lib.mm_crt_rule(0, 0.25, 0.25, ctypes.byref(b)) == -1
    assert lib.mm_crt_rule(10, 0.25, 0.25, None) == -1


def test_create_without_gpu_fails_cleanly(lib):
    h = ctypes.c_void_p()
    rc = lib.mm_create(ctypes.byref(h), 0, 0)
    assert rc in (0, 5, 9)  # no device here: MM_ERR_CUDA; on a GB300 machine: OK
    if rc == 0:
        lib.mm_destroy(h)
    assert lib.mm_create(None, 0, 0) == 2


def test_fill_argument_errors(lib):
    assert lib.mm_fill_uniform(None, 4, 4, 4, 1, 1, 0, 0, None) == 2
    assert lib.mm_fill_uniform(None, 0, 0, 0, 1, 1, 0, 0, None) == 0
    assert lib.mm_fill_uniform(ctypes.c_void_p(16), 4, 4, 3, 1, 1, 0, 0, None) == 2


def test_no_oracle_in_product_path():
    """The package never imports the oracle (test infrastructure only)."""
    pkg = os.path.join(ROOT, "paper_2408_15384_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "mm_oracle" not in txt, f
