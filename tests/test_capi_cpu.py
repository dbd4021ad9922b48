"""The C-ABI library builds, loads without a GPU and exports every function sylv.h declares.

Only host-side entry points are called (no device work): defaults, status strings and the
argument checks that run before any CUDA call.
"""

import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sylv.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\*?\s+\**(sylv_\w+)\s*\(", text, re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2204_08057_gb300 import binding, build
    if not os.path.exists(build.LIB):
        if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
            pytest.skip("library not built and nvcc unavailable")
        build.build()
    return binding.load()


def test_header_lists_the_boundary():
    names = declared_functions()
    for required in ("sylv_create", "sylv_rhs", "sylv_apply", "sylv_solve",
                     "sylv_solve_batched", "sylv_backward", "sylv_destroy", "sylv_strerror"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_2204_08057_gb300 import binding as B
    assert sorted(B.EXPORTED) == sorted(declared_functions())


def test_host_only_entry_points(lib):
    from paper_2204_08057_gb300 import binding as B
    o = B.sylv_opts_default()
    assert o.tol == 1e-8 and o.precision == B.SYLV_PREC_MIXED and o.use_graph == 1
    assert B.sylv_strerror(B.SYLV_OK) == "ok"
    assert B.sylv_strerror(B.SYLV_E_NOT_CONVERGED) == "not converged"
    assert B.sylv_strerror(12345) == "unknown status"
    # argument checks that precede any device work
    h = ctypes.c_void_p()
    assert lib.sylv_create(ctypes.byref(h), None, None) == B.SYLV_E_INVALID
    assert h.value is None
    p = B.sylv_problem()
    p.n, p.k, p.m, p.ld = 10, 9, 3, 10
    assert lib.sylv_create(ctypes.byref(h), ctypes.byref(p), None) == B.SYLV_E_UNSUPPORTED
    p.k, p.ld = 3, 5
    assert lib.sylv_create(ctypes.byref(h), ctypes.byref(p), None) == B.SYLV_E_INVALID
    assert "ld" in B.sylv_last_error()
    assert lib.sylv_solve(None, None, None, 1, None, None, None) == B.SYLV_E_INVALID
    assert lib.sylv_solve_host(None, None, None, 1, None, None, None) == B.SYLV_E_INVALID
    assert lib.sylv_apply(None, None, None, 1, 0, None) == B.SYLV_E_INVALID
    lib.sylv_destroy(None)


def test_host_solve_argument_checks(lib):
    """sylv_solve_host's binding checks its host buffers before any device work."""
    import torch
    from paper_2204_08057_gb300 import binding as B
    Y = torch.zeros((1, 3, 16), dtype=torch.float64)
    X = torch.zeros((1, 2, 16), dtype=torch.float64)
    with pytest.raises(TypeError):
        B.sylv_solve_host(0, Y.float(), X, 1, k=2, m=3, ld=16, n=16)
    with pytest.raises(ValueError):
        B.sylv_solve_host(0, Y[:, :, :8], X, 1, k=2, m=3, ld=16, n=16)
    with pytest.raises(ValueError):
        B.sylv_solve_host(0, Y, X.t() if X.dim() == 2 else X.transpose(1, 2), 1, k=2, m=3,
                          ld=16, n=16)
    assert lib.sylv_solve_host(None, ctypes.c_void_p(Y.data_ptr()),
                               ctypes.c_void_p(X.data_ptr()), 1, None, None,
                               None) == B.SYLV_E_INVALID


def test_struct_layouts_match_header():
    from paper_2204_08057_gb300 import binding as B
    # sizes implied by the header's field lists on an LP64 ABI
    assert ctypes.sizeof(B.sylv_opts) == 2 * 8 + 8 * 4
    assert ctypes.sizeof(B.sylv_info) == 4 * 4 + 5 * 8 + 4 * 4 + 6 * 4
    assert ctypes.sizeof(B.sylv_problem) == 8 + 4 + 4 + 8 + 3 * 8 + 8 + 2 * 8 + 5 * 8 + 8 + 2 * 4
