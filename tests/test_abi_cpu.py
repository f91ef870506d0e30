"""CPU-only checks of the C ABI boundary: the library loads, exports every
function declared in include/svlcov.h, and its host-side logic (workspace
sizing, argument validation, error strings) works without a GPU."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "svlcov.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(svlcov_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2401_09703_gb300 import _abi
    return _abi.lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["svlcov_init", "svlcov_add_cols", "svlcov_add_rows", "svlcov_update_weights",
                     "svlcov_get_factors", "svlcov_query_rows", "svlcov_status", "svlcov_destroy"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert missing == []


def test_bindings_cover_every_declared_symbol():
    from paper_2401_09703_gb300 import _abi
    assert sorted(_abi.SIGNATURES) == sorted(n for n in declared_functions())


def _desc(**kw):
    from paper_2401_09703_gb300 import _abi
    d = _abi.svlcov_init_desc()
    d.m, d.n, d.k = 100, 80, 8
    d.max_m, d.max_n, d.max_s, d.max_nnz = 200, 200, 16, 400
    d.storage, d.small = _abi.SVLCOV_FP32, _abi.SVLCOV_SMALL_MIXED
    for a, v in kw.items():
        setattr(d, a, v)
    return d


def test_workspace_size_host_only(lib):
    d = _desc()
    n1 = lib.svlcov_workspace_bytes(C.byref(d))
    assert n1 > 0 and n1 % 256 == 0
    d2 = _desc(max_s=64)
    assert lib.svlcov_workspace_bytes(C.byref(d2)) > n1
    for bad in (dict(k=0), dict(k=129), dict(max_s=0), dict(max_s=2000), dict(max_m=10), dict(storage=7),
                dict(small=9)):
        assert lib.svlcov_workspace_bytes(C.byref(_desc(**bad))) == 0, bad


def test_init_rejects_bad_arguments_without_cuda(lib):
    from paper_2401_09703_gb300 import _abi
    h = C.c_void_p()
    assert lib.svlcov_init(C.byref(h), C.byref(_desc(k=0)), None) == _abi.SVLCOV_ERR_INVALID_ARG
    assert lib.svlcov_init(C.byref(h), C.byref(_desc()), None) == _abi.SVLCOV_ERR_INVALID_ARG  # null buffers
    assert lib.svlcov_add_cols(None, None, None) == _abi.SVLCOV_ERR_INVALID_ARG
    assert lib.svlcov_get_shape(None, None, None, None) == _abi.SVLCOV_ERR_INVALID_ARG


def test_dgemm_engines_and_arguments_checked_without_cuda(lib):
    """svlcov_dgemm's engines 0 (FP64 pipe), 1 (tensor cores) and 2
    (double-float) share the host-side checks, which run before any CUDA call."""
    from paper_2401_09703_gb300 import _abi
    bad = _abi.SVLCOV_ERR_INVALID_ARG
    dummy = C.c_void_p(16)   # never dereferenced: every call below returns before a launch
    for engine in (-1, 3, 7):
        assert lib.svlcov_dgemm(0, 0, 4, 4, 4, 1.0, dummy, 4, dummy, 4, 0.0, dummy, 4, engine, None) == bad
    for engine in (0, 1, 2):
        assert lib.svlcov_dgemm(0, 0, 4, 4, 4, 1.0, dummy, 4, dummy, 4, 0.0, None, 4, engine, None) == bad   # no C
        assert lib.svlcov_dgemm(0, 0, 4, 4, 4, 1.0, dummy, 3, dummy, 4, 0.0, dummy, 4, engine, None) == bad  # lda < M
        assert lib.svlcov_dgemm(1, 0, 4, 4, 5, 1.0, dummy, 4, dummy, 5, 0.0, dummy, 4, engine, None) == bad  # lda < K (A^T)
        assert lib.svlcov_dgemm(0, 0, 4097, 4, 4, 1.0, dummy, 4097, dummy, 4, 0.0, dummy, 4097, engine, None) == bad
        assert lib.svlcov_dgemm(0, 0, 0, 4, 4, 1.0, None, 1, None, 4, 0.0, None, 1, engine, None) == _abi.SVLCOV_OK


def test_strerror(lib):
    assert lib.svlcov_strerror(0) == b"ok"
    assert b"CSR" in lib.svlcov_strerror(0x10)


def test_product_path_does_not_import_the_oracle():
    """The package and bench's GPU leg never import oracle/ (test
    infrastructure only)."""
    pkg = os.path.join(ROOT, "paper_2401_09703_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
