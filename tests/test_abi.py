"""The C-ABI library builds, loads without a GPU and exports every declared symbol."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bkrylov.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bkrylov_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2104_02494_gb300 import build, _lib
    path = build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 18
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_header():
    from paper_2104_02494_gb300 import _lib
    bound = {s[0] for s in _lib.SIGNATURES}
    assert bound == set(_declared())


def test_host_only_entry_points(lib):
    from paper_2104_02494_gb300 import _lib
    L = _lib.load()
    assert L.bkrylov_version() == 201
    assert L.bkrylov_status_string(_lib.BK_BREAKDOWN) == b"breakdown"
    o = _lib.default_opts()
    assert o.restart == 30 and o.eta == float("inf") and o.ortho == 1 and o.norm_mode == 0
    # argument validation happens before any device work
    assert L.bkrylov_create(None, 0, None) == _lib.BK_ERR_ARG
    assert L.bkrylov_destroy(None) == _lib.BK_ERR_ARG
    assert L.bkrylov_op_destroy(None) == _lib.BK_ERR_ARG


def test_opts_struct_layout_matches_header():
    from paper_2104_02494_gb300 import _lib
    # field order of bkrylov_opts / bkrylov_info in the header
    text = open(HEADER).read()
    for struct, cls in (("bkrylov_opts", _lib.bkrylov_opts), ("bkrylov_info", _lib.bkrylov_info)):
        body = re.search(r"typedef struct \{([^}]*)\}\s*" + struct + ";", text).group(1)
        body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
        fields = re.findall(r"([A-Za-z_][A-Za-z_0-9]*)\s*;", body)
        assert fields == [f[0] for f in cls._fields_], (struct, fields)


def test_no_gpu_create_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    from paper_2104_02494_gb300 import _lib
    L = _lib.load()
    h = ctypes.c_void_p()
    assert L.bkrylov_create(ctypes.byref(h), 0, None) == _lib.BK_ERR_ARG


def test_launches_per_iteration_counts():
    """Launches of one BCG iteration as the library enqueues them (host-only): at 128^3, s = 8
    the TSQR has a leaf level and two tree levels, so 3 factor launches, the root's sign fix
    and 3 two-launch applies = 10; the CholeskyQR2 iteration adds the SpMM, two s x s
    kernels, the update, two CholeskyQR2 s x s kernels, one row pass and the P update = 18
    (the count of the ncu launch list of the benchmark); the Householder iteration 6 + 10."""
    from paper_2104_02494_gb300 import _lib as L
    lib = L.load()
    assert lib.bkrylov_bcg_launches_per_iteration(2097152, 8, None) == 18
    o = L.default_opts()
    o.qr_mode = 1
    assert lib.bkrylov_bcg_launches_per_iteration(2097152, 8, ctypes.byref(o)) == 16
    o = L.default_opts()
    o.one_reduction = 1
    assert lib.bkrylov_bcg_launches_per_iteration(2097152, 8, ctypes.byref(o)) == 17
    assert lib.bkrylov_bcg_launches_per_iteration(0, 8, None) == -1
