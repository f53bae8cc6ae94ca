"""bkrylov_bdot_noalloc: the block inner product for callers that cannot allocate.

Such callers (a program under a fixed device-memory budget, a loop where an
allocation could block or fail) get G = X^T Y from static device scratch.  The
test calls it through the C ABI, twice in a row (the static scratch keeps the
previous call's contents, so the second call must not depend on them), and
compares with the handle-based bkrylov_bdot within the tolerance of the other
Gram tests (1e-13 of the entrywise magnitude bound |X|^T |Y|: its 512-CTA grid
orders the partial sums differently, so the two agree to rounding, not bit for
bit), checks that repeated calls agree bit for bit and that the device's free
memory does not move after one warm-up call per precision.  This file is
collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _call_noalloc(lib, X, Y, sym):
    n, s = X.shape
    G = torch.empty((s, s), dtype=torch.float64, device="cuda")
    prec = 0 if X.dtype == torch.float64 else 1
    st = lib.bkrylov_bdot_noalloc(n, s, C.c_void_p(X.data_ptr()), C.c_void_p(Y.data_ptr()),
                                  C.c_void_p(G.data_ptr()), int(sym), prec, None)
    assert st == 0, st
    torch.cuda.synchronize()
    return G.cpu().numpy()


def test_bdot_noalloc_matches_bdot_twice():
    from paper_2104_02494_gb300 import build, _lib
    from paper_2104_02494_gb300.api import Handle
    build()
    lib = _lib.load()
    g = np.random.default_rng(42)
    cases = [(100003, 7, False, np.float64), (4099, 32, True, np.float64),
             (20000, 8, False, np.float32)]
    with Handle(0) as h:
        data = []
        for n, s, sym, dt in cases:
            Xn = g.standard_normal((n, s)).astype(dt)
            Yn = g.standard_normal((n, s)).astype(dt)
            X, Y = torch.from_numpy(Xn).cuda(), torch.from_numpy(Yn).cuda()
            ref = h.bdot(X, Y, sym=sym).cpu().numpy()
            data.append((X, Y, sym, ref, Xn, Yn, dt, n, s))
        # one warm-up call per precision (module loading), then the device's free memory
        # must not move over the later calls
        _call_noalloc(lib, data[0][0], data[0][1], data[0][2])
        _call_noalloc(lib, data[2][0], data[2][1], data[2][2])
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        for X, Y, sym, ref, Xn, Yn, dt, n, s in data:
            bound = np.abs(Xn.astype(np.float64)).T @ np.abs(Yn.astype(np.float64))
            if sym:
                bound = bound + bound.T
            rtol = 1e-13 if dt == np.float64 else 2e-6
            prev = None
            for _ in range(2):                      # two calls in a row
                G = _call_noalloc(lib, X, Y, sym)
                assert np.all(np.abs(G - ref) <= rtol * bound), (n, s, sym)
                if prev is not None:                # reproducible from call to call
                    assert np.array_equal(G, prev)
                prev = G
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0


def test_bdot_noalloc_rejects_out_of_range():
    from paper_2104_02494_gb300 import build, _lib
    build()
    lib = _lib.load()
    X = torch.zeros((10, 33), dtype=torch.float64, device="cuda")
    G = torch.empty((33, 33), dtype=torch.float64, device="cuda")
    p = C.c_void_p(X.data_ptr())
    assert lib.bkrylov_bdot_noalloc(10, 33, p, p, C.c_void_p(G.data_ptr()), 0, 0, None) == 1
    assert lib.bkrylov_bdot_noalloc(0, 4, p, p, C.c_void_p(G.data_ptr()), 0, 0, None) == 1
    assert lib.bkrylov_bdot_noalloc(10, 4, p, p, C.c_void_p(G.data_ptr()), 0, 7, None) == 1
