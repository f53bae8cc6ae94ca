"""The thesis's worked example on the GPU (Ch. 2, Ex. "nonconverging_gmres", stored in
tests/golden/gmres_cyclic_shift.json): block GMRes with s = 1 on the cyclic shift with b = e_1
keeps X = 0 and a relative residual of 1 for k < n steps and is exact at k = n; BiCGStab breaks
down at once (r0^T A r0 = a_11 = 0).  The oracle's side is in tests/test_golden.py.
"""
import math

import numpy as np
import pytest

from test_golden import CYCLIC, _cyclic

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("ortho", ["mgs", "cgs2", "localized"])
def test_gpu_gmres_stalls_on_the_cyclic_shift(ortho):
    import torch
    from paper_2104_02494_gb300 import build
    from paper_2104_02494_gb300.api import Handle
    build()
    n = CYCLIC["n"][1]
    A = _cyclic(n, False)
    b = np.zeros((n, 1)); b[0, 0] = 1.0
    dv = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    with Handle(0) as h:
        op = h.op_csr(dv(A.row_ptr), dv(A.col), dv(A.val))
        for k in (1, n // 2, n - 1):
            X, info = h.solve("bgmres", op, dv(b), tol=0.0, maxit=k, restart=n, ortho=ortho)
            assert np.abs(X.cpu().numpy()).max() <= 1e-14 and abs(info.relres_max - 1.0) <= 1e-14
        X, info = h.solve("bgmres", op, dv(b), tol=1e-12, maxit=n, restart=n, ortho=ortho)
        sol = np.zeros(n); sol[1] = 1.0
        assert info.converged and info.iters == n
        assert np.abs(X.cpu().numpy()[:, 0] - sol).max() <= 1e-13
        X, info = h.solve("bbicgstab", op, dv(b), tol=1e-12, maxit=2 * n, eta=math.inf)
        assert info.status == 5 and np.all(X.cpu().numpy() == 0.0)
        op.close()
