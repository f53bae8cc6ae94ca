"""Planted-mistake tests: each mutation of the oracle must fail one of its pins.

A mutation is a one-token edit of the oracle's source (a dropped transpose, a
flipped sign, swapped operands).  The edited function is compiled in a copy
of its module's namespace and the relevant pin battery is run on it; the
test passes only if the battery rejects the mutant.  Nothing here touches a
GPU; the mistakes are planted in the CPU oracle only.
"""
import inspect
import math
import sys
import textwrap

import numpy as np
import pytest

import oracle  # noqa: F401  (loads the submodules)
import workloads as W

# planted mistakes are expected to overflow or divide by zero on the way to failing a pin
pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _mutant(modname, fname, old, new):
    mod = sys.modules[modname]
    src = textwrap.dedent(inspect.getsource(getattr(mod, fname)))
    assert src.count(old) >= 1, f"mutation anchor not found: {old!r}"
    src = src.replace(old, new, 1)
    ns = dict(vars(mod))
    exec(compile(src, f"<mutant {fname}>", "exec"), ns)
    return ns[fname]


def _spd(n, seed, cond=30.0):
    g = np.random.default_rng(seed)
    Qm, _ = np.linalg.qr(g.standard_normal((n, n)))
    return (Qm * np.geomspace(1.0, cond, n)) @ Qm.T


class _Dense:
    def __init__(self, M):
        n = M.shape[0]
        self.n = n
        self.row_ptr = np.arange(0, n * n + 1, n, dtype=np.int32)
        self.col = np.tile(np.arange(n, dtype=np.int32), n)
        self.val = M.ravel().copy()


def _bcg_battery_passes(bcg_fn):
    """Dense-solve pin, sigma-residual pin and invariants for a BCG implementation."""
    try:
        # eta = 1e-30 normalises R^0 but never again, so sigma != I throughout
        for eta in (math.inf, 0.0, 1e4, 1e-30):
            M = _spd(30, 1)
            B = np.random.default_rng(2).standard_normal((30, 5))
            r = bcg_fn(_Dense(M), B, tol=1e-12, maxit=60, eta=eta)
            if not r.converged:
                return False
            Xs = np.linalg.solve(M, B)
            if np.abs(r.X - Xs).max() > 1e-9 * np.abs(Xs).max():
                return False
            true = np.linalg.norm(B - M @ r.X, axis=0) / np.linalg.norm(B, axis=0)
            if np.abs(true - r.relres).max() > 1e-10:
                return False
            # mid-run: residual norms from sigma/rho equal the recomputed ones (relative)
            r3 = bcg_fn(_Dense(M), B, tol=0.0, maxit=3, eta=eta)
            true3 = np.linalg.norm(B - M @ r3.X, axis=0) / np.linalg.norm(B, axis=0)
            if np.abs(true3 / r3.relres - 1).max() > 1e-8:
                return False
        # s = 1 with eta = 0 is textbook CG, iterate for iterate
        A = W.lap2d5(9, 8)
        b = W.normal_block(A.n, 1, 3)
        r = bcg_fn(A, b, tol=1e-10, maxit=100, eta=0.0, record_iterates=20)
        _, _, _, xs = sys.modules["oracle.bcg"].scalar_cg(A, b[:, 0], tol=1e-10, maxit=100,
                                                          record_iterates=20)
        for k in range(20):
            if np.abs(r.iterates[k][:, 0] - xs[k]).max() > 1e-12 * np.abs(xs[k]).max():
                return False
        # Jacobi-preconditioned: the energy minimiser over K_k(M^{-1}A, M^{-1}R^0)
        # (Eq. "energy-minimizer") and Euclidean residual tracking
        kf = np.exp(1.5 * np.random.default_rng(5).standard_normal(125))
        A = W.diff3d7_var(5, 5, 5, kf)
        Ad = A.to_dense()
        w = 1.0 / np.diag(Ad)
        B = W.normal_block(A.n, 3, 4)
        for eta in (0.0, math.inf):
            r = bcg_fn(A, B, tol=0.0, maxit=4, eta=eta, Minv=w, record_iterates=4)
            blocks = [w[:, None] * B]
            for k in range(1, 5):
                V, _ = np.linalg.qr(np.hstack(blocks))
                Xk = V @ np.linalg.solve(V.T @ Ad @ V, V.T @ B)
                if np.abs(r.iterates[k - 1] - Xk).max() > 1e-9 * np.abs(Xk).max():
                    return False
                blocks.append(w[:, None] * (Ad @ blocks[-1]))
            true = np.linalg.norm(B - Ad @ r.X, axis=0) / np.linalg.norm(B, axis=0)
            if np.abs(true / r.relres - 1).max() > 1e-8:
                return False
        return True
    except Exception:
        return False


BCG_MUTATIONS = [
    ("oracle.bcg", "bcg", "gamma.T @ rho_new", "rho_new"),                 # dropped gamma^T in beta
    ("oracle.bcg", "bcg", "gamma.T @ rho_new", "gamma @ rho_new"),         # missing transpose
    ("oracle.bcg", "bcg", "sigma = gamma @ sigma", "sigma = sigma @ gamma"),  # operand order
    ("oracle.bcg", "bcg", "Rt = Rb - Q @ lam", "Rt = Rb + Q @ lam"),       # sign
    ("oracle.bcg", "bcg", "X += P @ (lam @ sigma)", "X += P @ (sigma @ lam)"),
    ("oracle.bcg", "bcg", "X += P @ (lam @ sigma)", "X += P @ lam"),       # dropped sigma
    ("oracle.bcg", "bcg", "P = Z + P @ beta", "P = Z + P @ beta.T"),
    ("oracle.bcg", "bcg", "P = Z + P @ beta", "P = Rb + P @ beta"),        # dropped M^{-1}
    ("oracle.bcg", "bcg", "rho_new = gram(Z, Rb, p)", "rho_new = gram(Rb, Rb, p)"),
    ("oracle.bcg", "bcg", "rho = gram(P, Rb, p)", "rho = G"),              # rho^0 without M^{-1}
    ("oracle.bcg", "bcg", "G = None if reo else gram(Rb, Rb, p)",          # M^{-1}-norm residual
     "G = None if reo else gram(Rb if prec is None else prec(Rb), Rb, p)"),
    ("oracle.bcg", "bcg", "lam = chol_solve(alpha, rho)", "lam = chol_solve(rho, alpha)"),
    ("oracle.bcg", "_resid_from", "sigma.T @ G @ sigma", "sigma @ G @ sigma.T"),
]


def test_unmutated_bcg_passes_battery():
    assert _bcg_battery_passes(sys.modules["oracle.bcg"].bcg)


@pytest.mark.parametrize("mod,fn,old,new", BCG_MUTATIONS)
def test_bcg_mutation_is_caught(mod, fn, old, new, monkeypatch):
    m = _mutant(mod, fn, old, new)
    bmod = sys.modules["oracle.bcg"]
    if fn == "bcg":
        assert not _bcg_battery_passes(m)
    else:
        monkeypatch.setattr(bmod, fn, m)
        assert not _bcg_battery_passes(bmod.bcg)


def _bcg1r_battery_passes(fn):
    """1R-BCG against the 2R oracle (iterates), with and without Jacobi, and at s = 1."""
    try:
        bmod = sys.modules["oracle.bcg"]
        kf = np.exp(0.5 * np.random.default_rng(5).standard_normal(216))
        for A in (W.lap2d5(12, 11), W.diff3d7_var(6, 6, 6, kf)):
            B = W.normal_block(A.n, 4, 2)
            for eta in (0.0, math.inf):
                for w in (None, sys.modules["oracle.precond"].jacobi_inverse_diagonal(A)):
                    a = bmod.bcg(A, B, tol=0.0, maxit=8, eta=eta, Minv=w, record_iterates=8)
                    b = fn(A, B, tol=0.0, maxit=8, eta=eta, Minv=w, record_iterates=8)
                    for k in range(8):
                        if np.abs(b.iterates[k] - a.iterates[k]).max() > 1e-10 * np.abs(a.iterates[k]).max():
                            return False
        return True
    except Exception:
        return False


BCG1R_MUTATIONS = [
    ("alpha = delta - beta.T @ alpha @ beta", "alpha = delta + beta.T @ alpha @ beta"),
    ("alpha = delta - beta.T @ alpha @ beta", "alpha = delta - beta @ alpha @ beta.T"),
    ("Q = U + Q @ beta.astype(dtype)", "Q = U + Q @ beta.T.astype(dtype)"),
    ("U = op(Z)", "U = op(Rb)"),
    ("delta = gram(Z, U)", "delta = gram(Rb, U)"),
    ("rho_new = gram(Z, Rb)", "rho_new = gram(Rb, Rb)"),
    ("X += P @ (lam @ sigma_old)", "X += P @ (lam @ sigma)"),
]


def test_unmutated_bcg1r_passes_battery():
    assert _bcg1r_battery_passes(sys.modules["oracle.bcg"].bcg_1r)


@pytest.mark.parametrize("old,new", BCG1R_MUTATIONS)
def test_bcg1r_mutation_is_caught(old, new):
    assert not _bcg1r_battery_passes(_mutant("oracle.bcg", "bcg_1r", old, new))


def _replace_battery_passes(fn):
    """1R-BCG with the replacement of Q and alpha: after every iteration (replace = 1) the
    iterates are the 2R oracle's and every iteration counts; replace = 5 replaces after
    iterations 5 and 10 of 12 without moving the (well-conditioned, FP64) iterates."""
    try:
        bmod = sys.modules["oracle.bcg"]
        A = W.lap2d5(12, 11)
        B = W.normal_block(A.n, 4, 2)
        a = bmod.bcg(A, B, tol=0.0, maxit=12, eta=math.inf, record_iterates=12)
        for m, count in ((1, 12), (5, 2)):
            b = fn(A, B, tol=0.0, maxit=12, eta=math.inf, record_iterates=12, replace=m)
            if b.replacements != count:
                return False
            for k in range(12):
                if np.abs(b.iterates[k] - a.iterates[k]).max() > 1e-10 * np.abs(a.iterates[k]).max():
                    return False
        return True
    except Exception:
        return False


REPLACE_MUTATIONS = [
    ("Q = op(P)                                   # Q^{k+1} = A P^{k+1}",
     "Q = op(Z)                                   # Q^{k+1} = A P^{k+1}"),          # wrong operand
    ("alpha = gram(P, Q)                          # alpha^{k+1}", "alpha = gram(Q, Q)                          # alpha^{k+1}"),
    ("(k + 1) % replace == 0", "k % replace == 0"),                                  # off by one
    ("or not _chol_ok(alpha)", "and not _chol_ok(alpha)"),                           # trigger inverted
]


def test_unmutated_replacement_passes_battery():
    assert _replace_battery_passes(sys.modules["oracle.bcg"].bcg_1r)


@pytest.mark.parametrize("old,new", REPLACE_MUTATIONS)
def test_replacement_mutation_is_caught(old, new):
    assert not _replace_battery_passes(_mutant("oracle.bcg", "bcg_1r", old, new))


def _localized_battery_passes(cls):
    """Distributed S-QR = LAPACK QR of the concatenated blocks (signs fixed), 1, 5 and 8 tiles."""
    try:
        for n, s, tile in ((200, 3, 200), (200, 3, 40), (301, 4, 40)):
            g = np.random.default_rng(n + tile)
            blocks = [g.standard_normal((n, s)) for _ in range(4)]
            la = cls(n, s, tile)
            Xs = [la.extend(Wb)[0] for Wb in blocks]
            Q, R = np.linalg.qr(np.hstack(blocks))
            d = np.sign(np.diag(R))
            if np.abs(np.hstack(Xs) - Q * d).max() > 1e-11:
                return False
        return True
    except Exception:
        return False


LOCALIZED_MUTATIONS = [
    ("S[q] = S[q] - zi[q] @ ri", "S[q] = S[q] + zi[q] @ ri"),
    ("ri = sum(zi[q].T @ S[q] for q in range(len(ch)))", "ri = sum(zi[q].T @ S[q] for q in range(1))"),
    ("acc += _pad(comp[q], L) @ rt[ii * s:(ii + 1) * s]", "acc += _pad(comp[q], L) @ rt[:s]"),
    ("Wp = Wp - self.P[p][j] @ zj", "Wp = Wp - self.P[p][j] @ zj.T"),
    ("coef = list(self.node_basis[(top, 0)][-1])", "coef = list(self.node_basis[(top, 0)][0])"),
]


def test_unmutated_localized_passes_battery():
    assert _localized_battery_passes(sys.modules["oracle.localized"].LocalizedArnoldi)


@pytest.mark.parametrize("old,new", LOCALIZED_MUTATIONS)
def test_localized_mutation_is_caught(old, new):
    assert not _localized_battery_passes(_mutant("oracle.localized", "LocalizedArnoldi", old, new))


def _qr_battery_passes(qr_fn):
    try:
        for (n, s) in ((40, 6), (12, 12)):
            X = np.random.default_rng(n).standard_normal((n, s))
            Y, R = qr_fn(X)
            if np.abs(Y.T @ Y - np.eye(s)).max() > 1e-12 or np.abs(Y @ R - X).max() > 1e-12:
                return False
            if np.any(np.diag(R) < 0) or not np.allclose(np.tril(R, -1), 0):
                return False
        return True
    except Exception:
        return False


QR_MUTATIONS = [
    ("tau = (beta - alpha) / beta", "tau = (alpha - beta) / beta"),
    ("v = x / (alpha - beta)", "v = x / (beta - alpha)"),
    ("A[j:, j + 1:] -= tau * np.outer(v, w)", "A[j:, j + 1:] += tau * np.outer(v, w)"),
    ("Y[j:, :] -= taus[j] * np.outer(v, w)", "Y[j:, :] += taus[j] * np.outer(v, w)"),
    ("for j in range(s - 1, -1, -1):", "for j in range(s):"),
]


def test_unmutated_qr_passes_battery():
    assert _qr_battery_passes(sys.modules["oracle.blockops"].householder_qr)


@pytest.mark.parametrize("old,new", QR_MUTATIONS)
def test_qr_mutation_is_caught(old, new):
    assert not _qr_battery_passes(_mutant("oracle.blockops", "householder_qr", old, new))


def test_gram_mirror_mutation_is_caught():
    m = _mutant("oracle.blockops", "gram", "np.triu(G) + np.triu(G, 1).T", "np.triu(G) + np.triu(G, 1)")
    X = np.random.default_rng(0).integers(-5, 5, (9, 4)).astype(float)
    G = m(X, X)
    assert not np.array_equal(G, X.T @ X)


def _textbook_bicgstab(M, b, nrec):
    x = np.zeros_like(b); r = b.copy(); rt = r.copy(); p = r.copy(); rho = rt @ r; xs = []
    for _ in range(nrec):
        v = M @ p; a = rho / (rt @ v); s_ = r - a * v; t = M @ s_; w = (t @ s_) / (t @ t)
        x = x + a * p + w * s_; r = s_ - w * t; xs.append(x.copy())
        rho_new = rt @ r; p = r + (rho_new / rho) * (a / w) * (p - w * v); rho = rho_new
    return xs


def _bbicg_battery_passes(fn):
    try:
        A1 = W.const7(6, 5, 4, W.convdiff3d7_coeffs(5, pe=40.0))
        b = W.normal_block(A1.n, 1, 0)
        r = fn(A1, b, tol=1e-14, maxit=8, eta=0.0, record_iterates=8)
        xs = _textbook_bicgstab(A1.to_dense(), b[:, 0], 8)
        for k in range(8):
            if np.abs(r.iterates[k][:, 0] - xs[k]).max() > 1e-11 * np.abs(xs[k]).max():
                return False
        A = W.const7(7, 6, 5, W.convdiff3d7_coeffs(6))
        Ad = A.to_dense()
        B = W.normal_block(A.n, 3, 0)
        for eta in (0.0, math.inf, 100.0):
            r = fn(A, B, tol=1e-10, maxit=300, eta=eta)
            if not r.converged:
                return False
            true = np.linalg.norm(B - Ad @ r.X, axis=0) / np.linalg.norm(B, axis=0)
            if true.max() > 1e-9 or np.abs(true - r.relres).max() > 1e-9:
                return False
        # the normalised iteration commutes with every change of basis C of the
        # right-hand sides: X_k(B C) = X_k(B) C
        C = np.eye(3) * 2.0 + 0.5 * np.random.default_rng(7).standard_normal((3, 3))
        a = fn(A, B, tol=0.0, maxit=6, eta=math.inf, record_iterates=6)
        c = fn(A, B @ C, tol=0.0, maxit=6, eta=math.inf, record_iterates=6)
        for k in range(6):
            ref = a.iterates[k] @ C
            if np.abs(c.iterates[k] - ref).max() > 1e-10 * np.abs(ref).max():
                return False
        return True
    except Exception:
        return False


BBICG_MUTATIONS = [
    ("X += omega * (Th @ sigma_new)", "X += omega * (Th @ sigma)"),      # the printed sigma^k
    ("X += Ph @ (lam @ sigma)", "X += Ph @ (sigma @ lam)"),
    ("beta = -lu_solve", "beta = lu_solve"),
    ("Ph = Rh + (Ph - omega * Qh) @ beta", "Ph = Rh + (Ph + omega * Qh) @ beta"),  # the derivation's "+omega"
    ("omega = float(np.sum(Uh * Sh)) / uu", "omega = float(np.sum(Uh * Sh)) / uu ** 0.5"),
    ("gram(R0s, Uh, sym=False)", "gram(Uh, R0s, sym=False)"),   # transposed shadow Gram in beta
    ("gram(R0s, Rh, sym=False)", "gram(Rh, R0s, sym=False)"),   # transposed shadow Gram in lambda
    ("sigma_new = gamma @ sigma", "sigma_new = sigma @ gamma"),
]


def test_unmutated_bbicgstab_passes_battery():
    assert _bbicg_battery_passes(sys.modules["oracle.bbicgstab"].bbicgstab)


@pytest.mark.parametrize("old,new", BBICG_MUTATIONS)
def test_bbicgstab_mutation_is_caught(old, new):
    assert not _bbicg_battery_passes(_mutant("oracle.bbicgstab", "bbicgstab", old, new))


def _bgmres_battery_passes(fn):
    try:
        A = W.const7(6, 5, 5, W.convdiff3d7_coeffs(6))
        Ad = A.to_dense()
        B = W.normal_block(A.n, 3, 1)
        r = fn(A, B, tol=1e-10, restart=8, maxit=200)
        if not r.converged:
            return False
        true = np.linalg.norm(B - Ad @ r.X, axis=0) / np.linalg.norm(B, axis=0)
        if true.max() > 1e-9 or np.abs(true - r.relres).max() > 1e-9:
            return False
        # X_k - X_0 is the column-wise least-squares solution over K_k(A, R0)
        X0 = 0.1 * W.normal_block(A.n, 3, 2)
        R0 = B - Ad @ X0
        blocks = [R0]
        for k in range(1, 5):
            V, _ = np.linalg.qr(np.hstack(blocks))
            ref = X0 + V @ np.linalg.lstsq(Ad @ V, R0, rcond=None)[0]
            for ortho in ("mgs", "cgs2"):
                got = fn(A, B, X0=X0, tol=0.0, restart=8, maxit=k, ortho=ortho).X
                if np.abs(got - ref).max() > 1e-9 * np.abs(ref).max():
                    return False
            blocks.append(Ad @ blocks[-1])
        return True
    except Exception:
        return False


BGMRES_MUTATIONS = [
    ("h[j * s:(j + 2) * s] = G[j].T @ blk", "h[j * s:(j + 2) * s] = G[j] @ blk"),
    ("W = W - V[j] @ hj", "W = W + V[j] @ hj"),
    ("sig[k * s:(k + 2) * s] = Qk.T @ pair", "sig[k * s:(k + 2) * s] = Qk @ pair"),
    ("for j in range(l + 1, k_done):", "for j in range(l + 2, k_done):"),
    ("h[:(k + 1) * s] += hp", "h[:(k + 1) * s] = hp"),          # CGS2 drops the first pass's coefficients
    ("for j in range(k):", "for j in range(k - 1):"),            # one earlier Givens factor not applied
]


def test_unmutated_bgmres_passes_battery():
    assert _bgmres_battery_passes(sys.modules["oracle.bgmres"].bgmres)


@pytest.mark.parametrize("old,new", BGMRES_MUTATIONS)
def test_bgmres_mutation_is_caught(old, new):
    assert not _bgmres_battery_passes(_mutant("oracle.bgmres", "bgmres", old, new))


# ---------------------------------------------------------------------------
# TSQR tree (Ch. 7.3): Y and sigma of the tree equal one Householder QR.

def _tsqr_battery_passes(fn):
    try:
        X = np.random.default_rng(3).standard_normal((300, 6))
        Y1, s1 = sys.modules["oracle.blockops"].householder_qr(X)
        for parts, fanin in ((2, 2), (7, 2), (9, 3)):
            Y, sig = fn(X, parts, fanin)
            if np.abs(sig - s1).max() > 1e-12 * np.abs(s1).max() or np.abs(Y - Y1).max() > 1e-12:
                return False
        return True
    except Exception:
        return False


TSQR_MUTATIONS = [
    ("_reduce", "T = node_Q[gi] @ up[gi]", "T = node_Q[gi]"),                 # scatter factor not carried down
    ("_reduce", "out.append(T[j * s:(j + 1) * s])", "out.append(T[:s])"),
    ("_reduce", "Qg, Rg = householder_qr(np.vstack(g))", "Qg, Rg = householder_qr(np.vstack(g[::-1]))"),
    ("tsqr", "Qs[i] @ Y_parts[i]", "Qs[i] @ Y_parts[i].T"),
]


def _tsqr_with(fname, old, new):
    mod = sys.modules["oracle.tsqr"]
    m = _mutant("oracle.tsqr", fname, old, new)
    if fname == "tsqr":
        return m
    saved = mod._reduce
    def run(X, parts, fanin):
        mod._reduce = m
        try:
            return mod.tsqr(X, parts, fanin)
        finally:
            mod._reduce = saved
    return run


def test_unmutated_tsqr_passes_battery():
    assert _tsqr_battery_passes(sys.modules["oracle.tsqr"].tsqr)


@pytest.mark.parametrize("fname,old,new", TSQR_MUTATIONS)
def test_tsqr_mutation_is_caught(fname, old, new):
    assert not _tsqr_battery_passes(_tsqr_with(fname, old, new))


# ---------------------------------------------------------------------------
# kappa_D (Ch. 4.3): closed forms and invariance under diagonal scaling.

def _kappa_battery_passes(fn):
    try:
        if abs(fn(np.diag([1.0, 7.0, 1e-6])) - 1.0) > 1e-12:
            return False
        for c in (0.3, -0.9):
            M = np.array([[1.0, c], [c, 1.0]])
            D = np.diag([3.0, 0.01])
            ref = (1 + abs(c)) / (1 - abs(c))
            for A in (M, D @ M @ D):
                if abs(fn(A) - ref) > 1e-12 * ref:
                    return False
        # 3 x 3: the eigenvalues of the unit-diagonal matrix by LAPACK
        C = np.array([[1.0, 0.5, 0.2], [0.5, 1.0, -0.3], [0.2, -0.3, 1.0]])
        ev = np.linalg.eigvalsh(C)
        D = np.diag([2.0, 0.5, 7.0])
        return abs(fn(D @ C @ D) - ev[-1] / ev[0]) <= 1e-12 * ev[-1] / ev[0]
    except Exception:
        return False


KAPPA_MUTATIONS = [
    ("r = 1.0 / np.sqrt(d)", "r = 1.0 / d"),
    ("M = alpha * r[:, None] * r[None, :]", "M = alpha * r[:, None] * r[:, None]"),
    ("return float(ev[-1] / ev[0])", "return float(ev[-1] / ev[1])"),
]


def test_unmutated_kappa_passes_battery():
    assert _kappa_battery_passes(sys.modules["oracle.blockops"].kappa_d)


@pytest.mark.parametrize("old,new", KAPPA_MUTATIONS)
def test_kappa_mutation_is_caught(old, new):
    assert not _kappa_battery_passes(_mutant("oracle.blockops", "kappa_d", old, new))


# ---------------------------------------------------------------------------
# Iterative refinement: reaches 1e-10 in a few outer steps, from zero and from X0.

def _ir_battery_passes(fn):
    try:
        N = 6
        k = np.exp(1.0 * np.random.default_rng(1).standard_normal(N ** 3))
        A = W.diff3d7_var(N, N, N, k)
        B = W.normal_block(A.n, 3, 0)
        for X0 in (None, 0.3 * W.normal_block(A.n, 3, 5)):
            r = fn(A, B, tol=1e-10, inner_tol=1e-5, max_outer=6, X0=X0)
            true = np.linalg.norm(B - A.to_dense() @ r.X, axis=0) / np.linalg.norm(B, axis=0)
            if not r.converged or true.max() > 1e-10 or np.abs(true - r.relres).max() > 1e-12:
                return False
        # the first outer step from X0 is X0 plus the zero-start step on B - A X0
        X0 = 0.3 * W.normal_block(A.n, 3, 5)
        a = fn(A, B, tol=0.0, max_outer=1, inner_maxit=4, X0=X0)
        b = fn(A, B - A.to_dense() @ X0, tol=0.0, max_outer=1, inner_maxit=4)
        return np.abs(a.X - (X0 + b.X)).max() <= 1e-12 * np.abs(a.X).max()
    except Exception:
        return False


IR_MUTATIONS = [
    ("X += inner.X.astype(np.float64) * scale[None, :]", "X += inner.X.astype(np.float64)"),
    ("Rs = (R / scale[None, :])", "Rs = (R * scale[None, :])"),
    ("out.relres = np.where(nb > 0, nr / nb_safe, 0.0)", "out.relres = np.where(nb > 0, nr / nb_safe ** 2, 0.0)"),
    ("X = np.zeros((n, s)) if X0 is None else", "X = np.zeros((n, s)) if True else"),
]


def test_unmutated_ir_passes_battery():
    assert _ir_battery_passes(sys.modules["oracle.ir"].bcg_ir)


@pytest.mark.parametrize("old,new", IR_MUTATIONS)
def test_ir_mutation_is_caught(old, new):
    assert not _ir_battery_passes(_mutant("oracle.ir", "bcg_ir", old, new))


# ---------------------------------------------------------------------------
# Adjoint: every edge's theta-gradient against central differences on a 3 x 3
# grid, the CSR scatter against the dense dL/dA, and the dense adjoint on a
# non-symmetric matrix (where A^T != A) against central differences.

def _edge_fd_battery_passes(grad_fn, scatter_fn):
    try:
        nx = ny = 3; s = 2
        g = np.random.default_rng(8)
        thx = 0.4 * g.standard_normal((ny, nx + 1)); thy = 0.4 * g.standard_normal((ny + 1, nx))
        B = g.standard_normal((nx * ny, s)); Xt = g.standard_normal((nx * ny, s))
        oracle_mod = sys.modules["oracle.adjoint"]

        def loss(tx, ty):
            return oracle_mod.dense_adjoint(W.edge2d5(nx, ny, np.exp(tx), np.exp(ty)).to_dense(), B, Xt)

        L, X, Lam, dA = loss(thx, thy)
        gx, gy = grad_fn(nx, ny, np.exp(thx), np.exp(thy), Lam, X)
        h = 1e-6
        for arr, gr, is_x in ((thx, gx, True), (thy, gy, False)):
            for idx in np.ndindex(arr.shape):
                p = arr.copy(); p[idx] += h
                m = arr.copy(); m[idx] -= h
                fd = ((loss(p, thy) if is_x else loss(thx, p))[0]
                      - (loss(m, thy) if is_x else loss(thx, m))[0]) / (2 * h)
                if abs(gr[idx] - fd) > 1e-6 * abs(fd) + 1e-9:
                    return False
        Acsr = W.edge2d5(nx, ny, np.exp(thx), np.exp(thy))
        rows = np.repeat(np.arange(Acsr.n), np.diff(Acsr.row_ptr))
        return np.allclose(scatter_fn(Acsr, Lam, X), dA[rows, Acsr.col], rtol=1e-13, atol=1e-13)
    except Exception:
        return False


def _dense_adjoint_nonsym_passes(fn):
    try:
        A = W.const7(3, 3, 2, W.convdiff3d7_coeffs(3, pe=20.0)).to_dense()
        g = np.random.default_rng(2)
        B = g.standard_normal((A.shape[0], 2)); Xt = g.standard_normal(B.shape)
        L, X, Lam, dA = fn(A, B, Xt)
        h = 1e-6
        for (i, j) in ((0, 0), (0, 1), (1, 0), (5, 4), (4, 5)):
            p = A.copy(); p[i, j] += h
            m = A.copy(); m[i, j] -= h
            fd = (fn(p, B, Xt)[0] - fn(m, B, Xt)[0]) / (2 * h)
            if abs(dA[i, j] - fd) > 1e-6 * abs(fd) + 1e-9:
                return False
        for idx in ((0, 0), (7, 1)):
            p = B.copy(); p[idx] += h
            m = B.copy(); m[idx] -= h
            fd = (fn(A, p, Xt)[0] - fn(A, m, Xt)[0]) / (2 * h)
            if abs(Lam[idx] - fd) > 1e-6 * abs(fd) + 1e-9:
                return False
        return True
    except Exception:
        return False


EDGE_GRAD_MUTATIONS = [
    ("gx[:, nx] = -ax[:, nx] * np.sum(L3[:, nx - 1, :] * X3[:, nx - 1, :], axis=1)",
     "gx[:, nx] = -ax[:, nx] * np.sum(L3[:, nx - 2, :] * X3[:, nx - 1, :], axis=1)"),
    ("gy[ny, :] = -ay[ny, :] * np.sum(L3[ny - 1, :, :] * X3[ny - 1, :, :], axis=1)",
     "gy[ny, :] = -ay[ny, :] * np.sum(L3[ny - 1, :, :] * X3[ny - 2, :, :], axis=1)"),
    ("dl = L3[:, 1:, :] - L3[:, :-1, :]", "dl = L3[:, 1:, :] + L3[:, :-1, :]"),
    ("gy[1:ny, :] = -ay[1:ny, :]", "gy[1:ny, :] = ay[1:ny, :]"),
    ("gy[0, :] = -ay[0, :] * np.sum(L3[0, :, :] * X3[0, :, :], axis=1)",
     "gy[0, :] = -ay[0, :] * np.sum(L3[0, :, :] * X3[1, :, :], axis=1)"),
]
SCATTER_MUTATIONS = [
    ("Lam[rows], X[cols]", "Lam[cols], X[rows]"),
    ("return -np.einsum", "return np.einsum"),
]
DENSE_ADJOINT_MUTATIONS = [
    ("Lam = np.linalg.solve(Adense.T, G)", "Lam = np.linalg.solve(Adense, G)"),
    ("dA = -Lam @ X.T", "dA = -X @ Lam.T"),
]


def test_unmutated_adjoint_passes_batteries():
    mod = sys.modules["oracle.adjoint"]
    assert _edge_fd_battery_passes(mod.edge_theta_grad, mod.adjoint_scatter)
    assert _dense_adjoint_nonsym_passes(mod.dense_adjoint)


@pytest.mark.parametrize("old,new", EDGE_GRAD_MUTATIONS)
def test_edge_grad_mutation_is_caught(old, new):
    mod = sys.modules["oracle.adjoint"]
    m = _mutant("oracle.adjoint", "edge_theta_grad", old, new)
    assert not _edge_fd_battery_passes(m, mod.adjoint_scatter)


@pytest.mark.parametrize("old,new", SCATTER_MUTATIONS)
def test_scatter_mutation_is_caught(old, new):
    mod = sys.modules["oracle.adjoint"]
    m = _mutant("oracle.adjoint", "adjoint_scatter", old, new)
    assert not _edge_fd_battery_passes(mod.edge_theta_grad, m)


@pytest.mark.parametrize("old,new", DENSE_ADJOINT_MUTATIONS)
def test_dense_adjoint_mutation_is_caught(old, new):
    assert not _dense_adjoint_nonsym_passes(_mutant("oracle.adjoint", "dense_adjoint", old, new))


# ---- CholeskyQR2 (the fast normaliser) ----------------------------------------------
def _cholqr_battery_passes(fn):
    """Householder agreement, orthogonality and the decline test for a CholeskyQR2."""
    try:
        g = np.random.default_rng(11)
        for n, s, cond in ((300, 4, 1e2), (2000, 8, 1e4), (500, 1, 1.0)):
            U, _ = np.linalg.qr(g.standard_normal((n, s)))
            V, _ = np.linalg.qr(g.standard_normal((s, s)))
            X = (U * np.geomspace(1.0, 1.0 / cond, s)) @ V.T
            out = fn(X)
            if out is None:
                return False
            Y, R = out
            Yh, Rh = oracle.householder_qr(X)
            if np.abs(Y.T @ Y - np.eye(s)).max() > 1e-13 or np.abs(Y @ R - X).max() > 1e-13:
                return False
            if np.abs(R - Rh).max() > 1e-9 * np.abs(Rh).max():
                return False
        Xd = g.standard_normal((100, 4))
        Xd[:, 2] = Xd[:, 0] + Xd[:, 1]
        if fn(Xd) is not None:
            return False
        # a column at sine ~3e-6 from the span of the others: below the 1e-5 threshold,
        # declined although CholeskyQR2 would still factor it (kappa ~ 3e5)
        Xe = g.standard_normal((400, 4))
        Xe[:, 3] = Xe[:, 1] + 3e-6 * np.linalg.norm(Xe[:, 1]) * g.standard_normal(400) / 20.0
        if fn(Xe) is not None:
            return False
        return True
    except Exception:
        return False


CHOLQR_MUTATIONS = [
    ("return Y, R2 @ R1", "return Y, R1 @ R2"),                          # factors in the wrong order
    ("Y1 = np.linalg.solve(R1.T, X.T).T", "Y1 = np.linalg.solve(R1, X.T).T"),   # dropped transpose
    ("Y = np.linalg.solve(R2.T, Y1.T).T", "Y = Y1"),                     # second pass dropped
    ("if not (d > floor * G[j, j])", "if not (d > -1.0)"),             # decline test dropped
    ("R[j, c] = (G[j, c] - float(np.dot(R[:j, j], R[:j, c]))) / R[j, j]",
     "R[j, c] = (G[j, c] + float(np.dot(R[:j, j], R[:j, c]))) / R[j, j]"),   # sign of the update
]


def test_unmutated_cholqr_passes_battery():
    assert _cholqr_battery_passes(oracle.cholesky_qr2)


@pytest.mark.parametrize("old,new", CHOLQR_MUTATIONS)
def test_cholqr_mutation_is_caught(old, new):
    assert not _cholqr_battery_passes(_mutant("oracle.blockops", "cholesky_qr2", old, new))
