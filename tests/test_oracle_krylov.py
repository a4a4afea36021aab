"""Pins of the oracle's ILU(0) preconditioner and left-preconditioned GMRES (Sec. 3).

ILU(0): a dense textbook IKJ elimination restricted to the sparsity pattern,
written here in numpy, must give the same factors; L U must reproduce the
still-water matrix on its pattern; with no dropped fill (pattern = full)
ILU(0) is the exact LU.
GMRES: the solution matches numpy.linalg.solve; the residual estimate is
monotone within each cycle; after j steps from x0 = 0 the preconditioned
residual is the least-squares minimum over the Krylov space K_j(M^-1 A, M^-1 b)
computed here with numpy.linalg.lstsq; an exact initial guess costs 0 steps.
"""
import math

import numpy as np
import pytest

import oracle as O


def _problem(nx=8, nz=7, bar=False, **kw):
    L = 2 * math.pi
    x = np.arange(nx) * (L / nx)
    h = 1.0 - (0.3 * np.exp(-4 * (x - 3) ** 2) if bar else 0.0 * x)
    return O.OracleProblem(nx, 1, nz, L, 0.0, h, **kw), x


def _perm_matrix(P):
    """Still-water matrix renumbered in the factorisation order, from scratch."""
    P.assemble()
    A = P.matrix().toarray()
    LU = P.ilu_factors().toarray()
    return A, LU


def _colour_order(nx, ny, nz):
    order = []
    for c in range(4):
        for iy in range(ny):
            for ix in range(nx):
                if (ix + iy) % 4 == c:
                    order += [((j + 1) * ny + iy) * nx + ix for j in range(-1, nz)]
    return np.array(order)


def _dense_ilu0(B, pattern):
    n = B.shape[0]
    A = B.copy()
    for i in range(1, n):
        for k in range(i):
            if not pattern[i, k]:
                continue
            A[i, k] /= A[k, k]
            for j in range(k + 1, n):
                if pattern[i, j]:
                    A[i, j] -= A[i, k] * A[k, j]
    return A


@pytest.mark.parametrize("bar", [False, True])
def test_ilu0_matches_dense_ikj(bar):
    P, _ = _problem(bar=bar)
    A, LU = _perm_matrix(P)
    order = _colour_order(P.nx, 1, P.nz)
    B = A[np.ix_(order, order)]
    # structural pattern: the still-water stencil (box pattern over a bar)
    P2, _ = _problem(bar=bar)
    patt = np.zeros_like(B, dtype=bool)
    csr = P.ilu_factors()
    for i in range(B.shape[0]):
        patt[i, csr.indices[csr.indptr[i]:csr.indptr[i + 1]]] = True
    assert np.all(patt[np.abs(B) > 1e-12 * np.abs(B).max()])   # pattern covers A0
    ref = _dense_ilu0(B, patt)
    np.testing.assert_allclose(LU[patt], ref[patt], rtol=1e-11, atol=1e-11 * np.abs(ref).max())
    L = np.tril(LU, -1) + np.eye(B.shape[0])
    U = np.triu(LU)
    prod = L @ U
    np.testing.assert_allclose(prod[patt], B[patt], rtol=1e-10, atol=1e-10 * np.abs(B).max())


def test_ilu0_full_pattern_is_exact_lu():
    # a dense "pattern" keeps all fill: ILU(0) of a full matrix is LU, so M^-1 A = I
    P, _ = _problem()
    A, _ = _perm_matrix(P)
    order = _colour_order(P.nx, 1, P.nz)
    B = A[np.ix_(order, order)]
    full = np.ones_like(B, dtype=bool)
    LU = _dense_ilu0(B, full)
    L = np.tril(LU, -1) + np.eye(B.shape[0])
    U = np.triu(LU)
    np.testing.assert_allclose(L @ U, B, rtol=1e-10, atol=1e-10 * np.abs(B).max())


def test_ilu_apply_inverts_factors():
    P, _ = _problem(nx=12, nz=9, bar=True)
    A, LU = _perm_matrix(P)
    order = _colour_order(P.nx, 1, P.nz)
    L = np.tril(LU, -1) + np.eye(LU.shape[0])
    U = np.triu(LU)
    v = np.random.default_rng(0).standard_normal(P.m)
    out = P.ilu_apply(v)
    # M = P^T L U P in the natural numbering
    y = np.linalg.solve(U, np.linalg.solve(L, v[order]))
    ref = np.empty_like(y)
    ref[order] = y
    np.testing.assert_allclose(out, ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max())


def _system(nx=12, nz=9, bar=True, **kw):
    P, x = _problem(nx=nx, nz=nz, bar=bar, **kw)
    e1 = 0.03 * np.sin(x)
    e2 = 0.03 * np.sin(x + 0.1)
    P.assemble(e1, e2)
    A = P.matrix().toarray()
    b = np.random.default_rng(1).standard_normal(P.m)
    b[P.index(0, 0, P.nz - 1):] = 0.0      # surface rows
    return P, A, b


def test_gmres_converges_to_dense_solve():
    P, A, b = _system(tol=1e-13, max_restarts=400)
    x, st, code = P.gmres(b)
    assert code == 0 and st["converged"]
    ref = np.linalg.solve(A, b)
    assert np.linalg.norm(x - ref) <= 1e-9 * np.linalg.norm(ref)
    assert st["true_res"] < 1e-10


def test_gmres_residual_monotone_within_cycles():
    P, A, b = _system(tol=1e-12, max_restarts=200, restart=20)
    x, st, code, tr = P.gmres(b, trace=True)
    assert code == 0
    for c0 in range(0, len(tr), 20):
        seg = tr[c0:c0 + 20]
        assert np.all(np.diff(seg) <= 1e-12 * seg[0]), seg


@pytest.mark.parametrize("j", [1, 3, 7])
def test_gmres_minimises_over_krylov_space(j):
    P, A, b = _system(tol=1e-300, max_restarts=0, restart=j)
    x, st, code = P.gmres(b)
    assert st["iterations"] == j
    # explicit Krylov basis of M^-1 A from r0 = M^-1 b
    Mb = P.ilu_apply(b)
    K = np.zeros((P.m, j))
    v = Mb / np.linalg.norm(Mb)
    for q in range(j):
        K[:, q] = v
        v = P.ilu_apply(A @ v)
        v /= np.linalg.norm(v)
    MA_K = np.column_stack([P.ilu_apply(A @ K[:, q]) for q in range(j)])
    z, *_ = np.linalg.lstsq(MA_K, Mb, rcond=None)
    best = np.linalg.norm(Mb - MA_K @ z) / np.linalg.norm(Mb)
    assert abs(st["res_final"] - best) <= 1e-8 * max(best, 1e-300) + 1e-13
    np.testing.assert_allclose(x, K @ z, rtol=1e-6, atol=1e-8 * np.abs(K @ z).max())


def test_exact_guess_takes_no_iterations():
    P, A, b = _system()
    x_exact = np.linalg.solve(A, b)
    x, st, code = P.gmres(b, x0=x_exact)
    assert code == 0 and st["iterations"] == 0 and st["res0"] < 1e-8


def test_iteration_cap_reports_not_converged():
    P, A, b = _system(tol=1e-14, max_restarts=0, restart=2)
    x, st, code = P.gmres(b)
    assert code == -3 and not st["converged"] and st["iterations"] == 2
