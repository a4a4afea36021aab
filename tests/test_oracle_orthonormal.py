"""Pins of the oracle's optional orthonormalisation V = Q of the subspace
sketch (the QR step of Algorithms 3 and 4).

1. The basis is the Q of Y = Q R: orthonormal columns spanning span(Y), equal
   column by column up to sign to numpy.linalg.qr's Q for a full-rank Y.
2. A dependent column is dropped and the span of the rest is kept whole (a
   Householder QR without pivoting would lose part of a later column).
3. V = Q and V = Y span the same space, so for a well-conditioned sketch the
   guesses agree (EWMA and range finder), and both equal the projection of b
   onto span(A Y) computed by numpy.linalg.lstsq over A Q_numpy.
4. On a sketch whose columns are nearly dependent (EWMA with a small
   forgetting rate, condition ~1e8) the basis stays orthonormal to 1e-13,
   which one Gram-Schmidt pass would not give (it loses orthogonality like
   eps cond^2: 1.7e-4 on this sketch), and the guess from Q leaves a residual
   within rounding of the exact minimum over the span and of the guess from Y.
5. Full solves with V = Q converge like V = Y on the Airy wave.
"""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W


def test_basis_is_q_of_qr():
    rng = np.random.default_rng(1)
    Y = rng.standard_normal((300, 6)) @ np.triu(rng.uniform(0.5, 2.0, (6, 6)))
    Q, r = O.orth_basis(Y)
    assert r == 6
    np.testing.assert_allclose(Q.T @ Q, np.eye(6), atol=1e-14)
    Qn, Rn = np.linalg.qr(Y)
    sign = np.sign(np.diag(Rn))
    np.testing.assert_allclose(Q, Qn * sign, atol=1e-12)


def test_dependent_column_dropped_span_kept():
    rng = np.random.default_rng(2)
    y1, y2, y3 = rng.standard_normal((3, 200))
    Y = np.column_stack([y1, 2.0 * y1, y2, y1 - 3.0 * y2, y3])
    Q, r = O.orth_basis(Y)
    assert r == 3
    np.testing.assert_allclose(Q.T @ Q, np.eye(3), atol=1e-14)
    for y in (y1, y2, y3):
        np.testing.assert_allclose(Q @ (Q.T @ y), y, atol=1e-12 * np.abs(y).max())
    Q0, r0 = O.orth_basis(np.zeros((50, 3)))
    assert r0 == 0


def _problem(guess, orth, **kw):
    nx, nz, L = 16, 7, 2 * math.pi
    x = np.arange(nx) * (L / nx)
    h = 1.0 - 0.2 * np.exp(-2 * (x - 3) ** 2)
    P = O.OracleProblem(nx, 1, nz, L, 0.0, h, guess=guess, orthonormalize=orth, **kw)
    return P, x


def _system(P, x, seed):
    rng = np.random.default_rng(seed)
    e1 = 0.02 * np.sin(x + rng.uniform(0, 6))
    e2 = e1 + 0.002 * np.cos(x)
    b = rng.standard_normal(P.m)
    b[P.index(0, 0, P.nz - 1):] = 0.0
    return e1, e2, b


@pytest.mark.parametrize("guess", ["ewma", "rrf"])
def test_same_guess_as_v_equals_y(guess):
    K, k = 6, 4
    runs = {}
    for orth in (False, True):
        P, x = _problem(guess, orth, k=k, history=K, n_init_solves=0, decay=0.9, tol=1e-12, max_restarts=200)
        for s in range(K + 2):
            e1, e2, b = _system(P, x, 10 + s)
            _, _, code = P.solve(e1, e2, b)
            assert code == 0
        e1, e2, b = _system(P, x, 99)
        P.assemble(e1, e2)
        Y = P.sketch() if guess == "ewma" else P.rrf_sketch()
        x0, _ = P.ewma_guess(b) if guess == "ewma" else P.rrf_guess(b)
        runs[orth] = (x0, Y, P.matrix(), b)
    x0y, Y, A, b = runs[False]
    x0q, Yq, _, _ = runs[True]
    # the same history either way, up to the rounding of solves to 1e-12
    np.testing.assert_allclose(Yq, Y, rtol=0, atol=1e-10 * np.abs(Y).max())
    np.testing.assert_allclose(x0q, x0y, rtol=0, atol=1e-9 * np.abs(x0y).max())
    Qn, _ = np.linalg.qr(Y)
    c, *_ = np.linalg.lstsq(A @ Qn, b, rcond=None)
    np.testing.assert_allclose(A @ x0q, A @ (Qn @ c), rtol=0, atol=1e-9 * np.abs(b).max())


def test_nearly_dependent_sketch():
    # r = 0.05: the sketch is dominated by the newest solution times omega^T, nearly rank one
    P, x = _problem("ewma", False, k=6, decay=0.05, n_init_solves=0, tol=1e-12, max_restarts=200)
    for s in range(8):
        e1, e2, b = _system(P, x, 30 + s)
        P.solve(e1, e2, b)
    Y = P.sketch()
    sv = np.linalg.svd(Y, compute_uv=False)
    assert sv[0] / sv[-1] > 1e6                          # ill-conditioned columns
    e1, e2, b = _system(P, x, 77)
    P.assemble(e1, e2)
    A = P.matrix()
    xy, _ = P.ewma_guess(b)
    Q, r = O.orth_basis(Y)
    assert r == 6
    np.testing.assert_allclose(Q.T @ Q, np.eye(r), atol=1e-13)
    np.testing.assert_allclose(Q @ (Q.T @ Y), Y, atol=1e-12 * np.abs(Y).max())
    c, *_ = np.linalg.lstsq(A @ Q, b, rcond=None)
    best = np.linalg.norm(b - A @ (Q @ c))
    Pq, _ = _problem("ewma", True, k=6, decay=0.05, n_init_solves=0)
    Pq.assemble(e1, e2)
    Pq.set_sketch(Y)
    xq, _ = Pq.ewma_guess(b)
    rq = np.linalg.norm(b - A @ xq)
    ry = np.linalg.norm(b - A @ xy)
    assert rq <= best * (1 + 1e-8) + 1e-14 * np.linalg.norm(b), (rq, best)
    assert abs(rq - ry) <= 1e-8 * ry, (rq, ry)


def test_airy_run_converges_like_v_equals_y():
    wl = W.airy_2d()
    its = {}
    for orth in (False, True):
        P = O.OracleProblem(wl["nx"], 1, wl["nz"], wl["lx"], 0.0, wl["h"], guess="ewma", k=8, decay=0.9,
                            n_init_solves=10, orthonormalize=orth)
        st = W.state_arrays(wl)
        n = []
        for step in range(6):
            for i in range(1, 6):
                _, s, code = P.stage((wl["g"], wl["rho"], wl["dt"]), i, st)
                assert code == 0
                n.append(s["iterations"])
        its[orth] = np.array(n)
    assert np.all(np.abs(its[True] - its[False]) <= 1), its
