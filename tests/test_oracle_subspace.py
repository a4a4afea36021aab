"""Pins of the oracle's subspace acceleration (Algorithms 2 and 4, Sec. 4).

- SplitMix64 reproduces the published reference outputs for seed 0.
- The Gaussian draws have mean 0 and variance 1 (statistical check).
- The least-squares solve by Householder QR agrees with numpy.linalg.lstsq, also
  for a rank-deficient basis (compared by residual, the unique quantity).
- After n rank-1 updates Y equals the closed-form weighted sum
  sum_l r^(n-1-l) x_l omega_l^T printed under Algorithm 4.
- When the solution lies in span(Y) the guess is exact and GMRES takes no
  step (Theorem 4.1 with epsilon = 0).
- Fischer's special case (Sec. 4): with A fixed and V = [x_1 .. x_K], A x0
  is the orthogonal projection of b onto span(b_1 .. b_K).
"""
import math

import numpy as np
import pytest

import oracle as O


def test_splitmix64_reference_outputs():
    # first outputs of SplitMix64 seeded with 0 (Steele, Lea & Flood 2014 reference code)
    assert O.splitmix64(0, 1) == 0xE220A8397B1DCDAF
    assert O.splitmix64(0, 2) == 0x6E789E6AA1B965F4
    assert O.splitmix64(0, 3) == 0x06C45D188009454F


def test_gaussian_draws_moments():
    w = np.concatenate([O.draw_omega(2511, s, 16) for s in range(4000)])
    assert abs(w.mean()) < 0.02 and abs(w.var() - 1.0) < 0.03
    # deterministic in (seed, solve index), distinct across solves
    np.testing.assert_array_equal(O.draw_omega(7, 5, 10), O.draw_omega(7, 5, 10))
    assert not np.allclose(O.draw_omega(7, 5, 10), O.draw_omega(7, 6, 10))


def test_lstsq_qr_matches_numpy():
    rng = np.random.default_rng(3)
    W = rng.standard_normal((300, 10))
    b = rng.standard_normal(300)
    z, rank = O.lstsq_qr(W, b)
    ref, *_ = np.linalg.lstsq(W, b, rcond=None)
    assert rank == 10
    np.testing.assert_allclose(z, ref, rtol=1e-11, atol=1e-12)


def test_lstsq_qr_rank_deficient_residual():
    rng = np.random.default_rng(4)
    W = rng.standard_normal((200, 6))
    W = np.column_stack([W, W[:, 1] + W[:, 2], 2 * W[:, 0]])
    b = rng.standard_normal(200)
    z, rank = O.lstsq_qr(W, b)
    ref, *_ = np.linalg.lstsq(W, b, rcond=None)
    assert rank == 6
    assert abs(np.linalg.norm(W @ z - b) - np.linalg.norm(W @ ref - b)) < 1e-10 * np.linalg.norm(b)


def _problem(k=4, decay=0.8, **kw):
    nx, nz, L = 16, 7, 2 * math.pi
    x = np.arange(nx) * (L / nx)
    h = 1.0 + 0.1 * np.cos(x)
    return O.OracleProblem(nx, 1, nz, L, 0.0, h, k=k, decay=decay, **kw), x


def test_ewma_rank1_updates_equal_closed_form():
    k, r = 5, 0.7
    P, _ = _problem(k=k, decay=r)
    rng = np.random.default_rng(5)
    xs = [rng.standard_normal(P.m) for _ in range(9)]
    for s, xv in enumerate(xs):
        P.ewma_update(xv, s)
    n = len(xs)
    closed = sum(r ** (n - 1 - l) * np.outer(xs[l], O.draw_omega(2511, l, k)) for l in range(n))
    np.testing.assert_allclose(P.sketch(), closed, rtol=1e-13, atol=1e-13 * np.abs(closed).max())


def test_guess_exact_when_solution_in_span():
    k = 4
    P, x = _problem(k=k, tol=1e-8)
    rng = np.random.default_rng(6)
    Y = rng.standard_normal((P.m, k))
    P.set_sketch(Y)
    P.assemble(0.02 * np.sin(x), 0.02 * np.sin(x + 0.2))
    A = P.matrix()
    c = rng.standard_normal(k)
    b = A @ (Y @ c)
    x0, rank = P.ewma_guess(b)
    assert rank == k
    np.testing.assert_allclose(x0, Y @ c, rtol=1e-9, atol=1e-10 * np.abs(Y @ c).max())
    xs, st, code = P.gmres(b, x0=x0)
    assert code == 0 and st["iterations"] == 0


def test_fischer_projection_special_case():
    K = 5
    P, x = _problem(k=K)
    P.assemble(0.02 * np.sin(x), 0.02 * np.sin(x))   # one fixed matrix A
    A = P.matrix()
    rng = np.random.default_rng(7)
    X = rng.standard_normal((P.m, K))        # previous solutions, V = X
    B = A @ X                                # their right-hand sides
    P.set_sketch(X)
    b = rng.standard_normal(P.m)
    x0, rank = P.ewma_guess(b)
    z, *_ = np.linalg.lstsq(B, b, rcond=None)
    proj = B @ z                             # orthogonal projection of b onto range(B)
    np.testing.assert_allclose(A @ x0, proj, rtol=1e-9, atol=1e-10 * np.abs(proj).max())


def test_solve_guess_modes_and_history():
    # EWMA mode runs the previous-solution guess during the first n_init solves
    P, x = _problem(k=3, guess="ewma", n_init_solves=2)
    rng = np.random.default_rng(8)
    e0 = 0.01 * np.sin(x)
    xs = []
    for s in range(4):
        e1 = 0.01 * np.sin(x + 0.05 * (s + 1))
        b = rng.standard_normal(P.m)
        b[P.index(0, 0, P.nz - 1):] = 0
        xv, st, code = P.solve(e0, e1, b)
        assert code == 0
        xs.append(xv)
        e0 = e1
    assert P.solve_count == 4
    closed = sum(0.8 ** (3 - l) * np.outer(xs[l], O.draw_omega(2511, l, 3)) for l in range(4))
    np.testing.assert_allclose(P.sketch(), closed, rtol=1e-12, atol=1e-12 * np.abs(closed).max())
