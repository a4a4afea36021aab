"""Pins of the oracle's randomized range finder (Algorithm 3, with V = Y in
Algorithm 2).

1. The sketch is X Omega for the K newest solutions of the run (newest
   first, including after the ring of K slots wraps around) and the Gaussian
   draws of the solve, built here from the recorded solutions with numpy.
2. With k = K, span(X Omega) = span(X) for any invertible Omega, so A x0 is
   the orthogonal projection of b onto span(A X): checked against
   numpy.linalg.lstsq over A X, which does not involve Omega at all.
3. A right-hand side whose solution lies in span(X) is solved by the guess,
   and GMRES takes no iterations (Theorem 4.1 with epsilon = 0).
4. On the linear Airy wave the range-finder guess needs fewer GMRES
   iterations per solve than the previous solution (the paper's baseline).
"""
import math

import numpy as np

import oracle as O
import workloads as W


def _problem(K, k, n_init=0, **kw):
    nx, nz, L = 16, 7, 2 * math.pi
    x = np.arange(nx) * (L / nx)
    h = 1.0 - 0.2 * np.exp(-2 * (x - 3) ** 2)
    P = O.OracleProblem(nx, 1, nz, L, 0.0, h, guess="rrf", k=k, history=K, n_init_solves=n_init, **kw)
    return P, x


def _system(P, x, seed):
    rng = np.random.default_rng(seed)
    e1 = 0.02 * np.sin(x + rng.uniform(0, 6))
    e2 = e1 + 0.002 * np.cos(x)
    b = rng.standard_normal(P.m)
    b[P.index(0, 0, P.nz - 1):] = 0.0
    return e1, e2, b


def test_sketch_is_x_times_omega_newest_first():
    K, k = 4, 3
    P, x = _problem(K, k, tol=1e-12, max_restarts=200)
    hist = []
    for s in range(7):
        if s > 0:
            Y = P.rrf_sketch()
            Ke = min(s, K)
            ke = min(k, Ke)
            Om = O.draw_omega(P.params.seed, s, K * k).reshape(K, k)
            X = np.column_stack(hist[::-1][:Ke])
            np.testing.assert_allclose(Y, X @ Om[:Ke, :ke], rtol=1e-13, atol=1e-13 * np.abs(X).max())
        e1, e2, b = _system(P, x, s)
        xs, st, code = P.solve(e1, e2, b)
        assert code == 0
        hist.append(xs.copy())


def test_full_sketch_guess_is_projection_onto_span():
    K = k = 4
    P, x = _problem(K, k, tol=1e-12, max_restarts=200)
    hist = []
    for s in range(K):
        e1, e2, b = _system(P, x, 20 + s)
        xs, st, code = P.solve(e1, e2, b)
        hist.append(xs.copy())
    e1, e2, b = _system(P, x, 99)
    P.assemble(e1, e2)
    A = P.matrix()
    x0, rank = P.rrf_guess(b)
    assert rank == k
    AX = np.column_stack([A @ h for h in hist])
    c, *_ = np.linalg.lstsq(AX, b, rcond=None)
    proj = AX @ c
    np.testing.assert_allclose(A @ x0, proj, rtol=1e-8, atol=1e-8 * np.abs(proj).max())


def test_solution_in_span_needs_no_iterations():
    K, k = 5, 5
    P, x = _problem(K, k, tol=1e-8, max_restarts=200)
    hist = []
    for s in range(K):
        e1, e2, b = _system(P, x, 40 + s)
        xs, st, code = P.solve(e1, e2, b)
        hist.append(xs.copy())
    e1, e2, _ = _system(P, x, 77)
    P.assemble(e1, e2)
    A = P.matrix()
    xt = np.column_stack(hist) @ np.array([0.3, -1.0, 0.5, 2.0, -0.7])
    b = A @ xt
    x0, rank = P.rrf_guess(b)
    assert np.linalg.norm(x0 - xt) <= 1e-8 * np.linalg.norm(xt)
    xs, st, code = P.solve(e1, e2, b)
    assert code == 0 and st["iterations"] == 0, st


def test_range_finder_beats_previous_solution_on_airy_wave():
    wl = W.airy_2d()
    its = {}
    for guess in ("previous", "rrf"):
        P = O.OracleProblem(wl["nx"], 1, wl["nz"], wl["lx"], 0.0, wl["h"], guess=guess, k=10, history=15,
                            n_init_solves=15)
        st = W.state_arrays(wl)
        n = 0
        for step in range(12):
            for i in range(1, 6):
                p, s, code = P.stage((wl["g"], wl["rho"], wl["dt"]), i, st)
                assert code == 0
                if step >= 4:
                    n += s["iterations"]
        its[guess] = n / 40
    assert its["rrf"] < 0.7 * its["previous"], its
