"""Pins of the oracle's discrete operator A(eta_prev, eta_cur) (Eq. 16-18).

1. Still water, flat bed, periodic x: A acting on cos(k x) g(sigma), g a
   polynomial of degree <= 6, equals (lambda(k) g + g''/h^2) cos(k x) with the
   Fourier symbol lambda(k) of the centred 7-point second difference, written
   out here from the textbook weights.  The ghost row equals -(1/h) g'(0) cos(kx).
2. General geometry: the mixed-stage operator grad^(i) . grad^(i-1) p is built
   in sympy directly from the push-forward of Eq. (9b) and the transform of
   Eq. (8) (sympy differentiates sigma(x, z) = (z+h)/(h+eta) itself; no
   hand-expanded coefficient is typed here), and the discrete rows must
   converge to it at the order of the stencils: 6 where the sigma stencil is
   centred, at least 5 next to bed and surface.
3. With eta_prev = eta_cur the operator is the physical Laplacian, which
   vanishes on the harmonic function cosh(k(z+1)) cos(k x).
"""
import math

import numpy as np
import pytest
import sympy as sp

import oracle as O


def _sig(nz):
    return np.arange(-1, nz) / (nz - 1.0)


def test_flat_still_water_fourier_symbol():
    nx, nz, L, H = 32, 9, 2 * math.pi, 0.7
    P = O.OracleProblem(nx, 1, nz, L, 0.0, np.full(nx, H))
    P.assemble()
    A = P.matrix()
    x = np.arange(nx) * (L / nx)
    s = _sig(nz)
    dx = L / nx
    for kk in [0, 1, 3, 7]:
        k = 2 * math.pi * kk / L
        th = k * dx
        lam = (2 * 2 * math.cos(3 * th) - 27 * 2 * math.cos(2 * th) + 270 * 2 * math.cos(th) - 490) / (180 * dx * dx)
        for q in range(7):
            g = s ** q
            g1 = q * s ** (q - 1) if q >= 1 else 0 * s
            g2 = q * (q - 1) * s ** (q - 2) if q >= 2 else 0 * s
            p = (g[:, None] * np.cos(k * x)[None, :]).ravel()
            y = (A @ p).reshape(nz + 1, nx)
            expect = (lam * g + g2 / H ** 2)[:, None] * np.cos(k * x)[None, :]
            scale = max(1.0, np.abs(expect).max())
            np.testing.assert_allclose(y[1:nz], expect[1:nz], atol=1e-9 * scale)   # interior rows
            np.testing.assert_allclose(y[nz], p.reshape(nz + 1, nx)[nz], atol=1e-14)  # surface: identity
            ghost = -(g1[1] / H) * np.cos(k * x)                                     # sigma = 0 is level index 1
            np.testing.assert_allclose(y[0], ghost, atol=1e-9 * max(1.0, abs(ghost).max()))


# ---- manufactured solution built from the definitions of the transform ----

_X, _S, _Z = sp.symbols("X S Z", real=True)
_H = 1.0 + 0.1 * sp.cos(_X)
_E1 = 0.05 * sp.sin(2 * _X)
_E2 = 0.05 * sp.sin(2 * _X + 0.3)
_P = sp.cos(_X) * sp.cosh(_S) + _S ** 3 - _S * sp.sin(_X) ** 2


def _pushforward_coefs(eta):
    """sigma_x and sigma_z of Eq. (8)-(9b) as functions of (chi, sigma)."""
    sig = (_Z + _H) / (_H + eta)
    sx = sp.diff(sig, _X)
    sz = sp.diff(sig, _Z)
    zs = _S * (_H + eta) - _H
    return sp.simplify(sx.subs(_Z, zs)), sp.simplify(sz.subs(_Z, zs))


def _manufactured():
    sx1, sz1 = _pushforward_coefs(_E1)
    sx2, sz2 = _pushforward_coefs(_E2)
    V1 = sp.diff(_P, _X) + sx1 * sp.diff(_P, _S)
    V2 = sz1 * sp.diff(_P, _S)
    Lp = sp.diff(V1, _X) + sx2 * sp.diff(V1, _S) + sz2 * sp.diff(V2, _S)
    hx = sp.diff(_H, _X)
    nrm = 1 / sp.sqrt(1 + hx ** 2)
    ghost = (-nrm * (hx * V1 + V2)).subs(_S, 0)
    f = sp.lambdify((_X, _S), Lp, "numpy")
    gfun = sp.lambdify((_X,), ghost, "numpy")
    return f, gfun, [sp.lambdify((_X,), e, "numpy") for e in (_H, _E1, _E2)], sp.lambdify((_X, _S), _P, "numpy")


_MAN = None


def _errors(nx, nz):
    global _MAN
    if _MAN is None:
        _MAN = _manufactured()
    f, gfun, (hf, e1f, e2f), pf = _MAN
    L = 2 * math.pi
    x = np.arange(nx) * (L / nx)
    s = _sig(nz)
    P = O.OracleProblem(nx, 1, nz, L, 0.0, hf(x) * np.ones(nx))
    P.assemble(e1f(x) * np.ones(nx), e2f(x) * np.ones(nx))
    A = P.matrix()
    p = pf(x[None, :], s[:, None]).ravel()
    y = (A @ p).reshape(nz + 1, nx)
    exact = f(x[None, :], s[:, None]) * np.ones((nz + 1, nx))
    err_rows = np.abs(y - exact).max(axis=1)
    centred = [j + 1 for j in range(2, nz - 3)]
    interior = list(range(1, nz))
    eg = np.abs(y[0] - gfun(x) * np.ones(nx)).max()
    return err_rows[centred].max(), err_rows[interior].max(), eg


def test_manufactured_convergence_order():
    res = [_errors(16 * 2 ** q, 8 * 2 ** q + 1) for q in range(3)]
    e_c = [r[0] for r in res]
    e_i = [r[1] for r in res]
    e_g = [r[2] for r in res]
    ord_c = [math.log2(e_c[q] / e_c[q + 1]) for q in range(2)]
    ord_i = [math.log2(e_i[q] / e_i[q + 1]) for q in range(2)]
    ord_g = [math.log2(e_g[q] / e_g[q + 1]) for q in range(2)]
    assert e_c[-1] < 1e-6 and e_i[-1] < 1e-5, res
    assert ord_c[-1] > 5.5, (ord_c, res)
    assert ord_i[-1] > 4.5, (ord_i, res)
    assert ord_g[-1] > 4.5, (ord_g, res)


def test_same_geometry_is_physical_laplacian():
    # harmonic P = cosh(k (z + 1)) cos(k x) with z = sigma d - h
    nx, nz, L = 64, 33, 2 * math.pi
    k = 1.0
    x = np.arange(nx) * (L / nx)
    h = 1.0 + 0.1 * np.cos(x)
    eta = 0.05 * np.sin(2 * x)
    P = O.OracleProblem(nx, 1, nz, L, 0.0, h)
    P.assemble(eta, eta)
    A = P.matrix()
    s = _sig(nz)
    z = s[:, None] * (h + eta)[None, :] - h[None, :]
    p = (np.cosh(k * (z + 1)) * np.cos(k * x)[None, :]).ravel()
    y = (A @ p).reshape(nz + 1, nx)
    assert np.abs(y[1:nz]).max() < 1e-5


def test_dense_matrix_structure_3d():
    # 3-D flat bed still water: interior row = D2x + D2y + D2s/h^2 only (19-point cross).
    nx = ny = 8
    nz = 7
    P = O.OracleProblem(nx, ny, nz, 2 * math.pi, 2 * math.pi, np.full(nx * ny, 1.0))
    assert not P.box
    P.assemble()
    A = P.matrix()
    r = P.index(3, 4, 3)
    row = A[r].toarray().ravel()
    # D_chi of a constant depth is zero up to rounding of the weights
    assert np.count_nonzero(np.abs(row) > 1e-12 * np.abs(row).max()) == 19
    # the preconditioner keeps only that cross pattern: ILU rows have 19 entries
    assert np.diff(P.ilu_factors().indptr).max() == 19
    eta = 0.01 * np.cos(np.arange(nx * ny) * 0.7)
    P.assemble(np.zeros(nx * ny), eta)
    assert np.count_nonzero(P.matrix()[r].toarray()) == 91
