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


# ---- 3-D: the y-terms of the operator --------------------------------------
#
# 4. Still water on a flat bed, periodic x and y: A acting on
#    cos(kx x + ky y) g(sigma) equals (lambda(kx) + lambda(ky)) g + g''/h^2 with
#    the two directions' own grid spacings (nx != ny, lx != ly, so a transposed
#    index or a swapped spacing fails).
# 5. The 3-D manufactured solution: h, eta^(i-1), eta^(i) and p all vary in x
#    and y; sympy builds grad^(i) . grad^(i-1) p from the push-forward of
#    Eq. (9b) with sigma(x, y, z) of Eq. (8), and the ghost row from the bed
#    normal -(h_x, h_y, 1)/|.|.  Observed order as in 2-D.
# 6. A problem that varies only in y is the 2-D problem turned by 90 degrees:
#    the 3-D rows must equal the 2-D oracle's rows along y (same spacing,
#    same depth profile), value for value.  This reaches every y-coefficient
#    (sigma_y at both stages, its chi- and sigma-derivatives, the mixed
#    D_gamma D_sigma term and the ghost row's h_y terms).

def test_flat_still_water_fourier_symbol_3d():
    nx, ny, nz, lx, ly, H = 16, 12, 9, 2 * math.pi, 3.0, 0.8
    P = O.OracleProblem(nx, ny, nz, lx, ly, np.full(nx * ny, H))
    P.assemble()
    A = P.matrix()
    x = np.arange(nx) * (lx / nx)
    y = np.arange(ny) * (ly / ny)
    X, Y = np.meshgrid(x, y, indexing="xy")
    X, Y = X.ravel(), Y.ravel()
    s = _sig(nz)
    dx, dy = lx / nx, ly / ny

    def lam(th, d):
        return (2 * 2 * math.cos(3 * th) - 27 * 2 * math.cos(2 * th) + 270 * 2 * math.cos(th) - 490) / (180 * d * d)

    for ix_, iy_ in [(0, 1), (1, 0), (2, 3), (5, 4)]:
        kx, ky = 2 * math.pi * ix_ / lx, 2 * math.pi * iy_ / ly
        lx_, ly_ = lam(kx * dx, dx), lam(ky * dy, dy)
        ph = np.cos(kx * X + ky * Y)
        for q in (0, 2, 5, 6):
            g = s ** q
            g1 = q * s ** (q - 1) if q >= 1 else 0 * s
            g2 = q * (q - 1) * s ** (q - 2) if q >= 2 else 0 * s
            p = (g[:, None] * ph[None, :]).ravel()
            yv = (A @ p).reshape(nz + 1, nx * ny)
            expect = ((lx_ + ly_) * g + g2 / H ** 2)[:, None] * ph[None, :]
            scale = max(1.0, np.abs(expect).max())
            np.testing.assert_allclose(yv[1:nz], expect[1:nz], atol=1e-9 * scale)
            np.testing.assert_allclose(yv[nz], p.reshape(nz + 1, -1)[nz], atol=1e-14)
            ghost = -(g1[1] / H) * ph
            np.testing.assert_allclose(yv[0], ghost, atol=1e-9 * max(1.0, abs(ghost).max()))


_Y = sp.symbols("Y", real=True)
_H3 = 1.0 + 0.1 * sp.cos(_X) + 0.08 * sp.sin(_Y) + 0.04 * sp.cos(_X - _Y)
_E13 = 0.05 * sp.sin(2 * _X) + 0.03 * sp.cos(_Y + 0.2) + 0.02 * sp.sin(_X + _Y)
_E23 = 0.05 * sp.sin(2 * _X + 0.3) + 0.04 * sp.cos(_Y - 0.4) + 0.02 * sp.cos(_X - 2 * _Y)
_P3 = sp.cos(_X) * sp.cosh(_S) + _S ** 3 - _S * sp.sin(_X) ** 2 + sp.cos(_Y) * sp.sinh(_S) \
    + _S ** 2 * sp.sin(_X + 2 * _Y)


def _pushforward_coefs_3d(eta):
    """sigma_x, sigma_y, sigma_z of Eq. (8)-(9b) as functions of (chi, gamma, sigma)."""
    sig = (_Z + _H3) / (_H3 + eta)
    zs = _S * (_H3 + eta) - _H3
    return tuple(sp.diff(sig, v).subs(_Z, zs) for v in (_X, _Y, _Z))


_MAN3 = None


def _manufactured_3d():
    sx1, sy1, sz1 = _pushforward_coefs_3d(_E13)
    sx2, sy2, sz2 = _pushforward_coefs_3d(_E23)
    # grad^(i-1) p, then grad^(i) . (that field), in (chi, gamma, sigma)
    V1 = sp.diff(_P3, _X) + sx1 * sp.diff(_P3, _S)
    V2 = sp.diff(_P3, _Y) + sy1 * sp.diff(_P3, _S)
    V3 = sz1 * sp.diff(_P3, _S)
    Lp = (sp.diff(V1, _X) + sx2 * sp.diff(V1, _S) + sp.diff(V2, _Y) + sy2 * sp.diff(V2, _S)
          + sz2 * sp.diff(V3, _S))
    hx, hy = sp.diff(_H3, _X), sp.diff(_H3, _Y)
    nrm = 1 / sp.sqrt(1 + hx ** 2 + hy ** 2)
    ghost = (-nrm * (hx * V1 + hy * V2 + V3)).subs(_S, 0)
    args = (_X, _Y, _S)
    return (sp.lambdify(args, Lp, "numpy"), sp.lambdify((_X, _Y), ghost, "numpy"),
            [sp.lambdify((_X, _Y), e, "numpy") for e in (_H3, _E13, _E23)], sp.lambdify(args, _P3, "numpy"))


def _errors_3d(n, nz):
    global _MAN3
    if _MAN3 is None:
        _MAN3 = _manufactured_3d()
    f, gfun, (hf, e1f, e2f), pf = _MAN3
    L = 2 * math.pi
    x = np.arange(n) * (L / n)
    X, Yg = np.meshgrid(x, x, indexing="xy")
    X, Yg = X.ravel(), Yg.ravel()
    s = _sig(nz)
    one = np.ones(X.size)
    P = O.OracleProblem(n, n, nz, L, L, hf(X, Yg) * one)
    P.assemble(e1f(X, Yg) * one, e2f(X, Yg) * one)
    p = (pf(X[None, :], Yg[None, :], s[:, None]) * np.ones((nz + 1, 1))).ravel()
    yv = P.matvec(p).reshape(nz + 1, n * n)
    exact = f(X[None, :], Yg[None, :], s[:, None]) * np.ones((nz + 1, X.size))
    err_rows = np.abs(yv - exact).max(axis=1)
    centred = [j + 1 for j in range(2, nz - 3)]
    interior = list(range(1, nz))
    eg = np.abs(yv[0] - gfun(X, Yg) * one).max()
    return err_rows[centred].max(), err_rows[interior].max(), eg


def test_manufactured_convergence_order_3d():
    res = [_errors_3d(16 * 2 ** q, 8 * 2 ** q + 1) for q in range(3)]
    e_c = [r[0] for r in res]
    e_i = [r[1] for r in res]
    e_g = [r[2] for r in res]
    ord_c = [math.log2(e_c[q] / e_c[q + 1]) for q in range(2)]
    ord_i = [math.log2(e_i[q] / e_i[q + 1]) for q in range(2)]
    ord_g = [math.log2(e_g[q] / e_g[q + 1]) for q in range(2)]
    assert e_c[-1] < 1e-5 and e_i[-1] < 1e-4, res
    assert ord_c[-1] > 5.5, (ord_c, res)
    assert ord_i[-1] > 4.5, (ord_i, res)
    assert ord_g[-1] > 4.5, (ord_g, res)


def test_y_only_problem_is_the_2d_problem_turned():
    # depth, both surfaces and the unknown vary along y only; nx columns in x are copies
    nx, ny, nz, L = 8, 24, 9, 2 * math.pi
    yv = np.arange(ny) * (L / ny)
    h1 = 1.0 + 0.15 * np.cos(yv) + 0.05 * np.sin(2 * yv)
    ep1 = 0.04 * np.sin(yv + 0.3)
    ec1 = 0.04 * np.sin(yv + 0.45) + 0.01 * np.cos(3 * yv)
    rng = np.random.default_rng(3)
    p2 = rng.standard_normal((nz + 1, ny))
    Q = O.OracleProblem(ny, 1, nz, L, 0.0, h1)
    Q.assemble(ep1, ec1)
    y2 = Q.matvec(p2.ravel()).reshape(nz + 1, ny)
    rep = lambda a: np.repeat(a[:, None], nx, axis=1).ravel()     # (iy, ix) layout, x fastest
    P = O.OracleProblem(nx, ny, nz, L, L, rep(h1))
    assert P.box
    P.assemble(rep(ep1), rep(ec1))
    p3 = np.repeat(p2[:, :, None], nx, axis=2).ravel()
    y3 = P.matvec(p3).reshape(nz + 1, ny, nx)
    scale = np.abs(y2).max()
    for ix in range(nx):
        np.testing.assert_allclose(y3[:, :, ix], y2, rtol=0, atol=1e-12 * scale)
    # and the x-only problem is the 2-D problem itself
    P = O.OracleProblem(ny, nx, nz, L, L, np.tile(h1, nx))
    P.assemble(np.tile(ep1, nx), np.tile(ec1, nx))
    p3 = np.repeat(p2[:, None, :], nx, axis=1).ravel()
    y3 = P.matvec(p3).reshape(nz + 1, nx, ny)
    for iy in range(nx):
        np.testing.assert_allclose(y3[:, iy, :], y2, rtol=0, atol=1e-12 * scale)
