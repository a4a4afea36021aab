"""Pins of the oracle's wall-bounded flume: walls with ghost columns, the
seven-group factorisation order, and the generation/absorption zones.

1. Still water over a flat bed: the off-centred 7-point x stencils next to
   the walls are exact on polynomials of degree <= 6, so A acting on
   x^a sigma^b (a, b <= 6) equals p_xx + p_ss/h^2 on every PDE row, n . grad p
   = +-p_x at the wall node on the ghost-column rows, -p_s/h on the bed rows.
2. General geometry: rows converge to the continuous operator built in
   sympy from the transform (same construction as the periodic pin), now with
   the wall rows n . grad^(i-1) p at the wall nodes.
3. ILU(0) in the seven-group order equals a dense IKJ elimination on the
   pattern; no two columns of one group are coupled (which lets a device sweep
   a whole group at once); GMRES reaches the dense solution.
4. A closed basin one wavelength long, started at rest from a cos(kx), is a
   standing wave: after half a period the surface is -a cos(kx), after a full
   period a cos(kx) again (linear theory), within 1 % of a; the volume under
   the surface is conserved (no flux through the walls).
5. Relaxation zones: weight Gamma(0) = 1, Gamma(1) = 0, monotone; the linear
   dispersion relation is solved to rounding; a flume driven by the
   generation zone carries the incident linear wave between the zones with
   the right amplitude and phase, and the absorption zone removes it.
"""
import math

import numpy as np
import pytest
import sympy as sp

import oracle as O
import workloads as W


def _sig(nz):
    return np.arange(-1, nz) / (nz - 1.0)


def _wall_problem(nx, nz, lx, h, **kw):
    return O.OracleProblem(nx, 1, nz, lx, 0.0, h, walls=True, **kw)


# ---- 1. exactness on polynomials ----

@pytest.mark.parametrize("ab", [(0, 0), (1, 0), (2, 3), (3, 1), (6, 0), (4, 2), (0, 6), (1, 5), (5, 1), (6, 6)])
def test_flat_still_water_exact_on_polynomials(ab):
    a, b = ab
    nx, nz, lx, H = 20, 9, 1.0, 0.7
    P = _wall_problem(nx, nz, lx, np.full(nx, H))
    x = P.xcoord()
    np.testing.assert_allclose(x[1], 0.0, atol=0)
    np.testing.assert_allclose(x[-2], lx, rtol=1e-15)
    P.assemble()
    A = P.matrix()
    s = _sig(nz)
    X, S = x[None, :], s[:, None]

    def mono(e, v):
        return e * v ** (e - 1) if e >= 1 else 0 * v

    def mono2(e, v):
        return e * (e - 1) * v ** (e - 2) if e >= 2 else 0 * v

    p = (X ** a * S ** b) * np.ones((nz + 1, nx))
    y = (A @ p.ravel()).reshape(nz + 1, nx)
    scale = max(1.0, np.abs(p).max()) * (nx - 3) ** 2
    lap = mono2(a, X) * S ** b + X ** a * mono2(b, S) / H ** 2
    phys = slice(1, nx - 1)
    np.testing.assert_allclose(y[1:nz, phys], lap[1:nz, phys], atol=1e-11 * scale)        # PDE rows
    bed = -(X ** a * mono(b, np.zeros_like(X))) / H
    np.testing.assert_allclose(y[0, phys], bed[0, phys], atol=1e-11 * scale)              # bed rows
    np.testing.assert_allclose(y[nz], p[nz], atol=1e-14)                                   # surface rows
    for ig, iw, sgn in [(0, 1, -1.0), (nx - 1, nx - 2, 1.0)]:                             # wall rows
        want = sgn * mono(a, x[iw]) * s[:nz] ** b
        np.testing.assert_allclose(y[:nz, ig], want, atol=1e-11 * scale)


# ---- 2. convergence to the continuous operator ----

_X, _S, _Z = sp.symbols("X S Z", real=True)
_H = 1.0 + 0.1 * sp.cos(_X)
_E1 = 0.05 * sp.sin(2 * _X)
_E2 = 0.05 * sp.sin(2 * _X + 0.3)
_P = sp.cos(_X) * sp.cosh(_S) + _S ** 3 - _S * sp.sin(_X) ** 2 + 0.2 * _X * _S


def _coefs(eta):
    sig = (_Z + _H) / (_H + eta)
    zs = _S * (_H + eta) - _H
    return sp.simplify(sp.diff(sig, _X).subs(_Z, zs)), sp.simplify(sp.diff(sig, _Z).subs(_Z, zs))


def _manufactured():
    sx1, sz1 = _coefs(_E1)
    sx2, sz2 = _coefs(_E2)
    V1 = sp.diff(_P, _X) + sx1 * sp.diff(_P, _S)      # x component of grad^(i-1) p
    V2 = sz1 * sp.diff(_P, _S)                        # z component
    Lp = sp.diff(V1, _X) + sx2 * sp.diff(V1, _S) + sz2 * sp.diff(V2, _S)
    hx = sp.diff(_H, _X)
    bed = (-(hx * V1 + V2) / sp.sqrt(1 + hx ** 2)).subs(_S, 0)
    lam = lambda e, *v: sp.lambdify(v, e, "numpy")
    return (lam(Lp, _X, _S), lam(bed, _X), lam(V1, _X, _S), lam(_H, _X), lam(_E1, _X), lam(_E2, _X),
            lam(_P, _X, _S))


_MAN = None


def _wall_errors(nphys, nz):
    global _MAN
    if _MAN is None:
        _MAN = _manufactured()
    Lf, bedf, V1f, hf, e1f, e2f, pf = _MAN
    lx = 3.0
    nx = nphys + 3
    x = W.wall_x(nx, lx)
    s = _sig(nz)
    one = np.ones(nx)
    P = _wall_problem(nx, nz, lx, hf(x) * one)
    P.assemble(e1f(x) * one, e2f(x) * one)
    p = (pf(x[None, :], s[:, None]) * np.ones((nz + 1, nx))).ravel()
    y = (P.matrix() @ p).reshape(nz + 1, nx)
    phys = slice(1, nx - 1)
    e_pde = np.abs(y[1:nz, phys] - (Lf(x[None, :], s[1:nz, None]) * np.ones((nz - 1, nx)))[:, phys]).max()
    e_bed = np.abs(y[0, phys] - (bedf(x) * one)[phys]).max()
    e_wall = 0.0
    for ig, iw, sgn in [(0, 1, -1.0), (nx - 1, nx - 2, 1.0)]:
        want = sgn * V1f(x[iw], s[:nz]) * np.ones(nz)
        e_wall = max(e_wall, np.abs(y[:nz, ig] - want).max())
    return e_pde, e_bed, e_wall


def test_walls_manufactured_convergence_order():
    res = [_wall_errors(24 * 2 ** q, 8 * 2 ** q + 1) for q in range(3)]
    for c in range(3):
        e = [r[c] for r in res]
        order = math.log2(e[1] / e[2])
        assert order > 4.5, (c, res)
    assert res[-1][0] < 1e-5 and res[-1][2] < 1e-6, res


# ---- 3. factorisation order, ILU(0), GMRES ----

def _group_order(nx, nz):
    cols = []
    for c in range(4):
        cols += [ix for ix in range(3, nx - 3) if ix % 4 == c]
    groups = [len(cols)]
    for e in range(3):
        cols += [e, nx - 1 - e]
    order = [(j + 1) * nx + ix for ix in cols for j in range(-1, nz)]
    return np.array(order), cols


def _dense_ilu0(B, pattern):
    A = B.copy()
    n = A.shape[0]
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
def test_walls_ilu0_matches_dense_ikj(bar):
    nx, nz, lx = 16, 7, 3.0
    x = W.wall_x(nx, lx)
    h = 1.0 - (0.3 * np.exp(-4 * (x - 1.5) ** 2) if bar else 0 * x)
    h[0], h[-1] = h[1], h[-2]
    P = _wall_problem(nx, nz, lx, h)
    assert P.box == bar
    P.assemble()
    A = P.matrix().toarray()
    order, cols = _group_order(nx, nz)
    B = A[np.ix_(order, order)]
    LU = P.ilu_factors().toarray()
    csr = P.ilu_factors()
    patt = np.zeros_like(B, dtype=bool)
    for i in range(B.shape[0]):
        patt[i, csr.indices[csr.indptr[i]:csr.indptr[i + 1]]] = True
    assert np.all(patt[np.abs(B) > 1e-12 * np.abs(B).max()])
    ref = _dense_ilu0(B, patt)
    np.testing.assert_allclose(LU[patt], ref[patt], rtol=1e-11, atol=1e-11 * np.abs(ref).max())
    L = np.tril(LU, -1) + np.eye(B.shape[0])
    U = np.triu(LU)
    np.testing.assert_allclose((L @ U)[patt], B[patt], rtol=1e-10, atol=1e-10 * np.abs(B).max())


def test_walls_groups_are_uncoupled():
    # the device sweeps all columns of a group at once: no pattern entry may join two of them
    for bar in (False, True):
        nx, nz, lx = 24, 7, 3.0
        x = W.wall_x(nx, lx)
        h = 1.0 - (0.3 * np.exp(-4 * (x - 1.5) ** 2) if bar else 0 * x)
        P = _wall_problem(nx, nz, lx, h)
        csr = P.ilu_factors()
        order, cols = _group_order(nx, nz)
        col_of_rank = np.repeat(np.array(cols), nz + 1)
        group = {}
        for c in range(4):
            for ix in range(3, nx - 3):
                if ix % 4 == c:
                    group[ix] = c
        for e in range(3):
            group[e] = group[nx - 1 - e] = 4 + e
        for i in range(P.m):
            ci = col_of_rank[i]
            for jj in csr.indices[csr.indptr[i]:csr.indptr[i + 1]]:
                cj = col_of_rank[jj]
                assert cj == ci or group[cj] != group[ci], (bar, ci, cj)


def test_walls_gmres_reaches_dense_solution():
    nx, nz, lx = 20, 9, 3.0
    x = W.wall_x(nx, lx)
    h = 1.0 - 0.3 * np.exp(-4 * (x - 1.5) ** 2)
    P = _wall_problem(nx, nz, lx, h, tol=1e-13, max_restarts=400)
    P.assemble(0.03 * np.sin(x), 0.03 * np.sin(x + 0.1))
    A = P.matrix().toarray()
    b = np.random.default_rng(3).standard_normal(P.m)
    b[P.index(0, 0, nz - 1):] = 0.0
    xs, st, code = P.gmres(b)
    assert code == 0
    ref = np.linalg.solve(A, b)
    assert np.linalg.norm(xs - ref) <= 1e-9 * np.linalg.norm(ref)


# ---- 4. standing wave in a closed basin ----

def _stage_time(n, i, dt, C):
    return (n + (C[i] if i < 5 else 1.0)) * dt


def test_closed_basin_standing_wave():
    # a/h = 0.002 keeps the second-order bound harmonic (~ka a) well below the bound
    wl = W.standing_wave_basin(a_over_h=0.002)
    P = _wall_problem(wl["nx"], wl["nz"], wl["lx"], wl["h"], guess="ewma", k=8, decay=0.9)
    st = W.state_arrays(wl)
    x = W.wall_x(wl["nx"], wl["lx"])
    a = 0.002
    phys = slice(1, wl["nx"] - 1)
    n = wl["steps"]
    dx = wl["lx"] / (wl["nx"] - 3)

    def mass(eta):   # trapezoid rule over the physical columns, wall to wall
        e = eta[phys]
        return dx * (e.sum() - 0.5 * (e[0] + e[-1]))

    m0 = mass(st["eta"])
    snaps = {}
    for step in range(n):
        for i in range(1, 6):
            p, stt, code = P.stage((wl["g"], wl["rho"], wl["dt"]), i, st)
            assert code == 0
        if step + 1 in (n // 2, n):
            snaps[step + 1] = st["eta"].copy()
    ref = a * np.cos(wl["k"] * x)
    assert np.abs(snaps[n // 2][phys] + ref[phys]).max() < 0.01 * a, np.abs(snaps[n // 2][phys] + ref[phys]).max()
    assert np.abs(snaps[n][phys] - ref[phys]).max() < 0.01 * a, np.abs(snaps[n][phys] - ref[phys]).max()
    # no flux through the walls: the volume of the surface stays put (to 1e-6 of a L)
    assert abs(mass(st["eta"]) - m0) < 1e-6 * a * wl["lx"], mass(st["eta"]) - m0
    # no flow through the walls: the wall-node horizontal velocity stays at rounding level
    u = st["u"].reshape(wl["nz"] + 1, wl["nx"])
    assert np.abs(u[1:, 1]).max() < 1e-3 * a * wl["omega"] / wl["k"], np.abs(u[1:, 1]).max()


# ---- 5. relaxation zones ----

def test_relaxation_weight_shape():
    xi = np.linspace(0, 1, 101)
    g = np.array([O.relax_weight(v) for v in xi])
    assert g[0] == 1.0 and g[-1] == 0.0
    assert np.all(np.diff(g) < 0)
    # smooth start: 1 - Gamma grows like xi^3.5 / (e - 1)
    small = 1e-2
    assert abs((1 - O.relax_weight(small)) / small ** 3.5 * (math.e - 1) - 1) < 1e-3


@pytest.mark.parametrize("T,h", [(2.02, 0.4), (1.0, 5.0), (20.0, 0.5)])
def test_wavenumber_solves_dispersion(T, h):
    om = 2 * math.pi / T
    k = O.wavenumber(om, h)
    assert abs(9.81 * k * math.tanh(k * h) - om * om) < 1e-12 * om * om
    if h * om * om / 9.81 > 10:                 # deep water
        assert abs(k / (om * om / 9.81) - 1) < 1e-6
    if k * h < 0.2:                             # shallow water: k ~ omega / sqrt(g h)
        assert abs(k / (om / math.sqrt(9.81 * h)) - 1) < 0.01


def test_relax_blends_only_inside_zones():
    wl = W.flume_2d(nx=67, nz=9, lx=12.0, depth=0.4, gen=(0.0, 3.0), absorb=(9.0, 12.0))
    P = _wall_problem(wl["nx"], wl["nz"], wl["lx"], wl["h"])
    rng = np.random.default_rng(4)
    st = dict(u=rng.standard_normal(P.m), w=rng.standard_normal(P.m), eta=0.01 * rng.standard_normal(P.nx))
    before = {k: v.copy() for k, v in st.items()}
    P.relax(wl["relax"], 3.3, st)
    x = W.wall_x(wl["nx"], wl["lx"])
    inside = (x >= 0) & (x <= 3.0) | (x >= 9.0) & (x <= 12.0)
    inside[0] = inside[-1] = False
    assert np.array_equal(st["eta"][~inside], before["eta"][~inside])
    u = st["u"].reshape(P.nz + 1, P.nx)
    ub = before["u"].reshape(P.nz + 1, P.nx)
    assert np.array_equal(u[:, ~inside], ub[:, ~inside])
    # at the far wall (xi = 1) the absorption target, still water, is taken exactly
    assert st["eta"][-2] == 0.0 and np.all(u[:, -2] == 0.0)
    # a state equal to the generation target is a fixed point of the blend
    k, om, a = wl["k"], wl["omega"], 0.01
    t = 10 * wl["relax"]["period"]
    eta_t = a * np.cos(k * x - om * t)
    z = _sig(P.nz)[:, None] * (wl["h"] + eta_t)[None, :] - wl["h"][None, :]
    ch = np.cosh(k * (z + 0.4)) / math.sinh(k * 0.4)
    sh = np.sinh(k * (z + 0.4)) / math.sinh(k * 0.4)
    st2 = dict(eta=eta_t.copy(), u=(a * om * ch * np.cos(k * x - om * t)).ravel(),
               w=(a * om * sh * np.sin(k * x - om * t)).ravel())
    ref = {kk: v.copy() for kk, v in st2.items()}
    P.relax(dict(wl["relax"], abs_x0=0.0, abs_x1=0.0), t, st2)
    gen = (x >= 0) & (x <= 3.0)
    np.testing.assert_allclose(st2["eta"][gen], ref["eta"][gen], atol=1e-15)
    np.testing.assert_allclose(st2["u"].reshape(P.nz + 1, P.nx)[:, gen], ref["u"].reshape(P.nz + 1, P.nx)[:, gen],
                               atol=1e-14)


def test_generated_wave_crosses_flume_and_is_absorbed():
    # H = 0.004 m (ka ~ 0.003) so that second-order harmonics stay near 1 % of a
    H = 0.004
    wl = W.flume_2d(nx=131, nz=9, lx=12.0, depth=0.4, gen=(0.0, 3.0), absorb=(8.6, 12.0), height=H)
    P = _wall_problem(wl["nx"], wl["nz"], wl["lx"], wl["h"], guess="ewma", k=8, decay=0.9)
    st = W.state_arrays(wl)
    _, _, C = O.lserk45()
    T = wl["relax"]["period"]
    n = int(round(8 * T / wl["dt"]))
    dt = 8 * T / n
    x = W.wall_x(wl["nx"], wl["lx"])
    a, k, om = H / 2, wl["k"], wl["omega"]
    mid = (x >= 3.5) & (x <= 8.0)
    rows, vals = [], []
    for step in range(n):
        for i in range(1, 6):
            p, stt, code = P.stage((wl["g"], wl["rho"], dt), i, st)
            assert code == 0
            P.relax(wl["relax"], _stage_time(step, i, dt, C), st)
        if step >= n - n // 8:                 # the last period: separate incident and reflected waves
            t = (step + 1) * dt
            xm = x[mid]
            rows.append(np.column_stack([np.cos(k * xm - om * t), np.sin(k * xm - om * t),
                                         np.cos(k * xm + om * t), np.sin(k * xm + om * t)]))
            vals.append(st["eta"][mid].copy())
    A, v = np.vstack(rows), np.concatenate(vals)
    c, *_ = np.linalg.lstsq(A, v, rcond=None)
    inc, refl = math.hypot(c[0], c[1]), math.hypot(c[2], c[3])
    assert abs(inc / a - 1) < 0.03, inc / a                      # incident linear wave, right amplitude
    assert abs(math.atan2(c[1], c[0])) < 0.05                    # and phase
    assert refl < 0.05 * a, refl / a                             # little comes back from the absorber
    assert np.abs(v - A @ c).max() < 0.05 * a
    quiet = (x >= 11.0) & (x <= 12.0)
    assert np.abs(st["eta"][quiet]).max() < 0.01 * a
