"""Pins of the oracle's time integration (Algorithm 1, Eq. 14-17, LSERK45).

- The LSERK45 coefficients (Carpenter & Kennedy 1994, not printed in the
  paper) satisfy the eight fourth-order conditions once the 2N-storage form of
  Eq. (15) is rewritten as a Butcher tableau, and their abscissae c_i are the
  row sums of that tableau; integrating y' = lambda y converges at order 4.
- The first-stage pressure of a small linear (Airy) wave matches linear wave
  theory, p = -rho g z + rho g a cosh(k(z+h))/cosh(kh) cos(kx), to O(ka).
- After one wave period the free surface returns to its initial shape: phase
  and amplitude errors below 1 % (linear dispersion relation).
"""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W


def _butcher():
    A2, B2, C2 = O.lserk45()
    s = 5
    a = np.zeros((s + 1, s))
    # y_i = y_0 + sum_{j<=i} dt f_j sum_{l=j..i} B_l prod_{q=j+1..l} A_q
    for i in range(1, s + 1):
        for j in range(1, i + 1):
            tot = 0.0
            for l in range(j, i + 1):
                pr = 1.0
                for q in range(j + 1, l + 1):
                    pr *= A2[q - 1]
                tot += B2[l - 1] * pr
            a[i, j - 1] = tot
    A = a[:s, :]        # stage i (1-based) evaluates f at y_{i-1}: rows 0..4
    b = a[s, :]
    return A, b, C2


def test_lserk45_order_conditions():
    A, b, C = _butcher()
    c = A.sum(axis=1)
    np.testing.assert_allclose(c, C, atol=1e-12)
    conds = [
        (b.sum(), 1.0),
        (b @ c, 1 / 2),
        (b @ c ** 2, 1 / 3),
        (b @ (A @ c), 1 / 6),
        (b @ c ** 3, 1 / 4),
        (b @ (c * (A @ c)), 1 / 8),
        (b @ (A @ c ** 2), 1 / 12),
        (b @ (A @ (A @ c)), 1 / 24),
    ]
    for got, want in conds:
        assert abs(got - want) < 1e-12, (got, want)


def test_lserk45_convergence_order():
    al, be, _ = O.lserk45()
    lam = -1.0 + 2.0j
    errs = []
    for n in [20, 40, 80]:
        dt = 1.0 / n
        y, K = 1.0 + 0j, 0j
        for _ in range(n):
            for i in range(5):
                K = al[i] * K + dt * lam * y
                y = y + be[i] * K
        errs.append(abs(y - np.exp(lam)))
    order = math.log2(errs[1] / errs[2])
    assert 3.8 < order < 4.3, errs


def _airy(nx=64, nz=9):
    return W.airy_2d(nx=nx, nz=nz)


def test_first_stage_pressure_matches_linear_theory():
    wl = _airy()
    P = O.OracleProblem(wl["nx"], 1, wl["nz"], wl["lx"], 0.0, wl["h"], tol=1e-12, max_restarts=200)
    st = W.state_arrays(wl)
    p, stt, code = P.stage((wl["g"], wl["rho"], wl["dt"]), 1, st)
    assert code == 0
    x = np.arange(wl["nx"]) * (wl["lx"] / wl["nx"])
    eta0 = wl["eta"]
    s = np.arange(-1, wl["nz"]) / (wl["nz"] - 1.0)
    z = s[:, None] * (1.0 + eta0)[None, :] - 1.0
    k, a, rho, g = 1.0, 0.01, wl["rho"], wl["g"]
    plin = -rho * g * z + rho * g * a * np.cosh(k * (z + 1)) / math.cosh(k) * np.cos(k * x)[None, :]
    pp = p.reshape(wl["nz"] + 1, wl["nx"])
    dyn = rho * g * a
    err = np.abs(pp[1:] - plin[1:]).max()       # physical levels sigma in [0, 1]
    assert err < 0.05 * dyn, (err, dyn)


def test_airy_wave_one_period():
    wl = _airy()
    k, h, g = 1.0, 1.0, wl["g"]
    om = math.sqrt(g * k * math.tanh(k * h))
    T = 2 * math.pi / om
    n = 128
    dt = T / n
    P = O.OracleProblem(wl["nx"], 1, wl["nz"], wl["lx"], 0.0, wl["h"], guess="ewma", k=8, decay=0.9)
    st = W.state_arrays(wl)
    for _ in range(n):
        for i in range(1, 6):
            p, stt, code = P.stage((g, wl["rho"], dt), i, st)
            assert code == 0
    x = np.arange(wl["nx"]) * (wl["lx"] / wl["nx"])
    eta = st["eta"]
    c1 = 2 * np.mean(eta * np.cos(k * x))
    s1 = 2 * np.mean(eta * np.sin(k * x))
    amp = math.hypot(c1, s1)
    phase = math.atan2(s1, c1)
    assert abs(amp / 0.01 - 1) < 0.01, amp
    assert abs(phase) / (2 * math.pi) < 0.01, phase


# ---- 3-D: the y-components of the stage driver ---------------------------

def test_first_stage_pressure_oblique_wave_3d():
    # wave vector (1, 2): most of the velocity is along y, so the v terms of
    # f_eta (Eq. 14b) and of the right-hand side (Eq. 16-17) carry the pressure
    wl = W.airy_3d(nx=32, ny=32, nz=9, kx_index=1, ky_index=2, a_over_h=0.01)
    P = O.OracleProblem(wl["nx"], wl["ny"], wl["nz"], wl["lx"], wl["ly"], wl["h"], tol=1e-12, max_restarts=400)
    st = W.state_arrays(wl)
    p, stt, code = P.stage((wl["g"], wl["rho"], wl["dt"]), 1, st)
    assert code == 0, stt
    x = np.arange(wl["nx"]) * (wl["lx"] / wl["nx"])
    y = np.arange(wl["ny"]) * (wl["ly"] / wl["ny"])
    X, Y = np.meshgrid(x, y, indexing="xy")
    th = (1.0 * X + 2.0 * Y).ravel()
    k, a, rho, g = math.sqrt(5.0), 0.01, wl["rho"], wl["g"]
    z = W.node_z(wl["h"], wl["eta"], wl["nz"])
    plin = -rho * g * z + rho * g * a * np.cosh(k * (z + 1)) / math.cosh(k) * np.cos(th)[None, :]
    pp = p.reshape(wl["nz"] + 1, -1)
    dyn = rho * g * a
    err = np.abs(pp[1:] - plin[1:]).max()
    assert err < 0.05 * dyn, (err, dyn)
    # the dynamic part has the wave's shape and size (not just the hydrostatic column)
    pd = pp[1:] + rho * g * z[1:]
    corr = np.corrcoef(pd[0], np.cos(th))[0, 1]
    assert corr > 0.99, corr


def test_stage_y_only_equals_2d_stage_turned():
    # a wave over a bar, both uniform in x and varying along y: every stage of
    # the 3-D driver must reproduce the 2-D driver (pinned above) run along y,
    # column by column, with v in the role of u.  The sloping bed reaches the
    # h_y terms of the ghost rows (operator and right-hand side).
    ny, nx, nz = 32, 8, 9
    w2 = W.periodic_bar_2d(nx=ny, nz=nz, kh=1.2, a_over_h=0.02, bar_height=0.4, seed=11)
    L = w2["lx"]
    rep = lambda a: np.repeat(np.asarray(a).reshape(-1, ny)[:, :, None], nx, axis=2).ravel()
    h3 = rep(w2["h"])
    st2 = W.state_arrays(w2)
    st3 = dict(u=np.zeros((nz + 1) * ny * nx), v=rep(w2["u"]), w=rep(w2["w"]), eta=rep(w2["eta"]))
    st3["Ku"], st3["Kv"], st3["Kw"] = (np.zeros_like(st3["u"]) for _ in range(3))
    st3["Keta"] = np.zeros_like(st3["eta"])
    phys = (w2["g"], w2["rho"], w2["dt"])
    kw = dict(tol=1e-13, max_restarts=400, guess="previous")
    P2 = O.OracleProblem(ny, 1, nz, L, 0.0, w2["h"], **kw)
    P3 = O.OracleProblem(nx, ny, nz, L, L, h3, **kw)
    assert P3.box
    dyn = w2["rho"] * w2["g"] * 0.02
    for i in range(1, 6):
        p2, _, c2 = P2.stage(phys, i, st2)
        p3, _, c3 = P3.stage(phys, i, st3)
        assert c2 == 0 and c3 == 0
        np.testing.assert_allclose(p3, rep(p2), rtol=0, atol=1e-9 * dyn)
        np.testing.assert_allclose(st3["eta"], rep(st2["eta"]), rtol=0, atol=1e-12)
        np.testing.assert_allclose(st3["v"], rep(st2["u"]), rtol=0, atol=1e-11)
        np.testing.assert_allclose(st3["w"], rep(st2["w"]), rtol=0, atol=1e-11)
        assert np.abs(st3["u"]).max() < 1e-12
