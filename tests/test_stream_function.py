"""Pins of the stream-function wave generator (Fenton's Fourier method, the
initial condition of the paper's Sec. 5.1 experiments) and, through it, of the
oracle's nonlinear time stepping.

1. Linear limit: at vanishing steepness the fields equal the Airy workload
   (linear theory) up to a difference that is first order in the steepness.
2. Stokes' third-order phase speed, c = c0 + eps^2 C2 (eps = kH/2, Stokes'
   first definition of c): the difference is O(eps^4), i.e. it drops 16-fold
   when eps halves.
3. Stokes' second-order bound harmonic, E_2 = E_1^2 (3 - sigma^2)/(4 sigma^3)
   (sigma = tanh kd): the relative difference is O(eps^2).
4. The free-surface conditions hold between the collocation points too, on
   the paper's kh x steepness grid.
5. Mean level, wave height and zero mean Eulerian current of the workload.
6. Battjes' limit tends to McCowan's solitary-wave limit H/h = 0.78 in
   shallow water and to 0.1401 in deep water.
7. The wave is a steady solution of the free-surface model: the oracle's
   LSERK45 stages carry the surface along at the phase speed c, with an error
   that falls by more than 50x from 64 x 9 to 128 x 17 nodes.
"""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W
from workloads.stream_function import FentonWave, battjes_max_steepness, converged_wave


@pytest.mark.parametrize("kh", [0.4, 1.0, 2.0])
def test_linear_limit_is_airy(kh):
    diffs = []
    for s in (1e-4, 5e-5):
        sf = W.stream_function_2d(nx=64, nz=9, kh=kh, steepness=s)
        ai = W.airy_2d(nx=64, nz=9, kh=kh, a_over_h=sf["height"] / 2)
        d = max(np.abs(sf[f] - ai[f]).max() / np.abs(ai[f]).max() for f in ("eta", "u", "w"))
        diffs.append(d)
    assert diffs[0] < 1e-3, diffs
    assert 1.8 < diffs[0] / diffs[1] < 2.2, diffs


@pytest.mark.parametrize("kd", [0.8, 1.0, 2.0, 4.0])
def test_phase_speed_is_stokes_third_order(kd):
    S = 1.0 / math.cosh(2 * kd)
    c0 = math.sqrt(math.tanh(kd))
    c2 = c0 * (2 + 7 * S * S) / (4 * (1 - S) ** 2)
    err = []
    for eps in (0.04, 0.02):
        w = FentonWave(kd, 2 * eps, n_modes=24)
        err.append(w.c - (c0 + eps * eps * c2))
        assert abs(err[-1]) < 0.01 * eps * eps * c2
    assert 14.0 < err[0] / err[1] < 18.0, err


@pytest.mark.parametrize("kd", [0.8, 1.0, 2.0, 4.0])
def test_second_harmonic_is_stokes_second_order(kd):
    sg = math.tanh(kd)
    rel = []
    for eps in (0.04, 0.02):
        w = FentonWave(kd, 2 * eps, n_modes=24)
        e2 = w.E[1] ** 2 * (3 - sg * sg) / (4 * sg ** 3)
        rel.append(abs(w.E[2] / e2 - 1.0))
    assert rel[1] < 1e-3, rel
    assert 3.0 < rel[0] / rel[1] < 5.0, rel


@pytest.mark.parametrize("kh", [0.4, 2.0, 4.0])
@pytest.mark.parametrize("frac", [0.01, 0.3, 0.7])
def test_surface_conditions_between_collocation_points(kh, frac):
    kH = 2 * math.pi * frac * battjes_max_steepness(kh)
    w = converged_wave(kh, kH)
    Xh = (np.arange(w.N) + 0.5) * math.pi / w.N
    eta = w.surface(Xh)
    kin = w._psi(Xh, eta, w.B, w.ubar) + w.Q
    u, v = w._velocities(Xh, eta, w.B, w.ubar)
    dyn = 0.5 * (u * u + v * v) + eta - w.R
    assert np.abs(kin).max() < 1e-9 * kH and np.abs(dyn).max() < 1e-9 * kH, (np.abs(kin).max(), np.abs(dyn).max())
    # the surface series reproduces the collocation heights
    np.testing.assert_allclose(w.surface(w.Xm), w.eta_m, rtol=0, atol=1e-12 * kh)


def test_workload_level_height_and_current():
    wl = W.stream_function_2d(nx=200, nz=20, kh=1.0, steepness=0.6)
    nx = wl["nx"]
    assert abs(wl["eta"].mean()) < 1e-12
    assert abs(wl["eta"][0] - wl["eta"][nx // 2] - wl["height"]) < 1e-12 * wl["height"] + 1e-14
    assert np.argmax(wl["eta"]) == 0
    # H/L = 0.6 (H/L)_max at kh = 1
    assert abs(wl["height"] / wl["lx"] - 0.6 * 0.1401 * math.tanh(0.8863)) < 1e-15
    # zero mean Eulerian current: the bed-level velocity averages to zero over a wavelength
    ub = wl["u"].reshape(wl["nz"] + 1, nx)[1]
    assert abs(ub.mean()) < 1e-12 * np.abs(ub).max()
    # the bed is a streamline: no vertical velocity there
    assert np.abs(wl["w"].reshape(wl["nz"] + 1, nx)[1]).max() < 1e-14


def test_battjes_limits():
    assert abs(battjes_max_steepness(50.0) - 0.1401) < 1e-12
    kh = 1e-4
    h_over_depth = 2 * math.pi * battjes_max_steepness(kh) / kh      # H / h = (H/L) L / h
    assert abs(h_over_depth - 0.78) < 0.01


def _propagate(nx, nz, kh, s, nsteps):
    wl = W.stream_function_2d(nx=nx, nz=nz, kh=kh, steepness=s)
    P = O.OracleProblem(nx, 1, nz, wl["lx"], 0.0, wl["h"], guess="previous", tol=1e-12, max_restarts=200)
    st = W.state_arrays(wl)
    for _ in range(nsteps):
        for i in range(1, 6):
            _, _, code = P.stage((wl["g"], wl["rho"], wl["dt"]), i, st)
            assert code == 0
    t = nsteps * wl["dt"]
    x = np.arange(nx) * (wl["lx"] / nx)
    exact = wl["wave"].surface(kh * (x - wl["c"] * t)) / kh - 1.0
    moved = np.abs(wl["eta"] - exact).max() / wl["height"]
    return np.abs(st["eta"] - exact).max() / wl["height"], moved


def test_oracle_carries_the_steady_wave_at_its_phase_speed():
    coarse, moved = _propagate(64, 9, 1.0, 0.3, 20)
    fine, _ = _propagate(128, 17, 1.0, 0.3, 20)
    assert moved > 0.2                       # the wave has travelled ten grid spacings
    assert coarse < 1e-4, coarse
    assert fine < coarse / 50, (coarse, fine)
