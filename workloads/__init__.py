"""Seeded synthetic inputs for the sigma-transformed Poisson solve.

This module only makes input data: bathymetry h, initial free surface eta and
initial velocities (u, v, w) from linear (Airy) wave theory, plus the grid sizes
and time step of each workload.  It contains none of the solver's arithmetic
and is shared by the tests, the benchmark and the oracle checks.

Stand-ins: the paper initialises stream-function waves from Fenton's Fourier
method and runs the Beji-Battjes flume (Sec. 5).  The stream-function waves
are computed here (workloads.stream_function, Fenton's method written out);
the flume's measured data are not available, and the other workloads use sums
of linear waves of the same wavenumber, depth and steepness class.
"""
import math

import numpy as np

G = 9.81
RHO = 1000.0


def sigma_levels(nz):
    """sigma_j = j/(nz-1) for j = -1 (ghost) .. nz-1."""
    return np.arange(-1, nz) / (nz - 1.0)


def node_z(h, eta, nz):
    """Physical z of every node, shape (nz+1, ncol): z = sigma d - h."""
    s = sigma_levels(nz)[:, None]
    d = (h + eta)[None, :]
    return s * d - h[None, :]


def dispersion_omega(k, h):
    return np.sqrt(G * k * np.tanh(k * h))


def airy_fields(x, y, h, nz, comps):
    """Linear superposition of progressive waves.

    comps: list of (kx, ky, amplitude, phase).  Returns eta (ncol,), u, v, w
    (each (nz+1)*ncol, x fastest then y then sigma, ghost level first).
    """
    X, Y = np.meshgrid(x, y, indexing="xy")
    X = X.ravel(); Y = Y.ravel()
    eta = np.zeros(X.size)
    for kx, ky, a, ph in comps:
        eta += a * np.cos(kx * X + ky * Y + ph)
    Z = node_z(h, eta, nz)
    u = np.zeros_like(Z); v = np.zeros_like(Z); w = np.zeros_like(Z)
    for kx, ky, a, ph in comps:
        k = math.hypot(kx, ky)
        om = dispersion_omega(k, h)[None, :]
        th = (kx * X + ky * Y + ph)[None, :]
        hz = (Z + h[None, :])
        ch = np.cosh(k * hz) / np.sinh(k * h)[None, :]
        sh = np.sinh(k * hz) / np.sinh(k * h)[None, :]
        u += a * om * (kx / k) * ch * np.cos(th)
        v += a * om * (ky / k) * ch * np.cos(th)
        w += a * om * sh * np.sin(th)
    return eta, u.ravel(), v.ravel(), w.ravel()


def courant_dt(dx, lmax, hmax, cr=0.5):
    """dt with Courant number cr for the phase speed of the longest periodic wave."""
    k = 2 * math.pi / lmax
    c = math.sqrt(G / k * math.tanh(k * hmax))
    return cr * dx / c


def _wl(nx, ny, nz, lx, ly, h, comps, steps, name, **extra):
    x = np.arange(nx) * (lx / nx)
    y = np.arange(ny) * (ly / ny) if ny > 1 else np.zeros(1)
    eta, u, v, w = airy_fields(x, y, h, nz, comps)
    dx = lx / nx
    if ny > 1:
        dx = min(dx, ly / ny)
    dt = courant_dt(dx, max(lx, ly if ny > 1 else 0.0), float(h.max()))
    d = dict(name=name, nx=nx, ny=ny, nz=nz, lx=lx, ly=(ly if ny > 1 else 0.0), h=h, eta=eta, u=u,
             v=(v if ny > 1 else None), w=w, dt=dt, steps=steps, g=G, rho=RHO, m=nx * ny * (nz + 1))
    d.update(extra)
    return d


def airy_2d(nx=64, nz=9, kh=1.0, a_over_h=0.01, depth=1.0, steps=50, waves=1):
    """Linear Airy wave in a periodic 2-D slice of `waves` wavelengths, flat bed
    (the 64 x 9 workload: one wavelength)."""
    k = kh / depth
    lx = waves * 2 * math.pi / k
    h = np.full(nx, depth)
    return _wl(nx, 1, nz, lx, 0.0, h, [(k, 0.0, a_over_h * depth, 0.0)], steps, "airy2d_%dx%d" % (nx, nz))


def airy_3d(nx=32, ny=32, nz=9, kx_index=1, ky_index=2, a_over_h=0.01, depth=1.0, lx=2 * math.pi,
            ly=2 * math.pi, steps=50):
    """Oblique linear Airy wave in a periodic 3-D box over a flat bed; the wave
    vector (kx, ky) = 2 pi (kx_index / lx, ky_index / ly) lies on the lattice."""
    kx, ky = 2 * math.pi * kx_index / lx, 2 * math.pi * ky_index / ly
    h = np.full(nx * ny, depth)
    return _wl(nx, ny, nz, lx, ly, h, [(kx, ky, a_over_h * depth, 0.0)], steps,
               "airy3d_%dx%dx%d_k%d_%d" % (nx, ny, nz, kx_index, ky_index))


def stokes_like_2d(nx=512, nz=17, kh=2.0, a1_over_h=0.08, depth=1.0, n_harm=4, ratio=0.3, seed=2511,
                   steps=1000):
    """Steep periodic wave: first n_harm harmonics a_n = a1 ratio^(n-1), seeded phases."""
    rng = np.random.default_rng(seed)
    k = kh / depth
    lx = 2 * math.pi / k
    phases = rng.uniform(0, 2 * math.pi, n_harm)
    comps = [(n * k, 0.0, a1_over_h * depth * ratio ** (n - 1), phases[n - 1]) for n in range(1, n_harm + 1)]
    h = np.full(nx, depth)
    return _wl(nx, 1, nz, lx, 0.0, h, comps, steps, "stokes2d_%dx%d" % (nx, nz))


def periodic_bar_2d(nx=256, nz=9, kh=1.5, a_over_h=0.02, depth=1.0, bar_frac=0.25, bar_height=0.5, seed=7,
                    steps=50, max_slope=None, waves=1):
    """Periodic 2-D slice of `waves` wavelengths over a trapezoidal bar
    (variable depth, box pattern).

    max_slope: if given, the ramps are widened (up to what keeps the bar off the
    domain's ends) and then the crest lowered until no ramp is steeper than it."""
    rng = np.random.default_rng(seed)
    k = kh / depth
    lx = waves * 2 * math.pi / k
    x = np.arange(nx) * (lx / nx)
    c0 = rng.uniform(0.3, 0.7) * lx
    top = bar_frac * lx * 0.3
    ramp = bar_frac * lx * 0.35
    if max_slope is not None:
        ramp = min(max(ramp, bar_height * depth / max_slope), 0.3 * lx - top)
        bar_height = min(bar_height, max_slope * ramp / depth)
    dist = np.abs(x - c0)
    prof = np.clip((top + ramp - dist) / ramp, 0.0, 1.0)
    h = depth * (1.0 - bar_height * prof)
    phase = rng.uniform(0, 2 * math.pi)
    return _wl(nx, 1, nz, lx, 0.0, h, [(k, 0.0, a_over_h * depth, phase)], steps, "bar2d_%dx%d" % (nx, nz))


def bumpy_3d(nx=256, ny=256, nz=17, depth=1.0, n_bumps=8, n_comp=16, amp_sum=0.03, seed=4, steps=500):
    """3-D periodic field over seeded Gaussian bumps (depth 1 + 0.2 * bumps)."""
    rng = np.random.default_rng(seed)
    L = 2 * math.pi
    x = np.arange(nx) * (L / nx)
    y = np.arange(ny) * (L / ny)
    X, Y = np.meshgrid(x, y, indexing="xy")
    bump = np.zeros_like(X)
    for _ in range(n_bumps):
        cx, cy = rng.uniform(0, L, 2)
        s = rng.uniform(0.3, 0.8)
        dxp = np.minimum(np.abs(X - cx), L - np.abs(X - cx))
        dyp = np.minimum(np.abs(Y - cy), L - np.abs(Y - cy))
        bump += np.exp(-(dxp ** 2 + dyp ** 2) / (2 * s * s))
    h = depth + 0.2 * depth * bump / bump.max()
    comps = []
    amps = rng.uniform(0.5, 1.0, n_comp)
    amps *= amp_sum * depth / amps.sum()
    for q in range(n_comp):
        while True:
            kx, ky = rng.integers(-4, 5, 2)
            if 1.0 <= math.hypot(kx, ky) <= 4.0:
                break
        comps.append((float(kx), float(ky), float(amps[q]), float(rng.uniform(0, 2 * math.pi))))
    return _wl(nx, ny, nz, L, L, h.ravel(), comps, steps, "bumpy3d_%dx%dx%d" % (nx, ny, nz))


def state_arrays(wl):
    """Fresh RK state for a workload: copies of u, v, w, eta and zero registers."""
    st = dict(u=wl["u"].copy(), v=None if wl["v"] is None else wl["v"].copy(), w=wl["w"].copy(),
              eta=wl["eta"].copy())
    st["Ku"] = np.zeros_like(st["u"])
    st["Kv"] = None if st["v"] is None else np.zeros_like(st["v"])
    st["Kw"] = np.zeros_like(st["w"])
    st["Keta"] = np.zeros_like(st["eta"])
    return st


def batch_members(n=512, seed=5, nxs=(128, 256, 512, 1024, 2048), nzs=(9, 17, 33), max_slope=0.5, ppw=128):
    """Uneven 2-D members: nx, nz drawn uniformly, kh ~ U[0.5, 3], a/h ~ U[0.005, 0.08],
    half flat-bottomed, half over a seeded periodic trapezoidal bar whose ramps
    are no steeper than max_slope.  Every member resolves its wave with ppw
    points per wavelength, so a member of nx columns spans nx / ppw
    wavelengths (uneven sizes are uneven domain lengths at one resolution).
    On one-wavelength domains of 2,048 columns the x spacing is far below the
    sigma spacing, and ramps of slope 2 appear on the shortest domains; in both
    cases restarted GMRES(20) with ILU(0) stagnates."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        nx = int(rng.choice(nxs))
        nz = int(rng.choice(nzs))
        kh = float(rng.uniform(0.5, 3.0))
        a = float(rng.uniform(0.005, 0.08))
        waves = max(1, nx // ppw)
        if i % 2 == 0:
            wl = airy_2d(nx=nx, nz=nz, kh=kh, a_over_h=a, steps=1, waves=waves)
        else:
            wl = periodic_bar_2d(nx=nx, nz=nz, kh=kh, a_over_h=a, seed=int(rng.integers(1 << 30)), steps=1,
                                 max_slope=max_slope, waves=waves)
        wl["name"] = "member%03d_%s" % (i, wl["name"])
        out.append(wl)
    return out


# ---------------------------------------------------------------------------
# Wave flume with walls: ghost columns 0 and nx-1 lie one spacing outside the
# walls at x = 0 and x = lx; physical columns 1..nx-2 at x = (ix-1) lx/(nx-3).
# ---------------------------------------------------------------------------
def wall_x(nx, lx):
    return (np.arange(nx) - 1.0) * (lx / (nx - 3))


def linear_wavenumber(omega, depth):
    k = omega * omega / G
    for _ in range(100):
        th = math.tanh(k * depth)
        dk = (G * k * th - omega * omega) / (G * th + G * k * depth * (1 - th * th))
        k -= dk
        if abs(dk) <= 1e-15 * k:
            break
    return k


def beji_bar_depth(x):
    """Trapezoidal submerged bar: 0.4 m, 1:20 up to 0.1 m over [6, 12], flat to 14, 1:10 down to 0.4 at 17."""
    h = np.full_like(x, 0.4)
    up = (x >= 6) & (x < 12)
    h[up] = 0.4 - (x[up] - 6) / 20
    h[(x >= 12) & (x < 14)] = 0.1
    dn = (x >= 14) & (x < 17)
    h[dn] = 0.1 + (x[dn] - 14) / 10
    return h


def flume_2d(nx=2048, nz=17, lx=40.0, depth="bar", height=0.02, period=2.02, gen=(0.0, 3.0), absorb=None,
             ramp_periods=2.0, steps=4000, cr=0.5):
    """Wave flume between walls, starting from rest; waves enter through a
    relaxation generation zone and leave through an absorption zone.

    depth: "bar" for the trapezoidal bar (0.4 m still-water depth away from it)
    or a number for a flat bed.  The time step has Courant number cr for the
    phase speed of the incident wave in 0.4 m (or the flat depth).
    """
    x = wall_x(nx, lx)
    h0 = 0.4 if depth == "bar" else float(depth)
    if depth == "bar":
        h = beji_bar_depth(np.clip(x, 0.0, lx))
    else:
        h = np.full(nx, h0)
    h[0], h[-1] = h[1], h[-2]
    if absorb is None:
        absorb = (lx - 4.0, lx)
    om = 2 * math.pi / period
    k = linear_wavenumber(om, h0)
    dx = lx / (nx - 3)
    dt = cr * dx / (om / k)
    m = nx * (nz + 1)
    relax = dict(gen_x0=gen[0], gen_x1=gen[1], abs_x0=absorb[0], abs_x1=absorb[1], height=height, period=period,
                 depth=h0, ramp_time=ramp_periods * period, g=G)
    return dict(name="flume2d_%dx%d_%s" % (nx, nz, "bar" if depth == "bar" else "flat"), nx=nx, ny=1, nz=nz,
                lx=lx, ly=0.0, h=h, eta=np.zeros(nx), u=np.zeros(m), v=None, w=np.zeros(m), dt=dt, steps=steps,
                g=G, rho=RHO, m=m, walls=True, relax=relax, k=k, omega=om)


def standing_wave_basin(nx=67, nz=9, depth=1.0, kh=1.0, a_over_h=0.01, steps=128):
    """Closed basin one wavelength long, free surface a cos(k x) at rest (a standing wave at its crest)."""
    k = kh / depth
    lx = 2 * math.pi / k
    x = wall_x(nx, lx)
    h = np.full(nx, depth)
    m = nx * (nz + 1)
    om = dispersion_omega(k, depth)
    T = 2 * math.pi / om
    return dict(name="basin2d_%dx%d" % (nx, nz), nx=nx, ny=1, nz=nz, lx=lx, ly=0.0, h=h,
                eta=a_over_h * depth * np.cos(k * x), u=np.zeros(m), v=None, w=np.zeros(m), dt=T / steps,
                steps=steps, g=G, rho=RHO, m=m, walls=True, relax=None, k=k, omega=float(om))


def stream_function_2d(nx=200, nz=20, kh=1.0, steepness=0.6, depth=1.0, steps=200, dt=None):
    """Periodic flat-bed slice one wavelength long holding a steady stream-function
    wave (Sec. 5.1): height H = steepness (H/L)_max L with Battjes' limit, crest at
    x = 0, no mean Eulerian current; nx x nz = 200 x 20 as in the paper's study.
    dt: Courant 0.5 by default, else the given step in seconds (the paper's study
    steps by 1e-4)."""
    from .stream_function import battjes_max_steepness, converged_wave, stream_function_fields
    k = kh / depth
    lx = 2 * math.pi / k
    x = np.arange(nx) * (lx / nx)
    h = np.full(nx, depth)
    h_over_l = steepness * battjes_max_steepness(kh)
    wave = converged_wave(kh, 2 * math.pi * h_over_l)
    eta, u, w = stream_function_fields(x, depth, nz, wave, k, G)
    dt = courant_dt(lx / nx, lx, depth) if dt is None else float(dt)
    return dict(name="sfwave2d_%dx%d_kh%g_s%g" % (nx, nz, kh, steepness), nx=nx, ny=1, nz=nz, lx=lx, ly=0.0,
                h=h, eta=eta, u=u, v=None, w=w, dt=dt, steps=steps, g=G, rho=RHO, m=nx * (nz + 1),
                kh=kh, steepness=steepness, height=h_over_l * lx, c=wave.c * math.sqrt(G / k), wave=wave)
