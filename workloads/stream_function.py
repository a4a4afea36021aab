"""Steady stream-function waves by Fenton's Fourier method (Rienecker & Fenton,
J. Fluid Mech. 104, 1981; Fenton, "The numerical solution of steady water wave
problems", Computers & Geosciences 14, 1988), the initial condition of the
paper's stream-function wave experiments (Sec. 5.1).

The wave is steady in a frame moving with the phase speed c.  In units where
k = 1 and g = 1, with y measured up from the bed (mean depth d = kh), the
stream function in the moving frame is

    psi(X, y) = -ubar y + sum_{j=1..N} B_j sinh(j y) / cosh(j d) cos(j X),

which satisfies Laplace's equation and the bed condition psi(X, 0) = 0 for any
B_j.  The unknowns are the surface heights eta_m at X_m = m pi / N (m = 0..N,
crest to trough), B_1..B_N, ubar, the flux Q and the Bernoulli constant R; the
equations are the two free-surface conditions at the N + 1 collocation points

    psi(X_m, eta_m) = -Q                                    (kinematic)
    (psi_y^2 + psi_X^2) / 2 + eta_m = R                     (dynamic)

plus mean depth d (trapezoidal mean of eta over the half period, exact for
cosine series of degree < 2N) and crest-to-trough height H.  Newton's method
with a finite-difference Jacobian solves the 2N + 4 equations, stepping the
height up from linear theory (Airy) in a few increments.  The phase speed
follows from the current criterion: c = ubar + c_E, and c_E = 0 here (no mean
Eulerian current, Stokes' first definition).

The result is input data only: the surface elevation and the fixed-frame
velocities at the sigma nodes at t = 0 (crest at x = 0).  The steepness limit
of Battjes (1974) that the paper uses to place the experiments is
(H/L)_max = 0.1401 tanh(0.8863 kh).
"""
import math

import numpy as np

G = 9.81


def battjes_max_steepness(kh):
    """(H/L)_max = 0.1401 tanh(0.8863 kh) (Battjes 1974, quoted in Sec. 5.1)."""
    return 0.1401 * math.tanh(0.8863 * kh)


def _ratios(j, y, d):
    """sinh(j y)/cosh(j d) and cosh(j y)/cosh(j d) without overflow."""
    den = 1.0 + np.exp(-2.0 * j * d)
    a = np.exp(j * (y - d))
    b = np.exp(-j * (y + d))
    return (a - b) / den, (a + b) / den


class FentonWave:
    """Converged Fourier solution for one (kd, kH); nondimensional (k = g = 1)."""

    def __init__(self, kd, kH, n_modes=32, height_steps=None, c_e=0.0, tol=1e-12, max_newton=40, start=None):
        if kd <= 0 or kH <= 0 or n_modes < 2:
            raise ValueError("need kd > 0, kH > 0, n_modes >= 2")
        self.kd, self.kH, self.N, self.c_e = float(kd), float(kH), int(n_modes), float(c_e)
        N = self.N
        self.Xm = np.arange(N + 1) * (math.pi / N)
        self.j = np.arange(1, N + 1, dtype=float)
        if start is not None and start.kd == self.kd and start.kH == self.kH:
            # a converged solution with fewer modes: its surface at the new points, its B padded with zeros
            z = np.zeros(2 * N + 4)
            z[:N + 1] = start.surface(self.Xm)
            nb = min(N, start.N)
            z[N + 1:N + 1 + nb] = start.B[:nb]
            z[2 * N + 1:] = [start.ubar, start.Q, start.R]
            self.height_steps = 0
            self._finish(self._newton(z, kH, tol, max_newton))
            return
        lim = 2 * math.pi * battjes_max_steepness(kd)
        if height_steps is None:
            height_steps = max(1, int(math.ceil(10.0 * kH / lim)))
        self.height_steps = height_steps
        sols = []
        for s in range(1, height_steps + 1):
            H = kH * s / height_steps
            if not sols:
                guess = self._linear_guess(H)
            elif len(sols) == 1:
                guess = sols[-1]
            else:
                guess = 2.0 * sols[-1] - sols[-2]       # linear extrapolation in the height
            sols.append(self._newton(guess, H, tol, max_newton))
        self._finish(sols[-1])

    def _finish(self, z):
        N = self.N
        self.z = z
        self.eta_m = z[:N + 1]
        self.B = z[N + 1:2 * N + 1]
        self.ubar, self.Q, self.R = z[2 * N + 1], z[2 * N + 2], z[2 * N + 3]
        self.c = self.ubar + self.c_e
        # cosine coefficients of eta (about the bed) from the N + 1 collocation values
        w = np.ones(N + 1)
        w[0] = w[-1] = 0.5
        E = np.array([(2.0 / N) * np.sum(w * self.eta_m * np.cos(jj * self.Xm)) for jj in range(N + 1)])
        E[0] *= 0.5
        E[N] *= 0.5
        self.E = E

    # ---- the nonlinear system ----
    def _unpack(self, z):
        N = self.N
        return z[:N + 1], z[N + 1:2 * N + 1], z[2 * N + 1], z[2 * N + 2], z[2 * N + 3]

    def _velocities(self, X, y, B, ubar):
        """Moving-frame u = psi_y and v = -psi_X at points (X, y)."""
        jj = self.j[:, None]
        sh, ch = _ratios(jj, y[None, :], self.kd)
        cs = np.cos(jj * X[None, :])
        sn = np.sin(jj * X[None, :])
        jb = (self.j * B)[:, None]
        u = -ubar + np.sum(jb * ch * cs, axis=0)
        v = np.sum(jb * sh * sn, axis=0)
        return u, v

    def _psi(self, X, y, B, ubar):
        jj = self.j[:, None]
        sh, _ = _ratios(jj, y[None, :], self.kd)
        return -ubar * y + np.sum(B[:, None] * sh * np.cos(jj * X[None, :]), axis=0)

    def residual(self, z, H):
        eta, B, ubar, Q, R = self._unpack(z)
        N = self.N
        kin = self._psi(self.Xm, eta, B, ubar) + Q
        u, v = self._velocities(self.Xm, eta, B, ubar)
        dyn = 0.5 * (u * u + v * v) + eta - R
        mean = (0.5 * eta[0] + eta[1:N].sum() + 0.5 * eta[N]) / N - self.kd
        return np.concatenate([kin, dyn, [mean, eta[0] - eta[N] - H]])

    def _linear_guess(self, H):
        N, d = self.N, self.kd
        c0 = math.sqrt(math.tanh(d))
        z = np.zeros(2 * N + 4)
        z[:N + 1] = d + 0.5 * H * np.cos(self.Xm)
        z[N + 1] = c0 * 0.5 * H / math.tanh(d)
        z[2 * N + 1] = c0
        z[2 * N + 2] = c0 * d
        z[2 * N + 3] = 0.5 * c0 * c0 + d
        return z

    def _newton(self, z, H, tol, max_newton):
        n = z.size
        for _ in range(max_newton):
            f = self.residual(z, H)
            if np.abs(f).max() < tol:
                return z
            J = np.empty((n, n))
            for i in range(n):
                hstep = 1e-7 * max(1.0, abs(z[i]))
                zp = z.copy()
                zp[i] += hstep
                zm = z.copy()
                zm[i] -= hstep
                J[:, i] = (self.residual(zp, H) - self.residual(zm, H)) / (2 * hstep)
            z = z - np.linalg.solve(J, f)
        f = self.residual(z, H)
        if np.abs(f).max() >= 1e3 * tol:
            raise RuntimeError("Fenton's Newton iteration did not converge (|f| = %.3e)" % np.abs(f).max())
        return z

    # ---- evaluation (nondimensional, fixed frame, t = 0, crest at x = 0) ----
    def surface(self, X):
        """Surface height above the bed at phase X."""
        X = np.asarray(X, dtype=float)
        return np.sum(self.E[:, None] * np.cos(np.arange(self.N + 1)[:, None] * X.ravel()[None, :]),
                      axis=0).reshape(X.shape)

    def fixed_frame_velocity(self, X, y):
        """Fixed-frame (u, w) = moving-frame (u + c, v) at phase X and height y above the bed."""
        X = np.asarray(X, dtype=float).ravel()
        y = np.asarray(y, dtype=float).ravel()
        u, v = self._velocities(X, y, self.B, self.ubar)
        return u + self.c, v


def converged_wave(kd, kH, tail=1e-10, modes=(32, 48, 64, 96)):
    """The first of the mode counts whose surface series has decayed to `tail`
    (|E_N| <= tail |E_1|); the shallow steep waves need the most.  Raises if
    none does (a wave too close to breaking for these mode counts)."""
    w = None
    for n in modes:
        w = FentonWave(kd, kH, n_modes=n, start=w)
        if abs(w.E[n]) <= tail * abs(w.E[1]):
            return w
    raise RuntimeError("stream-function series not converged with %d modes (|E_N|/|E_1| = %.1e)"
                       % (modes[-1], abs(w.E[-1] / w.E[1])))


def stream_function_fields(x, h, nz, wave, k, g=G):
    """eta (nx,) about the still level and fixed-frame u, w at every node
    ((nz + 1) * nx, ghost level first) of a flat-bed slice of depth h."""
    if abs(k * h - wave.kd) > 1e-12 * max(1.0, wave.kd):
        raise ValueError("the wave was computed for kh = %g, the grid has kh = %g" % (wave.kd, k * h))
    X = k * np.asarray(x, dtype=float)
    eta = wave.surface(X) / k - h
    s = np.arange(-1, nz) / (nz - 1.0)
    ynode = s[:, None] * (h + eta)[None, :]             # height above the bed of every node
    Xn = np.broadcast_to(X[None, :], ynode.shape)
    u, w = wave.fixed_frame_velocity(Xn, k * ynode)
    vs = math.sqrt(g / k)
    return eta, (u * vs).ravel(), (w * vs).ravel()
