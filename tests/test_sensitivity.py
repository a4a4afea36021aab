"""How far the oracle's iteration counts move under rounding-level
perturbations: the measurement behind the GPU-vs-oracle iteration bands.

The GPU and the oracle each run their own stage driver, so their trajectories
differ by rounding (different summation orders, a different least-squares
method).  Here the oracle is run against itself with the initial surface
perturbed by 1e-13 relative (seeded), on the two trajectories whose
iteration counts the GPU tests compare:

- the 512 x 17 steep wave of the benchmark (EWMA, k = 10, r = 0.9), window =
  solves 30..124 (after the history fill);
- the paper's stream-function run at kh = 2, 0.7 of the breaking limit
  (k = 10, r = 0.7, range finder K = 15), window = solves 30..119.

Findings (pinned below): single-solve counts are chaotic (a large share of the
window's solves change count, by up to tens of iterations), so counts along
independent trajectories are compared only as window means, and solve by solve
only on shared inputs (tests/test_gpu_iterations.py, test_gpu_parity.py).
Over 8 perturbations the window mean moved by up to 9.5 % on the 512 x 17 wave
(standard deviation 5.4 %) and up to 19.4 % (EWMA) and 19.1 % (range finder)
on the stream-function wave (standard deviations 6.2 % and 6.7 %).  The
stream-function GPU tests use a band of 25 % (about four standard deviations)
and the 512 x 17 GPU test compares nine-member ensemble means within 10 %;
the runs here check that the oracle stays inside these bands against itself,
so a band never asks more of the GPU than the oracle can meet.  On the
GPU machine, nine-member ensembles of the 512 x 17 window mean came out at 24.2
(persistent kernel), 24.6 (resident executor) and 25.3 (oracle), with
standard deviations 1.4-1.8 per run: no systematic difference.
"""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W

# largest move of one run's window mean under the perturbations: the 512 x 17
# wave, and the stream-function runs (the band of tests/test_gpu_stream_function.py)
BAND_HEADLINE = 0.15
BAND_STREAM = 0.25
# two nine-member ensembles of the 512 x 17 window mean: with a spread of at most
# 8 % per run (asserted below), the standard error of the difference of the two
# ensemble means is at most 8 % x sqrt(2/9) = 3.8 %; the band is 10 %
ENSEMBLE_BAND = 0.10


def _run(wl, kw, nsteps, eps, seed):
    P = O.OracleProblem(wl["nx"], 1, wl["nz"], wl["lx"], 0.0, wl["h"], **kw)
    st = W.state_arrays(wl)
    if eps:
        st["eta"] = st["eta"] * (1 + eps * np.random.default_rng(seed).standard_normal(st["eta"].size))
    phys = (wl["g"], wl["rho"], wl["dt"])
    its = []
    for _ in range(nsteps):
        for i in range(1, 6):
            _, so, code = P.stage(phys, i, st)
            assert code == 0
            its.append(so["iterations"])
    return np.array(its)


def _spread(wl, kw, nsteps, seeds):
    base = _run(wl, kw, nsteps, 0.0, 0)[30:]
    rel, frac, maxd = [], [], []
    for s in seeds:
        r = _run(wl, kw, nsteps, 1e-13, s)[30:]
        rel.append(r.mean() / base.mean() - 1)
        frac.append(np.mean(r != base))
        maxd.append(np.abs(r - base).max())
    return np.array(rel), np.array(frac), np.array(maxd), base


def test_headline_trajectory_sensitivity():
    wl = W.stokes_like_2d(nx=512, nz=17, kh=2.0, a1_over_h=0.08, steps=1000)
    kw = dict(restart=20, max_restarts=500, tol=1e-8, guess="ewma", k=10, decay=0.9, n_init_solves=30, seed=2511)
    rel, frac, maxd, base = _spread(wl, kw, 25, (1, 3, 5))
    # single solves: chaotic in the rounding
    assert frac.min() > 0.5 and maxd.max() >= 20, (frac, maxd)
    # window means: within the band the GPU test uses
    assert np.abs(rel).max() <= BAND_HEADLINE, rel
    # spread of one run's window mean (relative standard deviation of the four runs)
    means = np.concatenate([[1.0], 1.0 + rel])
    assert means.std(ddof=1) / means.mean() <= 0.08, means


@pytest.mark.parametrize("guess", ["ewma", "rrf"])
def test_stream_function_sensitivity(guess):
    wl = W.stream_function_2d(kh=2.0, steepness=0.7, dt=1e-4 * math.sqrt(1.0 / 9.81))
    kw = dict(restart=20, max_restarts=100, tol=1e-8, guess=guess, k=10, decay=0.7, n_init_solves=30)
    if guess == "rrf":
        kw["history"] = 15
    rel, frac, maxd, base = _spread(wl, kw, 24, (1, 2, 3, 4))
    assert frac.min() > 0.3 and maxd.max() >= 5, (frac, maxd)
    assert np.abs(rel).max() <= BAND_STREAM, rel
