"""Helpers for the GPU iteration tests: oracle runs of the 512 x 17 benchmark
trajectory under seeded 1e-13 relative perturbations of the initial surface,
run in spawned worker processes (test infrastructure; no GPU is used here)."""
import numpy as np

HEADLINE_KW = dict(restart=20, max_restarts=500, tol=1e-8, guess="ewma", k=10, decay=0.9, n_init_solves=30,
                   seed=2511)


def headline_workload(seed):
    """The benchmark's workload; seed 0 unperturbed, seed s > 0 with eta scaled by 1 + 1e-13 N(0, 1)."""
    import workloads as W
    wl = W.stokes_like_2d(nx=512, nz=17, kh=2.0, a1_over_h=0.08, steps=1000)
    if seed:
        wl["eta"] = wl["eta"] * (1 + 1e-13 * np.random.default_rng(seed).standard_normal(wl["eta"].size))
    return wl


def oracle_iterations(args):
    """Iteration count of every solve of an oracle run: (seed, steps) -> list."""
    seed, nsteps = args
    import oracle as O
    import workloads as W
    wl = headline_workload(seed)
    P = O.OracleProblem(wl["nx"], 1, wl["nz"], wl["lx"], 0.0, wl["h"], **HEADLINE_KW)
    st = W.state_arrays(wl)
    phys = (wl["g"], wl["rho"], wl["dt"])
    its = []
    for _ in range(nsteps):
        for i in range(1, 6):
            _, so, code = P.stage(phys, i, st)
            assert code == 0
            its.append(so["iterations"])
    return its
