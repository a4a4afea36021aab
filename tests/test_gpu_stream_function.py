"""GPU parity on the paper's stream-function wave runs (Sec. 5.1: a periodic
200 x 20 slice, K = 15, k = 10, r = 0.7, six steps on the previous solution
before the subspace guess; here with a step of 3.19e-5 s, a third of the
paper's): the library's stage driver, through the C ABI, against the oracle's
on the same Fenton initial condition.

Tolerances: with solves to 1e-12 the fields agree to 1e-9 relative after
every stage (as in test_gpu_parity.py).  With the paper's 1e-8 the fields agree
to 1e-6 after the run, the previous-solution warm-up solves to +-2 iterations
and the mean iteration count of the 90 subspace-guess solves to the band
BAND_STREAM (25 %).  Solve-by-solve counts are not compared on this run: they
are chaotic in the rounding.  The band comes from the oracle against itself
(tests/test_sensitivity.py): with eta perturbed by 1e-13 relative, the same
window's mean moved by up to 19 % (standard deviation 6-7 %) over 8 seeds.
The per-solve comparisons on shared systems are in test_gpu_parity.py and
test_gpu_iterations.py.
"""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W
from test_sensitivity import BAND_STREAM

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda"
DT = 1e-4 * math.sqrt(1.0 / 9.81)


@pytest.fixture(scope="module")
def sw():
    from paper_2511_18071_gb300 import build
    build.build()
    import paper_2511_18071_gb300 as sw
    assert torch.cuda.is_available()
    return sw


def _t(a):
    return torch.tensor(np.ascontiguousarray(a, dtype=np.float64), device=DEV)


def _run(sw, wl, nsteps, kw, executor, every_stage, tol):
    ora = O.OracleProblem(wl["nx"], 1, wl["nz"], wl["lx"], 0.0, wl["h"], **kw)
    gpu = sw.Problem(wl["nx"], 1, wl["nz"], wl["lx"], 0.0, wl["h"], executor=executor, **kw)
    st = W.state_arrays(wl)
    sw.set_physics(gpu.handle, sw.Physics(wl["g"], wl["rho"], wl["dt"]))
    sw.set_state(gpu.handle, _t(wl["u"]), None, _t(wl["w"]), _t(wl["eta"]))
    phys = (wl["g"], wl["rho"], wl["dt"])
    u = torch.empty(gpu.m, dtype=torch.float64, device=DEV)
    w = torch.empty_like(u)
    pr = torch.empty_like(u)
    eta = torch.empty(gpu.ncol, dtype=torch.float64, device=DEV)
    its = []
    for step in range(nsteps):
        for i in range(1, 6):
            p, so, code = ora.stage(phys, i, st)
            assert code == 0
            sw.advance_stage(gpu.handle)
            sg = gpu.stats()
            assert sg["status"] == 0, sg
            its.append((sg["iterations"], so["iterations"]))
            if every_stage or (step == nsteps - 1 and i == 5):
                sw.get_state(gpu.handle, u=u, w=w, eta=eta, pres=pr)
                torch.cuda.synchronize()
                for nm, g_, o_ in [("eta", eta, st["eta"]), ("u", u, st["u"]), ("w", w, st["w"]), ("p", pr, p)]:
                    err = np.abs(g_.cpu().numpy() - o_).max() / max(np.abs(o_).max(), 1e-300)
                    assert err < tol, (step, i, nm, err)
    gpu.close()
    return np.array(its)


@pytest.mark.parametrize("kh,steep", [(0.4, 0.7), (2.0, 0.7), (4.0, 0.3)])
@pytest.mark.parametrize("executor", ["persistent", "streamed"])
def test_stage_driver_tight(sw, kh, steep, executor):
    wl = W.stream_function_2d(kh=kh, steepness=steep, dt=DT)
    kw = dict(restart=20, max_restarts=200, tol=1e-12, guess="previous")
    _run(sw, wl, 2, kw, executor, True, 1e-9)


@pytest.mark.parametrize("guess", ["ewma", "rrf"])
@pytest.mark.parametrize("executor", ["persistent", "streamed"])
def test_paper_subspace_run_iterations(sw, guess, executor):
    wl = W.stream_function_2d(kh=2.0, steepness=0.7, dt=DT)
    kw = dict(restart=20, max_restarts=100, tol=1e-8, guess=guess, k=10, decay=0.7, n_init_solves=30)
    if guess == "rrf":
        kw["history"] = 15
    its = _run(sw, wl, 24, kw, executor, False, 1e-6)
    assert np.all(np.abs(its[:30, 0] - its[:30, 1]) <= 2), its[:30].T     # previous-solution warm-up
    g, o = its[30:, 0].mean(), its[30:, 1].mean()
    assert abs(g - o) <= BAND_STREAM * o, (g, o, its[30:].T)
