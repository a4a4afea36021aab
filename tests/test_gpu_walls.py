"""GPU parity for the wall-bounded flume (walls with ghost columns, the
seven-group ILU order, generation/absorption zones), through the C ABI,
against the oracle on the same seeded inputs.

Tolerances as in test_gpu_parity.py: operator 1e-12 (|A| |p|) element-wise;
preconditioner 1e-10 relative; solves to 1e-12 within 1e-10; iteration counts
+-1; stage-driver fields within 1e-9 relative per stage (solves to 1e-12).
The precision form (FP32 inner cycles, FP64 refinement) meets 1e-8 against the
FP64 oracle.
"""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda"


@pytest.fixture(scope="module")
def sw():
    from paper_2511_18071_gb300 import build
    build.build()
    import paper_2511_18071_gb300 as sw
    assert torch.cuda.is_available()
    return sw


def _t(a):
    return torch.tensor(np.ascontiguousarray(a, dtype=np.float64), device=DEV)


def _bar(x, lx):
    h = 1.0 - 0.3 * np.exp(-4 * (x - 0.5 * lx) ** 2)
    h[0], h[-1] = h[1], h[-2]
    return h


def _cases():
    out = []
    for name, nx, nz in [("flat_walls", 68, 9), ("bar_walls", 68, 9), ("bar_walls_nz17", 32, 17)]:
        lx = 3.0
        x = W.wall_x(nx, lx)
        h = np.ones(nx) if name.startswith("flat") else _bar(x, lx)
        out.append((name, nx, nz, lx, h))
    return out


def _surfaces(nx, lx, seed):
    rng = np.random.default_rng(seed)
    x = W.wall_x(nx, lx)
    e1 = 0.03 * np.cos(2 * x + rng.uniform(0, 6)) + 0.01 * np.sin(5 * x)
    e2 = e1 + 0.002 * np.cos(3 * x + rng.uniform(0, 6))
    return e1, e2


def _rhs(ora, nz, seed):
    b = np.random.default_rng(seed).standard_normal(ora.m)
    b[ora.index(0, 0, nz - 1):] = 0.0
    return b


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c[0])
def test_walls_apply_operator(sw, case):
    name, nx, nz, lx, h = case
    gpu = sw.Problem(nx, 1, nz, lx, 0.0, h, walls=True)
    ora = O.OracleProblem(nx, 1, nz, lx, 0.0, h, walls=True)
    e1, e2 = _surfaces(nx, lx, 1)
    p = np.random.default_rng(2).standard_normal(ora.m)
    ora.assemble(e1, e2)
    A = ora.matrix()
    ref = A @ p
    bound = abs(A) @ np.abs(p)
    y = torch.empty(gpu.m, dtype=torch.float64, device=DEV)
    sw.apply_operator(gpu.handle, _t(e1), _t(e2), _t(p), y)
    torch.cuda.synchronize()
    err = np.abs(y.cpu().numpy() - ref)
    assert np.all(err <= 1e-12 * bound + 1e-300), (name, (err / bound).max())


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c[0])
def test_walls_apply_preconditioner(sw, case):
    name, nx, nz, lx, h = case
    gpu = sw.Problem(nx, 1, nz, lx, 0.0, h, walls=True)
    ora = O.OracleProblem(nx, 1, nz, lx, 0.0, h, walls=True)
    v = np.random.default_rng(3).standard_normal(ora.m)
    ref = ora.ilu_apply(v)
    out = torch.empty(gpu.m, dtype=torch.float64, device=DEV)
    sw.apply_preconditioner(gpu.handle, _t(v), out)
    torch.cuda.synchronize()
    err = np.abs(out.cpu().numpy() - ref).max() / np.abs(ref).max()
    assert err < 1e-10, (name, err)


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c[0])
@pytest.mark.parametrize("executor", ["persistent", "streamed"])
def test_walls_cold_solve_tight(sw, case, executor):
    name, nx, nz, lx, h = case
    kw = dict(restart=20, max_restarts=300, tol=1e-12, guess="cold")
    gpu = sw.Problem(nx, 1, nz, lx, 0.0, h, walls=True, executor=executor, **kw)
    ora = O.OracleProblem(nx, 1, nz, lx, 0.0, h, walls=True, **kw)
    e1, e2 = _surfaces(nx, lx, 4)
    b = _rhs(ora, nz, 5)
    xo, so, co = ora.solve(e1, e2, b)
    x = torch.zeros(gpu.m, dtype=torch.float64, device=DEV)
    gpu.solve(_t(e1), _t(e2), _t(b), x)
    sg = gpu.stats()
    assert co == 0 and sg["status"] == 0, (so, sg)
    err = np.linalg.norm(x.cpu().numpy() - xo) / np.linalg.norm(xo)
    assert err <= 1e-10, (name, err, so, sg)
    assert abs(sg["iterations"] - so["iterations"]) <= 1, (sg, so)


@pytest.mark.parametrize("executor", ["persistent", "streamed"])
def test_walls_mixed_precision_solve(sw, executor):
    name, nx, nz, lx, h = _cases()[1]
    kw = dict(restart=20, max_restarts=300, tol=1e-10, guess="cold")
    gpu = sw.Problem(nx, 1, nz, lx, 0.0, h, walls=True, precision="mixed", executor=executor, **kw)
    ora = O.OracleProblem(nx, 1, nz, lx, 0.0, h, walls=True, **dict(kw, tol=1e-13))
    e1, e2 = _surfaces(nx, lx, 6)
    b = _rhs(ora, nz, 7)
    xo, so, co = ora.solve(e1, e2, b)
    x = torch.zeros(gpu.m, dtype=torch.float64, device=DEV)
    gpu.solve(_t(e1), _t(e2), _t(b), x)
    sg = gpu.stats()
    assert sg["status"] == 0, sg
    err = np.linalg.norm(x.cpu().numpy() - xo) / np.linalg.norm(xo)
    assert err <= 1e-8, err


def _flume_run(sw, wl, nsteps, kw, check_every_stage=True, tol=1e-9):
    """Advance the oracle and the library side by side; relaxation after every stage."""
    ora = O.OracleProblem(wl["nx"], 1, wl["nz"], wl["lx"], 0.0, wl["h"], walls=True, **kw)
    gpu = sw.Problem(wl["nx"], 1, wl["nz"], wl["lx"], 0.0, wl["h"], walls=True, **kw)
    st = W.state_arrays(wl)
    sw.set_physics(gpu.handle, sw.Physics(wl["g"], wl["rho"], wl["dt"]))
    sw.set_state(gpu.handle, _t(wl["u"]), None, _t(wl["w"]), _t(wl["eta"]))
    sw.set_relaxation(gpu.handle, wl["relax"])
    phys = (wl["g"], wl["rho"], wl["dt"])
    _, _, C = O.lserk45()
    u = torch.empty(gpu.m, dtype=torch.float64, device=DEV)
    w = torch.empty_like(u)
    pr = torch.empty_like(u)
    eta = torch.empty(gpu.ncol, dtype=torch.float64, device=DEV)
    diffs = []
    for step in range(nsteps):
        for i in range(1, 6):
            p, so, code = ora.stage(phys, i, st)
            assert code == 0
            ora.relax(wl["relax"], (step + (C[i] if i < 5 else 1.0)) * wl["dt"], st)
            sw.advance_stage(gpu.handle)
            sg = gpu.stats()
            assert sg["status"] == 0, sg
            diffs.append(sg["iterations"] - so["iterations"])
            if check_every_stage or (step == nsteps - 1 and i == 5):
                sw.get_state(gpu.handle, u=u, w=w, eta=eta, pres=pr)
                torch.cuda.synchronize()
                for nm, g_, o_ in [("eta", eta, st["eta"]), ("u", u, st["u"]), ("w", w, st["w"]), ("p", pr, p)]:
                    err = np.abs(g_.cpu().numpy() - o_).max() / max(np.abs(o_).max(), 1e-300)
                    assert err < tol, (step, i, nm, err)
    return np.array(diffs), st


def test_flume_stage_driver_with_relaxation(sw):
    # no time ramp, so the generation zone forces the full incident wave from the first stage
    wl = W.flume_2d(nx=132, nz=9, lx=12.0, depth=0.4, gen=(0.0, 3.0), absorb=(8.6, 12.0), ramp_periods=0.0)
    kw = dict(restart=20, max_restarts=200, tol=1e-12, guess="previous")
    diffs, st = _flume_run(sw, wl, 3, kw)
    assert np.abs(st["eta"]).max() > 1e-3          # the zone has driven a wave into the flume


def test_flume_trajectory_iterations_ewma(sw):
    wl = W.flume_2d(nx=132, nz=9, lx=12.0, depth=0.4, gen=(0.0, 3.0), absorb=(8.6, 12.0), ramp_periods=0.0)
    kw = dict(restart=20, max_restarts=100, tol=1e-8, guess="ewma", k=8, decay=0.9, n_init_solves=10)
    diffs, _ = _flume_run(sw, wl, 8, kw, check_every_stage=False, tol=1e-6)
    assert np.all(np.abs(diffs) <= 1), diffs
    assert np.count_nonzero(diffs) <= len(diffs) // 5, diffs


def test_bar_flume_full_size(sw):
    # the 2048 x 17 flume over the trapezoidal bar, x in [0, 40], two steps
    wl = W.flume_2d(ramp_periods=0.0)
    kw = dict(restart=20, max_restarts=200, tol=1e-12, guess="previous")
    _flume_run(sw, wl, 2, kw, check_every_stage=False)


def test_walls_reject_bad_grids(sw):
    h = np.ones(12)
    with pytest.raises(sw.SawaveError):
        sw.Problem(12, 1, 9, 1.0, 0.0, h, walls=True)            # nx < 16
    with pytest.raises(sw.SawaveError):
        sw.Problem(16, 8, 9, 1.0, 1.0, np.ones(128), walls=True)  # walls are 2-D only
