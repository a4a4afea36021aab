"""GPU parity at the benchmark's full sizes, in the launch configuration the
benchmark times (the executor chosen by size: the persistent kernel for the
512 x 17 steep wave, the streamed kernels for the 256 x 256 x 17 field), by
checks that hold at any size:

- operator apply: element-wise within 1e-12 (|A| |p|), the rounding bound of
  a sum of at most 91 products, as in test_gpu_parity.py;
- ILU(0) apply: within 1e-10 of max |out|;
- subspace guess on a fixed random sketch (sw_set_sketch): within 1e-8
  relative (CholeskyQR2 on the device, Householder QR in the oracle; the
  operator's condition grows with the grid);
- a solve in the benchmark's configuration meets the stopping test as the
  oracle evaluates it, ||M^-1 (b - A x)|| <= tol ||M^-1 b|| (x 1.01 in FP64,
  x 1.5 in the precision form, whose restart residual goes through the FP32
  factors);
- 512 x 17: two steps of the stage driver at tol 1e-12 agree with the
  oracle's within 1e-9 relative after every stage.

Iteration counts are not compared here: at these sizes single solves are
chaotic in the rounding (on the 512 x 17 wave the oracle's first solve takes
656, 714 or 809 iterations after relative perturbations of eta of 0, 1e-12
and 1e-11); per-solve counts are compared on shared systems in
test_gpu_parity.py.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda"
BENCH_KW = dict(restart=20, max_restarts=500, tol=1e-8, guess="ewma", k=10, decay=0.9, n_init_solves=30,
                seed=2511, executor="auto")


@pytest.fixture(scope="module")
def sw():
    from paper_2511_18071_gb300 import build
    build.build()
    import paper_2511_18071_gb300 as sw
    assert torch.cuda.is_available()
    return sw


def _t(a):
    return torch.tensor(np.ascontiguousarray(a, dtype=np.float64), device=DEV)


def surfaces(wl, seed):
    """eta of the workload and a second surface a small seeded step away."""
    e1 = wl["eta"]
    rng = np.random.default_rng(seed)
    e2 = e1 + 0.002 * np.cos(np.arange(e1.size) * (2 * np.pi / e1.size) * 3 + rng.uniform(0, 6))
    return e1, e2


def rhs(ora, seed):
    b = np.random.default_rng(seed).standard_normal(ora.m)
    b[ora.index(0, 0, ora.nz - 1):] = 0.0           # surface rows: Dirichlet
    return b


def operator_error(ora, p, y):
    """max over rows of |y - A p| / (|A| |p|)."""
    A = ora.matrix()
    ref = A @ p
    bound = abs(A) @ np.abs(p)
    return float((np.abs(y - ref) / (bound + 1e-300)).max())


def preconditioned_residual(ora, b, x):
    """||M^-1 (b - A x)|| / ||M^-1 b|| with the oracle's operator and factors."""
    r = b - ora.matvec(x)
    return float(np.linalg.norm(ora.ilu_apply(r)) / np.linalg.norm(ora.ilu_apply(b)))


def headline():
    return W.stokes_like_2d(nx=512, nz=17, kh=2.0, a1_over_h=0.08, steps=1000)


def field3d():
    return W.bumpy_3d(nx=256, ny=256, nz=17)


@pytest.fixture(scope="module")
def oracle_3d():
    wl = field3d()
    ora = O.OracleProblem(wl["nx"], wl["ny"], wl["nz"], wl["lx"], wl["ly"], wl["h"], guess="ewma", k=10)
    return wl, ora


def _check_operator_and_ilu(sw, wl, ora, gpu, seed):
    e1, e2 = surfaces(wl, seed)
    ora.assemble(e1, e2)
    p = np.random.default_rng(seed + 1).standard_normal(ora.m)
    y = torch.empty(gpu.m, dtype=torch.float64, device=DEV)
    sw.apply_operator(gpu.handle, _t(e1), _t(e2), _t(p), y)
    v = np.random.default_rng(seed + 2).standard_normal(ora.m)
    out = torch.empty(gpu.m, dtype=torch.float64, device=DEV)
    sw.apply_preconditioner(gpu.handle, _t(v), out)
    torch.cuda.synchronize()
    assert operator_error(ora, p, y.cpu().numpy()) <= 1e-12
    ref = ora.ilu_apply(v)
    assert np.abs(out.cpu().numpy() - ref).max() <= 1e-10 * np.abs(ref).max()


def _check_guess(sw, wl, ora, gpu, seed):
    k = BENCH_KW["k"]
    Y = np.random.default_rng(seed).standard_normal((ora.m, k))
    ora.set_sketch(Y)
    sw.set_sketch(gpu.handle, _t(Y.T.ravel()), 0)
    e1, e2 = surfaces(wl, seed + 1)
    b = rhs(ora, seed + 2)
    ora.assemble(e1, e2)
    x0o, rank = ora.ewma_guess(b)
    x0 = torch.empty(gpu.m, dtype=torch.float64, device=DEV)
    sw.subspace_guess(gpu.handle, _t(e1), _t(e2), _t(b), x0)
    torch.cuda.synchronize()
    err = np.linalg.norm(x0.cpu().numpy() - x0o) / np.linalg.norm(x0o)
    assert rank == k and err < 1e-8, err


def _check_solve(sw, wl, ora, gpu, seed, factor):
    e1, e2 = surfaces(wl, seed)
    b = rhs(ora, seed + 1)
    x = torch.zeros(gpu.m, dtype=torch.float64, device=DEV)
    gpu.solve(_t(e1), _t(e2), _t(b), x)
    sg = gpu.stats()
    assert sg["status"] == 0, sg
    ora.assemble(e1, e2)
    rel = preconditioned_residual(ora, b, x.cpu().numpy())
    assert rel <= factor * BENCH_KW["tol"], (rel, sg)


def test_headline_512x17_operator_ilu_guess_solve(sw):
    wl = headline()
    ora = O.OracleProblem(wl["nx"], 1, wl["nz"], wl["lx"], 0.0, wl["h"], guess="ewma", k=10)
    gpu = sw.Problem(wl["nx"], 1, wl["nz"], wl["lx"], 0.0, wl["h"], precision="fp64", **BENCH_KW)
    _check_operator_and_ilu(sw, wl, ora, gpu, 1)
    _check_guess(sw, wl, ora, gpu, 11)
    gpu.close()
    gpu = sw.Problem(wl["nx"], 1, wl["nz"], wl["lx"], 0.0, wl["h"], precision="fp64", **BENCH_KW)
    _check_solve(sw, wl, ora, gpu, 21, 1.01)
    gpu.close()


def test_headline_512x17_stage_driver_tight(sw):
    wl = headline()
    kw = dict(restart=20, max_restarts=200, tol=1e-12, guess="previous")
    ora = O.OracleProblem(wl["nx"], 1, wl["nz"], wl["lx"], 0.0, wl["h"], **kw)
    gpu = sw.Problem(wl["nx"], 1, wl["nz"], wl["lx"], 0.0, wl["h"], **kw)
    st = W.state_arrays(wl)
    sw.set_physics(gpu.handle, sw.Physics(wl["g"], wl["rho"], wl["dt"]))
    sw.set_state(gpu.handle, _t(wl["u"]), None, _t(wl["w"]), _t(wl["eta"]))
    phys = (wl["g"], wl["rho"], wl["dt"])
    u = torch.empty(gpu.m, dtype=torch.float64, device=DEV)
    w = torch.empty_like(u)
    pr = torch.empty_like(u)
    eta = torch.empty(gpu.ncol, dtype=torch.float64, device=DEV)
    for step in range(2):
        for i in range(1, 6):
            p, so, code = ora.stage(phys, i, st)
            assert code == 0
            sw.advance_stage(gpu.handle)
            assert gpu.stats()["status"] == 0
            sw.get_state(gpu.handle, u=u, w=w, eta=eta, pres=pr)
            torch.cuda.synchronize()
            for name, g_, o_ in [("eta", eta, st["eta"]), ("u", u, st["u"]), ("w", w, st["w"]), ("p", pr, p)]:
                err = np.abs(g_.cpu().numpy() - o_).max() / max(np.abs(o_).max(), 1e-300)
                assert err < 1e-9, (step, i, name, err)
    gpu.close()


def test_field_256x256x17_operator_ilu_guess(sw, oracle_3d):
    wl, ora = oracle_3d
    gpu = sw.Problem(wl["nx"], wl["ny"], wl["nz"], wl["lx"], wl["ly"], wl["h"], precision="fp64", **BENCH_KW)
    _check_operator_and_ilu(sw, wl, ora, gpu, 31)
    _check_guess(sw, wl, ora, gpu, 41)
    gpu.close()


def test_field_256x256x17_precision_form_solve(sw, oracle_3d):
    wl, ora = oracle_3d
    gpu = sw.Problem(wl["nx"], wl["ny"], wl["nz"], wl["lx"], wl["ly"], wl["h"], precision="mixed", **BENCH_KW)
    _check_solve(sw, wl, ora, gpu, 51, 1.5)
    gpu.close()
