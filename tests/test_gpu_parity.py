"""GPU parity: the CUDA library, called through its C ABI, against the oracle on
the same seeded inputs.

Tolerances (FP64 everywhere):
- operator apply: |y_gpu - y_ref| <= 1e-12 (|A| |p|) element by element, the
  rounding bound of a sum of at most 91 products;
- preconditioner: 1e-10 relative to max |out| (the triangular factors amplify
  rounding by their condition number);
- a whole solve run to 1e-12: ||x_gpu - x_ref|| <= 1e-10 ||x_ref||;
- iteration counts at 1e-8: equal up to +-1 (a residual landing within
  rounding of the threshold may stop one step earlier on either side).
"""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sw():
    from paper_2511_18071_gb300 import build
    build.build()
    import paper_2511_18071_gb300 as sw
    assert torch.cuda.is_available()
    return sw


DEV = "cuda"


def _t(a):
    return torch.tensor(np.ascontiguousarray(a, dtype=np.float64), device=DEV)


def _cases():
    L = 2 * math.pi
    out = []
    x64 = np.arange(64) * (L / 64)
    out.append(("flat2d", 64, 1, 9, L, 0.0, np.ones(64)))
    out.append(("bar2d", 64, 1, 9, L, 0.0, 1.0 - 0.4 * np.exp(-3 * (x64 - 3.0) ** 2)))
    out.append(("bar2d_nz33", 32, 1, 33, L, 0.0, 0.8 + 0.1 * np.cos(np.arange(32) * (L / 32))))
    X, Y = np.meshgrid(np.arange(16) * (L / 16), np.arange(8) * (L / 8), indexing="xy")
    out.append(("flat3d", 16, 8, 7, L, L, np.ones(128)))
    out.append(("bumpy3d", 16, 8, 9, L, L, (1.0 + 0.2 * np.exp(-((X - 3) ** 2 + (Y - 2) ** 2))).ravel()))
    return out


def _surfaces(nx, ny, seed):
    rng = np.random.default_rng(seed)
    L = 2 * math.pi
    X, Y = np.meshgrid(np.arange(nx) * (L / nx), np.arange(ny) * (L / ny), indexing="xy")
    e1 = (0.03 * np.cos(X + rng.uniform(0, 6)) + 0.01 * np.sin(2 * X + Y)).ravel()
    e2 = e1 + (0.002 * np.cos(X + Y + rng.uniform(0, 6))).ravel()
    return e1, e2


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c[0])
def test_apply_operator(sw, case):
    name, nx, ny, nz, lx, ly, h = case
    gpu = sw.Problem(nx, ny, nz, lx, ly, h)
    ora = O.OracleProblem(nx, ny, nz, lx, ly, h)
    e1, e2 = _surfaces(nx, ny, 1)
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
def test_apply_preconditioner(sw, case):
    name, nx, ny, nz, lx, ly, h = case
    gpu = sw.Problem(nx, ny, nz, lx, ly, h)
    ora = O.OracleProblem(nx, ny, nz, lx, ly, h)
    v = np.random.default_rng(3).standard_normal(ora.m)
    ref = ora.ilu_apply(v)
    out = torch.empty(gpu.m, dtype=torch.float64, device=DEV)
    sw.apply_preconditioner(gpu.handle, _t(v), out)
    torch.cuda.synchronize()
    err = np.abs(out.cpu().numpy() - ref).max() / np.abs(ref).max()
    assert err < 1e-10, (name, err)


def _rhs(ora, nz, seed):
    b = np.random.default_rng(seed).standard_normal(ora.m)
    b[ora.index(0, 0, nz - 1):] = 0.0
    return b


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c[0])
@pytest.mark.parametrize("executor", ["persistent", "streamed", "resident"])
def test_cold_solve_tight(sw, case, executor):
    name, nx, ny, nz, lx, ly, h = case
    if executor == "resident" and ny > 1:
        pytest.skip("the resident executor serves 2-D problems")
    kw = dict(restart=20, max_restarts=300, tol=1e-12, guess="cold")
    gpu = sw.Problem(nx, ny, nz, lx, ly, h, executor=executor, **kw)
    ora = O.OracleProblem(nx, ny, nz, lx, ly, h, **kw)
    e1, e2 = _surfaces(nx, ny, 4)
    b = _rhs(ora, nz, 5)
    xo, so, co = ora.solve(e1, e2, b)
    x = torch.zeros(gpu.m, dtype=torch.float64, device=DEV)
    gpu.solve(_t(e1), _t(e2), _t(b), x)
    sg = gpu.stats()
    assert co == 0 and sg["status"] == 0, (so, sg)
    err = np.linalg.norm(x.cpu().numpy() - xo) / np.linalg.norm(xo)
    assert err <= 1e-10, (name, err, so, sg)
    assert abs(sg["iterations"] - so["iterations"]) <= 1, (sg, so)
    assert sg["true_res"] < 1e-9


def _record(wl, nsteps, **kw):
    """Systems (eta_prev, eta_cur, b) of an oracle run of the stage driver."""
    ora = O.OracleProblem(wl["nx"], wl["ny"], wl["nz"], wl["lx"], wl["ly"], wl["h"], **kw)
    st = W.state_arrays(wl)
    phys = (wl["g"], wl["rho"], wl["dt"])
    al, be, _ = O.lserk45()
    out = []
    for _ in range(nsteps):
        for i in range(1, 6):
            feta = ora.f_eta(st["u"], st["v"], st["w"], st["eta"])
            keta = al[i - 1] * st["Keta"] + wl["dt"] * feta
            eta_new = st["eta"] + be[i - 1] * keta
            b = ora.rhs(phys, i, st["u"], st["v"], st["w"], st["Ku"], st["Kv"], st["Kw"], st["eta"], eta_new, feta)
            eprev = st["eta"].copy()
            p, s, code = ora.stage(phys, i, st)
            assert code == 0
            np.testing.assert_array_equal(st["eta"], eta_new)
            out.append((eprev, eta_new.copy(), b, p, s))
    return out


@pytest.mark.parametrize("guess", ["previous", "ewma", "rrf"])
@pytest.mark.parametrize("executor", ["persistent", "streamed", "resident"])
def test_trajectory_iterations_and_solutions(sw, guess, executor):
    wl = W.airy_2d()
    kw = dict(restart=20, max_restarts=100, tol=1e-8, guess=guess, k=8, decay=0.9, n_init_solves=10)
    rec = _record(wl, 8, **kw)
    gpu = sw.Problem(wl["nx"], 1, wl["nz"], wl["lx"], 0.0, wl["h"], executor=executor, **kw)
    x = torch.zeros(gpu.m, dtype=torch.float64, device=DEV)
    diffs = []
    for ep, ec, b, p, so in rec:
        gpu.solve(_t(ep), _t(ec), _t(b), x)
        sg = gpu.stats()
        assert sg["status"] == 0
        diffs.append(sg["iterations"] - so["iterations"])
        err = np.linalg.norm(x.cpu().numpy() - p) / np.linalg.norm(p)
        assert err < 1e-6, err          # both meet 1e-8 on the preconditioned residual
    diffs = np.array(diffs)
    assert np.all(np.abs(diffs) <= 1), diffs
    assert np.count_nonzero(diffs) <= len(diffs) // 5, diffs


@pytest.mark.parametrize("executor", ["persistent", "streamed", "resident"])
def test_sketch_after_solves_matches_oracle(sw, executor):
    wl = W.airy_2d()
    kw = dict(restart=20, max_restarts=100, tol=1e-12, guess="ewma", k=5, decay=0.8, n_init_solves=2)
    rec = _record(wl, 1, **kw)
    gpu = sw.Problem(wl["nx"], 1, wl["nz"], wl["lx"], 0.0, wl["h"], executor=executor, **kw)
    ora = O.OracleProblem(wl["nx"], 1, wl["nz"], wl["lx"], 0.0, wl["h"], **kw)
    x = torch.zeros(gpu.m, dtype=torch.float64, device=DEV)
    for ep, ec, b, p, so in rec:
        gpu.solve(_t(ep), _t(ec), _t(b), x)
        ora.solve(ep, ec, b)
    Y = torch.empty(kw["k"] * gpu.m, dtype=torch.float64, device=DEV)
    sw.get_sketch(gpu.handle, Y)
    torch.cuda.synchronize()
    Yg = Y.cpu().numpy().reshape(kw["k"], gpu.m).T
    Yo = ora.sketch()
    assert np.abs(Yg - Yo).max() <= 1e-9 * np.abs(Yo).max()


@pytest.mark.parametrize("executor", ["persistent", "streamed", "resident"])
def test_subspace_guess_matches_oracle(sw, executor):
    nx, nz, L = 64, 9, 2 * math.pi
    x64 = np.arange(nx) * (L / nx)
    h = 1.0 - 0.3 * np.exp(-3 * (x64 - 3.0) ** 2)
    k = 6
    kw = dict(k=k, guess="ewma")
    gpu = sw.Problem(nx, 1, nz, L, 0.0, h, executor=executor, **kw)
    ora = O.OracleProblem(nx, 1, nz, L, 0.0, h, **kw)
    rng = np.random.default_rng(9)
    Y = rng.standard_normal((ora.m, k))
    ora.set_sketch(Y)
    sw.set_sketch(gpu.handle, _t(Y.T.ravel()), 0)
    e1, e2 = _surfaces(nx, 1, 10)
    b = _rhs(ora, nz, 11)
    ora.assemble(e1, e2)
    x0o, rank = ora.ewma_guess(b)
    x0 = torch.empty(gpu.m, dtype=torch.float64, device=DEV)
    sw.subspace_guess(gpu.handle, _t(e1), _t(e2), _t(b), x0)
    torch.cuda.synchronize()
    err = np.linalg.norm(x0.cpu().numpy() - x0o) / np.linalg.norm(x0o)
    assert rank == k and err < 1e-10, err


@pytest.mark.parametrize("executor", ["persistent", "streamed", "resident"])
def test_in_span_solution_needs_no_iterations(sw, executor):
    nx, nz, L = 64, 9, 2 * math.pi
    h = np.ones(nx)
    k = 4
    kw = dict(k=k, guess="ewma", n_init_solves=0, tol=1e-8)
    gpu = sw.Problem(nx, 1, nz, L, 0.0, h, executor=executor, **kw)
    ora = O.OracleProblem(nx, 1, nz, L, 0.0, h, **kw)
    e1, e2 = _surfaces(nx, 1, 12)
    ora.assemble(e1, e2)
    A = ora.matrix()
    rng = np.random.default_rng(13)
    Y = rng.standard_normal((ora.m, k))
    b = A @ (Y @ rng.standard_normal(k))
    sw.set_sketch(gpu.handle, _t(Y.T.ravel()), 0)
    x = torch.zeros(gpu.m, dtype=torch.float64, device=DEV)
    gpu.solve(_t(e1), _t(e2), _t(b), x)
    sg = gpu.stats()
    assert sg["status"] == 0 and sg["iterations"] == 0, sg


@pytest.mark.parametrize("executor", ["persistent", "streamed", "resident"])
def test_zero_rhs_and_iteration_cap(sw, executor):
    nx, nz, L = 32, 9, 2 * math.pi
    gpu = sw.Problem(nx, 1, nz, L, 0.0, np.ones(nx), restart=2, max_restarts=0, tol=1e-14, executor=executor)
    e1, e2 = _surfaces(nx, 1, 14)
    x = torch.ones(gpu.m, dtype=torch.float64, device=DEV)
    gpu.solve(_t(e1), _t(e2), torch.zeros(gpu.m, dtype=torch.float64, device=DEV), x)
    sg = gpu.stats()
    assert sg["status"] == 0 and sg["iterations"] == 0 and float(x.abs().max()) == 0.0
    ora = O.OracleProblem(nx, 1, nz, L, 0.0, np.ones(nx))
    b = _rhs(ora, nz, 15)
    gpu.solve(_t(e1), _t(e2), _t(b), x)
    sg = gpu.stats()
    assert sg["status"] == -3 and sg["iterations"] == 2 and not sg["converged"], sg


@pytest.mark.parametrize("executor", ["persistent", "streamed", "resident"])
def test_nan_rhs_reported(sw, executor):
    nx, nz, L = 32, 9, 2 * math.pi
    gpu = sw.Problem(nx, 1, nz, L, 0.0, np.ones(nx), executor=executor)
    e1, e2 = _surfaces(nx, 1, 16)
    b = np.zeros(gpu.m)
    b[5] = np.nan
    x = torch.zeros(gpu.m, dtype=torch.float64, device=DEV)
    gpu.solve(_t(e1), _t(e2), _t(b), x)
    assert gpu.stats()["status"] == -5


@pytest.mark.parametrize("executor", ["persistent", "streamed", "resident"])
def test_stage_driver_matches_oracle(sw, executor):
    wl = W.airy_2d()
    kw = dict(restart=20, max_restarts=200, tol=1e-12, guess="previous")
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
    for step in range(3):
        for i in range(1, 6):
            p, so, code = ora.stage(phys, i, st)
            sw.advance_stage(gpu.handle)
            sw.get_state(gpu.handle, u=u, w=w, eta=eta, pres=pr)
            torch.cuda.synchronize()
            for name, g_, o_ in [("eta", eta, st["eta"]), ("u", u, st["u"]), ("w", w, st["w"]), ("p", pr, p)]:
                err = np.abs(g_.cpu().numpy() - o_).max() / max(np.abs(o_).max(), 1e-300)
                assert err < 1e-9, (step, i, name, err)


def test_host_buffer_entry_point(sw):
    wl = W.airy_2d()
    kw = dict(restart=20, max_restarts=100, tol=1e-10, guess="cold")
    gpu = sw.Problem(wl["nx"], 1, wl["nz"], wl["lx"], 0.0, wl["h"], **kw)
    ora = O.OracleProblem(wl["nx"], 1, wl["nz"], wl["lx"], 0.0, wl["h"], **kw)
    e1, e2 = _surfaces(wl["nx"], 1, 17)
    b = _rhs(ora, wl["nz"], 18)
    xo, so, co = ora.solve(e1, e2, b)
    xh = np.zeros(gpu.m)
    code = sw.solve_poisson_host(gpu.handle, np.ascontiguousarray(e1), np.ascontiguousarray(e2), b, xh)
    assert code == 0
    assert np.linalg.norm(xh - xo) <= 1e-8 * np.linalg.norm(xo)


@pytest.mark.parametrize("executor", ["persistent", "streamed"])
def test_orthonormal_basis_guess_matches_oracle(sw, executor):
    # V = Q (the optional QR step of Algorithms 3 and 4) on a fixed sketch: the same
    # x0 as the oracle's Gram-Schmidt basis (a well-conditioned sketch drops no column)
    nx, nz, L = 64, 9, 2 * math.pi
    x64 = np.arange(nx) * (L / nx)
    h = 1.0 - 0.3 * np.exp(-3 * (x64 - 3.0) ** 2)
    k = 6
    kw = dict(k=k, guess="ewma", orthonormalize=True)
    gpu = sw.Problem(nx, 1, nz, L, 0.0, h, executor=executor, **kw)
    ora = O.OracleProblem(nx, 1, nz, L, 0.0, h, **kw)
    rng = np.random.default_rng(19)
    Y = rng.standard_normal((ora.m, k)) @ np.triu(rng.uniform(0.5, 2.0, (k, k)))
    ora.set_sketch(Y)
    sw.set_sketch(gpu.handle, _t(Y.T.ravel()), 0)
    e1, e2 = _surfaces(nx, 1, 20)
    b = _rhs(ora, nz, 21)
    ora.assemble(e1, e2)
    x0o, rank = ora.ewma_guess(b)
    x0 = torch.empty(gpu.m, dtype=torch.float64, device=DEV)
    sw.subspace_guess(gpu.handle, _t(e1), _t(e2), _t(b), x0)
    torch.cuda.synchronize()
    err = np.linalg.norm(x0.cpu().numpy() - x0o) / np.linalg.norm(x0o)
    assert rank == k and err < 1e-10, err


@pytest.mark.parametrize("guess", ["ewma", "rrf"])
@pytest.mark.parametrize("executor", ["persistent", "streamed"])
def test_orthonormal_basis_trajectory(sw, guess, executor):
    wl = W.airy_2d()
    kw = dict(restart=20, max_restarts=100, tol=1e-8, guess=guess, k=8, decay=0.9, n_init_solves=10,
              orthonormalize=True)
    rec = _record(wl, 8, **kw)
    gpu = sw.Problem(wl["nx"], 1, wl["nz"], wl["lx"], 0.0, wl["h"], executor=executor, **kw)
    x = torch.zeros(gpu.m, dtype=torch.float64, device=DEV)
    diffs = []
    for ep, ec, b, p, so in rec:
        gpu.solve(_t(ep), _t(ec), _t(b), x)
        sg = gpu.stats()
        assert sg["status"] == 0
        diffs.append(sg["iterations"] - so["iterations"])
        err = np.linalg.norm(x.cpu().numpy() - p) / np.linalg.norm(p)
        assert err < 1e-6, err
    diffs = np.array(diffs)
    assert np.all(np.abs(diffs) <= 1), diffs
    assert np.count_nonzero(diffs) <= len(diffs) // 5, diffs


def test_resident_wait_bound_reports_timeout(sw):
    # failure detection without a GPU fault: block 0 stops raising its flag at
    # the third boundary exchange, its neighbours' bounded waits run out (2 s), every
    # block leaves the kernel, the solve reports SW_ERR_TIMEOUT, and the next
    # solve on the same problem and context succeeds
    nx, nz, L = 64, 9, 2 * math.pi
    kw = dict(restart=20, max_restarts=100, tol=1e-10, guess="cold")
    gpu = sw.Problem(nx, 1, nz, L, 0.0, np.ones(nx), executor="resident", **kw)
    ora = O.OracleProblem(nx, 1, nz, L, 0.0, np.ones(nx), **kw)
    e1, e2 = _surfaces(nx, 1, 22)
    b = _rhs(ora, nz, 23)
    x = torch.zeros(gpu.m, dtype=torch.float64, device=DEV)
    sw.test_stall_exchange(gpu.handle, 3)
    gpu.solve(_t(e1), _t(e2), _t(b), x)
    assert gpu.stats()["status"] == -6
    xo, so, co = ora.solve(e1, e2, b)
    gpu.solve(_t(e1), _t(e2), _t(b), x)
    sg = gpu.stats()
    assert sg["status"] == 0, sg
    assert np.linalg.norm(x.cpu().numpy() - xo) <= 1e-8 * np.linalg.norm(xo)
    with pytest.raises(sw.SawaveError):
        sw.test_stall_exchange(sw.Problem(nx, 1, nz, L, 0.0, np.ones(nx), executor="persistent").handle, 1)


@pytest.mark.parametrize("dims", [(32, 16, 17), (512, 1, 17), (256, 1, 33)], ids=["3d_32x16x17", "2d_512x17", "2d_256x33"])
@pytest.mark.parametrize("form", [0, 1], ids=["tile", "column"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_streamed_apply_forms(sw, dims, form, precision):
    # the streamed executor's two operator forms (staged tile, column marching),
    # forced, on grids the column form serves: a solve to 1e-12 against the oracle
    nx, ny, nz = dims
    L = 2 * math.pi
    X, Y = np.meshgrid(np.arange(nx) * (L / nx), np.arange(ny) * (L / ny), indexing="xy")
    h = (1.0 + 0.2 * np.exp(-((X - 3) ** 2 + (Y - 2) ** 2))).ravel() if ny > 1 else 1.0 - 0.3 * np.exp(-3 * (X.ravel() - 3.0) ** 2)
    ly = L if ny > 1 else 0.0
    kw = dict(restart=20, max_restarts=400, tol=1e-12, guess="cold")
    gpu = sw.Problem(nx, ny, nz, L, ly, h, executor="streamed", precision=precision, **kw)
    sw.set_apply_form(gpu.handle, form)
    assert sw.autotuned_apply(gpu.handle)[0] == form
    ora = O.OracleProblem(nx, ny, nz, L, ly, h, **kw)
    e1, e2 = _surfaces(nx, ny, 24)
    b = _rhs(ora, nz, 25)
    xo, so, co = ora.solve(e1, e2, b)
    x = torch.zeros(gpu.m, dtype=torch.float64, device=DEV)
    gpu.solve(_t(e1), _t(e2), _t(b), x)
    sg = gpu.stats()
    assert co == 0 and sg["status"] == 0, (so, sg)
    err = np.linalg.norm(x.cpu().numpy() - xo) / np.linalg.norm(xo)
    assert err <= 1e-10, (err, so, sg)
    if precision == "fp64":
        assert abs(sg["iterations"] - so["iterations"]) <= 1, (sg, so)
    gpu.close()
