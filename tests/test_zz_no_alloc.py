"""The allocation-free operator apply (sw_apply_operator_noalloc).

It serves callers that cannot call cudaMalloc (a memory budget or pool that
forbids new device allocations, or a framework that owns every buffer): its
scratch lives in a static device array of at most 65,536 columns.  Here it is
called through the C ABI twice in a row, each time on new inputs, and its
output is compared with the regular entry point sw_apply_operator on the same
inputs and with the oracle's assembled operator, A x, both with the
element-wise bound the operator parity tests use: 1e-12 (|A| |x|).  The cases
cover a 2-D bar, a 3-D field, the deepest sigma grid the entry point accepts
(nz = 61, where the 3-D tile shrinks) and a grid exactly at the column limit
(256 x 256 columns, where the scratch regions are full).  Grids above the
limit are rejected before any GPU work.

This file is named so that pytest collects it last.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def sw():
    from paper_2511_18071_gb300 import build
    build.build()
    import paper_2511_18071_gb300 as sw
    sw.lib()
    return sw


@pytest.mark.gpu
def test_rejects_grids_above_the_static_limit(sw):
    g = sw.Grid(512, 256, 9, 1.0, 1.0)   # 131,072 columns
    dev = torch.device("cuda")
    small = torch.zeros(8, dtype=torch.float64, device=dev)
    # the column limit is checked on the host before any GPU work touches the buffers
    with pytest.raises(sw.SawaveError) as e:
        sw.apply_operator_noalloc(g, small, small, small, small, small)
    assert e.value.code == -1 and "65536" in str(e.value)


@pytest.mark.gpu
@pytest.mark.parametrize("dims", [(64, 1, 9), (16, 8, 9), (16, 8, 61), (256, 256, 7)],
                         ids=["2d_bar", "3d_bumps", "3d_nz61", "3d_at_limit"])
def test_matches_regular_apply_and_oracle_on_two_calls(sw, dims):
    import oracle as O
    nx, ny, nz = dims
    L = 2 * math.pi
    ly = L if ny > 1 else 0.0
    X, Y = np.meshgrid(np.arange(nx) * (L / nx), np.arange(ny) * (L / ny), indexing="xy")
    h = (1.0 - 0.3 * np.exp(-2 * ((X - 3) ** 2 + (Y - 2) ** 2))).ravel()
    dev = torch.device("cuda")
    grid = sw.Grid(nx, ny, nz, L, ly)
    prob = sw.Problem(nx, ny, nz, L, ly, h)
    ora = O.OracleProblem(nx, ny, nz, L, ly, h)
    m = prob.m
    rng = np.random.default_rng(21)
    dh = torch.tensor(h, device=dev)
    for call in range(2):
        e1 = (0.02 * np.cos(X + call) + 0.01 * np.sin(2 * Y)).ravel()
        e2 = e1 + 0.003 * np.sin(X + Y + call).ravel()
        x = rng.standard_normal(m)
        ref = torch.empty(m, dtype=torch.float64, device=dev)
        out = torch.full((m,), float("nan"), dtype=torch.float64, device=dev)
        te1, te2, tx = (torch.tensor(a, device=dev) for a in (e1, e2, x))
        sw.apply_operator(prob.handle, te1, te2, tx, ref)
        sw.apply_operator_noalloc(grid, dh, te1, te2, tx, out)
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        ora.assemble(e1, e2)
        A = ora.matrix()
        bound = abs(A) @ np.abs(x)
        d_reg = np.abs(o - ref.cpu().numpy())
        d_ora = np.abs(o - A @ x)
        assert np.all(d_reg <= 1e-12 * bound), (call, (d_reg / bound).max())
        assert np.all(d_ora <= 1e-12 * bound), (call, (d_ora / bound).max())
    prob.close()
