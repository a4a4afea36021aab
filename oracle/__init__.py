"""Reference oracle (plain FP64 C, serial) for the subspace-accelerated
sigma-transformed Poisson solve.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``.  The product package never imports
it, and it shares no code with the CUDA library.  See ``oracle/oracle.h`` for the
paper passages each function follows and ``oracle/README.md`` for what pins each
one.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
        ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
        vp = C.c_void_p
        L.or_fornberg.argtypes = [C.c_double, dp, C.c_int, C.c_int, dp]
        L.or_sigma_window.argtypes = [C.c_int, C.c_int]
        L.or_sigma_window.restype = C.c_int
        L.or_create.argtypes = [C.POINTER(Grid), C.POINTER(Params), dp, C.POINTER(C.c_int)]
        L.or_create.restype = vp
        L.or_destroy.argtypes = [vp]
        L.or_size.argtypes = [vp]
        L.or_size.restype = C.c_int
        L.or_is_box_pattern.argtypes = [vp]
        L.or_is_box_pattern.restype = C.c_int
        L.or_assemble.argtypes = [vp, vp, vp]
        L.or_assemble.restype = C.c_int
        L.or_export_matrix.argtypes = [vp, ip, ip, dp]
        L.or_matvec.argtypes = [vp, dp, dp]
        L.or_build_ilu.argtypes = [vp, vp]
        L.or_build_ilu.restype = C.c_int
        L.or_ilu_nnz.argtypes = [vp]
        L.or_ilu_nnz.restype = C.c_int
        L.or_export_ilu.argtypes = [vp, ip, ip, dp]
        L.or_ilu_apply.argtypes = [vp, dp, dp]
        L.or_gmres.argtypes = [vp, dp, dp, C.POINTER(Stats)]
        L.or_gmres.restype = C.c_int
        L.or_gmres_trace.argtypes = [vp, dp, dp, C.POINTER(Stats), dp, C.c_int]
        L.or_gmres_trace.restype = C.c_int
        L.or_splitmix64.argtypes = [C.c_uint64, C.c_uint64]
        L.or_splitmix64.restype = C.c_uint64
        L.or_draw_omega.argtypes = [C.c_uint64, C.c_long, C.c_int, dp]
        L.or_lstsq_qr.argtypes = [C.c_int, C.c_int, dp, dp, dp]
        L.or_lstsq_qr.restype = C.c_int
        L.or_ewma_guess.argtypes = [vp, dp, dp]
        L.or_ewma_guess.restype = C.c_int
        L.or_ewma_update.argtypes = [vp, dp, C.c_long]
        L.or_rrf_sketch.argtypes = [vp, dp]
        L.or_rrf_sketch.restype = C.c_int
        L.or_rrf_guess.argtypes = [vp, dp, dp]
        L.or_rrf_guess.restype = C.c_int
        L.or_orth_basis.argtypes = [C.c_int, C.c_int, dp, dp]
        L.or_orth_basis.restype = C.c_int
        L.or_get_sketch.argtypes = [vp, dp]
        L.or_set_sketch.argtypes = [vp, dp]
        L.or_solve.argtypes = [vp, vp, vp, dp, dp, C.POINTER(Stats)]
        L.or_solve.restype = C.c_int
        L.or_solve_count.argtypes = [vp]
        L.or_solve_count.restype = C.c_long
        L.or_lserk45.argtypes = [dp, dp, dp]
        L.or_f_eta.argtypes = [vp, dp, vp, dp, dp, dp]
        L.or_rhs.argtypes = [vp, C.POINTER(Physics), C.c_int, dp, vp, dp, dp, vp, dp, dp, dp, dp, dp]
        L.or_stage.argtypes = [vp, C.POINTER(Physics), C.c_int, dp, vp, dp, dp, dp, vp, dp, dp, dp,
                               C.POINTER(Stats)]
        L.or_stage.restype = C.c_int
        L.or_xcoord.argtypes = [vp, C.c_int]
        L.or_xcoord.restype = C.c_double
        L.or_relax_weight.argtypes = [C.c_double]
        L.or_relax_weight.restype = C.c_double
        L.or_wavenumber.argtypes = [C.c_double, C.c_double, C.c_double]
        L.or_wavenumber.restype = C.c_double
        L.or_relax.argtypes = [vp, C.POINTER(Relaxation), C.c_double, dp, dp, dp]
        _lib = L
    return _lib


class Grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("lx", C.c_double), ("ly", C.c_double),
                ("walls", C.c_int)]


class Relaxation(C.Structure):
    _fields_ = [("gen_x0", C.c_double), ("gen_x1", C.c_double), ("abs_x0", C.c_double), ("abs_x1", C.c_double),
                ("height", C.c_double), ("period", C.c_double), ("depth", C.c_double), ("ramp_time", C.c_double),
                ("g", C.c_double)]


class Params(C.Structure):
    _fields_ = [("restart", C.c_int), ("max_restarts", C.c_int), ("tol", C.c_double), ("guess", C.c_int),
                ("k", C.c_int), ("decay", C.c_double), ("n_init_solves", C.c_int), ("seed", C.c_uint64),
                ("history", C.c_int), ("orthonormalize", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("iterations", C.c_int), ("restarts", C.c_int), ("converged", C.c_int), ("res0", C.c_double),
                ("res_final", C.c_double), ("true_res", C.c_double), ("guess_res", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class Physics(C.Structure):
    _fields_ = [("g", C.c_double), ("rho", C.c_double), ("dt", C.c_double)]


GUESS = {"cold": 0, "previous": 1, "ewma": 2, "rrf": 3}
STATUS = {0: "OK", -1: "BAD_ARG", -3: "NOT_CONVERGED", -4: "SINGULAR", -5: "NAN"}


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def fornberg(z, xs, mmax):
    xs = _f64(xs)
    out = np.zeros((mmax + 1) * len(xs))
    lib().or_fornberg(float(z), xs, len(xs), mmax, out)
    return out.reshape(mmax + 1, len(xs))


def sigma_window(nz, j):
    return lib().or_sigma_window(nz, j)


def splitmix64(seed, i):
    return lib().or_splitmix64(seed, i)


def draw_omega(seed, solve_index, k):
    out = np.zeros(k)
    lib().or_draw_omega(seed, solve_index, k, out)
    return out


def lstsq_qr(W, b):
    W = np.asfortranarray(W, dtype=np.float64)
    m, k = W.shape
    z = np.zeros(k)
    rank = lib().or_lstsq_qr(m, k, _f64(W.ravel(order="F")), _f64(b), z)
    return z, rank


def orth_basis(Y):
    """Orthonormal basis of span(Y) (Gram-Schmidt twice, dependent columns dropped): (Q, r)."""
    Y = np.asfortranarray(Y, dtype=np.float64)
    m, k = Y.shape
    Q = np.zeros(m * max(k, 1))
    r = lib().or_orth_basis(m, k, _f64(Y.ravel(order="F")), Q)
    return Q[:m * r].reshape(r, m).T.copy(), r


def relax_weight(xi):
    return lib().or_relax_weight(float(xi))


def wavenumber(omega, depth, g=9.81):
    return lib().or_wavenumber(float(omega), float(depth), float(g))


def lserk45():
    a, b, c = np.zeros(5), np.zeros(5), np.zeros(5)
    lib().or_lserk45(a, b, c)
    return a, b, c


class OracleProblem:
    """One sigma-grid problem: operator, ILU(0), GMRES, EWMA history, stage driver."""

    def __init__(self, nx, ny, nz, lx, ly, h, restart=20, max_restarts=50, tol=1e-8, guess="cold", k=10,
                 decay=0.9, n_init_solves=30, seed=2511, walls=False, history=15, orthonormalize=False):
        self.grid = Grid(nx, ny, nz, lx, ly if ny > 1 else 0.0, int(bool(walls)))
        self.walls = bool(walls)
        self.params = Params(restart, max_restarts, tol, GUESS[guess], k, decay, n_init_solves, seed, history,
                             int(bool(orthonormalize)))
        st = C.c_int(0)
        h = _f64(h).ravel()
        assert h.size == nx * ny
        self._h = h
        self._p = lib().or_create(C.byref(self.grid), C.byref(self.params), h, C.byref(st))
        if not self._p:
            raise RuntimeError("oracle create failed: %s" % STATUS.get(st.value, st.value))
        self.nx, self.ny, self.nz = nx, ny, nz
        self.m = lib().or_size(self._p)
        self.ncol = nx * ny
        self.box = bool(lib().or_is_box_pattern(self._p))
        self.k = k

    def __del__(self):
        if getattr(self, "_p", None) and _lib is not None:
            _lib.or_destroy(self._p)
            self._p = None

    def index(self, ix, iy, j):
        return ((j + 1) * self.ny + iy) * self.nx + ix

    # operator
    def assemble(self, eta_prev=None, eta_cur=None):
        ep = None if eta_prev is None else _f64(eta_prev).ravel()
        ec = None if eta_cur is None else _f64(eta_cur).ravel()
        self._nnz = lib().or_assemble(self._p, _ptr(ep), _ptr(ec))
        return self._nnz

    def matrix(self):
        import scipy.sparse as sp
        rp = np.zeros(self.m + 1, dtype=np.int32)
        col = np.zeros(self._nnz, dtype=np.int32)
        val = np.zeros(self._nnz)
        lib().or_export_matrix(self._p, rp, col, val)
        return sp.csr_matrix((val, col, rp), shape=(self.m, self.m))

    def matvec(self, x):
        y = np.zeros(self.m)
        lib().or_matvec(self._p, _f64(x), y)
        return y

    # preconditioner and solver
    def build_ilu(self, order=None):
        o = None if order is None else np.ascontiguousarray(order, dtype=np.int32)
        st = lib().or_build_ilu(self._p, _ptr(o))
        if st != 0:
            raise RuntimeError("ILU failed: %s" % STATUS.get(st, st))
        self._order = o

    def ilu_factors(self):
        """L (unit lower) and U of the permuted still-water matrix, as one CSR."""
        import scipy.sparse as sp
        nnz = lib().or_ilu_nnz(self._p)
        rp = np.zeros(self.m + 1, dtype=np.int32)
        col = np.zeros(nnz, dtype=np.int32)
        val = np.zeros(nnz)
        lib().or_export_ilu(self._p, rp, col, val)
        return sp.csr_matrix((val, col, rp), shape=(self.m, self.m))

    def ilu_apply(self, v):
        out = np.zeros(self.m)
        lib().or_ilu_apply(self._p, _f64(v), out)
        return out

    def gmres(self, b, x0=None, trace=False):
        x = np.zeros(self.m) if x0 is None else _f64(x0).copy()
        st = Stats()
        if trace:
            tr = np.zeros(4096)
            code = lib().or_gmres_trace(self._p, _f64(b), x, C.byref(st), tr, len(tr))
            return x, st.as_dict(), code, tr[:st.iterations]
        code = lib().or_gmres(self._p, _f64(b), x, C.byref(st))
        return x, st.as_dict(), code

    def solve(self, eta_prev, eta_cur, b):
        x = np.zeros(self.m)
        st = Stats()
        code = lib().or_solve(self._p, _ptr(_f64(eta_prev).ravel()), _ptr(_f64(eta_cur).ravel()), _f64(b), x,
                              C.byref(st))
        return x, st.as_dict(), code

    @property
    def solve_count(self):
        return lib().or_solve_count(self._p)

    # subspace
    def ewma_guess(self, b):
        x0 = np.zeros(self.m)
        rank = lib().or_ewma_guess(self._p, _f64(b), x0)
        return x0, rank

    def ewma_update(self, x, solve_index):
        lib().or_ewma_update(self._p, _f64(x), solve_index)

    def sketch(self):
        Y = np.zeros(self.m * self.k)
        lib().or_get_sketch(self._p, Y)
        return Y.reshape(self.k, self.m).T.copy()

    def rrf_sketch(self):
        """Y = X Omega of the range finder for the next solve (m x k_e)."""
        Y = np.zeros(self.m * self.k)
        ke = lib().or_rrf_sketch(self._p, Y)
        return Y[:ke * self.m].reshape(ke, self.m).T.copy()

    def rrf_guess(self, b):
        x0 = np.zeros(self.m)
        rank = lib().or_rrf_guess(self._p, _f64(b), x0)
        return x0, rank

    def set_sketch(self, Y):
        lib().or_set_sketch(self._p, _f64(np.asarray(Y).T.ravel()))

    # physics
    def f_eta(self, u, v, w, eta):
        out = np.zeros(self.ncol)
        vv = None if v is None else _f64(v)
        lib().or_f_eta(self._p, _f64(u), _ptr(vv), _f64(w), _f64(eta).ravel(), out)
        return out

    def rhs(self, phys, stage, u, v, w, Ku, Kv, Kw, eta_prev, eta_cur, deta_dt):
        b = np.zeros(self.m)
        ph = Physics(*phys)
        vv = None if v is None else _f64(v)
        kv = None if Kv is None else _f64(Kv)
        lib().or_rhs(self._p, C.byref(ph), stage, _f64(u), _ptr(vv), _f64(w), _f64(Ku), _ptr(kv), _f64(Kw),
                     _f64(eta_prev).ravel(), _f64(eta_cur).ravel(), _f64(deta_dt).ravel(), b)
        return b

    def stage(self, phys, stage, state):
        """Advance ``state`` (dict of float64 arrays u, v|None, w, eta, Ku, Kv|None, Kw, Keta) by one stage."""
        ph = Physics(*phys)
        p = np.zeros(self.m)
        st = Stats()
        code = lib().or_stage(self._p, C.byref(ph), stage, state["u"], _ptr(state.get("v")), state["w"],
                              state["eta"], state["Ku"], _ptr(state.get("Kv")), state["Kw"], state["Keta"], p,
                              C.byref(st))
        return p, st.as_dict(), code

    def xcoord(self):
        """x of every column (walls: the ghost columns lie one spacing outside [0, lx])."""
        return np.array([lib().or_xcoord(self._p, i) for i in range(self.nx)])

    def relax(self, relaxation, t, state):
        """Blend eta, u, w of ``state`` towards the zone targets at time t, in place (2-D)."""
        rl = relaxation if isinstance(relaxation, Relaxation) else Relaxation(**relaxation)
        lib().or_relax(self._p, C.byref(rl), float(t), state["u"], state["w"], state["eta"])
