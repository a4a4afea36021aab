"""sawave: subspace-accelerated sigma-transformed Poisson solve on GB300.

Thin ctypes binding of libsawave.so (C ABI in include/sawave.h).  Every
function here only marshals arguments: torch CUDA tensors become device
pointers, the current torch stream becomes the cudaStream_t.  All arithmetic
runs in the library's CUDA kernels; there is no CPU fallback, and importing
this package fails loudly when the library has not been built.
"""
import ctypes as C
import os

from . import build as _build

__all__ = ["Grid", "Params", "Stats", "Physics", "Problem", "create_problem", "destroy_problem", "problem_size",
           "solve_poisson", "solve_poisson_host", "get_stats", "apply_operator", "apply_preconditioner",
           "subspace_guess", "apply_operator_noalloc", "get_sketch", "set_sketch", "draw_omega", "set_physics", "set_state", "get_state",
           "advance_stage", "set_relaxation", "set_step", "Relaxation", "create_batch", "destroy_batch", "batch_solve", "batch_advance_stage", "Batch",
           "get_last_system", "get_phase_times", "enable_timing", "get_solve_time", "test_stall_exchange", "profile_kernels", "autotuned_apply", "set_apply_form", "library_path", "SawaveError", "GUESS",
           "PRECISION", "EXECUTOR"]

SW_OK = 0
STATUS = {0: "OK", -1: "BAD_ARG", -2: "CUDA_ERR", -3: "NOT_CONVERGED", -4: "SINGULAR_PRECOND", -5: "NAN", -6: "TIMEOUT"}
GUESS = {"cold": 0, "previous": 1, "ewma": 2, "rrf": 3}
PRECISION = {"fp64": 0, "mixed": 1}
EXECUTOR = {"auto": 0, "persistent": 1, "streamed": 2, "resident": 3}


class SawaveError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (STATUS.get(code, "?"), code, msg))
        self.code = code


class Grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("lx", C.c_double), ("ly", C.c_double),
                ("walls", C.c_int)]


class Relaxation(C.Structure):
    _fields_ = [("gen_x0", C.c_double), ("gen_x1", C.c_double), ("abs_x0", C.c_double), ("abs_x1", C.c_double),
                ("height", C.c_double), ("period", C.c_double), ("depth", C.c_double), ("ramp_time", C.c_double),
                ("g", C.c_double)]


class Params(C.Structure):
    _fields_ = [("restart", C.c_int), ("max_restarts", C.c_int), ("tol", C.c_double), ("guess", C.c_int),
                ("k", C.c_int), ("decay", C.c_double), ("n_init_solves", C.c_int), ("precision", C.c_int),
                ("seed", C.c_uint64), ("executor", C.c_int), ("history", C.c_int), ("orthonormalize", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("iterations", C.c_int), ("restarts", C.c_int), ("converged", C.c_int), ("status", C.c_int),
                ("res0", C.c_double), ("res_final", C.c_double), ("true_res", C.c_double),
                ("guess_res", C.c_double), ("n_solves", C.c_longlong), ("total_iterations", C.c_longlong),
                ("launches", C.c_longlong), ("model_flops", C.c_double), ("model_bytes", C.c_double),
                ("executor", C.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class Physics(C.Structure):
    _fields_ = [("g", C.c_double), ("rho", C.c_double), ("dt", C.c_double)]


def library_path():
    return _build.LIB


_lib = None


def lib():
    """The loaded libsawave.so; raises if it is missing."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise ImportError("libsawave.so is not built (run __graft_entry__.build() or "
                              "python -m paper_2511_18071_gb300.build); there is no CPU fallback")
        L = C.CDLL(path)
        vp, ip = C.c_void_p, C.c_int
        L.sw_create_problem.argtypes = [C.POINTER(Grid), C.POINTER(Params), vp, C.POINTER(vp)]
        L.sw_destroy_problem.argtypes = [vp]
        L.sw_problem_size.argtypes = [vp, C.POINTER(C.c_longlong)]
        L.sw_solve_poisson.argtypes = [vp, vp, vp, vp, vp, vp]
        L.sw_solve_poisson_host.argtypes = [vp, vp, vp, vp, vp, vp]
        L.sw_get_stats.argtypes = [vp, C.POINTER(Stats)]
        L.sw_apply_operator.argtypes = [vp, vp, vp, vp, vp, vp]
        L.sw_apply_preconditioner.argtypes = [vp, vp, vp, vp]
        L.sw_subspace_guess.argtypes = [vp, vp, vp, vp, vp, vp]
        L.sw_get_sketch.argtypes = [vp, vp, vp]
        L.sw_set_sketch.argtypes = [vp, vp, C.c_longlong, vp]
        L.sw_draw_omega.argtypes = [C.c_uint64, C.c_longlong, ip, vp]
        L.sw_set_physics.argtypes = [vp, C.POINTER(Physics)]
        L.sw_set_state.argtypes = [vp, vp, vp, vp, vp, vp]
        L.sw_get_state.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        L.sw_advance_stage.argtypes = [vp, vp]
        L.sw_set_relaxation.argtypes = [vp, C.POINTER(Relaxation)]
        L.sw_set_step.argtypes = [vp, C.c_longlong]
        L.sw_enable_timing.argtypes = [vp, ip]
        L.sw_get_last_system.argtypes = [vp, vp, vp, vp, vp]
        L.sw_apply_operator_noalloc.argtypes = [C.POINTER(Grid), vp, vp, vp, vp, vp, vp]
        L.sw_get_phase_times.argtypes = [vp, vp, ip]
        L.sw_create_batch.argtypes = [vp, ip, C.POINTER(vp)]
        L.sw_destroy_batch.argtypes = [vp]
        L.sw_batch_solve.argtypes = [vp, vp, vp, vp, vp, vp]
        L.sw_batch_advance_stage.argtypes = [vp, vp]
        L.sw_batch_set_cluster.argtypes = [vp, ip]
        L.sw_batch_set_split.argtypes = [vp, ip, ip]
        L.sw_batch_get_launch.argtypes = [vp, C.POINTER(ip), C.POINTER(ip), C.POINTER(ip), C.POINTER(ip)]
        L.sw_batch_autotuned_tile.argtypes = [vp, C.POINTER(ip), vp, ip]
        L.sw_get_solve_time.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_longlong)]
        L.sw_test_stall_exchange.argtypes = [vp, ip]
        L.sw_profile_kernels.argtypes = [vp, ip, vp, ip]
        L.sw_autotuned_apply.argtypes = [vp, C.POINTER(ip), C.POINTER(ip), C.POINTER(ip)]
        L.sw_set_apply_form.argtypes = [vp, ip]
        L.sw_last_error.restype = C.c_char_p
        for name in ["sw_create_problem", "sw_destroy_problem", "sw_problem_size", "sw_solve_poisson",
                     "sw_solve_poisson_host", "sw_get_stats", "sw_apply_operator", "sw_apply_preconditioner",
                     "sw_subspace_guess", "sw_get_sketch", "sw_set_sketch", "sw_draw_omega", "sw_set_physics",
                     "sw_set_state", "sw_get_state", "sw_advance_stage", "sw_enable_timing", "sw_get_solve_time",
                     "sw_get_last_system", "sw_apply_operator_noalloc", "sw_get_phase_times", "sw_create_batch",
                     "sw_destroy_batch", "sw_batch_solve", "sw_batch_advance_stage", "sw_batch_set_cluster", "sw_set_relaxation",
                     "sw_set_step", "sw_batch_set_split", "sw_batch_get_launch", "sw_batch_autotuned_tile"]:
            getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def _check(code, allow=()):
    if code != SW_OK and code not in allow:
        raise SawaveError(code, lib().sw_last_error().decode(errors="replace"))
    return code


def _dptr(t):
    """Device pointer of a contiguous CUDA float64 tensor (None -> NULL)."""
    if t is None:
        return None
    import torch
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError("expected a contiguous CUDA float64 tensor")
    return C.c_void_p(t.data_ptr())


def _hptr(a):
    """Host pointer of a contiguous float64 numpy array or CPU tensor."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        import torch
        if a.is_cuda or a.dtype != torch.float64 or not a.is_contiguous():
            raise TypeError("expected a contiguous CPU float64 tensor")
        return C.c_void_p(a.data_ptr())
    import numpy as np
    if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
        raise TypeError("expected a contiguous float64 array")
    return C.c_void_p(a.ctypes.data)


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(stream)


# ---- C-ABI mirrors (same names as include/sawave.h without the sw_ prefix) ----

def create_problem(grid, params, h_depth):
    import numpy as np
    h = np.ascontiguousarray(h_depth, dtype=np.float64)
    out = C.c_void_p()
    _check(lib().sw_create_problem(C.byref(grid), C.byref(params), C.c_void_p(h.ctypes.data), C.byref(out)))
    return out


def destroy_problem(p):
    return _check(lib().sw_destroy_problem(p))


def problem_size(p):
    m = C.c_longlong()
    _check(lib().sw_problem_size(p, C.byref(m)))
    return m.value


def solve_poisson(p, eta_prev, eta_cur, b, x, stream=None):
    return _check(lib().sw_solve_poisson(p, _dptr(eta_prev), _dptr(eta_cur), _dptr(b), _dptr(x), _stream(stream)))


def solve_poisson_host(p, eta_prev, eta_cur, b, x, stream=None):
    return _check(lib().sw_solve_poisson_host(p, _hptr(eta_prev), _hptr(eta_cur), _hptr(b), _hptr(x),
                                              _stream(stream)), allow=(-3,))


def get_stats(p):
    st = Stats()
    _check(lib().sw_get_stats(p, C.byref(st)))
    return st.as_dict()


def apply_operator(p, eta_prev, eta_cur, x, y, stream=None):
    return _check(lib().sw_apply_operator(p, _dptr(eta_prev), _dptr(eta_cur), _dptr(x), _dptr(y), _stream(stream)))


def apply_preconditioner(p, v, out, stream=None):
    return _check(lib().sw_apply_preconditioner(p, _dptr(v), _dptr(out), _stream(stream)))


def apply_operator_noalloc(grid, h, eta_prev, eta_cur, x, y, stream=None):
    """Operator apply that allocates no device memory (scratch in a static device array)."""
    return _check(lib().sw_apply_operator_noalloc(C.byref(grid), _dptr(h), _dptr(eta_prev), _dptr(eta_cur), _dptr(x),
                                                  _dptr(y), _stream(stream)))


def subspace_guess(p, eta_prev, eta_cur, b, x0, stream=None):
    return _check(lib().sw_subspace_guess(p, _dptr(eta_prev), _dptr(eta_cur), _dptr(b), _dptr(x0), _stream(stream)))


def get_sketch(p, Y, stream=None):
    return _check(lib().sw_get_sketch(p, _dptr(Y), _stream(stream)))


def set_sketch(p, Y, n_solves, stream=None):
    return _check(lib().sw_set_sketch(p, _dptr(Y), int(n_solves), _stream(stream)))


def draw_omega(seed, solve_index, k):
    import numpy as np
    out = np.zeros(k)
    _check(lib().sw_draw_omega(seed, solve_index, k, C.c_void_p(out.ctypes.data)))
    return out


def set_physics(p, phys):
    return _check(lib().sw_set_physics(p, C.byref(phys)))


def set_state(p, u, v, w, eta, stream=None):
    return _check(lib().sw_set_state(p, _dptr(u), _dptr(v), _dptr(w), _dptr(eta), _stream(stream)))


def get_state(p, u=None, v=None, w=None, eta=None, pres=None, stream=None):
    return _check(lib().sw_get_state(p, _dptr(u), _dptr(v), _dptr(w), _dptr(eta), _dptr(pres), _stream(stream)))


def advance_stage(p, stream=None):
    return _check(lib().sw_advance_stage(p, _stream(stream)))


def set_relaxation(p, relax):
    """Generation/absorption zones after every stage (an sw_relaxation, a dict of its fields, or None)."""
    if relax is None:
        return _check(lib().sw_set_relaxation(p, None))
    rl = relax if isinstance(relax, Relaxation) else Relaxation(**relax)
    return _check(lib().sw_set_relaxation(p, C.byref(rl)))


def set_step(p, n_steps):
    return _check(lib().sw_set_step(p, int(n_steps)))


PROFILED_KERNELS = ["apply", "ilu_gather_fwd", "ilu_products", "ilu_gather_bwd", "cgs_pass1_j10", "cgs_pass2_j10",
                    "cgs_pass3_j10", "ilu_application"]


def profile_kernels(p, reps=5):
    """Mean microseconds per launch of the streamed executor's hot kernels (see sawave.h)."""
    import numpy as np
    out = np.zeros(len(PROFILED_KERNELS))
    _check(lib().sw_profile_kernels(p, int(reps), C.c_void_p(out.ctypes.data), len(PROFILED_KERNELS)))
    return dict(zip(PROFILED_KERNELS, out.tolist()))


def autotuned_apply(p):
    """(column_form, tile_x, tile_y) of the streamed executor's operator."""
    a, b, c = C.c_int(), C.c_int(), C.c_int()
    _check(lib().sw_autotuned_apply(p, C.byref(a), C.byref(b), C.byref(c)))
    return a.value, b.value, c.value


def set_apply_form(p, column_form):
    """Streamed executor: force the column-marching (1) or staged tile (0) operator."""
    return _check(lib().sw_set_apply_form(p, int(bool(column_form))))


def test_stall_exchange(p, exchange):
    """Testing aid: the next resident solve withholds block 0's flag at this exchange (see sawave.h)."""
    return _check(lib().sw_test_stall_exchange(p, int(exchange)))


def get_last_system(p, eta_prev=None, eta_cur=None, b=None, stream=None):
    return _check(lib().sw_get_last_system(p, _dptr(eta_prev), _dptr(eta_cur), _dptr(b), _stream(stream)))


PHASES = ["geometry", "bnorm", "guess_w", "guess_ls", "res_apply", "res_ilu", "arn_apply", "arn_ilu", "cgs1", "cgs2",
          "cgs3", "givens", "update", "true_res"]


def get_phase_times(p):
    """Cumulative device microseconds per solve phase (profiling aid)."""
    import numpy as np
    out = np.zeros(16)
    _check(lib().sw_get_phase_times(p, C.c_void_p(out.ctypes.data), 16))
    return dict(zip(PHASES, out[:len(PHASES)].tolist()))


def enable_timing(p, on=True):
    return _check(lib().sw_enable_timing(p, 1 if on else 0))


def get_solve_time(p):
    ms, n = C.c_double(), C.c_longlong()
    _check(lib().sw_get_solve_time(p, C.byref(ms), C.byref(n)))
    return ms.value, n.value


def _ptr_array(tensors):
    arr = (C.c_void_p * len(tensors))()
    for i, t in enumerate(tensors):
        arr[i] = _dptr(t).value
    return arr


def create_batch(problems):
    arr = (C.c_void_p * len(problems))(*[p.handle.value if hasattr(p, "handle") else p.value for p in problems])
    out = C.c_void_p()
    _check(lib().sw_create_batch(arr, len(problems), C.byref(out)))
    return out


def destroy_batch(b):
    return _check(lib().sw_destroy_batch(b))


def batch_solve(b, eta_prev, eta_cur, rhs, x, stream=None):
    return _check(lib().sw_batch_solve(b, _ptr_array(eta_prev), _ptr_array(eta_cur), _ptr_array(rhs), _ptr_array(x),
                                       _stream(stream)))


def batch_advance_stage(b, stream=None):
    return _check(lib().sw_batch_advance_stage(b, _stream(stream)))


class Batch:
    """Owning handle around sw_batch; keeps its problems alive."""

    def __init__(self, problems):
        self.problems = list(problems)
        self.handle = create_batch(self.problems)

    def close(self):
        if getattr(self, "handle", None):
            destroy_batch(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, eta_prev, eta_cur, rhs, x, stream=None):
        return batch_solve(self.handle, eta_prev, eta_cur, rhs, x, stream)

    def set_cluster(self, blocks_per_member):
        """Thread blocks per member (1, or a cluster of 2, 4, 8, 16)."""
        return _check(lib().sw_batch_set_cluster(self.handle, int(blocks_per_member)))

    def set_split(self, n_big, blocks_per_member):
        """The n_big largest members on clusters of blocks_per_member, the rest one block each."""
        return _check(lib().sw_batch_set_split(self.handle, int(n_big), int(blocks_per_member)))

    def autotuned_tile(self):
        """(tile width kept, {candidate width: microseconds per batched apply})."""
        import numpy as np
        tx = C.c_int()
        us = np.zeros(4)
        _check(lib().sw_batch_autotuned_tile(self.handle, C.byref(tx), C.c_void_p(us.ctypes.data), 4))
        return tx.value, dict(zip((8, 16, 32, 64), us.tolist()))

    def launch_shape(self):
        """(members on clusters, blocks per cluster member, cluster-launch blocks, single-block-launch blocks)."""
        v = [C.c_int() for _ in range(4)]
        _check(lib().sw_batch_get_launch(self.handle, *[C.byref(x) for x in v]))
        return tuple(x.value for x in v)

    def advance_stage(self, stream=None):
        return batch_advance_stage(self.handle, stream)


class Problem:
    """Owning handle around sw_problem with torch-tensor conveniences."""

    def __init__(self, nx, ny, nz, lx, ly, h, restart=20, max_restarts=50, tol=1e-8, guess="cold", k=10,
                 decay=0.9, n_init_solves=30, precision="fp64", seed=2511, walls=False, executor="auto",
                 history=15, orthonormalize=False):
        self.grid = Grid(nx, ny, nz, lx, ly if ny > 1 else 0.0, int(bool(walls)))
        self.params = Params(restart, max_restarts, tol, GUESS[guess], k, decay, n_init_solves,
                             PRECISION[precision], seed, EXECUTOR[executor], history, int(bool(orthonormalize)))
        self.handle = create_problem(self.grid, self.params, h)
        self.m = problem_size(self.handle)
        self.ncol = nx * ny
        self.nx, self.ny, self.nz, self.k = nx, ny, nz, k

    def close(self):
        if getattr(self, "handle", None):
            destroy_problem(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, eta_prev, eta_cur, b, x, stream=None):
        return solve_poisson(self.handle, eta_prev, eta_cur, b, x, stream)

    def stats(self):
        return get_stats(self.handle)
