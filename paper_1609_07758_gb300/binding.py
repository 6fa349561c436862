"""ctypes binding of include/hofem.h -- argument marshalling only.

Functions carry the C names.  Array arguments accept ``torch.Tensor`` (CUDA, float64,
contiguous; the data pointer is passed) or raw integer device pointers; ``stream``
accepts a ``torch.cuda.Stream``, an integer handle or None (legacy default stream).
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_NAME = "libhofem.so"

HOFEM_FP64 = 0
HOFEM_FP32 = 1
HOFEM_BF16 = 2
HOFEM_FP16 = 3
HOFEM_FP32_REFINED = 4
HOFEM_BF16_REFINED = 5
HOFEM_FP16_REFINED = 6

EXPORTED = (
    "hofem_plan", "hofem_set_refinement", "hofem_reserve", "hofem_solve", "hofem_apply",
    "hofem_residual", "hofem_transform1d", "hofem_get_eigen", "hofem_get_info",
    "hofem_destroy", "hofem_status_string", "hofem_last_error", "hofem_profile", "hofem_get_profile",
    "hofem_apply_static", "hofem_autotune", "hofem_batch_plan", "hofem_batch_tune", "hofem_batch_solve",
    "hofem_batch_get_info", "hofem_batch_get_plan", "hofem_batch_destroy", "hofem_batch_partition",
    "hofem_quadrature_points",
    "hofem_load", "hofem_lift_dirichlet", "hofem_mass", "hofem_heat_steps", "hofem_solve_banded", "hofem_plan_orders",
    "hofem_apply_varcoef", "hofem_pcg", "hofem_sweep", "hofem_copy_block", "hofem_residual_slab",
    "hofem_axpy",
)


class HofemError(RuntimeError):
    def __init__(self, status, where, message):
        self.status = status
        super().__init__(f"{where}: {status_name(status)}: {message}")


class hofem_info(ctypes.Structure):
    _fields_ = [
        ("N", ctypes.c_int), ("n", ctypes.c_int), ("K", ctypes.c_int * 3), ("M", ctypes.c_int * 3),
        ("dtype", ctypes.c_int), ("refine_iters", ctypes.c_int), ("iterations", ctypes.c_int),
        ("converged", ctypes.c_int), ("last_rel_update", ctypes.c_double), ("plan_ms", ctypes.c_double),
        ("table_bytes", ctypes.c_size_t), ("workspace_bytes", ctypes.c_size_t),
        ("lines_per_cta", ctypes.c_int * 3), ("threads_per_cta", ctypes.c_int),
        ("kernel_launches", ctypes.c_longlong), ("tuned_shapes", ctypes.c_longlong),
        ("orders", ctypes.c_int * 3), ("fft_len", ctypes.c_int * 3),
    ]


class hofem_problem(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("K", ctypes.c_int * 3), ("n", ctypes.c_int), ("X", ctypes.c_double * 3),
                ("alpha", ctypes.c_double), ("nrhs", ctypes.c_int)]


class hofem_batch_info(ctypes.Structure):
    _fields_ = [("count", ctypes.c_int), ("streams", ctypes.c_int), ("unknowns", ctypes.c_longlong),
                ("graph_nodes", ctypes.c_longlong), ("captures", ctypes.c_int), ("plan_ms", ctypes.c_double),
                ("tune_ms", ctypes.c_double), ("table_bytes", ctypes.c_size_t), ("workspace_bytes", ctypes.c_size_t)]


class hofem_kernel_time(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int), ("total_ms", ctypes.c_double)]


_lib = None


def library_path():
    return os.environ.get("HOFEM_LIBRARY", os.path.join(HERE, "lib", _LIB_NAME))


def load_library():
    """Load libhofem.so (raises HofemError if it is missing -- no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise HofemError(2, "load_library", f"{path} not found; run paper_1609_07758_gb300/build.py")
    lib = ctypes.CDLL(path)
    P, I, D, L, V = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_long, ctypes.c_void_p
    lib.hofem_plan.argtypes = [I, ctypes.POINTER(I), I, ctypes.POINTER(D), I, D, ctypes.POINTER(P)]
    lib.hofem_plan_orders.argtypes = [I, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(D), I, D,
                                      ctypes.POINTER(P)]
    lib.hofem_set_refinement.argtypes = [P, I, D]
    lib.hofem_reserve.argtypes = [P, I]
    lib.hofem_solve.argtypes = [P, V, V, I, V]
    lib.hofem_apply.argtypes = [P, V, V, I, V]
    lib.hofem_residual.argtypes = [P, V, V, V, I, V]
    lib.hofem_apply_static.argtypes = [P, V, V, I, V]
    lib.hofem_transform1d.argtypes = [P, I, I, V, V, L, V]
    lib.hofem_get_eigen.argtypes = [P, I, V, V, V]
    lib.hofem_get_info.argtypes = [P, ctypes.POINTER(hofem_info)]
    lib.hofem_profile.argtypes = [P, I]
    lib.hofem_get_profile.argtypes = [P, ctypes.POINTER(hofem_kernel_time), I, ctypes.POINTER(I)]
    lib.hofem_destroy.argtypes = [P]
    lib.hofem_destroy.restype = None
    lib.hofem_status_string.argtypes = [I]
    lib.hofem_status_string.restype = ctypes.c_char_p
    lib.hofem_last_error.argtypes = []
    lib.hofem_last_error.restype = ctypes.c_char_p
    lib.hofem_autotune.argtypes = [P, I, V]
    lib.hofem_quadrature_points.argtypes = [P, I, ctypes.POINTER(D)]
    lib.hofem_load.argtypes = [P, V, V, I, V]
    lib.hofem_lift_dirichlet.argtypes = [P, V, V, I, V]
    lib.hofem_mass.argtypes = [P, V, V, I, V]
    lib.hofem_solve_banded.argtypes = [P, V, V, I, V]
    lib.hofem_apply_varcoef.argtypes = [P, V, V, V, V]
    lib.hofem_pcg.argtypes = [P, V, V, V, D, I, ctypes.POINTER(I), ctypes.POINTER(D), V]
    lib.hofem_heat_steps.argtypes = [P, V, V, I, I, V]
    lib.hofem_batch_plan.argtypes = [I, ctypes.POINTER(hofem_problem), I, ctypes.POINTER(P)]
    lib.hofem_batch_tune.argtypes = [P, V]
    lib.hofem_batch_solve.argtypes = [P, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p), V]
    lib.hofem_batch_get_info.argtypes = [P, ctypes.POINTER(hofem_batch_info)]
    lib.hofem_batch_get_plan.argtypes = [P, I, ctypes.POINTER(P)]
    lib.hofem_batch_partition.argtypes = [I, ctypes.POINTER(hofem_problem), I, I, ctypes.POINTER(I),
                                          ctypes.POINTER(D)]
    LL = ctypes.c_longlong
    lib.hofem_sweep.argtypes = [P, I, I, V, V, LL, LL, LL, V]
    lib.hofem_copy_block.argtypes = [V, V, LL, LL, LL, LL, LL, LL, LL, V]
    lib.hofem_residual_slab.argtypes = [P, I, LL, LL, V, V, V, V, V, I, I, V]
    lib.hofem_axpy.argtypes = [V, D, V, LL, V]
    lib.hofem_batch_destroy.argtypes = [P]
    lib.hofem_batch_destroy.restype = None
    for name in ("hofem_plan", "hofem_set_refinement", "hofem_reserve", "hofem_solve", "hofem_apply",
                 "hofem_residual", "hofem_transform1d", "hofem_get_eigen", "hofem_get_info",
                 "hofem_profile", "hofem_get_profile", "hofem_apply_static", "hofem_autotune",
                 "hofem_batch_plan", "hofem_batch_tune", "hofem_batch_solve", "hofem_batch_get_info",
                 "hofem_batch_get_plan", "hofem_batch_partition", "hofem_quadrature_points", "hofem_load",
                 "hofem_lift_dirichlet", "hofem_mass",
                 "hofem_heat_steps", "hofem_solve_banded", "hofem_plan_orders", "hofem_apply_varcoef",
                 "hofem_pcg", "hofem_sweep", "hofem_copy_block", "hofem_residual_slab", "hofem_axpy"):
        getattr(lib, name).restype = I
    _lib = lib
    return lib


_NAMES = {0: "HOFEM_OK", 1: "HOFEM_ERR_INVALID_ARG", 2: "HOFEM_ERR_UNSUPPORTED", 3: "HOFEM_ERR_OOM",
          4: "HOFEM_ERR_CUDA", 5: "HOFEM_ERR_NOT_CONVERGED", 6: "HOFEM_ERR_TIMEOUT"}


def status_name(status):
    return _NAMES.get(int(status), str(status))


def hofem_status_string(status):
    return load_library().hofem_status_string(int(status)).decode()


def hofem_last_error():
    return load_library().hofem_last_error().decode()


def _check(status, where):
    if status != 0:
        raise HofemError(status, where, hofem_last_error())


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        import torch
        if not x.is_cuda or x.dtype != torch.float64 or not x.is_contiguous():
            raise HofemError(1, "argument", "arrays must be contiguous CUDA float64 tensors")
        return x.data_ptr()
    raise TypeError(f"cannot pass {type(x)} as a device pointer")


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def hofem_plan(N, K, n, X, dtype=HOFEM_FP64, alpha=0.0):
    """n: one order for every axis, or a sequence of N orders (hofem_plan_orders)."""
    lib = load_library()
    out = ctypes.c_void_p()
    Ka = (ctypes.c_int * N)(*[int(k) for k in K])
    Xa = (ctypes.c_double * N)(*[float(x) for x in X])
    if isinstance(n, (list, tuple)):
        Na = (ctypes.c_int * N)(*[int(v) for v in n])
        _check(lib.hofem_plan_orders(int(N), Ka, Na, Xa, int(dtype), float(alpha), ctypes.byref(out)),
               "hofem_plan_orders")
    else:
        _check(lib.hofem_plan(int(N), Ka, int(n), Xa, int(dtype), float(alpha), ctypes.byref(out)), "hofem_plan")
    return out.value


def hofem_set_refinement(plan, iters, tol=0.0):
    _check(load_library().hofem_set_refinement(plan, int(iters), float(tol)), "hofem_set_refinement")


def hofem_reserve(plan, nrhs):
    _check(load_library().hofem_reserve(plan, int(nrhs)), "hofem_reserve")


def hofem_solve(plan, f, u, nrhs, stream=None):
    _check(load_library().hofem_solve(plan, _ptr(f), _ptr(u), int(nrhs), _stream(stream)), "hofem_solve")


def hofem_apply(plan, u, r, nrhs, stream=None):
    _check(load_library().hofem_apply(plan, _ptr(u), _ptr(r), int(nrhs), _stream(stream)), "hofem_apply")


def hofem_apply_static(plan, u, r, nrhs, stream=None):
    """r = A u with the library's fixed device scratch (allocates nothing)."""
    _check(load_library().hofem_apply_static(plan, _ptr(u), _ptr(r), int(nrhs), _stream(stream)),
           "hofem_apply_static")


def hofem_residual(plan, f, u, r, nrhs, stream=None):
    _check(load_library().hofem_residual(plan, _ptr(f), _ptr(u), _ptr(r), int(nrhs), _stream(stream)),
           "hofem_residual")


def hofem_transform1d(plan, axis, inverse, x, y, lines, stream=None):
    _check(load_library().hofem_transform1d(plan, int(axis), int(inverse), _ptr(x), _ptr(y), int(lines),
                                            _stream(stream)), "hofem_transform1d")


HOFEM_SWEEP_FORWARD, HOFEM_SWEEP_FUSED, HOFEM_SWEEP_INVERSE = 0, 1, 2


def hofem_sweep(plan, axis, mode, x, y, outer, inner, line_offset=0, stream=None):
    _check(load_library().hofem_sweep(plan, int(axis), int(mode), _ptr(x), _ptr(y), int(outer), int(inner),
                                      int(line_offset), _stream(stream)), "hofem_sweep")


def hofem_residual_slab(plan, stage, e0, e1, a, b, f, out0, out1, out_fp32, nrhs, stream=None):
    _check(load_library().hofem_residual_slab(plan, int(stage), int(e0), int(e1), _ptr(a), _ptr(b), _ptr(f),
                                              _ptr(out0), _ptr(out1), int(out_fp32), int(nrhs), _stream(stream)),
           "hofem_residual_slab")


def hofem_axpy(y, c, x, count, stream=None):
    _check(load_library().hofem_axpy(_ptr(y), float(c), _ptr(x), int(count), _stream(stream)), "hofem_axpy")


def hofem_copy_block(src, dst, batch, rows, cols, src_ld, dst_ld, src_bs, dst_bs, stream=None):
    """dst[b][r][c] = src[b][r][c] (element offsets b *_bs + r *_ld + c); src, dst: device
    pointers or tensors (an int is an address, e.g. a tensor's data_ptr plus an offset)."""
    _check(load_library().hofem_copy_block(_ptr(src), _ptr(dst), int(batch), int(rows), int(cols), int(src_ld),
                                           int(dst_ld), int(src_bs), int(dst_bs), _stream(stream)),
           "hofem_copy_block")


def hofem_get_eigen(plan, axis):
    """Host copies (lam[M], mix[K-1, n, n], evec[n-1, n-1]) of one axis' eigen-data."""
    import numpy as np
    info = hofem_get_info(plan)
    n, K, M = info.n, info.K[axis], info.M[axis]
    lam = np.zeros(M)
    mix = np.zeros((K - 1, n, n))
    evec = np.zeros((max(n - 1, 1), max(n - 1, 1)))
    _check(load_library().hofem_get_eigen(plan, int(axis), lam.ctypes.data, mix.ctypes.data,
                                          evec.ctypes.data), "hofem_get_eigen")
    return lam, mix, evec[: n - 1, : n - 1]


def hofem_get_info(plan):
    info = hofem_info()
    _check(load_library().hofem_get_info(plan, ctypes.byref(info)), "hofem_get_info")
    return info


def hofem_profile(plan, enable):
    _check(load_library().hofem_profile(plan, int(enable)), "hofem_profile")


def hofem_get_profile(plan):
    """{kernel kind: (launches, total_ms)} since the last hofem_profile call (synchronises)."""
    arr = (hofem_kernel_time * 16)()
    cnt = ctypes.c_int()
    _check(load_library().hofem_get_profile(plan, arr, 16, ctypes.byref(cnt)), "hofem_get_profile")
    return {arr[i].name.decode(): (arr[i].launches, arr[i].total_ms) for i in range(min(cnt.value, 16))}


def hofem_destroy(plan):
    if plan:
        load_library().hofem_destroy(plan)


def hofem_autotune(plan, nrhs, stream=None):
    _check(load_library().hofem_autotune(plan, int(nrhs), _stream(stream)), "hofem_autotune")


class Plan:
    """Owns a hofem plan handle (destroyed with the object)."""

    def __init__(self, N, K, n, X, dtype=HOFEM_FP64, alpha=0.0):
        self.handle = hofem_plan(N, K, n, X, dtype, alpha)
        self.N, self.K, self.n, self.X, self.dtype, self.alpha = N, list(K), n, list(X), dtype, alpha
        self.ns = list(n) if isinstance(n, (list, tuple)) else [n] * N
        self.M = [nn * k - 1 for nn, k in zip(self.ns, K)]

    def solve(self, f, u, nrhs, stream=None):
        hofem_solve(self.handle, f, u, nrhs, stream)

    def apply(self, u, r, nrhs, stream=None):
        hofem_apply(self.handle, u, r, nrhs, stream)

    def residual(self, f, u, r, nrhs, stream=None):
        hofem_residual(self.handle, f, u, r, nrhs, stream)

    def transform1d(self, axis, inverse, x, y, lines, stream=None):
        hofem_transform1d(self.handle, axis, inverse, x, y, lines, stream)

    def sweep(self, axis, mode, x, y, outer, inner, line_offset=0, stream=None):
        hofem_sweep(self.handle, axis, mode, x, y, outer, inner, line_offset, stream)

    def set_refinement(self, iters, tol=0.0):
        hofem_set_refinement(self.handle, iters, tol)

    def reserve(self, nrhs):
        hofem_reserve(self.handle, nrhs)

    def info(self):
        return hofem_get_info(self.handle)

    def autotune(self, nrhs, stream=None):
        hofem_autotune(self.handle, nrhs, stream)

    def quadrature_points(self, axis):
        """The K (n+1) Gauss-Legendre points of the load vector along `axis` (numpy)."""
        import numpy as np
        x = np.zeros(self.K[axis] * (self.ns[axis] + 1))
        _check(load_library().hofem_quadrature_points(self.handle, int(axis),
                                                      x.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
               "hofem_quadrature_points")
        return x

    def solve_banded(self, f, u, nrhs, stream=None):
        """Algorithm (b): transforms along x_2..x_N, banded solves along x_1 (FP64)."""
        _check(load_library().hofem_solve_banded(self.handle, _ptr(f), _ptr(u), int(nrhs), _stream(stream)),
               "hofem_solve_banded")

    def apply_varcoef(self, aq, u, r, stream=None):
        _check(load_library().hofem_apply_varcoef(self.handle, _ptr(aq), _ptr(u), _ptr(r), _stream(stream)),
               "hofem_apply_varcoef")

    def pcg(self, aq, f, u, tol=1e-10, maxit=100, stream=None):
        """CG on -div(a grad u) = f preconditioned by this plan's solve; returns (iters, relres)."""
        it, rr = ctypes.c_int(), ctypes.c_double()
        _check(load_library().hofem_pcg(self.handle, _ptr(aq), _ptr(f), _ptr(u), float(tol), int(maxit),
                                        ctypes.byref(it), ctypes.byref(rr), _stream(stream)), "hofem_pcg")
        return it.value, rr.value

    def mass(self, u, out, nrhs, stream=None):
        _check(load_library().hofem_mass(self.handle, _ptr(u), _ptr(out), int(nrhs), _stream(stream)), "hofem_mass")

    def heat_steps(self, u, steps, nrhs, g=None, stream=None):
        """Backward Euler steps of u_t - Lap u = g in place (plan alpha = 1 / tau)."""
        _check(load_library().hofem_heat_steps(self.handle, _ptr(u), _ptr(g), int(steps), int(nrhs),
                                               _stream(stream)), "hofem_heat_steps")

    def load(self, fq, fh, nrhs, stream=None):
        """fh = f^h from samples fq of f at the tensor product of the quadrature points."""
        _check(load_library().hofem_load(self.handle, _ptr(fq), _ptr(fh), int(nrhs), _stream(stream)), "hofem_load")

    def lift_dirichlet(self, vb, f, nrhs, stream=None):
        """f -= (full-space operator, interior rows x boundary columns) vb: the Dirichlet
        data vb, given on the full grid (nrhs, M_1 + 2, ..), moved into the right-hand side."""
        _check(load_library().hofem_lift_dirichlet(self.handle, _ptr(vb), _ptr(f), int(nrhs), _stream(stream)),
               "hofem_lift_dirichlet")

    def profile(self, enable):
        hofem_profile(self.handle, enable)

    def get_profile(self):
        return hofem_get_profile(self.handle)

    def eigen(self, axis):
        return hofem_get_eigen(self.handle, axis)

    def close(self):
        if getattr(self, "handle", None):
            hofem_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _problem_array(problems):
    arr = (hofem_problem * len(problems))()
    for i, q in enumerate(problems):
        arr[i].N = int(q["N"])
        for a in range(int(q["N"])):
            arr[i].K[a] = int(q["K"][a])
            arr[i].X[a] = float(q["X"][a])
        arr[i].n = int(q["n"])
        arr[i].alpha = float(q.get("alpha", 0.0))
        arr[i].nrhs = int(q.get("nrhs", 1))
    return arr


def batch_partition(problems, dtype, parts):
    """(part_of, cost): hofem_batch_partition of a list of problem dicts over `parts` GPUs."""
    n = len(problems)
    part_of = (ctypes.c_int * n)()
    cost = (ctypes.c_double * n)()
    _check(load_library().hofem_batch_partition(n, _problem_array(problems), int(dtype), int(parts), part_of, cost),
           "hofem_batch_partition")
    return list(part_of), list(cost)


class Batch:
    """Owns a hofem batch: problems = list of dicts with keys N, K, n, X, alpha, nrhs."""

    def __init__(self, problems, dtype=HOFEM_FP32_REFINED):
        lib = load_library()
        arr = _problem_array(problems)
        out = ctypes.c_void_p()
        _check(lib.hofem_batch_plan(len(problems), arr, int(dtype), ctypes.byref(out)), "hofem_batch_plan")
        self.handle = out
        self.count = len(problems)

    def tune(self, stream=None):
        _check(load_library().hofem_batch_tune(self.handle, _stream(stream)), "hofem_batch_tune")

    def solve(self, fs, us, stream=None):
        """fs, us: sequences of device FP64 tensors (one per problem)."""
        if len(fs) != self.count or len(us) != self.count:
            raise HofemError(1, "Batch.solve", "one f and one u per problem")
        F = (ctypes.c_void_p * self.count)(*[_ptr(x) for x in fs])
        U = (ctypes.c_void_p * self.count)(*[_ptr(x) for x in us])
        _check(load_library().hofem_batch_solve(self.handle, F, U, _stream(stream)), "hofem_batch_solve")

    def info(self):
        inf = hofem_batch_info()
        _check(load_library().hofem_batch_get_info(self.handle, ctypes.byref(inf)), "hofem_batch_get_info")
        return inf

    def plan_info(self, i):
        p = ctypes.c_void_p()
        _check(load_library().hofem_batch_get_plan(self.handle, int(i), ctypes.byref(p)), "hofem_batch_get_plan")
        return hofem_get_info(p)

    def close(self):
        if getattr(self, "handle", None):
            load_library().hofem_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
