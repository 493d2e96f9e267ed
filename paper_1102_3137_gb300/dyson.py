"""Thin Python binding of include/dyson.h (argument marshalling only).

Every function keeps the C name and forwards to libdyson.so; all arithmetic
runs in the CUDA kernels behind the C ABI.  Arrays may be numpy arrays or
torch tensors (CPU or CUDA): complex arrays are complex128 (interleaved
re/im), real arrays float64.  Host arrays select DYSON_MEM_HOST, CUDA tensors
DYSON_MEM_DEVICE; one call may not mix the two.

If libdyson.so is missing or cannot be loaded every call raises: there is no
fallback implementation.

Typical use (128 x 128 lattice, 4 strips, rank 32, 64 Matsubara frequencies):

    from paper_1102_3137_gb300 import build, dyson as D
    build.build()                                   # once: nvcc, sm_103a
    plan = D.Plan((128, 128), t=-1.0, mu=0.0, p=4, k_max=32,
                  precision=D.DYSON_MIXED, max_freqs=64)
    diagG = plan.solve(omega, V, sigma, q1)         # complex128 [64][16384]

Geometry options beyond the positional ones (keyword arguments of Plan and
make_geometry): krylov_tol, krylov_maxit, refine_tol, refine_max, eta (> 0:
real axis), block_size (2..4: block Lanczos, q1 then [block_size][N]),
precond (DYSON_PRECOND_AUTO / _BANDED / _LAYER), freq_groups (0: default).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libdyson.so")

DYSON_OK = 0
DYSON_FP64 = 0
DYSON_MIXED = 1
DYSON_PRECOND_AUTO = 0
DYSON_PRECOND_BANDED = 1
DYSON_PRECOND_LAYER = 2
DYSON_MEM_HOST = 0
DYSON_MEM_DEVICE = 1
DYSON_ST_TERMINATED = 1
DYSON_ST_BREAKDOWN = 2
DYSON_ST_NO_CONVERGENCE = 4
DYSON_ST_WAIT_TIMEOUT = 16
DYSON_CUT_X = 0
DYSON_CUT_Y = 1


class dyson_geometry(C.Structure):
    _fields_ = [("dim", C.c_int), ("L", C.c_int * 3), ("t", C.c_double), ("mu", C.c_double),
                ("p", C.c_int), ("k_max", C.c_int), ("precision", C.c_int),
                ("krylov_tol", C.c_double), ("krylov_maxit", C.c_int),
                ("refine_tol", C.c_double), ("refine_max", C.c_int), ("max_freqs", C.c_int),
                ("eta", C.c_double), ("block_size", C.c_int), ("precond", C.c_int),
                ("freq_groups", C.c_int)]


class dyson_request(C.Structure):
    _fields_ = [("geom", dyson_geometry), ("K", C.c_int), ("omega", C.c_void_p), ("V", C.c_void_p),
                ("sigma", C.c_void_p), ("q1", C.c_void_p), ("diagG", C.c_void_p),
                ("status", C.c_void_p)]


class dyson_server_stats_t(C.Structure):
    _fields_ = [("queued", C.c_int), ("running", C.c_int), ("resident_plans", C.c_int),
                ("peak_running", C.c_int), ("bytes_in_use", C.c_size_t), ("peak_bytes", C.c_size_t),
                ("admitted", C.c_uint64), ("completed", C.c_uint64),
                ("plans_created", C.c_uint64), ("plans_evicted", C.c_uint64), ("fused", C.c_uint64)]


class DysonError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"dyson error {code}: {msg}")
        self.code = code


_lib = None


def load(path: str = LIB_PATH):
    """Load libdyson.so (built by paper_1102_3137_gb300.build); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} not found: build it with `python -m paper_1102_3137_gb300.build` "
                           "(the solver has no CPU fallback)")
    lib = C.CDLL(path)
    P = C.c_void_p
    I = C.c_int
    sig = {
        "dyson_version": ([], C.c_char_p),
        "dyson_last_error": ([], C.c_char_p),
        "dyson_partition": ([C.POINTER(dyson_geometry), P, P, P, P], I),
        "dyson_plan_footprint": ([C.POINTER(dyson_geometry), C.POINTER(C.c_size_t)], I),
        "dyson_plan_create": ([C.POINTER(dyson_geometry), C.POINTER(P)], I),
        "dyson_plan_destroy": ([P], I),
        "dyson_plan_tuning": ([P, P, P, P, P, P, P], I),
        "dyson_solve": ([P, I, P, P, P, P, P, P, I, P], I),
        "dyson_solve_info": ([P, I, P, P, P, P], I),
        "dyson_block_info": ([P, I, P, P], I),
        "dyson_apply_H": ([P, I, P, P, P, P, P, I, P], I),
        "dyson_apply_H_c64": ([P, I, P, P, P, P, P, I, P], I),
        "dyson_subdomain_diag": ([P, I, P, P, P, P, I, P], I),
        "dyson_subdomain_solve": ([P, I, P, P, P, P, P, I, P], I),
        "dyson_xmatvec": ([P, I, P, P, P, P, P, I, P], I),
        "dyson_plan_set_profiling": ([P, I], I),
        "dyson_profile_read": ([P, I, P, P, P], I),
        "dyson_profile_spans": ([P, I, P, P, P], I),
        "dyson_work_counters": ([P, I, P], I),
        "dyson_lanczos_basis": ([P, I, I, P], I),
        "dyson_subdomain_diag_noalloc": ([C.POINTER(dyson_geometry), I, P, P, P, P, P], I),
        "dyson_wait_selftest": ([C.c_double, P, P], I),
        "dyson_server_create": ([C.c_size_t, I, C.POINTER(P)], I),
        "dyson_server_destroy": ([P], I),
        "dyson_submit": ([P, C.POINTER(dyson_request), C.POINTER(C.c_uint64)], I),
        "dyson_poll": ([P, C.c_uint64, C.POINTER(I)], I),
        "dyson_wait": ([P, C.c_uint64, C.POINTER(C.c_double), C.POINTER(C.c_double)], I),
        "dyson_server_stats": ([P, C.POINTER(dyson_server_stats_t)], I),
        "dyson_recursive_plan_create": ([C.POINTER(dyson_geometry), I, I, I, C.POINTER(P)], I),
        "dyson_recursive_plan_destroy": ([P], I),
        "dyson_recursive_plan_info": ([P, P, P, P, P, P], I),
        "dyson_recursive_solve": ([P, I, P, P, P, P, P, P, I, P], I),
        "dyson_recursive_boxes": ([C.POINTER(dyson_geometry), I, I, C.POINTER(I), P], I),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _check(rc):
    if rc != DYSON_OK:
        raise DysonError(rc, load().dyson_last_error().decode())


def _kind(x):
    try:
        import torch
        if isinstance(x, torch.Tensor):
            return DYSON_MEM_DEVICE if x.is_cuda else DYSON_MEM_HOST
    except ImportError:
        pass
    return DYSON_MEM_HOST


def _ptr(x, dtype, n=None):
    """Data pointer of a contiguous numpy array or torch tensor of the given dtype name."""
    if x is None:
        return None
    try:
        import torch
        if isinstance(x, torch.Tensor):
            want = {"f8": torch.float64, "c16": torch.complex128, "f4": torch.float32,
                    "c8": torch.complex64, "i4": torch.int32}[dtype]
            if x.dtype != want or not x.is_contiguous():
                raise TypeError(f"expected a contiguous {want} tensor, got {x.dtype}")
            if n is not None and x.numel() < n:
                raise ValueError(f"tensor has {x.numel()} elements, need {n}")
            return x.data_ptr()
    except ImportError:
        pass
    a = x
    if not isinstance(a, np.ndarray) or a.dtype != np.dtype(dtype) or not a.flags.c_contiguous:
        raise TypeError(f"expected a C-contiguous numpy array of dtype {dtype}")
    if n is not None and a.size < n:
        raise ValueError(f"array has {a.size} elements, need {n}")
    return a.ctypes.data


def _kinds(*xs):
    ks = {_kind(x) for x in xs if x is not None}
    if len(ks) != 1:
        raise TypeError("all buffers of one call must be host arrays or all CUDA tensors")
    return ks.pop()


def _stream(stream):
    if stream is not None:
        return int(stream)
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except ImportError:
        pass
    return 0


def make_geometry(L, t=-1.0, mu=0.0, p=1, k_max=16, precision=DYSON_FP64, max_freqs=1,
                  krylov_tol=0.0, krylov_maxit=0, refine_tol=0.0, refine_max=0, eta=0.0,
                  block_size=1, precond=0, freq_groups=0):
    g = dyson_geometry()
    g.dim = len(L)
    for d in range(3):
        g.L[d] = int(L[d]) if d < len(L) else 1
    g.t, g.mu, g.p, g.k_max, g.precision = float(t), float(mu), int(p), int(k_max), int(precision)
    g.krylov_tol, g.krylov_maxit = float(krylov_tol), int(krylov_maxit)
    g.refine_tol, g.refine_max, g.max_freqs = float(refine_tol), int(refine_max), int(max_freqs)
    g.eta = float(eta)
    g.block_size = int(block_size)
    g.precond = int(precond)
    g.freq_groups = int(freq_groups)
    return g


def dyson_version():
    return load().dyson_version().decode()


def dyson_last_error():
    return load().dyson_last_error().decode()


def dyson_partition(geom):
    """(heights, m, dd2nat) of the domain-decomposition ordering; host only."""
    lib = load()
    ndd = C.c_int()
    m = C.c_int()
    heights = np.zeros(16, dtype=np.int32)
    _check(lib.dyson_partition(C.byref(geom), heights.ctypes.data, C.addressof(m), C.addressof(ndd), None))
    dd2nat = np.zeros(ndd.value, dtype=np.int32)
    _check(lib.dyson_partition(C.byref(geom), None, None, None, dd2nat.ctypes.data))
    return heights[:geom.p].copy(), m.value, dd2nat


def dyson_plan_tuning(plan):
    """Ring slots, chunk rows, X-matvec threads per CTA, configurations timed, heuristic
    and kept launch ms of a plan."""
    s, cr, n, nt = C.c_int(), C.c_int(), C.c_int(), C.c_int()
    mh, mb = C.c_float(), C.c_float()
    _check(load().dyson_plan_tuning(plan, C.addressof(s), C.addressof(cr), C.addressof(n),
                                    C.addressof(mh), C.addressof(mb), C.addressof(nt)))
    return dict(ring_slots=s.value, chunk_rows=cr.value, threads=nt.value, candidates=n.value,
                ms_heuristic=mh.value, ms_best=mb.value)


def dyson_plan_footprint(geom):
    b = C.c_size_t()
    _check(load().dyson_plan_footprint(C.byref(geom), C.byref(b)))
    return b.value


def dyson_plan_create(geom):
    h = C.c_void_p()
    _check(load().dyson_plan_create(C.byref(geom), C.byref(h)))
    return h


def dyson_plan_destroy(plan):
    _check(load().dyson_plan_destroy(plan))


def dyson_solve(plan, K, omega, V, sigma, q1, diagG, status=None, stream=None, block_size=1):
    """q1: [N] start vector, or [block_size][N] start block for a block plan."""
    N = V.shape[0] if hasattr(V, "shape") else len(V)
    nb = max(1, int(block_size))
    mk = _kinds(omega, V, sigma, q1, diagG, status)
    _check(load().dyson_solve(plan, K, _ptr(omega, "f8", K), _ptr(V, "f8", N), _ptr(sigma, "c16", K * N),
                              _ptr(q1, "f8", nb * N), _ptr(diagG, "c16", K * N), _ptr(status, "i4", K),
                              mk, _stream(stream)))


def dyson_solve_info(plan, K, k_max):
    ab = np.zeros((K, k_max, 2), dtype=np.complex128)
    steps = np.zeros(K, dtype=np.int32)
    iters = np.zeros(K, dtype=np.int32)
    refines = np.zeros(K, dtype=np.int32)
    _check(load().dyson_solve_info(plan, K, ab.ctypes.data, steps.ctypes.data, iters.ctypes.data,
                                   refines.ctypes.data))
    return dict(alpha=ab[:, :, 0].copy(), beta=ab[:, :, 1].copy(), steps=steps, iters=iters,
                refines=refines)


def dyson_block_info(plan, K, k_max, nb):
    """Block plans: (A[K][k_max/nb][nb][nb], B[K][k_max/nb][nb][nb], steps[K])."""
    ab = np.zeros((K, k_max // nb, 2, nb, nb), dtype=np.complex128)
    steps = np.zeros(K, dtype=np.int32)
    _check(load().dyson_block_info(plan, K, ab.ctypes.data, steps.ctypes.data))
    return ab[:, :, 0].copy(), ab[:, :, 1].copy(), steps


def _row_call(fn, plan, K, omega, V, sigma, x, y, xdt="c16", stream=None):
    N = V.shape[0] if hasattr(V, "shape") else len(V)
    mk = _kinds(omega, V, sigma, x, y)
    _check(fn(plan, K, _ptr(omega, "f8", K), _ptr(V, "f8", N), _ptr(sigma, "c16", K * N),
              _ptr(x, xdt, K * N), _ptr(y, xdt, K * N), mk, _stream(stream)))


def dyson_apply_H(plan, K, omega, V, sigma, x, y, stream=None):
    _row_call(load().dyson_apply_H, plan, K, omega, V, sigma, x, y, "c16", stream)


def dyson_apply_H_c64(plan, K, omega, V, sigma, x, y, stream=None):
    _row_call(load().dyson_apply_H_c64, plan, K, omega, V, sigma, x, y, "c8", stream)


def dyson_subdomain_diag(plan, K, omega, V, sigma, diagB, stream=None):
    N = V.shape[0] if hasattr(V, "shape") else len(V)
    mk = _kinds(omega, V, sigma, diagB)
    _check(load().dyson_subdomain_diag(plan, K, _ptr(omega, "f8", K), _ptr(V, "f8", N),
                                       _ptr(sigma, "c16", K * N), _ptr(diagB, "c16", K * N), mk,
                                       _stream(stream)))


def dyson_subdomain_solve(plan, K, omega, V, sigma, q, w, stream=None):
    _row_call(load().dyson_subdomain_solve, plan, K, omega, V, sigma, q, w, "c16", stream)


def dyson_xmatvec(plan, K, omega, V, sigma, q, u, stream=None):
    _row_call(load().dyson_xmatvec, plan, K, omega, V, sigma, q, u, "c16", stream)


KERNEL_NAMES = {0: "init", 1: "factor", 2: "precond", 3: "xmatvec", 4: "lanczos",
                5: "finalize", 6: "status"}


def dyson_plan_set_profiling(plan, on):
    _check(load().dyson_plan_set_profiling(plan, int(bool(on))))


def dyson_profile_read(plan, max_kernels=4096):
    kinds = np.zeros(max_kernels, np.int32)
    ms = np.zeros(max_kernels, np.float32)
    n = C.c_int()
    _check(load().dyson_profile_read(plan, max_kernels, kinds.ctypes.data, ms.ctypes.data,
                                     C.addressof(n)))
    k = min(n.value, max_kernels)
    return kinds[:k].copy(), ms[:k].astype(np.float64)


def dyson_profile_spans(plan, max_kernels=4096):
    """(start_ms, end_ms) of every profiled kernel of the last solve, from its earliest start."""
    a = np.zeros(max_kernels, np.float32)
    e = np.zeros(max_kernels, np.float32)
    n = C.c_int()
    _check(load().dyson_profile_spans(plan, max_kernels, a.ctypes.data, e.ctypes.data, C.addressof(n)))
    k = min(n.value, max_kernels)
    return a[:k].astype(np.float64), e[:k].astype(np.float64)


def dyson_work_counters(plan, K, p):
    out = np.zeros((K, p), np.uint64)
    _check(load().dyson_work_counters(plan, K, out.ctypes.data))
    return out


def dyson_subdomain_diag_noalloc(geom, K, omega, V, sigma, diagB, stream=None):
    """Allocation-free diag(blkdiag(B^-1, 0)): CUDA tensors only, no plan (see dyson.h).

    Every tensor must live on one CUDA device; the call runs with that device
    current, and with no stream given, on that device's current torch stream.
    N is the site count of the geometry: V needs N elements, sigma and diagB K*N.
    """
    import torch
    ts = (omega, V, sigma, diagB)
    if not all(isinstance(x, torch.Tensor) and x.is_cuda for x in ts):
        raise TypeError("dyson_subdomain_diag_noalloc takes CUDA tensors only")
    dev = diagB.device
    if any(x.device != dev for x in ts):
        raise TypeError("dyson_subdomain_diag_noalloc: every tensor must be on one CUDA device")
    N = int(np.prod([geom.L[d] for d in range(geom.dim)]))
    with torch.cuda.device(dev):
        s = int(stream) if stream is not None else torch.cuda.current_stream(dev).cuda_stream
        _check(load().dyson_subdomain_diag_noalloc(C.byref(geom), K, _ptr(omega, "f8", K), _ptr(V, "f8", N),
                                                   _ptr(sigma, "c16", K * N), _ptr(diagB, "c16", K * N), s))


def dyson_wait_selftest(limit_s):
    """Run the copy rings' bounded wait on an mbarrier nothing arrives on; (timed_out, waited_s)."""
    to, ws = C.c_int(), C.c_double()
    _check(load().dyson_wait_selftest(float(limit_s), C.byref(to), C.byref(ws)))
    return bool(to.value), ws.value


def dyson_lanczos_basis(plan, k, nvec, N):
    Q = np.zeros((nvec, N), np.complex128)
    _check(load().dyson_lanczos_basis(plan, int(k), int(nvec), Q.ctypes.data))
    return Q


def dyson_server_create(hbm_budget, max_inflight=8):
    h = C.c_void_p()
    _check(load().dyson_server_create(int(hbm_budget), int(max_inflight), C.byref(h)))
    return h


def dyson_server_destroy(server):
    _check(load().dyson_server_destroy(server))


def dyson_submit(server, geom, K, omega, V, sigma, q1, diagG, status=None):
    """Queue one request (host numpy arrays; keep them alive until dyson_wait)."""
    N = V.shape[0]
    req = dyson_request()
    req.geom = geom
    req.K = int(K)
    req.omega, req.V = _ptr(omega, "f8", K), _ptr(V, "f8", N)
    req.sigma, req.q1 = _ptr(sigma, "c16", K * N), _ptr(q1, "f8", max(1, geom.block_size) * N)
    req.diagG, req.status = _ptr(diagG, "c16", K * N), _ptr(status, "i4", K)
    t = C.c_uint64()
    _check(load().dyson_submit(server, C.byref(req), C.byref(t)))
    return t.value


def dyson_poll(server, ticket):
    d = C.c_int()
    _check(load().dyson_poll(server, C.c_uint64(ticket), C.byref(d)))
    return bool(d.value)


def dyson_wait(server, ticket):
    """Block until done; returns (latency_ms from submission, run_ms from admission)."""
    lat, run = C.c_double(), C.c_double()
    _check(load().dyson_wait(server, C.c_uint64(ticket), C.byref(lat), C.byref(run)))
    return lat.value, run.value


def dyson_server_stats(server):
    st = dyson_server_stats_t()
    _check(load().dyson_server_stats(server, C.byref(st)))
    return {f: getattr(st, f) for f, _ in st._fields_}


def dyson_recursive_plan_create(geom, min_sites, first_cut=DYSON_CUT_X, streams=0):
    h = C.c_void_p()
    _check(load().dyson_recursive_plan_create(C.byref(geom), int(min_sites), int(first_cut), int(streams),
                                              C.byref(h)))
    return h


def dyson_recursive_boxes(geom, min_sites, first_cut=DYSON_CUT_X):
    """Box tree of the recursive decomposition, host only: int array [n][8] of
    (x0, y0, nx, ny, level, leaf, cut axis (0 x, 1 y) or -1, cut line coordinate or -1)."""
    lib = load()
    n = C.c_int()
    _check(lib.dyson_recursive_boxes(C.byref(geom), int(min_sites), int(first_cut), C.byref(n), None))
    out = np.zeros((n.value, 8), dtype=np.int32)
    _check(lib.dyson_recursive_boxes(C.byref(geom), int(min_sites), int(first_cut), C.byref(n), out.ctypes.data))
    return out


def dyson_recursive_plan_destroy(rplan):
    _check(load().dyson_recursive_plan_destroy(rplan))


def dyson_recursive_plan_info(rplan):
    lv, bx, lf, pl = C.c_int(), C.c_int(), C.c_int(), C.c_int()
    by = C.c_size_t()
    _check(load().dyson_recursive_plan_info(rplan, C.addressof(lv), C.addressof(bx), C.addressof(lf),
                                            C.addressof(pl), C.addressof(by)))
    return dict(levels=lv.value, boxes=bx.value, leaves=lf.value, plans=pl.value, bytes=by.value)


def dyson_recursive_solve(rplan, K, N, omega, V, sigma, q1, diagG, status=None, stream=None):
    """Arguments as dyson_solve; N = Lx * Ly of the recursive plan's lattice."""
    mk = _kinds(omega, V, sigma, q1, diagG, status)
    _check(load().dyson_recursive_solve(rplan, K, _ptr(omega, "f8", K), _ptr(V, "f8", N), _ptr(sigma, "c16", K * N),
                                        _ptr(q1, "f8", N), _ptr(diagG, "c16", K * N), _ptr(status, "i4", K),
                                        mk, _stream(stream)))


class RecursivePlan:
    """Owning wrapper of a recursive-decomposition plan (2D)."""

    def __init__(self, L, t=-1.0, mu=0.0, k_max=16, precision=DYSON_FP64, max_freqs=1, min_sites=64,
                 first_cut=DYSON_CUT_X, streams=0, **kw):
        if len(L) != 2:
            raise ValueError("the recursive decomposition is defined for 2D lattices")
        self.geom = make_geometry(L, t, mu, 2, k_max, precision, max_freqs, **kw)
        self.L, self.N = tuple(L), int(np.prod(L))
        self.handle = dyson_recursive_plan_create(self.geom, min_sites, first_cut, streams)

    def close(self):
        if self.handle is not None:
            dyson_recursive_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        return dyson_recursive_plan_info(self.handle)

    def solve(self, omega, V, sigma, q1, diagG=None, status=None, stream=None):
        K = len(omega)
        if diagG is None:
            diagG = np.zeros((K, self.N), dtype=np.complex128)
        dyson_recursive_solve(self.handle, K, self.N, omega, V, sigma, q1, diagG, status, stream)
        return diagG


class Plan:
    """Owning wrapper: creates the plan on construction, destroys it on close()."""

    def __init__(self, L, t=-1.0, mu=0.0, p=1, k_max=16, precision=DYSON_FP64, max_freqs=1, **kw):
        self.geom = make_geometry(L, t, mu, p, k_max, precision, max_freqs, **kw)
        self.L, self.N, self.k_max = tuple(L), int(np.prod(L)), k_max
        self.nb = max(1, self.geom.block_size)
        self.handle = dyson_plan_create(self.geom)

    def close(self):
        if self.handle is not None:
            dyson_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, omega, V, sigma, q1, diagG=None, status=None, stream=None):
        K = len(omega)
        if diagG is None:
            diagG = np.zeros((K, self.N), dtype=np.complex128)
        dyson_solve(self.handle, K, omega, V, sigma, q1, diagG, status, stream, self.nb)
        return diagG

    def info(self, K):
        if self.nb > 1:
            A, B, steps = dyson_block_info(self.handle, K, self.k_max, self.nb)
            return dict(A=A, B=B, steps=steps)
        return dyson_solve_info(self.handle, K, self.k_max)
