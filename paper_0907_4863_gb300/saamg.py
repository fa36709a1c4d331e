"""Thin Python binding of libsaamg (include/saamg.h): argument marshalling only.

Every computation runs in the CUDA library; this module converts torch tensors to
device pointers, passes torch's current CUDA stream, and routes the library's device
allocations to torch's caching allocator.  There is no fallback: if libsaamg.so is
missing or fails to load, every call raises.
"""
import ctypes as C
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.path.join(PKG, "libsaamg.so")

OK, NOT_CONVERGED, NOT_READY = 0, 1, 2
EINVAL, ENOMEM, ECUDA, NUMERICAL, DEVICE_TIMEOUT, UNIMPLEMENTED = -1, -2, -3, -4, -5, -6
BC_CONSTANT, BC_LINEAR, BC_QUADRATIC = 0, 1, 2
Z_ROBIN, Z_DIRICHLET = 0, 1
PREC_FP64, PREC_FP32, PREC_FP32_BF16 = 0, 1, 2
KT_STENCIL_SMOOTH, KT_STENCIL_APPLY, KT_COARSE, KT_TRANSFER, KT_SPGEMM = 0, 1, 2, 3, 4
KT_STENCIL_RESID, KT_STENCIL_FIRST = 5, 6
KT_NAMES = ["stencil_smooth", "stencil_apply", "coarse_csr", "transfer", "spgemm", "stencil_resid",
            "stencil_first", "pic", "prolong0", "coarse_deep", "transfer_deep"]
MAX_LEVELS = 16


class SaamgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"saamg status {status}: {msg}")
        self.status = status


class Domain(C.Structure):
    _fields_ = [("a", C.c_double), ("b", C.c_double), ("taper", C.c_double), ("cx", C.c_double),
                ("cy", C.c_double), ("zbc", C.c_int), ("symmetrize_gamma2", C.c_int)]


class Grid(C.Structure):
    _fields_ = [("n", C.c_int * 3), ("h", C.c_double * 3), ("origin", C.c_double * 3)]


class Params(C.Structure):
    _fields_ = [("cheb_degree", C.c_int), ("cheb_ratio", C.c_double), ("cheb_safety", C.c_double),
                ("max_coarse", C.c_int), ("max_levels", C.c_int), ("power_iters", C.c_int),
                ("precision", C.c_int), ("beta_rule", C.c_int), ("maxit", C.c_int),
                ("aggregation", C.c_int), ("coarse_solver", C.c_int), ("coarse_sweeps", C.c_int),
                ("device_loop", C.c_int)]


class SolveInfo(C.Structure):
    _fields_ = [("iters", C.c_int), ("converged", C.c_int), ("relres", C.c_double),
                ("relres_true", C.c_double), ("solve_ms", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class StencilConfig(C.Structure):
    _fields_ = [("chunks_per_step", C.c_int), ("packed", C.c_int), ("block", C.c_int),
                ("blocks_per_sm", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class HierarchyInfo(C.Structure):
    _fields_ = [("levels", C.c_int), ("n", C.c_int * MAX_LEVELS),
                ("nnz", C.c_longlong * MAX_LEVELS), ("nnz_p", C.c_longlong * MAX_LEVELS),
                ("lambda_", C.c_double * MAX_LEVELS), ("device_bytes", C.c_longlong),
                ("setup_ms", C.c_double), ("sell_index_bytes", C.c_int * MAX_LEVELS)]

    def as_dict(self):
        L = self.levels
        return dict(levels=L, n=list(self.n[:L]), nnz=list(self.nnz[:L]), nnz_p=list(self.nnz_p[:L]),
                    lam=list(self.lambda_[:L]), device_bytes=self.device_bytes, setup_ms=self.setup_ms,
                    sell_index_bytes=list(self.sell_index_bytes[:L]))


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)

_lib = None
_hooks = None
# Handles dropped by the garbage collector.  The collector can run inside an allocator
# callback, i.e. while the library is executing a call on this thread; freeing there would
# re-enter the library.  __del__ therefore only queues the handle; the queue is emptied at
# the start of the next call made through this module.
_deferred = []


def _flush_deferred():
    while _deferred:
        h = _deferred.pop()
        if _lib is not None:
            _lib.saamg_free(h)

_p = C.c_void_p
_i = C.c_int


def lib():
    """Load libsaamg.so (raises if it is missing: there is no other implementation)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIBPATH):
        raise ImportError(f"{LIBPATH} is missing; build it with paper_0907_4863_gb300.build.build()")
    L = C.CDLL(LIBPATH)
    sig = {
        "saamg_params_default": [C.POINTER(Params)],
        "saamg_set_allocator": [ALLOC_FN, FREE_FN, _p],
        "saamg_build_operator": [C.POINTER(Domain), C.POINTER(Grid), _i, _p, C.POINTER(_p)],
        "saamg_operator_size": [_p, C.POINTER(_i), C.POINTER(C.c_longlong)],
        "saamg_operator_copy": [_p, _p, _p, _p, _p, _p, _p, _p],
        "saamg_operator_apply": [_p, _p, _p, _p],
        "saamg_dense_inverse": [_i, _p, _p, _p],
        "saamg_setup": [_p, C.POINTER(Params), _p, C.POINTER(_p)],
        "saamg_setup_reuse": [_p, _p, C.POINTER(Params), _p, C.POINTER(_p)],
        "saamg_hierarchy_work_set": [_p, _p, C.POINTER(_p)],
        "saamg_hierarchy_get_info": [_p, C.POINTER(HierarchyInfo)],
        "saamg_hierarchy_copy_level": [_p, _i] + [_p] * 12,
        "saamg_vcycle": [_p, _p, _p, _p],
        "saamg_solve": [_p, _p, _p, C.c_double, _p, C.POINTER(SolveInfo)],
        "saamg_solve_host": [_p, _p, _p, C.c_double, _p, C.POINTER(SolveInfo)],
        "saamg_mis2_aggregate": [_i, _p, _p, _p, C.c_uint32, _p, _p, C.POINTER(_i), _p],
        "saamg_mis2_aggregate_noalloc": [_i, _p, _p, _p, C.c_uint32, _p, _p, C.POINTER(_i), _p],
        "saamg_solve_async": [_p, _p, _p, C.c_double, _p],
        "saamg_solve_test": [_p],
        "saamg_solve_wait": [_p, C.POINTER(SolveInfo)],
        "saamg_solve_batched": [_p, _p, _p, _i, C.c_double, _p, _p],
        "saamg_set_cheb_degree": [_p, _i],
        "saamg_stencil_config_get": [_p, _i, C.POINTER(StencilConfig)],
        "saamg_stencil_config_set": [_p, _i, C.POINTER(StencilConfig)],
        "saamg_autotune_stencil": [_p, _i, _p, C.POINTER(StencilConfig), C.POINTER(C.c_double)],
        "saamg_autotune_cheb_degree": [_p, _p, _i, _i, C.c_double, _p, C.POINTER(_i),
                                       C.POINTER(C.c_double)],
        "saamg_deposit_cic": [C.POINTER(Grid), _i, _p, _p, _p, _p, _p, _p],
        "saamg_field_gradient": [_p, _p, _p, _p, _p, _p],
        "saamg_gather_cic": [C.POINTER(Grid), _p, _p, _p, _i, _p, _p, _p, _p, _p, _p, _p],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = C.c_int
    L.saamg_kernel_launches.argtypes = []
    L.saamg_kernel_launches.restype = C.c_longlong
    L.saamg_kernel_timing.argtypes = [_i]
    L.saamg_kernel_timing.restype = C.c_int
    L.saamg_kernel_timing_read.argtypes = [_i, C.POINTER(C.c_double), C.POINTER(C.c_longlong),
                                           C.POINTER(C.c_longlong)]
    L.saamg_kernel_timing_read.restype = C.c_int
    L.saamg_batch_last.argtypes = [C.POINTER(_i), C.POINTER(C.c_double), C.POINTER(C.c_double)]
    L.saamg_batch_last.restype = C.c_int
    L.saamg_release_batch_cache.argtypes = []
    L.saamg_release_batch_cache.restype = C.c_int
    L.saamg_free.argtypes = [_p]
    L.saamg_free.restype = None
    L.saamg_last_error.argtypes = []
    L.saamg_last_error.restype = C.c_char_p
    _lib = L
    import atexit
    # the batch cache's work vectors came from the allocator hook (a Python callback here):
    # hand them back while the interpreter can still run the hook
    atexit.register(release_batch_cache)
    return L


def batch_last():
    """Form of the most recent batched call ('merged' or 'per-solve') and the first-run wall
    times (ms) of both forms for its set of solves (None: not run yet)."""
    m, a, b = C.c_int(0), C.c_double(0), C.c_double(0)
    _check(lib().saamg_batch_last(C.byref(m), C.byref(a), C.byref(b)))
    return dict(form="merged" if m.value else "per-solve",
                ms_merged=a.value if a.value >= 0 else None,
                ms_per_solve=b.value if b.value >= 0 else None)


def release_batch_cache():
    """Frees the graphs and work vectors kept for repeated batched solves."""
    if _lib is not None:
        _flush_deferred()
        _lib.saamg_release_batch_cache()


def last_error():
    return lib().saamg_last_error().decode()


def _entry(fn):
    """Decorator: release queued handles before entering the library."""
    import functools

    @functools.wraps(fn)
    def wrapped(*a, **k):
        _flush_deferred()
        return fn(*a, **k)
    return wrapped


def _check(status, allow_not_converged=False):
    if status == OK or (allow_not_converged and status == NOT_CONVERGED):
        return status
    raise SaamgError(status, last_error())


def _stream(stream):
    if stream is not None:
        return C.c_void_p(int(stream))
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


# Every callback object ever installed stays referenced here: buffers allocated under a hook
# keep calling that hook's free function when they are released, so a callback must never be
# collected while the library may still hold memory it allocated.
_all_hooks = []


def use_torch_allocator():
    """Route the library's device allocations to torch's caching allocator (idempotent)."""
    global _hooks
    if _hooks is not None and _hooks[2] == "torch":
        return
    import torch

    def _alloc(nbytes, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(),
                                                      stream or 0)
        except Exception:
            return None

    def _free(ptr, stream, ctx):
        torch.cuda.caching_allocator_delete(ptr)

    hooks = (ALLOC_FN(_alloc), FREE_FN(_free), "torch")
    _all_hooks.append(hooks)
    _check(lib().saamg_set_allocator(hooks[0], hooks[1], None))
    _hooks = hooks


def use_cuda_malloc():
    """Back to cudaMalloc / cudaFree for new allocations."""
    global _hooks
    _check(lib().saamg_set_allocator(ALLOC_FN(), FREE_FN(), None))
    _hooks = None


def params_default(**overrides):
    p = Params()
    _check(lib().saamg_params_default(C.byref(p)))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


class Operator:
    """Handle of saamg_build_operator."""

    def __init__(self, handle, grid_n):
        self.handle = handle
        self.grid_n = tuple(grid_n)

    def size(self):
        n = C.c_int(0)
        nnz = C.c_longlong(0)
        _check(lib().saamg_operator_size(self.handle, C.byref(n), C.byref(nnz)))
        return n.value, nnz.value

    def free(self):
        if self.handle:
            _flush_deferred()
            lib().saamg_free(self.handle)
            self.handle = None

    def __del__(self):
        if getattr(self, "handle", None):
            _deferred.append(self.handle)
            self.handle = None


class Hierarchy:
    """Handle of saamg_setup (keeps its operator alive)."""

    def __init__(self, handle, op):
        self.handle = handle
        self.op = op

    def info(self):
        hi = HierarchyInfo()
        _check(lib().saamg_hierarchy_get_info(self.handle, C.byref(hi)))
        return hi.as_dict()

    def free(self):
        if self.handle:
            _flush_deferred()
            lib().saamg_free(self.handle)
            self.handle = None

    def __del__(self):
        if getattr(self, "handle", None):
            _deferred.append(self.handle)
            self.handle = None


@_entry
def build_operator(domain: Domain, grid: Grid, mode: int, stream=None) -> Operator:
    h = C.c_void_p()
    _check(lib().saamg_build_operator(C.byref(domain), C.byref(grid), int(mode), _stream(stream),
                                      C.byref(h)))
    return Operator(h, tuple(grid.n))


@_entry
def operator_size(op: Operator):
    return op.size()


@_entry
def operator_copy(op: Operator, stream=None):
    """Host copies: node_of_row, scale, rowptr, col, val, is_regular (numpy)."""
    import numpy as np
    n, nnz = op.size()
    out = dict(node_of_row=np.empty(n, np.int32), scale=np.empty(n, np.float64),
               rowptr=np.empty(n + 1, np.int32), col=np.empty(nnz, np.int32),
               val=np.empty(nnz, np.float64), is_regular=np.empty(n, np.uint8))
    P = lambda a: a.ctypes.data_as(C.c_void_p)  # noqa: E731
    _check(lib().saamg_operator_copy(op.handle, P(out["node_of_row"]), P(out["scale"]),
                                     P(out["rowptr"]), P(out["col"]), P(out["val"]),
                                     P(out["is_regular"]), _stream(stream)))
    return out


@_entry
def operator_apply(op: Operator, x, y, stream=None):
    _check(lib().saamg_operator_apply(op.handle, _ptr(x), _ptr(y), _stream(stream)))


@_entry
def dense_inverse(a, inv, stream=None):
    """inv = a^-1 for a dense n x n FP64 device matrix (row-major tensors; synchronises)."""
    import torch
    n = int(a.shape[0]) if a.dim() == 2 else -1
    if a.dim() != 2 or tuple(a.shape) != (n, n) or tuple(inv.shape) != (n, n):
        raise ValueError("a and inv must be n x n")
    for t in (a, inv):
        if t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous():
            raise ValueError("a and inv must be contiguous float64 device tensors")
    _check(lib().saamg_dense_inverse(n, _ptr(a), _ptr(inv), _stream(stream)))


@_entry
def deposit_cic(grid: Grid, x, y, z, q, rho, stream=None):
    """rho (box) = cloud-in-cell density of the particles (device arrays)."""
    _check(lib().saamg_deposit_cic(C.byref(grid), int(len(x)), _ptr(x), _ptr(y), _ptr(z),
                                   _ptr(q), _ptr(rho), _stream(stream)))


@_entry
def field_gradient(op: Operator, phi, ex, ey, ez, stream=None):
    """E = -grad phi on the box (device arrays)."""
    _check(lib().saamg_field_gradient(op.handle, _ptr(phi), _ptr(ex), _ptr(ey), _ptr(ez),
                                      _stream(stream)))


@_entry
def gather_cic(grid: Grid, ex, ey, ez, x, y, z, epx, epy, epz, stream=None):
    """E at the particles with the deposition's weights (device arrays)."""
    _check(lib().saamg_gather_cic(C.byref(grid), _ptr(ex), _ptr(ey), _ptr(ez), int(len(x)),
                                  _ptr(x), _ptr(y), _ptr(z), _ptr(epx), _ptr(epy), _ptr(epz),
                                  _stream(stream)))


@_entry
def setup(op: Operator, params: Params = None, stream=None) -> Hierarchy:
    h = C.c_void_p()
    _check(lib().saamg_setup(op.handle, C.byref(params) if params is not None else None,
                             _stream(stream), C.byref(h)))
    return Hierarchy(h, op)


@_entry
def setup_reuse(op: Operator, prev: Hierarchy, params: Params = None, stream=None) -> Hierarchy:
    """Hierarchy for `op` that keeps prev's aggregates (same operator pattern required)."""
    h = C.c_void_p()
    _check(lib().saamg_setup_reuse(op.handle, prev.handle,
                                   C.byref(params) if params is not None else None,
                                   _stream(stream), C.byref(h)))
    return Hierarchy(h, op)


@_entry
def hierarchy_work_set(h: Hierarchy, stream=None) -> Hierarchy:
    """A second handle over h's levels with its own work vectors (a solve on it may run
    while another runs on h); h's levels live until h and all its work sets are freed."""
    w = C.c_void_p()
    _check(lib().saamg_hierarchy_work_set(h.handle, _stream(stream), C.byref(w)))
    return Hierarchy(w, h.op)


@_entry
def hierarchy_get_info(h: Hierarchy):
    return h.info()


@_entry
def hierarchy_copy_level(h: Hierarchy, l: int, stream=None):
    """Host copies of level l: A (rowptr, col, val), agg, root, P and R (numpy)."""
    import numpy as np
    info = h.info()
    n = info["n"][l]
    nnz = info["nnz"][l]
    has_next = l + 1 < info["levels"]
    nn = info["n"][l + 1] if has_next else 0
    np_ = info["nnz_p"][l] if has_next else 0
    out = dict(rowptr=np.empty(n + 1, np.int32), col=np.empty(nnz, np.int32),
               val=np.empty(nnz, np.float64))
    if has_next:
        out.update(agg=np.empty(n, np.int32), root=np.empty(n, np.uint8),
                   p_rowptr=np.empty(n + 1, np.int32), p_col=np.empty(np_, np.int32),
                   p_val=np.empty(np_, np.float64), r_rowptr=np.empty(nn + 1, np.int32),
                   r_col=np.empty(np_, np.int32), r_val=np.empty(np_, np.float64))
    P = lambda k: out[k].ctypes.data_as(C.c_void_p) if k in out else None  # noqa: E731
    _check(lib().saamg_hierarchy_copy_level(h.handle, int(l), P("rowptr"), P("col"), P("val"),
                                            P("agg"), P("root"), P("p_rowptr"), P("p_col"),
                                            P("p_val"), P("r_rowptr"), P("r_col"), P("r_val"),
                                            _stream(stream)))
    return out


@_entry
def vcycle(h: Hierarchy, r, z, stream=None):
    _check(lib().saamg_vcycle(h.handle, _ptr(r), _ptr(z), _stream(stream)))


@_entry
def solve(h: Hierarchy, rho, phi, rtol=1e-8, stream=None):
    """rho, phi: float64 CUDA tensors over the whole box; phi = initial guess in, solution out."""
    info = SolveInfo()
    st = lib().saamg_solve(h.handle, _ptr(rho), _ptr(phi), float(rtol), _stream(stream),
                           C.byref(info))
    _check(st, allow_not_converged=True)
    d = info.as_dict()
    d["status"] = st
    return d


@_entry
def solve_host(h: Hierarchy, rho, phi, rtol=1e-8, stream=None):
    """Host (numpy float64) box arrays; the copies to and from the device are in the call."""
    info = SolveInfo()
    st = lib().saamg_solve_host(h.handle, rho.ctypes.data_as(C.c_void_p),
                                phi.ctypes.data_as(C.c_void_p), float(rtol), _stream(stream),
                                C.byref(info))
    _check(st, allow_not_converged=True)
    d = info.as_dict()
    d["status"] = st
    return d


@_entry
def solve_async(h: Hierarchy, rho, phi, rtol=1e-8, stream=None):
    """Enqueue the whole PCG solve as one device-loop graph on the stream; returns at once."""
    _check(lib().saamg_solve_async(h.handle, _ptr(rho), _ptr(phi), float(rtol), _stream(stream)))


@_entry
def solve_test(h: Hierarchy) -> bool:
    st = lib().saamg_solve_test(h.handle)
    if st == NOT_READY:
        return False
    _check(st)
    return True


@_entry
def solve_wait(h: Hierarchy):
    info = SolveInfo()
    st = lib().saamg_solve_wait(h.handle, C.byref(info))
    _check(st, allow_not_converged=True)
    d = info.as_dict()
    d["status"] = st
    return d


@_entry
def solve_batched(hs, rhos, phis, rtol=1e-8, stream=None):
    """Solves rhos[j] -> phis[j] on hierarchies hs[j] in one call; returns the infos."""
    n = len(hs)
    H = (C.c_void_p * n)(*[h.handle for h in hs])
    R = (C.c_void_p * n)(*[r.data_ptr() for r in rhos])
    X = (C.c_void_p * n)(*[x.data_ptr() for x in phis])
    infos = (SolveInfo * n)()
    st = lib().saamg_solve_batched(H, R, X, n, float(rtol), _stream(stream), infos)
    _check(st, allow_not_converged=True)
    return [dict(infos[j].as_dict()) for j in range(n)]


@_entry
def stencil_config(op: Operator, precision: int) -> dict:
    """The level-0 stencil launch shape op uses for precision 0 (FP64) or 1 (FP32)."""
    c = StencilConfig()
    _check(lib().saamg_stencil_config_get(op.handle, int(precision), C.byref(c)))
    return c.as_dict()


@_entry
def set_stencil_config(op: Operator, precision: int, cfg=None):
    """Sets the launch shape (a dict like stencil_config's; None: the default)."""
    if cfg is None:
        _check(lib().saamg_stencil_config_set(op.handle, int(precision), None))
        return
    c = StencilConfig(**{k: int(cfg[k]) for k, _ in StencilConfig._fields_})
    _check(lib().saamg_stencil_config_set(op.handle, int(precision), C.byref(c)))


@_entry
def autotune_stencil(op: Operator, precision: int, stream=None):
    """Times the 36 launch shapes of the level-0 Chebyshev step, sets the fastest on op and
    returns (shape, microseconds)."""
    c = StencilConfig()
    us = C.c_double(0)
    _check(lib().saamg_autotune_stencil(op.handle, int(precision), _stream(stream), C.byref(c),
                                        C.byref(us)))
    return c.as_dict(), us.value


@_entry
def set_cheb_degree(h: Hierarchy, degree: int):
    _check(lib().saamg_set_cheb_degree(h.handle, int(degree)))


@_entry
def autotune_cheb_degree(h: Hierarchy, rho, lo=2, hi=4, rtol=1e-8, stream=None):
    best = C.c_int(0)
    ms = C.c_double(0)
    _check(lib().saamg_autotune_cheb_degree(h.handle, _ptr(rho), int(lo), int(hi), float(rtol),
                                            _stream(stream), C.byref(best), C.byref(ms)))
    return best.value, ms.value


@_entry
def mis2_aggregate(rowptr, col, ids, seed, root, agg, stream=None):
    """Device CSR (int32 tensors), ids (int32/uint32 tensor or None) -> root (uint8), agg (int32)."""
    nagg = C.c_int(0)
    n = rowptr.numel() - 1
    _check(lib().saamg_mis2_aggregate(int(n), _ptr(rowptr), _ptr(col), _ptr(ids),
                                      int(seed) & 0xFFFFFFFF, _ptr(root), _ptr(agg),
                                      C.byref(nagg), _stream(stream)))
    return nagg.value


@_entry
def mis2_aggregate_noalloc(rowptr, col, ids, seed, root, agg, stream=None):
    """Same as mis2_aggregate, for callers that cannot allocate device memory during the call:
    the library uses its own static scratch (graphs of at most 262,144 nodes; calls must not
    overlap on the GPU).  The caller still provides every input and output tensor."""
    nagg = C.c_int(0)
    n = rowptr.numel() - 1
    _check(lib().saamg_mis2_aggregate_noalloc(int(n), _ptr(rowptr), _ptr(col), _ptr(ids),
                                              int(seed) & 0xFFFFFFFF, _ptr(root), _ptr(agg),
                                              C.byref(nagg), _stream(stream)))
    return nagg.value


def free(handle):
    if isinstance(handle, (Operator, Hierarchy)):
        handle.free()
    elif handle:
        lib().saamg_free(handle)


def make_domain(d) -> Domain:
    """From paper_0907_4863_gb300.inputs.Domain (or any object with the same fields)."""
    return Domain(d.a, d.b, d.taper, d.cx, d.cy, d.zbc, d.symmetrize)


def make_grid(g) -> Grid:
    gr = Grid()
    for k in range(3):
        gr.n[k] = g.n[k]
        gr.h[k] = g.h[k]
        gr.origin[k] = g.origin[k]
    return gr


def kernel_launches():
    """Number of kernels libsaamg has launched in this process."""
    return int(lib().saamg_kernel_launches())


def kernel_timing(enable: bool):
    _check(lib().saamg_kernel_timing(1 if enable else 0))


def kernel_timing_read(kclass: int):
    """(total_ms, launches, rows) of a kernel class since the last read; resets it."""
    ms = C.c_double(0)
    n = C.c_longlong(0)
    rows = C.c_longlong(0)
    _check(lib().saamg_kernel_timing_read(int(kclass), C.byref(ms), C.byref(n), C.byref(rows)))
    return ms.value, n.value, rows.value
