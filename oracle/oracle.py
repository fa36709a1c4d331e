"""ctypes wrapper of the FP64 CPU oracle (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  It loads ``oracle/liboracle.so`` (plain C,
built by ``oracle/build.py``) and shares nothing with the CUDA library.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None

CONSTANT, LINEAR, QUADRATIC = 0, 1, 2
Z_ROBIN, Z_DIRICHLET = 0, 1

_i = C.c_int
_l = C.c_long
_d = C.c_double
_p = C.c_void_p


def lib():
    """The sequential oracle (parity), or the OpenMP baseline build when the environment
    variable SAAMG_ORACLE_OPENMP is 1 when the library is first loaded."""
    global _lib
    if _lib is None:
        path = None
        if os.environ.get("SAAMG_ORACLE_OPENMP") == "1":
            path = _build.build_omp()
            if path is None:
                raise RuntimeError("the OpenMP build of the oracle is not available")
        path = path or _build.build()
        L = C.CDLL(path)
        L.orc_build_operator.restype = _p
        L.orc_build_operator.argtypes = [_i, _i, _i, _d, _d, _d, _d, _d, _d, _d, _d, _d, _d, _d,
                                         _i, _i, _i]
        L.orc_op_free.argtypes = [_p]
        L.orc_op_n.argtypes = [_p]
        L.orc_op_n.restype = _i
        L.orc_op_nnz.argtypes = [_p]
        L.orc_op_nnz.restype = _l
        L.orc_op_get.argtypes = [_p] + [_p] * 7
        L.orc_op_fractions.argtypes = [_p, _p]
        L.orc_node_inside.argtypes = [_p, _i, _i, _i]
        L.orc_node_inside.restype = _i
        L.orc_setup.restype = _p
        L.orc_setup.argtypes = [_p, _i, _d, _d, _i, _i, _i]
        L.orc_setup_agg.restype = _p
        L.orc_setup_agg.argtypes = [_p, _i, _d, _d, _i, _i, _i, _i]
        L.orc_setup_ex.restype = _p
        L.orc_setup_ex.argtypes = [_p, _i, _d, _d, _i, _i, _i, _i, _i, _i]
        L.orc_hier_colours.argtypes = [_p, _p]
        L.orc_hier_colours.restype = _i
        L.orc_colour.argtypes = [_i, _p, _p, _p, C.c_uint, _p]
        L.orc_colour.restype = _i
        L.orc_sgs.argtypes = [_i, _p, _p, _p, _p, _p, _i, _i, _p, _p]
        L.orc_cube_aggregate.argtypes = [_i, _p, _p, _p, _p, _p, _p]
        L.orc_cube_aggregate.restype = _i
        L.orc_hier_free.argtypes = [_p]
        for f in ("orc_hier_levels", "orc_hier_status"):
            getattr(L, f).argtypes = [_p]
            getattr(L, f).restype = _i
        L.orc_hier_n.argtypes = [_p, _i]
        L.orc_hier_n.restype = _i
        for f in ("orc_hier_nnz", "orc_hier_nnz_p"):
            getattr(L, f).argtypes = [_p, _i]
            getattr(L, f).restype = _l
        for f in ("orc_hier_get_a", "orc_hier_get_p", "orc_hier_get_r"):
            getattr(L, f).argtypes = [_p, _i, _p, _p, _p]
        L.orc_hier_get_agg.argtypes = [_p, _i, _p, _p]
        for f in ("orc_hier_lambda", "orc_hier_omega"):
            getattr(L, f).argtypes = [_p, _i]
            getattr(L, f).restype = _d
        L.orc_deposit_cic.argtypes = [_i, _i, _i, _d, _d, _d, _d, _d, _d, _i, _p, _p, _p, _p, _p]
        L.orc_field_gradient.argtypes = [_p, _p, _p, _p, _p]
        L.orc_gather_cic.argtypes = [_i, _i, _i, _d, _d, _d, _d, _d, _d, _p, _p, _p, _i, _p, _p,
                                     _p, _p, _p, _p]
        L.orc_fmix32.argtypes = [C.c_uint]
        L.orc_fmix32.restype = C.c_uint
        L.orc_mis2.argtypes = [_i, _p, _p, _p, C.c_uint, _p]
        L.orc_aggregate.argtypes = [_i, _p, _p, _p, C.c_uint, _p, _p]
        L.orc_aggregate.restype = _i
        L.orc_power_lambda.argtypes = [_i, _p, _p, _p, _p, _i]
        L.orc_power_lambda.restype = _d
        L.orc_cheb_smooth.argtypes = [_i, _p, _p, _p, _p, _d, _d, _d, _i, _p, _p, _i]
        L.orc_dense_lu_solve.argtypes = [_i, _p, _p, _p]
        L.orc_dense_lu_solve.restype = _i
        L.orc_vcycle.argtypes = [_p, _p, _p]
        L.orc_pcg.argtypes = [_p, _p, _p, _d, _i, _i, _p, _p]
        L.orc_pcg.restype = _i
        L.orc_solve.argtypes = [_p, _p, _p, _d, _i, _i, _p, _p, _p]
        L.orc_solve.restype = _i
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _csr_arrays(rowptr, col, val=None):
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = None if val is None else np.ascontiguousarray(val, dtype=np.float64)
    return rowptr, col, val


class Operator:
    """Finite-difference operator of Sec. 2 on a box grid (see saamg_oracle.h)."""

    def __init__(self, n, h, origin, a, b, taper=1.0, cx=0.0, cy=0.0, zbc=Z_ROBIN,
                 symmetrize=1, mode=LINEAR):
        self.shape = tuple(int(v) for v in n)
        self.h = tuple(float(v) for v in h)
        self.origin = tuple(float(v) for v in origin)
        L = lib()
        self._h = L.orc_build_operator(self.shape[0], self.shape[1], self.shape[2], *self.h,
                                       *self.origin, float(a), float(b), float(taper), float(cx),
                                       float(cy), int(zbc), int(symmetrize), int(mode))
        if not self._h:
            raise ValueError("oracle rejected the operator arguments")
        self.n = L.orc_op_n(self._h)
        self.nnz = L.orc_op_nnz(self._h)
        n_, nnz = self.n, self.nnz
        self.node_of_row = np.empty(n_, np.int32)
        self.scale = np.empty(n_, np.float64)
        self.bfac = np.empty(n_, np.float64)
        self.rowptr = np.empty(n_ + 1, np.int32)
        self.col = np.empty(nnz, np.int32)
        self.aval = np.empty(nnz, np.float64)
        self.ahat = np.empty(nnz, np.float64)
        L.orc_op_get(self._h, _ptr(self.node_of_row), _ptr(self.scale), _ptr(self.bfac),
                     _ptr(self.rowptr), _ptr(self.col), _ptr(self.aval), _ptr(self.ahat))

    def fractions(self):
        f = np.empty(6 * self.n, np.float64)
        lib().orc_op_fractions(self._h, _ptr(f))
        return f.reshape(self.n, 6)

    def inside(self, i, j, k):
        return bool(lib().orc_node_inside(self._h, i, j, k))

    def scipy(self, scaled=True):
        import scipy.sparse as sp
        v = self.ahat if scaled else self.aval
        return sp.csr_matrix((v, self.col, self.rowptr), shape=(self.n, self.n))

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.orc_op_free(self._h)
            self._h = None


class Hierarchy:
    """SA-AMG hierarchy of Sec. 3.2 built on the scaled operator."""

    AGG_MIS2, AGG_CUBES = 0, 1
    COARSE_LU, COARSE_GS = 0, 1

    def __init__(self, op, cheb_degree=2, cheb_ratio=30.0, cheb_safety=1.1, max_coarse=1000,
                 max_levels=10, power_iters=10, aggregation=0, coarse_solver=0,
                 coarse_sweeps=3):
        self.op = op
        L = lib()
        self._h = L.orc_setup_ex(op._h, int(cheb_degree), float(cheb_ratio),
                                 float(cheb_safety), int(max_coarse), int(max_levels),
                                 int(power_iters), int(aggregation), int(coarse_solver),
                                 int(coarse_sweeps))
        self.status = L.orc_hier_status(self._h)
        self.levels = L.orc_hier_levels(self._h)

    def n(self, l):
        return lib().orc_hier_n(self._h, l)

    def nnz(self, l):
        return lib().orc_hier_nnz(self._h, l)

    def _get(self, fn, l, n, nnz):
        rowptr = np.empty(n + 1, np.int32)
        col = np.empty(nnz, np.int32)
        val = np.empty(nnz, np.float64)
        fn(self._h, l, _ptr(rowptr), _ptr(col), _ptr(val))
        return rowptr, col, val

    def A(self, l):
        return self._get(lib().orc_hier_get_a, l, self.n(l), self.nnz(l))

    def P(self, l):
        return self._get(lib().orc_hier_get_p, l, self.n(l), lib().orc_hier_nnz_p(self._h, l))

    def R(self, l):
        return self._get(lib().orc_hier_get_r, l, self.n(l + 1), lib().orc_hier_nnz_p(self._h, l))

    def agg(self, l):
        n = self.n(l)
        agg = np.empty(n, np.int32)
        root = np.empty(n, np.uint8)
        lib().orc_hier_get_agg(self._h, l, _ptr(agg), _ptr(root))
        return agg, root

    def colours(self):
        """Colour of each row of the coarsest level (Gauss-Seidel coarse solver), or None."""
        c = np.empty(self.n(self.levels - 1), np.int32)
        k = lib().orc_hier_colours(self._h, _ptr(c))
        return (c, k) if k else None

    def lam(self, l):
        return lib().orc_hier_lambda(self._h, l)

    def omega(self, l):
        return lib().orc_hier_omega(self._h, l)

    def vcycle(self, r):
        r = np.ascontiguousarray(r, np.float64)
        z = np.zeros_like(r)
        lib().orc_vcycle(self._h, _ptr(r), _ptr(z))
        return z

    def pcg(self, bhat, x0=None, rtol=1e-8, maxit=1000, beta_rule=0):
        bhat = np.ascontiguousarray(bhat, np.float64)
        x = np.zeros_like(bhat) if x0 is None else np.array(x0, np.float64, copy=True)
        it = C.c_int(0)
        rr = C.c_double(0)
        rc = lib().orc_pcg(self._h, _ptr(bhat), _ptr(x), rtol, maxit, beta_rule, C.byref(it),
                           C.byref(rr))
        return x, rc, it.value, rr.value

    def solve(self, rho_box, phi0_box=None, rtol=1e-8, maxit=1000, beta_rule=0):
        rho = np.ascontiguousarray(rho_box, np.float64).ravel()
        phi = np.zeros_like(rho) if phi0_box is None else np.array(phi0_box, np.float64).ravel().copy()
        it = C.c_int(0)
        rr = C.c_double(0)
        rt = C.c_double(0)
        rc = lib().orc_solve(self._h, _ptr(rho), _ptr(phi), rtol, maxit, beta_rule, C.byref(it),
                             C.byref(rr), C.byref(rt))
        return phi, dict(rc=rc, iters=it.value, relres=rr.value, relres_true=rt.value)

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.orc_hier_free(self._h)
            self._h = None


def deposit_cic(grid, x, y, z, q):
    """Cloud-in-cell charge density on the box (Sec. 4.1)."""
    (nx, ny, nz), h, o = grid.n, grid.h, grid.origin
    x, y, z, q = (np.ascontiguousarray(a, np.float64) for a in (x, y, z, q))
    rho = np.empty(nx * ny * nz)
    lib().orc_deposit_cic(nx, ny, nz, h[0], h[1], h[2], o[0], o[1], o[2], len(x), _ptr(x),
                          _ptr(y), _ptr(z), _ptr(q), _ptr(rho))
    return rho


def field_gradient(op, phi):
    """E = -grad phi on the box (zero outside the unknowns)."""
    phi = np.ascontiguousarray(phi, np.float64).ravel()
    e = [np.empty_like(phi) for _ in range(3)]
    lib().orc_field_gradient(op._h, _ptr(phi), _ptr(e[0]), _ptr(e[1]), _ptr(e[2]))
    return e


def gather_cic(grid, e, x, y, z):
    """E at the particles with the CIC weights of the deposition."""
    (nx, ny, nz), h, o = grid.n, grid.h, grid.origin
    e = [np.ascontiguousarray(a, np.float64) for a in e]
    x, y, z = (np.ascontiguousarray(a, np.float64) for a in (x, y, z))
    out = [np.empty(len(x)) for _ in range(3)]
    lib().orc_gather_cic(nx, ny, nz, h[0], h[1], h[2], o[0], o[1], o[2], _ptr(e[0]), _ptr(e[1]),
                         _ptr(e[2]), len(x), _ptr(x), _ptr(y), _ptr(z), _ptr(out[0]),
                         _ptr(out[1]), _ptr(out[2]))
    return out


def fmix32(x):
    return lib().orc_fmix32(int(x) & 0xFFFFFFFF)


def mis2(rowptr, col, ids, seed):
    rowptr, col, _ = _csr_arrays(rowptr, col)
    n = len(rowptr) - 1
    ids = np.ascontiguousarray(ids, np.uint32)
    root = np.zeros(n, np.uint8)
    lib().orc_mis2(n, _ptr(rowptr), _ptr(col), _ptr(ids), int(seed) & 0xFFFFFFFF, _ptr(root))
    return root


def aggregate(rowptr, col, ids, seed, root):
    rowptr, col, _ = _csr_arrays(rowptr, col)
    n = len(rowptr) - 1
    ids = np.ascontiguousarray(ids, np.uint32)
    root = np.ascontiguousarray(root, np.uint8)
    agg = np.empty(n, np.int32)
    nagg = lib().orc_aggregate(n, _ptr(rowptr), _ptr(col), _ptr(ids), int(seed) & 0xFFFFFFFF,
                               _ptr(root), _ptr(agg))
    return agg, nagg


def cube_aggregate(ids, dims):
    """Cubes of 3 x 3 x 3 lattice nodes (Sec. 3.2): (agg, root, next_ids, next_dims)."""
    ids = np.ascontiguousarray(ids, np.uint32)
    n = len(ids)
    d = np.ascontiguousarray(dims, np.int32)
    agg = np.empty(n, np.int32)
    root = np.empty(n, np.uint8)
    nxt = np.empty(max(n, 1), np.uint32)
    nd = np.zeros(3, np.int32)
    nagg = lib().orc_cube_aggregate(n, _ptr(ids), _ptr(d), _ptr(agg), _ptr(root), _ptr(nxt),
                                    _ptr(nd))
    return agg, root, nxt[:nagg].copy(), tuple(int(v) for v in nd)


def colour(rowptr, col, ids, seed=0x2545F491):
    rowptr, col, _ = _csr_arrays(rowptr, col)
    n = len(rowptr) - 1
    ids = np.ascontiguousarray(ids, np.uint32)
    c = np.empty(n, np.int32)
    k = lib().orc_colour(n, _ptr(rowptr), _ptr(col), _ptr(ids), int(seed) & 0xFFFFFFFF, _ptr(c))
    return c, k


def sgs(rowptr, col, val, colours, ncolours, steps, b):
    rowptr, col, val = _csr_arrays(rowptr, col, val)
    n = len(rowptr) - 1
    invd = np.empty(n)
    for i in range(n):
        s, e = rowptr[i], rowptr[i + 1]
        invd[i] = 1.0 / val[s:e][col[s:e] == i][0]
    colours = np.ascontiguousarray(colours, np.int32)
    b = np.ascontiguousarray(b, np.float64)
    x = np.empty(n)
    lib().orc_sgs(n, _ptr(rowptr), _ptr(col), _ptr(val), _ptr(invd), _ptr(colours),
                  int(ncolours), int(steps), _ptr(b), _ptr(x))
    return x


def power_lambda(rowptr, col, val, ids, iters=10):
    rowptr, col, val = _csr_arrays(rowptr, col, val)
    ids = np.ascontiguousarray(ids, np.uint32)
    return lib().orc_power_lambda(len(rowptr) - 1, _ptr(rowptr), _ptr(col), _ptr(val), _ptr(ids),
                                  int(iters))


def cheb_smooth(rowptr, col, val, invd, lam, b, x=None, degree=2, ratio=30.0, safety=1.1):
    rowptr, col, val = _csr_arrays(rowptr, col, val)
    n = len(rowptr) - 1
    invd = np.ascontiguousarray(invd, np.float64)
    b = np.ascontiguousarray(b, np.float64)
    xz = x is None
    x = np.zeros(n) if xz else np.array(x, np.float64, copy=True)
    lib().orc_cheb_smooth(n, _ptr(rowptr), _ptr(col), _ptr(val), _ptr(invd), float(lam),
                          float(ratio), float(safety), int(degree), _ptr(b), _ptr(x), int(xz))
    return x


def dense_lu_solve(a, b):
    a = np.ascontiguousarray(a, np.float64)
    b = np.ascontiguousarray(b, np.float64)
    x = np.empty_like(b)
    rc = lib().orc_dense_lu_solve(len(b), _ptr(a), _ptr(b), _ptr(x))
    if rc != 0:
        raise ZeroDivisionError("zero pivot")
    return x
