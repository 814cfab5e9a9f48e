"""ctypes wrapper of the plain C FP64 oracle (``oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py``; never by the library.  The shared object is compiled
with the host C compiler on first use (or by ``build()``), into ``oracle/_build/``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SO = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

MASS, LAPLACE, HELMHOLTZ, KAPPA_DIFFUSION = 1, 2, 3, 4

_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``_build/liboracle.so`` (plain gcc, -O2, no fast-math)."""
    with _lock:
        if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
            os.makedirs(os.path.dirname(_SO), exist_ok=True)
            tmp = _SO + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fPIC", "-shared",
                                   "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = C.CDLL(build())
    lib.oracle_set_mutation.argtypes = [C.c_int]
    lib.oracle_num_nodes.argtypes = [C.c_int, C.c_int]
    lib.oracle_nodes.argtypes = [C.c_int, C.c_int, _i32p]
    lib.oracle_gauss_legendre01.argtypes = [C.c_int, _f64p, _f64p]
    lib.oracle_quadrature.argtypes = [C.c_int, C.c_int, _f64p, _f64p]
    lib.oracle_element_matrix.argtypes = [C.c_int, C.c_int, C.c_int, _f64p, _f64p, _f64p]
    lib.oracle_element_vector.argtypes = [C.c_int, C.c_int, C.c_int, _f64p, _f64p, _f64p]
    lib.oracle_sparsity.restype = C.c_int64
    lib.oracle_sparsity.argtypes = [C.c_int64, C.c_int, _i32p, C.c_int, _i32p, C.c_int64, C.c_int64,
                                    _i64p, C.c_void_p]
    lib.oracle_assemble_mat.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int64, _i32p, _f64p, _i32p,
                                        C.c_void_p, _i64p, _i32p, _f64p, _f64p]
    lib.oracle_assemble_vec.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int64, _i32p, _f64p, _i32p,
                                        _f64p, _i32p, _f64p, _f64p]
    lib.oracle_action.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int64, _i32p, _f64p, _i32p, C.c_void_p,
                                  _f64p, _f64p, _f64p]
    lib.oracle_assemble_rows.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int64, _i32p, _f64p, _i32p,
                                         C.c_void_p, C.c_int64, _i64p, C.c_int64, _i64p, _i32p, _f64p,
                                         _f64p]
    lib.oracle_eval_function.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int64, _i32p, _f64p, _i32p,
                                         _f64p, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.oracle_dirichlet_apply.argtypes = [C.c_int64, _i64p, _i32p, _f64p, _f64p,
                                           np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS"), C.c_void_p]
    lib.oracle_cg_jacobi.argtypes = [C.c_int64, _i64p, _i32p, _f64p, _f64p, _f64p, C.c_double, C.c_int,
                                     C.POINTER(C.c_double), C.POINTER(C.c_double)]
    lib.oracle_wave_steps.argtypes = [C.c_int, C.c_int, C.c_int64, _i32p, _f64p, _i32p, C.c_int64, C.c_void_p,
                                      _f64p, _f64p, C.c_double, C.c_double, C.c_int]
    _lib = lib
    return lib


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def set_mutation(code: int) -> None:
    """Plant a known mistake in the oracle (0 = none). Test use only."""
    _load().oracle_set_mutation(int(code))


def num_nodes(dim: int, p: int) -> int:
    return int(_load().oracle_num_nodes(dim, p))


def nodes(dim: int, p: int) -> np.ndarray:
    nd = num_nodes(dim, p)
    out = np.zeros(nd * (dim + 1), dtype=np.int32)
    if _load().oracle_nodes(dim, p, out) != nd:
        raise RuntimeError("oracle_nodes failed")
    return out.reshape(nd, dim + 1)


def gauss_legendre01(m: int):
    x, w = np.zeros(m), np.zeros(m)
    if _load().oracle_gauss_legendre01(m, x, w) != m:
        raise RuntimeError("bad m")
    return x, w


def quadrature(dim: int, m: int):
    pts, wts = np.zeros(m ** dim * dim), np.zeros(m ** dim)
    nq = _load().oracle_quadrature(dim, m, pts, wts)
    if nq < 0:
        raise RuntimeError("bad quadrature request")
    return pts.reshape(nq, dim), wts


def element_matrix(dim: int, p: int, form: int, xv, kv=None) -> np.ndarray:
    nd = num_nodes(dim, p)
    K = np.zeros(nd * nd)
    kv = _c(np.ones(dim + 1) if kv is None else kv, np.float64)
    if _load().oracle_element_matrix(dim, p, form, _c(xv, np.float64).ravel(), kv, K) != nd:
        raise RuntimeError("oracle_element_matrix failed")
    return K.reshape(nd, nd)


def element_vector(dim: int, p: int, pf: int, xv, fe) -> np.ndarray:
    nd = num_nodes(dim, p)
    b = np.zeros(nd)
    if _load().oracle_element_vector(dim, p, pf, _c(xv, np.float64).ravel(), _c(fe, np.float64), b) != nd:
        raise RuntimeError("oracle_element_vector failed")
    return b


def sparsity(rmap, cmap, nrows: int, ncols: int):
    """CSR pattern (rowptr int64, colidx int32) of the union of map pairs."""
    rmap, cmap = _c(rmap, np.int32), _c(cmap, np.int32)
    ncell = rmap.shape[0]
    rowptr = np.zeros(nrows + 1, dtype=np.int64)
    lib = _load()
    nnz = lib.oracle_sparsity(ncell, rmap.shape[1], rmap.ravel(), cmap.shape[1], cmap.ravel(),
                              nrows, ncols, rowptr, None)
    if nnz < 0:
        raise ValueError("map value out of range")
    colidx = np.zeros(max(nnz, 1), dtype=np.int32)
    lib.oracle_sparsity(ncell, rmap.shape[1], rmap.ravel(), cmap.shape[1], cmap.ravel(),
                        nrows, ncols, rowptr, colidx.ctypes.data)
    return rowptr, colidx[:nnz]


def _kappa_ptr(kappa):
    if kappa is None:
        return None, None
    k = _c(kappa, np.float64)
    return k, k.ctypes.data


def assemble_mat(dim, p, form, cmap, coords, coord_map, rowptr, colidx, kappa=None):
    """Global CSR values and absolute-contribution sums for the bilinear form."""
    cmap = _c(cmap, np.int32)
    vals = np.zeros(colidx.size)
    absv = np.zeros(colidx.size)
    keep, kp = _kappa_ptr(kappa)
    rc = _load().oracle_assemble_mat(dim, p, form, cmap.shape[0], cmap.ravel(), _c(coords, np.float64).ravel(),
                                     _c(coord_map, np.int32).ravel(), kp, _c(rowptr, np.int64),
                                     _c(colidx, np.int32), vals, absv)
    if rc != 0:
        raise RuntimeError("oracle_assemble_mat failed")
    return vals, absv


def assemble_vec(dim, p, pf, cmap, nrows, coords, coord_map, f, fmap):
    cmap = _c(cmap, np.int32)
    b, absb = np.zeros(nrows), np.zeros(nrows)
    rc = _load().oracle_assemble_vec(dim, p, pf, cmap.shape[0], cmap.ravel(), _c(coords, np.float64).ravel(),
                                     _c(coord_map, np.int32).ravel(), _c(f, np.float64),
                                     _c(fmap, np.int32).ravel(), b, absb)
    if rc != 0:
        raise RuntimeError("oracle_assemble_vec failed")
    return b, absb


def action(dim, p, form, cmap, coords, coord_map, x, kappa=None):
    cmap = _c(cmap, np.int32)
    x = _c(x, np.float64)
    y, absy = np.zeros(x.size), np.zeros(x.size)
    keep, kp = _kappa_ptr(kappa)
    rc = _load().oracle_action(dim, p, form, cmap.shape[0], cmap.ravel(), _c(coords, np.float64).ravel(),
                               _c(coord_map, np.int32).ravel(), kp, x, y, absy)
    if rc != 0:
        raise RuntimeError("oracle_action failed")
    return y, absy


def assemble_rows(dim, p, form, cmap, coords, coord_map, nrows, rows, sel_rowptr, sel_colidx, kappa=None):
    """Values of the selected rows (sorted unique ``rows``) on a caller-given pattern."""
    cmap = _c(cmap, np.int32)
    vals = np.zeros(sel_colidx.size)
    absv = np.zeros(sel_colidx.size)
    keep, kp = _kappa_ptr(kappa)
    rc = _load().oracle_assemble_rows(dim, p, form, cmap.shape[0], cmap.ravel(), _c(coords, np.float64).ravel(),
                                      _c(coord_map, np.int32).ravel(), kp, nrows, _c(rows, np.int64),
                                      len(rows), _c(sel_rowptr, np.int64), _c(sel_colidx, np.int32), vals, absv)
    if rc != 0:
        raise RuntimeError("oracle_assemble_rows failed")
    return vals, absv


def functional(dim, p, form, cmap, coords, coord_map, x, kappa=None):
    """A form of rank 0 (a Global, Sec. 4.3): the bilinear form with both arguments the Function x,
    a(x, x) = sum_e x_e^T K_e x_e = x . (A x), from the oracle's cell-by-cell action.  Returns the
    value and its scale sum_i |x_i| (sum_e |K_e| |x_e|)_i, which bounds the rounding of any
    summation order."""
    y, absy = action(dim, p, form, cmap, coords, coord_map, x, kappa=kappa)
    return float(np.dot(x, y)), float(np.dot(np.abs(x), absy))


def linear_functional(dim, p, pf, cmap, coords, coord_map, f, fmap, x):
    """The linear form with its test argument the Function x: L(x) = sum_e b_e . x_e = b . x (b the
    assembled f v dx), and its scale sum_i |x_i| (sum_e |b_e|)_i."""
    x = _c(x, np.float64)
    b, absb = assemble_vec(dim, p, pf, cmap, x.size, coords, coord_map, f, fmap)
    return float(np.dot(b, x)), float(np.dot(absb, np.abs(x)))


def cell_volumes(dim, coords, coord_map):
    """|T| of every cell: the oracle's quadrature weights w |det J| of each cell added up (its rule
    integrates constants exactly)."""
    cv = _c(coord_map, np.int32)
    _, w, _ = eval_function(dim, 1, 1, cv, coords, cv, np.zeros(_c(coords, np.float64).shape[0]))
    return w.reshape(cv.shape[0], -1).sum(axis=1)


def eval_function(dim, p, qdeg, cmap, coords, coord_map, u):
    """Physical quadrature points, weights (w |detJ|) and values of the P_p function u."""
    cmap = _c(cmap, np.int32)
    lib = _load()
    args = (dim, p, qdeg, cmap.shape[0], cmap.ravel(), _c(coords, np.float64).ravel(),
            _c(coord_map, np.int32).ravel(), _c(u, np.float64))
    nq = lib.oracle_eval_function(*args, None, None, None)
    ncell = cmap.shape[0]
    xq, wq, uq = np.zeros(ncell * nq * dim), np.zeros(ncell * nq), np.zeros(ncell * nq)
    lib.oracle_eval_function(*args, xq.ctypes.data, wq.ctypes.data, uq.ctypes.data)
    return xq.reshape(-1, dim), wq, uq


def dirichlet_apply(rowptr, colidx, vals, b, is_bc, g=None):
    """Symmetric elimination of u = g on the rows flagged in is_bc; returns new (vals, b)."""
    vals = np.array(vals, dtype=np.float64, copy=True)
    b = np.array(b, dtype=np.float64, copy=True)
    gk = None if g is None else _c(g, np.float64)
    _load().oracle_dirichlet_apply(b.size, _c(rowptr, np.int64), _c(colidx, np.int32), vals, b,
                                   _c(is_bc, np.uint8), None if gk is None else gk.ctypes.data)
    return vals, b


def cg_jacobi(rowptr, colidx, vals, b, x0=None, rtol=1e-8, maxit=100000):
    """Jacobi-preconditioned CG; returns (x, iterations, ||r||, ||b||). iterations = -1: not SPD."""
    b = _c(b, np.float64)
    x = np.zeros(b.size) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    rn, bn = C.c_double(), C.c_double()
    it = _load().oracle_cg_jacobi(b.size, _c(rowptr, np.int64), _c(colidx, np.int32), _c(vals, np.float64), b, x,
                                  float(rtol), int(maxit), C.byref(rn), C.byref(bn))
    return x, it, rn.value, bn.value


def wave_steps(dim, p, cmap, coords, coord_map, nnodes, phi, pv, t0, dt, nsteps, is_bc=None):
    """Explicit lumped-mass wave steps; returns new (phi, p)."""
    cmap = _c(cmap, np.int32)
    phi = np.array(phi, dtype=np.float64, copy=True)
    pv = np.array(pv, dtype=np.float64, copy=True)
    bc = None if is_bc is None else _c(is_bc, np.uint8)
    rc = _load().oracle_wave_steps(dim, p, cmap.shape[0], cmap.ravel(), _c(coords, np.float64).ravel(),
                                   _c(coord_map, np.int32).ravel(), int(nnodes),
                                   None if bc is None else bc.ctypes.data, phi, pv, float(t0), float(dt), int(nsteps))
    if rc != 0:
        raise RuntimeError("oracle_wave_steps failed")
    return phi, pv
