"""Thin ctypes binding of libfe (include/fe.h): argument marshalling only.

Every function here forwards to the C entry point of the same name (without the ``fe_``
prefix); all computation runs in libfe's CUDA kernels.  PyTorch provides device memory
(tensors passed in are borrowed; library-owned buffers come from torch's caching allocator
through fe_ctx_set_allocator) and the CUDA stream (torch's current stream by default).
There is no CPU fallback: importing this module without a built libfe.so raises, and so does
creating a context without a CUDA device.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "libfe.so")

FE_OK, FE_EINVAL, FE_EHANDLE, FE_ERANGE, FE_EARITY, FE_ENOMEM, FE_ECUDA, FE_ETIMEOUT, FE_EUNSUPPORTED = \
    0, -1, -2, -3, -4, -5, -6, -7, -8
FORM_MASS, FORM_LAPLACE, FORM_HELMHOLTZ, FORM_KAPPA_DIFFUSION, FORM_SOURCE = 1, 2, 3, 4, 5
PREC_FP64, PREC_F32X2, PREC_FP32, PREC_TF32X3 = 0, 1, 2, 3
STRATEGY_AUTO, STRATEGY_PUSH, STRATEGY_PULL = 0, 1, 2
REDUCE_SUM, REDUCE_MIN, REDUCE_MAX = 0, 1, 2

SYMBOLS = [
    "fe_last_error", "fe_version", "fe_ctx_create", "fe_ctx_set_stream", "fe_ctx_set_allocator",
    "fe_ctx_set_checks", "fe_sync", "fe_ctx_destroy", "fe_set_create", "fe_set_size", "fe_set_destroy",
    "fe_map_create", "fe_map_destroy", "fe_dat_create", "fe_dat_destroy", "fe_sparsity_build",
    "fe_sparsity_rebuild", "fe_sparsity_changed", "fe_sparsity_track_columns", "fe_sparsity_build_noalloc", "fe_sparsity_csr", "fe_sparsity_lut", "fe_sparsity_destroy", "fe_mat_create",
    "fe_mat_values", "fe_mat_zero", "fe_mat_destroy", "fe_kernel_create", "fe_kernel_destroy",
    "fe_assemble_mat", "fe_assemble_vec", "fe_action", "fe_assemble_mat_action", "fe_global_create", "fe_global_data", "fe_global_destroy",
    "fe_assemble_global", "fe_reduce_cell_volume", "fe_elem_matrices", "fe_action_stored", "fe_batch_create",
    "fe_batch_values", "fe_batch_tune",
    "fe_batch_assemble", "fe_batch_destroy", "fe_dirichlet_apply", "fe_cg_create", "fe_cg_add", "fe_cg_iterate",
    "fe_cg_poll", "fe_cg_remove", "fe_cg_destroy", "fe_server_create", "fe_server_submit", "fe_server_run",
    "fe_server_result", "fe_server_stats_get", "fe_server_destroy", "fe_wave_steps",
]


class FeError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class fe_form_desc(C.Structure):
    _fields_ = [("form", C.c_int), ("dim", C.c_int), ("degree", C.c_int), ("coeff_degree", C.c_int),
                ("precision", C.c_int), ("strategy", C.c_int)]


class fe_arg(C.Structure):
    _fields_ = [("dat", C.c_void_p), ("map", C.c_void_p)]


class fe_batch_item(C.Structure):
    _fields_ = [("kmat", C.c_void_p), ("kvec", C.c_void_p), ("cells", C.c_void_p), ("sp", C.c_void_p),
                ("coords", C.c_void_p), ("coord_map", C.c_void_p), ("f", fe_arg)]


class fe_server_config(C.Structure):
    _fields_ = [("hbm_budget", C.c_size_t), ("max_active", C.c_int), ("iters_per_tick", C.c_int),
                ("rtol", C.c_double), ("maxit", C.c_int), ("precision", C.c_int)]


class fe_solve_request(C.Structure):
    _fields_ = [("degree", C.c_int), ("ncell", C.c_int64), ("nnodes", C.c_int64), ("nvert", C.c_int64),
                ("cell_node", C.c_void_p), ("cell_vertex", C.c_void_p), ("coords", C.c_void_p), ("f", C.c_void_p),
                ("is_bc", C.c_void_p), ("x_out", C.c_void_p), ("arrival_s", C.c_double), ("mesh_key", C.c_uint64)]


class fe_solve_result(C.Structure):
    _fields_ = [("status", C.c_int), ("iters", C.c_int), ("rnorm", C.c_double), ("bnorm", C.c_double),
                ("admitted_s", C.c_double), ("finished_s", C.c_double), ("bytes", C.c_size_t),
                ("estimate", C.c_size_t)]


class fe_server_stats(C.Structure):
    _fields_ = [("peak_bytes", C.c_size_t), ("live_bytes", C.c_size_t), ("base_bytes", C.c_size_t),
                ("submitted", C.c_int), ("converged", C.c_int), ("refused", C.c_int), ("estimate_misses", C.c_int),
                ("run_s", C.c_double), ("cg_launches", C.c_int64), ("admit_s", C.c_double), ("tick_s", C.c_double),
                ("retire_s", C.c_double), ("cache_hits", C.c_int), ("cache_misses", C.c_int),
                ("cache_evictions", C.c_int), ("sparsity_builds", C.c_int), ("cache_bytes", C.c_size_t)]


CG_RUNNING, CG_CONVERGED, CG_MAXIT, CG_BREAKDOWN = 0, 1, 2, 3
SOLVE_PENDING, SOLVE_CONVERGED, SOLVE_MAXIT, SOLVE_BREAKDOWN, SOLVE_REFUSED = 0, 1, 2, 3, 4

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)

_lib = None


def library_path() -> str:
    return _LIB_PATH


def load():
    """Loads libfe.so (built by ``paper_1501_01809_gb300.build``); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"libfe.so is not built ({_LIB_PATH}); run `python -m paper_1501_01809_gb300.build`")
    lib = C.CDLL(_LIB_PATH)
    P, I64, I = C.c_void_p, C.c_int64, C.c_int
    PP = C.POINTER(C.c_void_p)
    sig = {
        "fe_last_error": (C.c_char_p, []), "fe_version": (C.c_char_p, []),
        "fe_ctx_create": (I, [I, P, PP]), "fe_ctx_set_stream": (I, [P, P]),
        "fe_ctx_set_allocator": (I, [P, ALLOC_FN, FREE_FN, P]), "fe_ctx_set_checks": (I, [P, I]),
        "fe_sync": (I, [P]), "fe_ctx_destroy": (I, [P]),
        "fe_set_create": (I, [P, I64, PP]), "fe_set_size": (I, [P, C.POINTER(I64)]), "fe_set_destroy": (I, [P]),
        "fe_map_create": (I, [P, P, P, I, P, I, PP]), "fe_map_destroy": (I, [P]),
        "fe_dat_create": (I, [P, P, I, P, PP]), "fe_dat_destroy": (I, [P]),
        "fe_sparsity_build": (I, [P, P, P, PP]), "fe_sparsity_rebuild": (I, [P]), "fe_sparsity_changed": (I, [P, PP]), "fe_sparsity_track_columns": (I, [P, I]),
        "fe_sparsity_build_noalloc": (I, [P, I, P, I, I64, I64, I64, P, P, I64, P, C.POINTER(I64), P]),
        "fe_sparsity_csr": (I, [P, C.POINTER(I64), C.POINTER(I64), C.POINTER(I64), PP, PP]),
        "fe_sparsity_lut": (I, [P, PP]), "fe_sparsity_destroy": (I, [P]),
        "fe_mat_create": (I, [P, P, PP]), "fe_mat_values": (I, [P, PP]), "fe_mat_zero": (I, [P]),
        "fe_mat_destroy": (I, [P]),
        "fe_kernel_create": (I, [P, C.POINTER(fe_form_desc), PP]), "fe_kernel_destroy": (I, [P]),
        "fe_assemble_mat": (I, [P, P, P, P, I, P, P, C.POINTER(fe_arg), I]),
        "fe_assemble_vec": (I, [P, P, P, P, P, I, P, P, C.POINTER(fe_arg), I, P]),
        "fe_action": (I, [P, P, P, P, P, P, I, P, P, C.POINTER(fe_arg), I, P]),
        "fe_assemble_mat_action": (I, [P, P, P, P, P, P, P, I, P, P, C.POINTER(fe_arg), I]),
        "fe_global_create": (I, [P, I, PP]), "fe_global_data": (I, [P, PP]), "fe_global_destroy": (I, [P]),
        "fe_assemble_global": (I, [P, P, P, P, I, P, P, P, P, C.POINTER(fe_arg), I]),
        "fe_reduce_cell_volume": (I, [P, P, P, I, I, P, P]),
        "fe_elem_matrices": (I, [P, P, P, P, P, P, C.POINTER(fe_arg), I]),
        "fe_action_stored": (I, [P, P, P, P, P, P, P, I]),
        "fe_batch_create": (I, [P, I, C.POINTER(fe_batch_item), PP]),
        "fe_batch_values": (I, [P, I, PP, C.POINTER(I64), PP, C.POINTER(I64)]),
        "fe_batch_tune": (I, [P, I, C.POINTER(I), C.POINTER(I), C.POINTER(C.c_float)]),
        "fe_batch_assemble": (I, [P, I]), "fe_batch_destroy": (I, [P]),
        "fe_dirichlet_apply": (I, [P, P, P, P, P]),
        "fe_wave_steps": (I, [P, P, P, P, P, P, P, P, P, P, P, C.c_double, C.c_double, I]),
        "fe_cg_create": (I, [P, I, PP]), "fe_cg_add": (I, [P, P, P, P, C.c_double, I, C.POINTER(I)]),
        "fe_cg_iterate": (I, [P, I, I]),
        "fe_cg_poll": (I, [P, I, P, P, P, P]), "fe_cg_remove": (I, [P, I]), "fe_cg_destroy": (I, [P]),
        "fe_server_create": (I, [P, C.POINTER(fe_server_config), PP]),
        "fe_server_submit": (I, [P, C.POINTER(fe_solve_request), C.POINTER(I64)]),
        "fe_server_run": (I, [P]), "fe_server_result": (I, [P, I64, C.POINTER(fe_solve_result)]),
        "fe_server_stats_get": (I, [P, C.POINTER(fe_server_stats)]), "fe_server_destroy": (I, [P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(rc: int):
    if rc != FE_OK:
        raise FeError(rc, load().fe_last_error().decode())


def version() -> str:
    return load().fe_version().decode()


class _CudaView:
    """__cuda_array_interface__ wrapper so torch can view library-owned device memory."""

    def __init__(self, ptr, shape, typestr, owner):
        self.owner = owner
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 3, "strides": None}


def _view(ptr, n, dtype, owner, device):
    typestr = {torch.int64: "<i8", torch.int32: "<i4", torch.uint8: "|u1", torch.float64: "<f8"}[dtype]
    if n == 0:
        return torch.empty(0, dtype=dtype, device=device)
    return torch.as_tensor(_CudaView(ptr, (n,), typestr, owner), device=device)


class Handle:
    _destroy = None

    def __init__(self, ptr, ctx, keep=()):
        self.ptr = ptr
        self.ctx = ctx
        self._keep = list(keep)

    def destroy(self):
        if self.ptr is not None and self._destroy and _lib is not None:
            getattr(_lib, self._destroy)(self.ptr)
        self.ptr = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


class Ctx(Handle):
    _destroy = "fe_ctx_destroy"

    def __init__(self, ptr, device, stream, alloc_cbs):
        super().__init__(ptr, None)
        self.device = device
        self.stream = stream
        self._alloc_cbs = alloc_cbs


class Set(Handle):
    _destroy = "fe_set_destroy"


class Map(Handle):
    _destroy = "fe_map_destroy"


class Dat(Handle):
    _destroy = "fe_dat_destroy"


class Sparsity(Handle):
    _destroy = "fe_sparsity_destroy"


class Mat(Handle):
    _destroy = "fe_mat_destroy"


class Kernel(Handle):
    _destroy = "fe_kernel_destroy"


class Global(Handle):
    _destroy = "fe_global_destroy"


class Batch(Handle):
    _destroy = "fe_batch_destroy"


class Cg(Handle):
    _destroy = "fe_cg_destroy"


class Server(Handle):
    _destroy = "fe_server_destroy"


def _torch_alloc(nbytes, user):
    try:
        return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device())
    except Exception:
        return None


def _torch_free(ptr, user):
    try:
        torch.cuda.caching_allocator_delete(int(ptr))
    except Exception:
        pass


# ----------------------------------------------------------------------------------- C entry points

def ctx_create(device: int = 0, stream=None, torch_allocator: bool = True, checks: bool = False) -> Ctx:
    """fe_ctx_create (+ fe_ctx_set_allocator with torch's caching allocator, fe_ctx_set_checks)."""
    lib = load()
    if not torch.cuda.is_available():
        raise RuntimeError("libfe needs a CUDA device; there is no CPU fallback")
    if stream is None:
        stream = torch.cuda.current_stream(device)
    out = C.c_void_p()
    _check(lib.fe_ctx_create(device, C.c_void_p(stream.cuda_stream), C.byref(out)))
    cbs = None
    if torch_allocator:
        cbs = (ALLOC_FN(_torch_alloc), FREE_FN(_torch_free))
        _check(lib.fe_ctx_set_allocator(out, cbs[0], cbs[1], None))
    if checks:
        _check(lib.fe_ctx_set_checks(out, 1))
    return Ctx(out, device, stream, cbs)


def ctx_set_stream(ctx: Ctx, stream) -> None:
    _check(load().fe_ctx_set_stream(ctx.ptr, C.c_void_p(stream.cuda_stream)))
    ctx.stream = stream


def ctx_set_checks(ctx: Ctx, checks: bool) -> None:
    _check(load().fe_ctx_set_checks(ctx.ptr, int(bool(checks))))


def sync(ctx: Ctx) -> None:
    """fe_sync: waits for the stream and raises on device-side errors (FE_ERANGE ...)."""
    _check(load().fe_sync(ctx.ptr))


def set_create(ctx: Ctx, size: int) -> Set:
    out = C.c_void_p()
    _check(load().fe_set_create(ctx.ptr, int(size), C.byref(out)))
    return Set(out, ctx)


def set_size(s: Set) -> int:
    v = C.c_int64()
    _check(load().fe_set_size(s.ptr, C.byref(v)))
    return v.value


def _dev_tensor(t, dtype, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous CUDA tensor of dtype {dtype}")
    return t


def map_create(ctx: Ctx, frm: Set, to: Set, values: torch.Tensor, validate: bool = False) -> Map:
    """fe_map_create: values is a device int32 tensor [frm.size, arity] (borrowed)."""
    values = _dev_tensor(values, torch.int32, "map values")
    arity = values.shape[1] if values.dim() == 2 else 1
    out = C.c_void_p()
    _check(load().fe_map_create(ctx.ptr, frm.ptr, to.ptr, int(arity), C.c_void_p(values.data_ptr()),
                                int(bool(validate)), C.byref(out)))
    m = Map(out, ctx, keep=(values, frm, to))
    m.arity = arity
    return m


def dat_create(ctx: Ctx, s: Set, data: torch.Tensor) -> Dat:
    """fe_dat_create: data is a device float64 tensor [s.size] or [s.size, dim] (borrowed)."""
    data = _dev_tensor(data, torch.float64, "dat data")
    dim = data.shape[1] if data.dim() == 2 else 1
    out = C.c_void_p()
    _check(load().fe_dat_create(ctx.ptr, s.ptr, int(dim), C.c_void_p(data.data_ptr()), C.byref(out)))
    d = Dat(out, ctx, keep=(data, s))
    d.data = data
    return d


def sparsity_build(ctx: Ctx, rmap: Map, cmap: Map) -> Sparsity:
    out = C.c_void_p()
    _check(load().fe_sparsity_build(ctx.ptr, rmap.ptr, cmap.ptr, C.byref(out)))
    return Sparsity(out, ctx, keep=(rmap, cmap))


def sparsity_rebuild(sp: Sparsity) -> None:
    _check(load().fe_sparsity_rebuild(sp.ptr))


def sparsity_changed(sp: Sparsity) -> torch.Tensor:
    """fe_sparsity_changed: a device view of the two flags of the last rebuild (int32 [2]: a row
    changed length; a row's columns changed, or columns are not tracked)."""
    p = C.c_void_p()
    _check(load().fe_sparsity_changed(sp.ptr, C.byref(p)))
    return _view(p.value, 2, torch.int32, sp, torch.device("cuda", sp.ctx.device))


def sparsity_track_columns(sp: Sparsity, on: bool = True) -> None:
    """fe_sparsity_track_columns: rebuilds compare the columns they write in place (exact flags[1])."""
    _check(load().fe_sparsity_track_columns(sp.ptr, int(bool(on))))


def sparsity_build_noalloc(rmap: torch.Tensor, cmap: torch.Tensor, nrows: int, ncols: int, rowptr: torch.Tensor,
                           colidx: torch.Tensor | None, lut: torch.Tensor, stream=None) -> int:
    """fe_sparsity_build_noalloc: pattern and lookup table into caller buffers, no device allocation.

    For callers that must not allocate device memory; scratch is a static device array with fixed
    size limits (see include/fe.h).  colidx None = size query.  Returns nnz.
    """
    rmap = _dev_tensor(rmap, torch.int32, "rmap")
    cmap = _dev_tensor(cmap, torch.int32, "cmap")
    rowptr = _dev_tensor(rowptr, torch.int64, "rowptr")
    lut = _dev_tensor(lut, torch.uint8, "lut")
    # the C entry point sees raw pointers only: every buffer's extent is checked here
    if rmap.dim() != 2 or cmap.dim() != 2 or rmap.shape[0] != cmap.shape[0]:
        raise ValueError(f"rmap and cmap must be [ncell][arity] with equal ncell, got {tuple(rmap.shape)} "
                         f"and {tuple(cmap.shape)}")
    if rowptr.numel() < int(nrows) + 1:
        raise ValueError(f"rowptr holds {rowptr.numel()} entries, needs nrows + 1 = {int(nrows) + 1}")
    need = rmap.shape[0] * rmap.shape[1] * cmap.shape[1]
    if lut.numel() < need:
        raise ValueError(f"lut holds {lut.numel()} bytes, needs ncell * arity_r * arity_c = {need}")
    cap = 0
    cptr = None
    if colidx is not None:
        colidx = _dev_tensor(colidx, torch.int32, "colidx")
        cap, cptr = colidx.numel(), C.c_void_p(colidx.data_ptr())
    if stream is None:
        stream = torch.cuda.current_stream()
    nnz = C.c_int64(0)
    ncell = rmap.shape[0]
    _check(load().fe_sparsity_build_noalloc(C.c_void_p(rmap.data_ptr()), int(rmap.shape[1]), C.c_void_p(cmap.data_ptr()),
                                            int(cmap.shape[1]), int(ncell), int(nrows), int(ncols),
                                            C.c_void_p(rowptr.data_ptr()), cptr, int(cap), C.c_void_p(lut.data_ptr()),
                                            C.byref(nnz), C.c_void_p(stream.cuda_stream)))
    return nnz.value


def sparsity_csr(sp: Sparsity):
    """(nrows, ncols, nnz, rowptr view int64 [nrows+1], colidx view int32 [nnz]) -- zero-copy views."""
    nr, nc, nnz = C.c_int64(), C.c_int64(), C.c_int64()
    rp, ci = C.c_void_p(), C.c_void_p()
    _check(load().fe_sparsity_csr(sp.ptr, C.byref(nr), C.byref(nc), C.byref(nnz), C.byref(rp), C.byref(ci)))
    dev = torch.device("cuda", sp.ctx.device)
    return (nr.value, nc.value, nnz.value, _view(rp.value, nr.value + 1, torch.int64, sp, dev),
            _view(ci.value, nnz.value, torch.int32, sp, dev))


def sparsity_lut(sp: Sparsity, ncell: int, ndr: int, ndc: int) -> torch.Tensor:
    p = C.c_void_p()
    _check(load().fe_sparsity_lut(sp.ptr, C.byref(p)))
    return _view(p.value, ncell * ndr * ndc, torch.uint8, sp, torch.device("cuda", sp.ctx.device))


def mat_create(ctx: Ctx, sp: Sparsity) -> Mat:
    out = C.c_void_p()
    _check(load().fe_mat_create(ctx.ptr, sp.ptr, C.byref(out)))
    return Mat(out, ctx, keep=(sp,))


def mat_values(A: Mat) -> torch.Tensor:
    p = C.c_void_p()
    _check(load().fe_mat_values(A.ptr, C.byref(p)))
    nnz = sparsity_csr(A._keep[0])[2]
    return _view(p.value, nnz, torch.float64, A, torch.device("cuda", A.ctx.device))


def mat_zero(A: Mat) -> None:
    _check(load().fe_mat_zero(A.ptr))


def kernel_create(ctx: Ctx, form: int, dim: int, degree: int, coeff_degree: int = 1,
                  precision: int = PREC_FP64, strategy: int = STRATEGY_AUTO) -> Kernel:
    d = fe_form_desc(form, dim, degree, coeff_degree, precision, strategy)
    out = C.c_void_p()
    _check(load().fe_kernel_create(ctx.ptr, C.byref(d), C.byref(out)))
    k = Kernel(out, ctx)
    k.nd = (degree + 1) * (degree + 2) // 2 if dim == 2 else (degree + 1) * (degree + 2) * (degree + 3) // 6
    return k


def _args(coeffs):
    coeffs = list(coeffs or [])
    arr = (fe_arg * max(1, len(coeffs)))()
    for i, (d, m) in enumerate(coeffs):
        arr[i].dat, arr[i].map = d.ptr, m.ptr
    return arr, len(coeffs)


def assemble_mat(ctx: Ctx, k: Kernel, cells: Set, A: Mat, coords: Dat, coord_map: Map,
                 coeffs=(), zero_first: bool = True) -> None:
    """fe_assemble_mat: A(INC) over cells; coeffs = [(Dat, Map), ...] READ."""
    arr, n = _args(coeffs)
    _check(load().fe_assemble_mat(ctx.ptr, k.ptr, cells.ptr, A.ptr, int(bool(zero_first)), coords.ptr,
                                  coord_map.ptr, arr, n))


def assemble_vec(ctx: Ctx, k: Kernel, cells: Set, b: Dat, test_map: Map, coords: Dat, coord_map: Map,
                 coeffs=(), zero_first: bool = True, sp: Sparsity | None = None) -> None:
    arr, n = _args(coeffs)
    _check(load().fe_assemble_vec(ctx.ptr, k.ptr, cells.ptr, b.ptr, test_map.ptr, int(bool(zero_first)),
                                  coords.ptr, coord_map.ptr, arr, n, sp.ptr if sp is not None else None))


def action(ctx: Ctx, k: Kernel, cells: Set, x: Dat, y: Dat, map_: Map, coords: Dat, coord_map: Map,
           coeffs=(), zero_first: bool = True, sp: Sparsity | None = None) -> None:
    arr, n = _args(coeffs)
    _check(load().fe_action(ctx.ptr, k.ptr, cells.ptr, x.ptr, y.ptr, map_.ptr, int(bool(zero_first)),
                            coords.ptr, coord_map.ptr, arr, n, sp.ptr if sp is not None else None))


def assemble_mat_action(ctx: Ctx, k: Kernel, cells: Set, A: Mat, x: Dat, y: Dat, map_: Map, coords: Dat,
                        coord_map: Map, coeffs=(), zero_first: bool = True) -> None:
    """fe_assemble_mat_action: A(INC) += K_e and y(INC) += K_e x_e in one pass over the cells."""
    arr, n = _args(coeffs)
    _check(load().fe_assemble_mat_action(ctx.ptr, k.ptr, cells.ptr, A.ptr, x.ptr, y.ptr, map_.ptr,
                                         int(bool(zero_first)), coords.ptr, coord_map.ptr, arr, n))


def global_create(ctx: Ctx, dim: int = 1) -> Global:
    """fe_global_create: dim FP64 values on the device, zeroed."""
    out = C.c_void_p()
    _check(load().fe_global_create(ctx.ptr, int(dim), C.byref(out)))
    g = Global(out, ctx)
    g.dim = int(dim)
    return g


def global_values(g: Global) -> torch.Tensor:
    """A device view of the Global's values (read after sync)."""
    p = C.c_void_p()
    _check(load().fe_global_data(g.ptr, C.byref(p)))
    return _view(p.value, g.dim, torch.float64, g, torch.device("cuda", g.ctx.device))


def assemble_global(ctx: Ctx, k: Kernel, cells: Set, g: Global, x: Dat, map_: Map, coords: Dat, coord_map: Map,
                    coeffs=(), zero_first: bool = True) -> None:
    """fe_assemble_global: g[0] (+)= a(x, x) for a bilinear kernel, or L(x) for a linear one (SUM)."""
    arr, n = _args(coeffs)
    _check(load().fe_assemble_global(ctx.ptr, k.ptr, cells.ptr, g.ptr, int(bool(zero_first)), x.ptr, map_.ptr,
                                     coords.ptr, coord_map.ptr, arr, n))


def reduce_cell_volume(ctx: Ctx, cells: Set, g: Global, op: int, coords: Dat, coord_map: Map,
                       zero_first: bool = True) -> None:
    """fe_reduce_cell_volume: g[0] (op)= SUM, MIN or MAX over the cells of their volumes."""
    _check(load().fe_reduce_cell_volume(ctx.ptr, cells.ptr, g.ptr, int(op), int(bool(zero_first)), coords.ptr,
                                        coord_map.ptr))


def _stored_tensor(Ke, k: Kernel, cells: Set):
    Ke = _dev_tensor(Ke, torch.float64, "Ke")
    nup, ncell = k.nd * (k.nd + 1) // 2, set_size(cells)
    if Ke.numel() != nup * ncell:
        raise ValueError(f"Ke must hold nd(nd+1)/2 * ncell = {nup} * {ncell} values")
    return Ke


def elem_matrices(ctx: Ctx, k: Kernel, cells: Set, Ke: torch.Tensor, coords: Dat, coord_map: Map, coeffs=()) -> None:
    """fe_elem_matrices: each cell's element matrix, upper triangle in FP64, entry-major (Ke[u, e])."""
    Ke = _stored_tensor(Ke, k, cells)
    arr, n = _args(coeffs)
    _check(load().fe_elem_matrices(ctx.ptr, k.ptr, cells.ptr, C.c_void_p(Ke.data_ptr()), coords.ptr, coord_map.ptr,
                                   arr, n))


def action_stored(ctx: Ctx, k: Kernel, cells: Set, Ke: torch.Tensor, x: Dat, y: Dat, map_: Map,
                  zero_first: bool = True) -> None:
    """fe_action_stored: y(INC) += K_e x_e cell by cell from matrices stored by elem_matrices."""
    Ke = _stored_tensor(Ke, k, cells)
    _check(load().fe_action_stored(ctx.ptr, k.ptr, cells.ptr, C.c_void_p(Ke.data_ptr()), x.ptr, y.ptr, map_.ptr,
                                   int(bool(zero_first))))


def batch_create(ctx: Ctx, items) -> Batch:
    """fe_batch_create: items = [dict(kmat=, kvec=None, cells=, sp=, coords=, coord_map=, f=(Dat, Map) or None)]."""
    arr = (fe_batch_item * max(1, len(items)))()
    keep = []
    for i, it in enumerate(items):
        f = it.get("f")
        arr[i].kmat = it["kmat"].ptr
        arr[i].kvec = it["kvec"].ptr if it.get("kvec") is not None else None
        arr[i].cells, arr[i].sp = it["cells"].ptr, it["sp"].ptr
        arr[i].coords, arr[i].coord_map = it["coords"].ptr, it["coord_map"].ptr
        if f is not None:
            arr[i].f.dat, arr[i].f.map = f[0].ptr, f[1].ptr
        keep.append(it)
    out = C.c_void_p()
    _check(load().fe_batch_create(ctx.ptr, len(items), arr, C.byref(out)))
    return Batch(out, ctx, keep=(keep,))


def batch_values(b: Batch, item: int):
    """(values view [nnz] float64, rhs view [nrows] float64) of one item."""
    v, r = C.c_void_p(), C.c_void_p()
    nnz, nr = C.c_int64(), C.c_int64()
    _check(load().fe_batch_values(b.ptr, int(item), C.byref(v), C.byref(nnz), C.byref(r), C.byref(nr)))
    dev = torch.device("cuda", b.ctx.device)
    return _view(v.value, nnz.value, torch.float64, b, dev), _view(r.value, nr.value, torch.float64, b, dev)


def batch_tune(b: Batch, reps: int = 3):
    t, g, ms = C.c_int(), C.c_int(), C.c_float()
    _check(load().fe_batch_tune(b.ptr, int(reps), C.byref(t), C.byref(g), C.byref(ms)))
    return t.value, g.value, ms.value


def batch_assemble(b: Batch, use_graph: bool = True) -> None:
    _check(load().fe_batch_assemble(b.ptr, int(bool(use_graph))))


def batch_buffers(b: Batch):
    """(all CSR values, all right-hand sides) of the batch as two flat views, items back to back."""
    lib, n = load(), len(b._keep[0]) if b._keep else 0
    dev = torch.device("cuda", b.ctx.device)
    if n == 0:
        return torch.empty(0, dtype=torch.float64, device=dev), torch.empty(0, dtype=torch.float64, device=dev)
    v0, r0, vl, rl = C.c_void_p(), C.c_void_p(), C.c_void_p(), C.c_void_p()
    nnz, nr = C.c_int64(), C.c_int64()
    _check(lib.fe_batch_values(b.ptr, 0, C.byref(v0), None, C.byref(r0), None))
    _check(lib.fe_batch_values(b.ptr, n - 1, C.byref(vl), C.byref(nnz), C.byref(rl), C.byref(nr)))
    nv = (vl.value - v0.value) // 8 + nnz.value
    nrr = (rl.value - r0.value) // 8 + nr.value
    return _view(v0.value, nv, torch.float64, b, dev), _view(r0.value, nrr, torch.float64, b, dev)


# ----------------------------------------------------------------------------------- boundary conditions, CG

def dirichlet_apply(ctx: Ctx, A: Mat, b: Dat, is_bc: torch.Tensor, g: torch.Tensor | None = None) -> None:
    """fe_dirichlet_apply: is_bc device uint8 [nrows]; g device float64 [nrows] or None (g = 0)."""
    is_bc = _dev_tensor(is_bc, torch.uint8, "is_bc")
    gp = None if g is None else _dev_tensor(g, torch.float64, "g").data_ptr()
    _check(load().fe_dirichlet_apply(ctx.ptr, A.ptr, b.ptr, is_bc.data_ptr(), gp))


def cg_create(ctx: Ctx, max_systems: int) -> Cg:
    out = C.c_void_p()
    _check(load().fe_cg_create(ctx.ptr, int(max_systems), C.byref(out)))
    return Cg(out, ctx)


def cg_add(cg: Cg, A: Mat, b: Dat, x: Dat, rtol: float = 1e-8, maxit: int = 100000) -> int:
    slot = C.c_int()
    _check(load().fe_cg_add(cg.ptr, A.ptr, b.ptr, x.ptr, float(rtol), int(maxit), C.byref(slot)))
    cg._keep.append((A, b, x))
    return slot.value


def cg_iterate(cg: Cg, iters: int, use_graph: bool = True) -> None:
    _check(load().fe_cg_iterate(cg.ptr, int(iters), int(bool(use_graph))))


def cg_poll(cg: Cg, nslots: int):
    """(status, iterations, ||r||, ||b||) arrays over slots 0..nslots-1 (synchronises)."""
    st, it = np.zeros(nslots, np.int32), np.zeros(nslots, np.int32)
    rn, bn = np.zeros(nslots), np.zeros(nslots)
    _check(load().fe_cg_poll(cg.ptr, int(nslots), st.ctypes.data, it.ctypes.data, rn.ctypes.data, bn.ctypes.data))
    return st, it, rn, bn


def cg_remove(cg: Cg, slot: int) -> None:
    _check(load().fe_cg_remove(cg.ptr, int(slot)))


# ----------------------------------------------------------------------------------- serving

def server_create(ctx: Ctx, hbm_budget: int, max_active: int = 64, iters_per_tick: int = 16, rtol: float = 1e-8,
                  maxit: int = 100000, precision: int = PREC_FP64) -> Server:
    cfg = fe_server_config(int(hbm_budget), int(max_active), int(iters_per_tick), float(rtol), int(maxit),
                           int(precision))
    out = C.c_void_p()
    _check(load().fe_server_create(ctx.ptr, C.byref(cfg), C.byref(out)))
    return Server(out, ctx, keep=([],))


def server_submit(srv: Server, degree: int, cell_node, cell_vertex, coords, f, is_bc, x_out, arrival_s: float,
                  mesh_key: int = 0) -> int:
    """Queue one Poisson solve; the host arrays are kept alive by the server handle until it is destroyed.
    Requests with the same non-zero mesh_key must be on the same mesh; they share its device copy and
    sparsity."""
    arrs = [np.ascontiguousarray(cell_node, np.int32), np.ascontiguousarray(cell_vertex, np.int32),
            np.ascontiguousarray(coords, np.float64), np.ascontiguousarray(f, np.float64),
            np.ascontiguousarray(is_bc, np.uint8)]
    if not (isinstance(x_out, np.ndarray) and x_out.dtype == np.float64 and x_out.flags.c_contiguous):
        raise TypeError("x_out must be a C-contiguous float64 numpy array")
    if x_out.size != arrs[3].size:
        raise ValueError("x_out must hold one value per node")
    req = fe_solve_request(int(degree), arrs[0].shape[0], arrs[3].size, arrs[2].shape[0], arrs[0].ctypes.data,
                           arrs[1].ctypes.data, arrs[2].ctypes.data, arrs[3].ctypes.data, arrs[4].ctypes.data,
                           x_out.ctypes.data, float(arrival_s), int(mesh_key))
    rid = C.c_int64()
    _check(load().fe_server_submit(srv.ptr, C.byref(req), C.byref(rid)))
    srv._keep[0].append((arrs, x_out))
    return rid.value


def server_run(srv: Server) -> None:
    _check(load().fe_server_run(srv.ptr))


def server_result(srv: Server, rid: int) -> dict:
    r = fe_solve_result()
    _check(load().fe_server_result(srv.ptr, int(rid), C.byref(r)))
    return {k: getattr(r, k) for k, _ in fe_solve_result._fields_}


def server_stats(srv: Server) -> dict:
    r = fe_server_stats()
    _check(load().fe_server_stats_get(srv.ptr, C.byref(r)))
    return {k: getattr(r, k) for k, _ in fe_server_stats._fields_}


def wave_steps(ctx: Ctx, k: Kernel, cells: Set, phi: Dat, p: Dat, mass: torch.Tensor, is_bc, map_: Map,
               coords: Dat, coord_map: Map, sp: Sparsity, t0: float, dt: float, nsteps: int) -> None:
    """fe_wave_steps: mass device float64 [nrows]; is_bc device uint8 [nrows] or None."""
    mass = _dev_tensor(mass, torch.float64, "mass")
    bc = None if is_bc is None else _dev_tensor(is_bc, torch.uint8, "is_bc").data_ptr()
    _check(load().fe_wave_steps(ctx.ptr, k.ptr, cells.ptr, phi.ptr, p.ptr, mass.data_ptr(), bc, map_.ptr,
                                coords.ptr, coord_map.ptr, sp.ptr, float(t0), float(dt), int(nsteps)))
