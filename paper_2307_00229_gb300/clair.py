"""Thin Python binding of ``libclair.so`` (the C ABI in include/clair.h).

Argument marshalling only: every function has the name of the C entry point it calls,
takes torch CUDA tensors where the C call takes device pointers, and raises ``ClairError``
when the call returns a non-zero status.  No computation happens here; when the library
is missing the import of this module fails loudly (there is no fallback path).
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import _build

_lib = None

CLAIR_OK = 0
CLAIR_ERR_ARG = 1
CLAIR_ERR_CUDA = 2
CLAIR_ERR_SINGULAR_BLOCK = 3
CLAIR_ERR_NONFINITE = 4
CLAIR_ERR_NOT_CONVERGED = 5
CLAIR_ERR_CAPACITY = 6
CLAIR_ERR_UNSUPPORTED = 7
CLAIR_COARSEN_FC = 0
CLAIR_COARSEN_AGG = 1
CLAIR_FP64 = 0
CLAIR_MIXED = 1
CLAIR_INVERSE_EXACT = 0
CLAIR_INVERSE_DIAG = 1
CLAIR_KRYLOV_FGMRES = 0
CLAIR_KRYLOV_PCG = 1
CLAIR_KMAX = 4


class ClairError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"clair status {status}: {msg}")
        self.status = status


class clair_params(ctypes.Structure):
    _fields_ = [
        ("theta_coarsen", ctypes.c_double),
        ("theta_interp", ctypes.c_double),
        ("degree", ctypes.c_int),
        ("coarsen", ctypes.c_int),
        ("b_smooth_iters", ctypes.c_int),
        ("arnoldi_iters", ctypes.c_int),
        ("post_weighted", ctypes.c_int),
        ("coarse_max", ctypes.c_int),
        ("max_levels", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("gmres_restart", ctypes.c_int),
        ("gmres_maxit", ctypes.c_int),
        ("rtol", ctypes.c_double),
        ("seed", ctypes.c_uint64),
        ("inverse", ctypes.c_int),
        ("iterations", ctypes.c_int),
        ("symmetric", ctypes.c_int),
        ("krylov", ctypes.c_int),
    ]


class clair_stats_t(ctypes.Structure):
    _fields_ = [
        ("levels", ctypes.c_int),
        ("n", ctypes.c_int64 * 32),
        ("nnz", ctypes.c_int64 * 32),
        ("nnz_R", ctypes.c_int64 * 32),
        ("nnz_P", ctypes.c_int64 * 32),
        ("omega", ctypes.c_double * 32),
        ("operator_complexity", ctypes.c_double),
        ("r_rows", ctypes.c_int64),
        ("p_cols", ctypes.c_int64),
        ("t_hist", ctypes.c_int64 * 9),
        ("singular_blocks", ctypes.c_int64),
        ("empty_constraints", ctypes.c_int64),
        ("setup_ms", ctypes.c_double),
        ("phase_ms", ctypes.c_double * 10),
        ("solve_phase_ms", ctypes.c_double * 10),
        ("lsolve_flops", ctypes.c_double),
        ("lsolve_min_bytes", ctypes.c_double),
        ("lsolve_gathered", ctypes.c_int64),
        ("fp64_cycle_from", ctypes.c_int64),
        ("k", ctypes.c_int),
        ("lsolve_kind_b1", ctypes.c_int),
        ("lsolve_kind_b3", ctypes.c_int),
        ("lsolve_blocks_per_sm", ctypes.c_int),
        ("lsolve_tuned", ctypes.c_int),
        ("cycle_short_lanes", ctypes.c_int),
        ("cycle64_from", ctypes.c_int),
        ("level_span_ms", ctypes.c_double * 32),
        ("level_phase_ms", (ctypes.c_double * 8) * 32),
    ]


PHASES = ["split", "weight", "smooth", "pattern", "local_solve", "projection", "galerkin",
          "coarse", "vcycle", "krylov"]


_P = ctypes.c_void_p
_I = ctypes.c_int
_PI = ctypes.POINTER(ctypes.c_int)
_PD = ctypes.POINTER(ctypes.c_double)
_PI64 = ctypes.POINTER(ctypes.c_int64)

_SIGNATURES = {
    "clair_params_default": (_I, [ctypes.POINTER(clair_params)]),
    "clair_setup": (_I, [_I, _I, _P, _P, _P, _I, _P, _P, ctypes.POINTER(clair_params), _P,
                         ctypes.POINTER(_P)]),
    "clair_solve": (_I, [_P, _P, _P, _I, _P, _PI, _PD]),
    "clair_solve_detail": (_I, [_P, _PI, _PI, _PD]),
    "clair_vcycle": (_I, [_P, _I, _P, _P, _P]),
    "clair_stats": (_I, [_P, ctypes.POINTER(clair_stats_t)]),
    "clair_level_view": (_I, [_P, _I, _PI, _PI, _PI, ctypes.POINTER(_P), ctypes.POINTER(_P),
                              ctypes.POINTER(_P), _PI, ctypes.POINTER(_P), ctypes.POINTER(_P),
                              ctypes.POINTER(_P), _PI, ctypes.POINTER(_P), ctypes.POINTER(_P),
                              ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_P),
                              ctypes.POINTER(_P), _PD]),
    "clair_free": (_I, [_P]),
    "clair_local_weights": (_I, [_I, _P, _P, _P, _P, _I, _P, _P, _P, _I, _P, _P, _PI64, _PI64]),
    "clair_local_weights_noalloc": (_I, [_I, _P, _P, _P, _P, _I, _P, _P, _P, _I, _P, _P, _PI64,
                                         _PI64]),
    "clair_setup_batched": (_I, [_I, _P, _I, _I, _P, _P, _P, _I, _P, _P,
                                 ctypes.POINTER(clair_params), _P, ctypes.POINTER(_P)]),
    "clair_batch_view": (_I, [_P, _I, _PI, _P, _P, _P]),
    "clair_setup_adjoint": (_I, [_P, _P, ctypes.POINTER(_P)]),
    "clair_sddmm_grad": (_I, [_I, _I, _P, _P, _I, _P, _P, _P, _P]),
    "clair_advdiff2d_param_grad": (_I, [_I, ctypes.c_double, _P, _P, _P, _P, _P, _I, _P, _P, _P,
                                        _P, _P]),
    "clair_last_error": (ctypes.c_char_p, []),
    "clair_kernel_launches": (ctypes.c_int64, []),
    "clair_compiled_arch": (ctypes.c_int, []),
    "clair_spgemm": (_I, [_I, _I, _I, _P, _P, _P, _P, _P, _P, _P, _P, _PI64, ctypes.c_int64, _P, _P]),
    "clair_lsolve_config": (_I, [_I, _I, _PI, _PI, _PI, _PI]),
}


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Loads ``libclair.so`` (building it in-tree first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError(f"CUDA library not found at {_build.LIB}; run __graft_entry__.build()")
    lib = ctypes.CDLL(_build.LIB)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status: int):
    if status != CLAIR_OK:
        raise ClairError(status, clair_last_error())


def _dptr(t: torch.Tensor, dtype: torch.dtype) -> ctypes.c_void_p:
    if not (t.is_cuda and t.is_contiguous() and t.dtype == dtype):
        raise TypeError(f"expected a contiguous CUDA {dtype} tensor, got {t.dtype} on {t.device}")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def clair_last_error() -> str:
    return load().clair_last_error().decode()


def clair_kernel_launches() -> int:
    return int(load().clair_kernel_launches())


def clair_compiled_arch() -> int:
    return int(load().clair_compiled_arch())


def clair_lsolve_config(precision: int, kind_b1: int | None = None, kind_b3: int = 3,
                        blocks_per_sm: int = 0, tuned: int = 2) -> dict:
    """Reads, or with ``kind_b1`` set installs, the persistent local-solve configuration
    of the current device for one precision."""
    k, k3 = ctypes.c_int(kind_b1 or 0), ctypes.c_int(kind_b3)
    b, t = ctypes.c_int(blocks_per_sm), ctypes.c_int(tuned)
    _check(load().clair_lsolve_config(precision, 0 if kind_b1 is None else 1, ctypes.byref(k),
                                      ctypes.byref(k3), ctypes.byref(b), ctypes.byref(t)))
    return {"kind_b1": k.value, "kind_b3": k3.value, "blocks_per_sm": b.value, "tuned": t.value}


def clair_spgemm(A_rowptr, A_col, A_val, B_rowptr, B_col, B_val, ncols: int, stream=None):
    """C = A B on the device; returns (rowptr, col, val) torch tensors."""
    m, kdim = A_rowptr.numel() - 1, B_rowptr.numel() - 1
    rp = torch.empty(m + 1, dtype=torch.int32, device=A_rowptr.device)
    nnz = ctypes.c_int64()
    args = [m, kdim, ncols, _dptr(A_rowptr, torch.int32), _dptr(A_col, torch.int32),
            _dptr(A_val, torch.float64), _dptr(B_rowptr, torch.int32), _dptr(B_col, torch.int32),
            _dptr(B_val, torch.float64), _stream(stream), _dptr(rp, torch.int32), ctypes.byref(nnz)]
    _check(load().clair_spgemm(*args, 0, None, None))
    col = torch.empty(max(nnz.value, 1), dtype=torch.int32, device=A_rowptr.device)
    val = torch.empty(max(nnz.value, 1), dtype=torch.float64, device=A_rowptr.device)
    _check(load().clair_spgemm(*args, nnz.value, _dptr(col, torch.int32), _dptr(val, torch.float64)))
    return rp, col[:nnz.value], val[:nnz.value]


def clair_params_default() -> clair_params:
    p = clair_params()
    _check(load().clair_params_default(ctypes.byref(p)))
    return p


def _modes(B, n: int) -> tuple[int, ctypes.c_void_p]:
    """B as (n,) for one mode or (k, n) for k modes (row a = mode a: the column-major n x k
    array the C call takes)."""
    if B.dim() == 1:
        if B.numel() != n:
            raise ValueError("B must have n entries")
        return 1, _dptr(B, torch.float64)
    if B.dim() != 2 or B.shape[1] != n:
        raise ValueError("B must be (n,) or (k, n)")
    return B.shape[0], _dptr(B, torch.float64)


def _cf(cf_marker):
    return None if cf_marker is None else _dptr(cf_marker, torch.int8)


def clair_setup(rowptr, col, val, B, params: clair_params | None = None, stream=None,
                cf_marker=None) -> ctypes.c_void_p:
    """Hierarchy of A (device CSR).  ``B``: (n,) or (k, n) mode vectors; ``cf_marker``:
    optional int8 (n,) fine-level splitting (1 = C)."""
    n = rowptr.numel() - 1
    k, bp = _modes(B, n)
    h = ctypes.c_void_p()
    _check(load().clair_setup(n, col.numel(), _dptr(rowptr, torch.int32), _dptr(col, torch.int32),
                              _dptr(val, torch.float64), k, bp, _cf(cf_marker),
                              ctypes.byref(params) if params is not None else None,
                              _stream(stream), ctypes.byref(h)))
    return h


def clair_setup_batched(offsets, rowptr, col, val, B, params: clair_params | None = None,
                        stream=None, cf_marker=None) -> ctypes.c_void_p:
    """Setup of a batch: block-diagonal CSR, instance i owning rows offsets[i]..offsets[i+1]-1."""
    off = (ctypes.c_int * len(offsets))(*[int(x) for x in offsets])
    n = rowptr.numel() - 1
    k, bp = _modes(B, n)
    h = ctypes.c_void_p()
    _check(load().clair_setup_batched(len(offsets) - 1, off, n, col.numel(), _dptr(rowptr, torch.int32),
                                      _dptr(col, torch.int32), _dptr(val, torch.float64), k, bp,
                                      _cf(cf_marker),
                                      ctypes.byref(params) if params is not None else None,
                                      _stream(stream), ctypes.byref(h)))
    return h


def clair_batch_view(h, level: int) -> dict:
    """Per-instance row ranges, weights and frozen flags of level ``level`` (host lists)."""
    ninst = ctypes.c_int()
    _check(load().clair_batch_view(h, level, ctypes.byref(ninst), None, None, None))
    k = ninst.value
    off = (ctypes.c_int * (k + 1))()
    om = (ctypes.c_double * k)()
    fz = (ctypes.c_int8 * k)()
    _check(load().clair_batch_view(h, level, ctypes.byref(ninst), off, om, fz))
    return {"ninst": k, "offsets": list(off), "omega": list(om), "frozen": [int(x) for x in fz]}


def clair_solve(h, f, u, stream=None, raise_not_converged: bool = True):
    """Solves for one right-hand side (f, u of shape (n,)) or several (shape (nrhs, n)).

    Returns ``(status, iterations, relative residual)``: scalars for one right-hand side,
    lists (one entry per right-hand side) for several."""
    single = f.dim() == 1
    nrhs = 1 if single else f.shape[0]
    if u.shape != f.shape:
        raise ValueError("clair_solve: u and f must have the same shape")
    its = (ctypes.c_int * nrhs)()
    rel = (ctypes.c_double * nrhs)()
    st = load().clair_solve(h, _dptr(f, torch.float64), _dptr(u, torch.float64), nrhs, _stream(stream),
                            its, rel)
    if st != CLAIR_OK and (st != CLAIR_ERR_NOT_CONVERGED or raise_not_converged):
        _check(st)
    if single:
        return st, its[0], rel[0]
    return st, list(its), list(rel)


def clair_solve_detail(h) -> tuple[list, list]:
    """Iterations and relative residuals of every (right-hand side, instance) process of
    the last solve, index r * ninst + i."""
    nseg = ctypes.c_int()
    _check(load().clair_solve_detail(h, ctypes.byref(nseg), None, None))
    its = (ctypes.c_int * nseg.value)()
    rel = (ctypes.c_double * nseg.value)()
    _check(load().clair_solve_detail(h, ctypes.byref(nseg), its, rel))
    return list(its), list(rel)


def clair_vcycle(h, level: int, b, x, stream=None):
    _check(load().clair_vcycle(h, level, _dptr(b, torch.float64), _dptr(x, torch.float64),
                               _stream(stream)))


def clair_stats(h) -> clair_stats_t:
    s = clair_stats_t()
    _check(load().clair_stats(h, ctypes.byref(s)))
    return s


class _DeviceArray:
    """Zero-copy view of library-owned device memory through __cuda_array_interface__."""

    def __init__(self, ptr: int, count: int, typestr: str):
        self.__cuda_array_interface__ = {"shape": (count,), "typestr": typestr,
                                         "data": (ptr, False), "version": 3, "strides": None}


def _view(ptr: ctypes.c_void_p, count: int, dtype: torch.dtype):
    if not ptr.value or count <= 0:
        return torch.empty(0, dtype=dtype, device="cuda")
    ts = {torch.int32: "<i4", torch.float64: "<f8", torch.int8: "|i1"}[dtype]
    return torch.as_tensor(_DeviceArray(ptr.value, count, ts), device="cuda")


def clair_level_view(h, level: int) -> dict:
    """Zero-copy torch views of level ``level`` (valid until ``clair_free``)."""
    n, nc, nnzA, nnzR, nnzP = (ctypes.c_int() for _ in range(5))
    ptrs = [ctypes.c_void_p() for _ in range(12)]
    om = ctypes.c_double()
    _check(load().clair_level_view(
        h, level, ctypes.byref(n), ctypes.byref(nc), ctypes.byref(nnzA), *(ctypes.byref(p) for p in ptrs[:3]),
        ctypes.byref(nnzR), *(ctypes.byref(p) for p in ptrs[3:6]), ctypes.byref(nnzP),
        *(ctypes.byref(p) for p in ptrs[6:9]), *(ctypes.byref(p) for p in ptrs[9:12]), ctypes.byref(om)))
    N, NC = n.value, nc.value
    K = clair_stats(h).k
    out = {"n": N, "nc": NC, "omega": om.value, "k": K,
           "A_rowptr": _view(ptrs[0], N + 1, torch.int32), "A_col": _view(ptrs[1], nnzA.value, torch.int32),
           "A_val": _view(ptrs[2], nnzA.value, torch.float64)}
    if NC:
        out.update({
            "R_rowptr": _view(ptrs[3], NC + 1, torch.int32), "R_col": _view(ptrs[4], nnzR.value, torch.int32),
            "R_val": _view(ptrs[5], nnzR.value, torch.float64),
            "P_rowptr": _view(ptrs[6], N + 1, torch.int32), "P_col": _view(ptrs[7], nnzP.value, torch.int32),
            "P_val": _view(ptrs[8], nnzP.value, torch.float64),
            "cf": _view(ptrs[9], N, torch.int8),
            "B_P": _view(ptrs[10], N * K, torch.float64).view(K, N).squeeze(0),
            "B_R": _view(ptrs[11], N * K, torch.float64).view(K, N).squeeze(0)})
    return out


def clair_free(h):
    _check(load().clair_free(h))


def clair_local_weights(Ahat_rowptr, Ahat_col, Ahat_val, cf, nc: int, Z_rowptr, Z_col, B,
                        precision: int, Z_val, stream=None, raise_singular: bool = True):
    """Returns ``(status, singular blocks, skipped F-points)``."""
    sing, empty = ctypes.c_int64(0), ctypes.c_int64(0)
    n = Ahat_rowptr.numel() - 1
    st = load().clair_local_weights(
        n, _dptr(Ahat_rowptr, torch.int32), _dptr(Ahat_col, torch.int32), _dptr(Ahat_val, torch.float64),
        _dptr(cf, torch.int8), nc, _dptr(Z_rowptr, torch.int32), _dptr(Z_col, torch.int32),
        _dptr(B, torch.float64), precision, _dptr(Z_val, torch.float64), _stream(stream),
        ctypes.byref(sing), ctypes.byref(empty))
    if st != CLAIR_OK and (st != CLAIR_ERR_SINGULAR_BLOCK or raise_singular):
        _check(st)
    return st, sing.value, empty.value


def clair_local_weights_noalloc(Ahat_rowptr, Ahat_col, Ahat_val, cf, nc: int, Z_rowptr, Z_col, B,
                                precision: int, Z_val, stream=None, raise_singular: bool = True):
    """Same as ``clair_local_weights`` but the library allocates no device memory (its
    temporaries live in one fixed static device array).  Returns ``(status, singular
    blocks, skipped F-points)``."""
    sing, empty = ctypes.c_int64(0), ctypes.c_int64(0)
    n = Ahat_rowptr.numel() - 1
    st = load().clair_local_weights_noalloc(
        n, _dptr(Ahat_rowptr, torch.int32), _dptr(Ahat_col, torch.int32), _dptr(Ahat_val, torch.float64),
        _dptr(cf, torch.int8), nc, _dptr(Z_rowptr, torch.int32), _dptr(Z_col, torch.int32),
        _dptr(B, torch.float64), precision, _dptr(Z_val, torch.float64), _stream(stream),
        ctypes.byref(sing), ctypes.byref(empty))
    if st != CLAIR_OK and (st != CLAIR_ERR_SINGULAR_BLOCK or raise_singular):
        _check(st)
    return st, sing.value, empty.value


# ---- adjoint path -------------------------------------------------------------------------

def clair_setup_adjoint(h, stream=None) -> ctypes.c_void_p:
    """Hierarchy for A^T of the hierarchy ``h`` (same parameters and mode vector)."""
    adj = ctypes.c_void_p()
    _check(load().clair_setup_adjoint(h, _stream(stream), ctypes.byref(adj)))
    return adj


def clair_sddmm_grad(rowptr, col, lam, u, dA, stream=None):
    """``dA[e] = -sum_r lam[r, row(e)] u[r, col(e)]`` on A's pattern; lam, u: (nrhs, n)."""
    n = rowptr.numel() - 1
    if lam.shape != u.shape or lam.dim() != 2 or lam.shape[1] != n or dA.numel() != col.numel():
        raise ValueError("clair_sddmm_grad: lam and u must be (nrhs, n) and dA must be (nnz,)")
    _check(load().clair_sddmm_grad(n, col.numel(), _dptr(rowptr, torch.int32), _dptr(col, torch.int32),
                                   lam.shape[0], _dptr(lam, torch.float64), _dptr(u, torch.float64),
                                   _dptr(dA, torch.float64), _stream(stream)))


def clair_advdiff2d_param_grad(nside: int, h: float, eps, vx, vy, rowptr, col, dA, stream=None):
    """Chain rule of the 5-point upwind operator: returns ``(deps, dvx, dvy)`` per node."""
    deps, dvx, dvy = (torch.empty(nside * nside, dtype=torch.float64, device="cuda") for _ in range(3))
    _check(load().clair_advdiff2d_param_grad(
        nside, float(h), _dptr(eps, torch.float64), _dptr(vx, torch.float64), _dptr(vy, torch.float64),
        _dptr(rowptr, torch.int32), _dptr(col, torch.int32), col.numel(), _dptr(dA, torch.float64),
        _dptr(deps, torch.float64), _dptr(dvx, torch.float64), _dptr(dvy, torch.float64),
        _stream(stream)))
    return deps, dvx, dvy


class Hierarchy:
    """Owns a library hierarchy handle and frees it with the object."""

    def __init__(self, handle):
        self.handle = handle

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.clair_free(self.handle)
            self.handle = None


class ClairSolve(torch.autograd.Function):
    """``U[r] = A(val)^{-1} F[r]`` for every row of F with CLAIR-preconditioned FGMRES,
    differentiable in the values of A and in F.

    Backward builds the hierarchy of A^T (clair_setup_adjoint), solves
    ``A^T Lam[r] = dL/dU[r]`` and returns ``dL/dval = -sum_r Lam[r, row] U[r, col]``
    (clair_sddmm_grad) and ``dL/dF = Lam``.  Every step runs in the CUDA library; this
    class only moves pointers.

    Arguments: ``val`` (nnz,) float64; ``F`` (nrhs, n) float64; ``rowptr``/``col`` int32
    CSR pattern; ``B`` (n,) float64 mode vector; ``params`` a ``clair_params`` or None.
    """

    @staticmethod
    def forward(ctx, val, F, rowptr, col, B, params):
        F = F.detach().contiguous()
        fwd = Hierarchy(clair_setup(rowptr, col, val.detach().contiguous(), B, params))
        U = torch.zeros_like(F)
        clair_solve(fwd.handle, F, U)  # every right-hand side in one call
        ctx.fwd = fwd
        ctx.pattern = (rowptr, col)
        ctx.save_for_backward(U)
        return U

    @staticmethod
    def backward(ctx, gU):
        (U,) = ctx.saved_tensors
        rowptr, col = ctx.pattern
        adj = Hierarchy(clair_setup_adjoint(ctx.fwd.handle))
        gU = gU.detach().contiguous()
        Lam = torch.zeros_like(gU)
        clair_solve(adj.handle, gU, Lam)
        dval = torch.empty(col.numel(), dtype=torch.float64, device=U.device)
        clair_sddmm_grad(rowptr, col, Lam, U, dval)
        del adj
        return dval, Lam, None, None, None, None
