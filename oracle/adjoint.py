"""Plain float64 oracle of the adjoint gradient through the advection-diffusion solve.

TEST INFRASTRUCTURE ONLY (see the package docstring): the product path never imports it.

The paper solves A u = f; the gradient of a loss of the solutions with respect to the
operator follows from the implicit-function theorem and is not in the paper.  The
definitions written out here:

* loss ``L = sum_r ||u_r - t_r||_2^2`` with ``A u_r = f_r`` (r over the right-hand sides);
* adjoint ``A^T lam_r = dL/du_r = 2 (u_r - t_r)``;
* operator gradient on the stored entries of A:
  ``dL/da_ij = -sum_r lam_r[i] u_r[j]`` (differentiate ``A u_r = f_r``: ``A du = -dA u``);
* parameter gradient: the chain rule through the first-order upwind finite-difference
  discretization of the paper's advection-diffusion problem (Section 4.2, Eq. 4.1),
  i.e. the operator ``workloads.advdiff_2d`` assembles (per-node eps, harmonic-mean
  faces, per-node velocity).

The solves here are exact sparse LU factorizations (scipy's SuperLU), so the oracle is
independent of the AMG solver whose gradient it checks.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import workloads


def solve_exact(A, F: np.ndarray, transpose: bool = False) -> np.ndarray:
    """Rows of ``F`` (nrhs x n) solved with ``A`` (or ``A^T``) by sparse LU."""
    A = sp.csc_matrix(A.to_scipy() if hasattr(A, "to_scipy") else A)
    lu = spla.splu(A)
    F = np.atleast_2d(F)
    return np.stack([lu.solve(np.ascontiguousarray(f), trans="T" if transpose else "N") for f in F])


def loss(A, F: np.ndarray, T: np.ndarray) -> float:
    """``sum_r ||u_r - t_r||^2`` with ``u_r = A^{-1} f_r``."""
    U = solve_exact(A, F)
    return float(np.sum((U - np.atleast_2d(T)) ** 2))


def operator_gradient(A, U: np.ndarray, Lam: np.ndarray) -> np.ndarray:
    """``dL/da_e = -sum_r Lam[r, row(e)] U[r, col(e)]`` over the stored entries of A, in
    the CSR order of A (the outer product of adjoint and state sampled on the pattern)."""
    A = sp.csr_matrix(A.to_scipy() if hasattr(A, "to_scipy") else A)
    rows = np.repeat(np.arange(A.shape[0]), np.diff(A.indptr))
    Lam, U = np.atleast_2d(Lam), np.atleast_2d(U)
    return -np.einsum("re,re->e", Lam[:, rows], U[:, A.indices])


def adjoint_gradient(A, F: np.ndarray, T: np.ndarray):
    """State, adjoint and operator gradient of the loss, with exact solves.

    Returns ``(U, Lam, dA)``: ``U`` and ``Lam`` are nrhs x n, ``dA`` follows A's CSR order.
    """
    U = solve_exact(A, F)
    Lam = solve_exact(A, 2.0 * (U - np.atleast_2d(T)), transpose=True)
    return U, Lam, operator_gradient(A, U, Lam)


def advdiff2d_param_gradient(nside: int, eps: np.ndarray, vx: np.ndarray, vy: np.ndarray,
                             A, dA: np.ndarray, h: float | None = None):
    """Chain rule from the entries of the 5-point upwind operator to its per-node fields.

    Per node k, face toward a valid neighbour Q: ``e_f = 2 e_k e_Q / (e_k + e_Q)`` adds
    ``e_f/h^2`` to ``a_kk`` and ``a_QQ`` and ``-e_f/h^2`` to ``a_kQ`` and ``a_Qk``; a
    boundary face adds ``e_k/h^2`` to ``a_kk`` only.  Advection: ``|v_x,k|/h`` on
    ``a_kk``, ``-max(v_x,k, 0)/h`` on the west entry and ``-max(-v_x,k, 0)/h`` on the east
    entry (likewise y with south/north).  Entries not stored in A carry no gradient.

    Returns ``(deps, dvx, dvy)``, each of length ``nside^2``; the derivative of ``|v|`` is
    taken as ``sign(v)`` (0 at v = 0, where the upwind operator is not differentiable).
    """
    A = sp.csr_matrix(A.to_scipy() if hasattr(A, "to_scipy") else A)
    n = nside * nside
    if h is None:
        h = 1.0 / (nside + 1)
    eps = np.broadcast_to(np.asarray(eps, dtype=np.float64), (n,))
    vx = np.broadcast_to(np.asarray(vx, dtype=np.float64), (n,))
    vy = np.broadcast_to(np.asarray(vy, dtype=np.float64), (n,))
    # stencil view of dA: g[k, s] = dL/da_{k, k + off[s]} (0 where not stored)
    off = np.array([-nside, -1, 0, 1, nside])
    rows = np.repeat(np.arange(n), np.diff(A.indptr))
    slot = np.searchsorted(off, A.indices - rows)
    assert np.all(off[slot] == A.indices - rows), "not a 5-point operator"
    g = np.zeros((n, 5))
    g[rows, slot] = dA
    S, W, C, E, N = range(5)
    k = np.arange(n)
    ix, iy = k % nside, k // nside
    deps = np.zeros(n)
    for s_kq, s_qk, valid, q in ((S, N, iy > 0, k - nside), (W, E, ix > 0, k - 1),
                                 (E, W, ix < nside - 1, k + 1), (N, S, iy < nside - 1, k + nside)):
        qq = np.where(valid, q, 0)
        ek, eq = eps, eps[qq]
        dface = 2.0 * eq * eq / (ek + eq) ** 2           # d e_f / d e_k on interior faces
        interior = (g[k, C] - g[k, s_kq] + g[qq, C] - g[qq, s_qk]) * dface
        deps += np.where(valid, interior, g[k, C]) / (h * h)
    dvx = g[:, C] * np.sign(vx) / h
    dvy = g[:, C] * np.sign(vy) / h
    dvx -= np.where((vx > 0) & (ix > 0), g[:, W], 0.0) / h
    dvx += np.where((vx < 0) & (ix < nside - 1), g[:, E], 0.0) / h
    dvy -= np.where((vy > 0) & (iy > 0), g[:, S], 0.0) / h
    dvy += np.where((vy < 0) & (iy < nside - 1), g[:, N], 0.0) / h
    return deps, dvx, dvy


def advdiff2d_loss(nside: int, eps, vx, vy, F: np.ndarray, T: np.ndarray) -> float:
    """The loss as a function of the discretization's fields (assembly + exact solves)."""
    return loss(workloads.advdiff_2d(nside, vx, vy, eps), F, T)
