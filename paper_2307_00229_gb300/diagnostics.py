"""Approximation-property diagnostics of a built hierarchy (Appendix A of the paper).

An offline analysis on the host with dense linear algebra, for small problems (the paper
uses a 32 x 32 grid, 1024 unknowns): it reads transfer operators out of a hierarchy
(``clair_level_view``) and measures how well their range captures the near-nullspace of a
nonsymmetric operator.  It is not part of setup or solve and runs no kernel.

For a nonsingular A = U S V^T (singular values ascending), the SPD matrices
sqrt(A^T A) = V S V^T and sqrt(A A^T) = U S U^T stand in for the energy norm: the first
for interpolation (T = P), the second for the restriction (T = R^T).  The fractional
approximation property FAP(beta, eta) of T with respect to such an SPD matrix M holds with
constant

    K_max = ||M||^(2 beta - eta) * || M^(eta/2) (I - Pi_eta) M^(-beta) ||_2^2,
    Pi_eta = T (T^T M^eta T)^-1 T^T M^eta   (the M^eta-orthogonal projection onto range T),

and for a single vector v

    K(v) = ||M||^(2 beta - eta) * ||(I - Pi_eta) v||^2_{M^eta} / ||v||^2_{M^(2 beta)}.

The weak approximation property is FAP(1/2, 0), the strong one FAP(1, 1).
"""
from __future__ import annotations

import numpy as np


def _spd_power(U: np.ndarray, s: np.ndarray, p: float) -> np.ndarray:
    """U diag(s^p) U^T for the orthonormal U and positive s of an SPD matrix."""
    return (U * s ** p) @ U.T


def energy_matrix(A: np.ndarray, side: str):
    """(U, s) with M = U diag(s) U^T: sqrt(A^T A) for side 'P' (right singular vectors),
    sqrt(A A^T) for side 'R' (left singular vectors); s ascending."""
    Uf, s, Vt = np.linalg.svd(np.asarray(A, dtype=np.float64))
    order = np.argsort(s)
    s = s[order]
    if side == "P":
        return Vt.T[:, order], s
    if side == "R":
        return Uf[:, order], s
    raise ValueError(side)


def fap_constants(A: np.ndarray, T: np.ndarray, beta: float, eta: float, side: str,
                  vectors: np.ndarray | None = None):
    """``(K_max, K_of_vectors)`` of the transfer T (n x n_c dense: P, or R^T for side 'R').

    ``vectors`` (n x q) defaults to the singular vectors that span the energy matrix's
    eigenvectors (in ascending singular value), as plotted in Appendix A."""
    U, s = energy_matrix(A, side)
    T = np.asarray(T, dtype=np.float64)
    Meta = _spd_power(U, s, eta)
    Mb_inv = _spd_power(U, s, -beta)
    Meta_half = _spd_power(U, s, eta / 2.0)
    Pi = T @ np.linalg.solve(T.T @ Meta @ T, T.T @ Meta)
    E = np.eye(A.shape[0]) - Pi
    norm = s[-1] ** (2.0 * beta - eta)
    kmax = norm * np.linalg.norm(Meta_half @ E @ Mb_inv, 2) ** 2
    V = U if vectors is None else np.asarray(vectors, dtype=np.float64)
    M2b = _spd_power(U, s, 2.0 * beta)
    EV = E @ V
    num = np.einsum("ij,ij->j", EV, Meta @ EV)
    den = np.einsum("ij,ij->j", V, M2b @ V)
    return float(kmax), norm * num / den


def wap(A, T, side: str, vectors=None):
    """Weak approximation property, FAP(1/2, 0)."""
    return fap_constants(A, T, 0.5, 0.0, side, vectors)


def sap(A, T, side: str, vectors=None):
    """Strong approximation property, FAP(1, 1)."""
    return fap_constants(A, T, 1.0, 1.0, side, vectors)
