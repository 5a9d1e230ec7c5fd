"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This module holds no arithmetic of the CLAIR method.  It only builds the
inputs the method is run on:

* a counter-based splitmix64 generator (Steele, Lea & Flood, "Fast splittable
  pseudorandom number generators", OOPSLA 2014): output ``i`` of a stream
  seeded with ``s`` is ``mix(s + (i + 1) * 0x9E3779B97F4A7C15)``, which is
  exactly the ``i``-th draw of the sequential splitmix64 generator seeded with
  ``s``;
* first-order upwind finite-difference advection-diffusion operators in CSR
  form (int32 row pointers and columns, float64 values, columns sorted and
  unique, explicit zeros dropped).  They stand in for the paper's upwind DG
  advection-diffusion discretizations (Section 4.2, Eq. 4.1), which are not
  available here;
* the five workloads the method is measured on (2D constant-direction
  advection-diffusion at 64^2 and 1024^2, 3D recirculating advection at 128^3,
  64 independent 2D instances, and a 512^2 problem with a variable diffusion
  field and a stream-function velocity).

The discretization (one row per interior node, Dirichlet values eliminated):
``a_PP = sum_faces eps_face/h^2 + sum_axes |v_axis|/h``; a neighbour ``Q`` on
axis ``d`` gets ``-eps_face/h^2`` plus ``-|v_d|/h`` when ``Q`` is the upwind
neighbour (``v_d > 0`` -> the lower neighbour, ``v_d < 0`` -> the upper one).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Draws ``offset .. offset+count-1`` of the splitmix64 stream seeded with ``seed``."""
    with np.errstate(over="ignore"):
        ctr = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + ctr * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Doubles in [0, 1): the top 53 bits of each draw times 2^-53 (exact)."""
    z = splitmix64(seed, count, offset)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def uniform_pm1(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Doubles in [-1, 1): ``2u - 1`` with ``u`` from :func:`uniform01` (exact)."""
    return 2.0 * uniform01(seed, count, offset) - 1.0


def normal(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Standard normals by Box-Muller from two uniform streams (draws 2i, 2i+1)."""
    u = uniform01(seed, 2 * count, 2 * offset)
    u1 = 1.0 - u[0::2]           # in (0, 1]
    u2 = u[1::2]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


# ----------------------------------------------------------------------------------
# CSR container
# ----------------------------------------------------------------------------------
@dataclass
class CSR:
    """Square sparse matrix in CSR form (host arrays)."""
    n: int
    rowptr: np.ndarray  # int32 [n+1]
    col: np.ndarray     # int32 [nnz]
    val: np.ndarray     # float64 [nnz]

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.val, self.col, self.rowptr), shape=(self.n, self.n))


def _assemble(n: int, rows: list, cols: list, vals: list) -> CSR:
    """Builds a CSR from per-stencil-point (row, col, value) arrays.

    Entries are listed in increasing column order within a row because the
    stencil points are passed in increasing index offset.  Zeros are dropped.
    """
    r = np.stack(rows, axis=1).reshape(-1)
    c = np.stack(cols, axis=1).reshape(-1)
    v = np.stack(vals, axis=1).reshape(-1)
    keep = (c >= 0) & (v != 0.0)
    r, c, v = r[keep], c[keep], v[keep]
    counts = np.bincount(r, minlength=n)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    assert rowptr[-1] < 2**31
    return CSR(n, rowptr.astype(np.int32), c.astype(np.int32), v.astype(np.float64))


def advdiff_2d(nside: int, vx, vy, eps, h: float | None = None) -> CSR:
    """5-point upwind advection-diffusion on the unit square, ``nside^2`` interior nodes.

    ``vx, vy`` are scalars or per-node arrays (lexicographic order, x fastest).
    ``eps`` is a scalar or a per-node array; a per-node field uses the harmonic
    mean of the two nodal values on interior faces and the node's own value on
    boundary faces.
    """
    n = nside * nside
    if h is None:
        h = 1.0 / (nside + 1)
    idx = np.arange(n, dtype=np.int64)
    ix, iy = idx % nside, idx // nside
    vx = np.broadcast_to(np.asarray(vx, dtype=np.float64), (n,))
    vy = np.broadcast_to(np.asarray(vy, dtype=np.float64), (n,))
    scalar_eps = np.ndim(eps) == 0
    e = np.broadcast_to(np.asarray(eps, dtype=np.float64), (n,))
    inv_h2 = 1.0 / (h * h)
    inv_h = 1.0 / h

    def face(nbr, valid):
        if scalar_eps:
            return e
        en = e[np.where(valid, nbr, 0)]
        s = e + en
        hm = 2.0 * e * en / np.where(s > 0, s, 1.0)
        return np.where(valid, hm, e)

    okS, okW, okE, okN = iy > 0, ix > 0, ix < nside - 1, iy < nside - 1
    fS, fW, fE, fN = face(idx - nside, okS), face(idx - 1, okW), face(idx + 1, okE), face(idx + nside, okN)
    upx = np.maximum(vx, 0.0) * inv_h
    dnx = np.maximum(-vx, 0.0) * inv_h
    upy = np.maximum(vy, 0.0) * inv_h
    dny = np.maximum(-vy, 0.0) * inv_h
    diag = (fS + fW + fE + fN) * inv_h2 + np.abs(vx) * inv_h + np.abs(vy) * inv_h
    rows = [idx] * 5
    cols = [np.where(okS, idx - nside, -1), np.where(okW, idx - 1, -1), idx,
            np.where(okE, idx + 1, -1), np.where(okN, idx + nside, -1)]
    vals = [-fS * inv_h2 - upy, -fW * inv_h2 - upx, diag, -fE * inv_h2 - dnx, -fN * inv_h2 - dny]
    return _assemble(n, rows, cols, vals)


def advdiff_3d(nside: int, vel, eps: float, lo: float = -1.0, hi: float = 1.0) -> CSR:
    """7-point upwind advection-diffusion on ``[lo,hi]^3``, ``nside^3`` interior nodes.

    ``vel(x, y, z) -> (vx, vy, vz)`` is evaluated at the nodes.
    """
    n = nside ** 3
    h = (hi - lo) / (nside + 1)
    idx = np.arange(n, dtype=np.int64)
    ix, iy, iz = idx % nside, (idx // nside) % nside, idx // (nside * nside)
    x, y, z = lo + (ix + 1) * h, lo + (iy + 1) * h, lo + (iz + 1) * h
    vx, vy, vz = (np.broadcast_to(np.asarray(a, dtype=np.float64), (n,)) for a in vel(x, y, z))
    dif = eps / (h * h)
    inv_h = 1.0 / h
    s2 = nside * nside
    ok = {"zm": iz > 0, "ym": iy > 0, "xm": ix > 0, "xp": ix < nside - 1,
          "yp": iy < nside - 1, "zp": iz < nside - 1}
    off = {"zm": -s2, "ym": -nside, "xm": -1, "xp": 1, "yp": nside, "zp": s2}
    adv = {"zm": np.maximum(vz, 0), "ym": np.maximum(vy, 0), "xm": np.maximum(vx, 0),
           "xp": np.maximum(-vx, 0), "yp": np.maximum(-vy, 0), "zp": np.maximum(-vz, 0)}
    diag = 6.0 * dif + (np.abs(vx) + np.abs(vy) + np.abs(vz)) * inv_h
    order = ["zm", "ym", "xm", "P", "xp", "yp", "zp"]
    rows, cols, vals = [], [], []
    for k in order:
        rows.append(idx)
        if k == "P":
            cols.append(idx)
            vals.append(diag)
        else:
            cols.append(np.where(ok[k], idx + off[k], -1))
            vals.append(-dif - adv[k] * inv_h)
    return _assemble(n, rows, cols, vals)


# ----------------------------------------------------------------------------------
# Workloads
# ----------------------------------------------------------------------------------
@dataclass
class Problem:
    """One linear system ``A u = f`` plus its near-nullspace candidate ``B``."""
    name: str
    A: CSR
    f: np.ndarray
    B: np.ndarray                       # [n] (k = 1: the constant vector)
    coarsen: str = "FC"                 # "FC" or "AGG"
    degree: int = 2                     # sparsity pattern degree m
    meta: dict = field(default_factory=dict)


def constdir_2d(nside: int, angle: float, eps: float, seed: int, degree: int = 2,
                name: str | None = None) -> Problem:
    """2D constant-direction advection-diffusion, velocity (cos a, sin a)."""
    A = advdiff_2d(nside, math.cos(angle), math.sin(angle), eps)
    f = uniform_pm1(seed, A.n)
    return Problem(name or f"constdir2d_{nside}_eps{eps:g}_m{degree}", A, f,
                   np.ones(A.n), "FC", degree,
                   {"nside": nside, "angle": angle, "eps": eps, "seed": seed})


def config1() -> Problem:
    """64x64 interior grid, velocity angle pi/6, eps = 1e-2, seed 0, m = 2."""
    return constdir_2d(64, math.pi / 6, 1e-2, seed=0, degree=2, name="constdir2d_64")


def config2(eps: float = 1e-2, degree: int = 2, nside: int = 1024) -> Problem:
    """1024x1024 interior grid, angle pi/6, eps in {0, 1e-4, 1e-2, 1}, seed 1, m in {1, 2}."""
    return constdir_2d(nside, math.pi / 6, eps, seed=1, degree=degree,
                       name=f"constdir2d_{nside}_eps{eps:g}_m{degree}")


CONFIG2_EPS = (0.0, 1e-4, 1e-2, 1.0)


def recirc_velocity(x, y, z):
    return 2.0 * y * (1.0 - x * x), -2.0 * x * (1.0 - y * y), 0.5 + 0.0 * z


def config3(nside: int = 128) -> Problem:
    """128^3 on [-1,1]^3, v = (2y(1-x^2), -2x(1-y^2), 0.5), eps = 1e-3, seed 2, AGG, m = 2."""
    A = advdiff_3d(nside, recirc_velocity, 1e-3)
    f = uniform_pm1(2, A.n)
    return Problem(f"recirc3d_{nside}", A, f, np.ones(A.n), "AGG", 2,
                   {"nside": nside, "eps": 1e-3, "seed": 2})


def config4_params(count: int = 64, seed: int = 3):
    """Per-instance (side, angle, eps): side ~ U{64..512}, angle ~ U(0, 2pi), log10 eps ~ U(-5, 0)."""
    u = uniform01(seed, 3 * count)
    sides = 64 + np.floor(u[0::3] * 449).astype(np.int64)
    angles = 2.0 * np.pi * u[1::3]
    eps = 10.0 ** (-5.0 + 5.0 * u[2::3])
    return [(int(s), float(a), float(e)) for s, a, e in zip(sides, angles, eps)]


def config4(count: int = 64, seed: int = 3, max_side: int | None = None) -> list[Problem]:
    """64 independent 2D problems; RHS of instance k is stream ``seed`` at offset sum of earlier sizes."""
    probs, offset = [], 0
    for k, (s, a, e) in enumerate(config4_params(count, seed)):
        if max_side is not None:
            s = min(s, max_side)
        A = advdiff_2d(s, math.cos(a), math.sin(a), e)
        f = uniform_pm1(seed + 1, A.n, offset)
        offset += A.n
        probs.append(Problem(f"inst{k}_{s}", A, f, np.ones(A.n), "FC", 2,
                             {"nside": s, "angle": a, "eps": e}))
    return probs


def block_diagonal(mats) -> tuple[CSR, np.ndarray]:
    """Stacks square CSR operators into one block-diagonal CSR; returns it and the row
    offsets of the blocks (length len(mats) + 1)."""
    offs = np.zeros(len(mats) + 1, dtype=np.int64)
    for i, M in enumerate(mats):
        offs[i + 1] = offs[i] + M.n
    rowptr = [np.zeros(1, dtype=np.int64)]
    cols, vals = [], []
    base_nnz = 0
    for i, M in enumerate(mats):
        rowptr.append(M.rowptr[1:].astype(np.int64) + base_nnz)
        cols.append(M.col.astype(np.int64) + offs[i])
        vals.append(M.val)
        base_nnz += M.nnz
    A = CSR(int(offs[-1]), np.concatenate(rowptr).astype(np.int32),
            np.concatenate(cols).astype(np.int32), np.concatenate(vals))
    return A, offs


def config5_fields(nside: int = 512, seed: int = 4):
    """Per-node eps = 10^(-3 + N(0, 0.5)) and velocity from psi = sin(pi x) sin(pi y)."""
    n = nside * nside
    h = 1.0 / (nside + 1)
    idx = np.arange(n)
    x, y = (idx % nside + 1) * h, (idx // nside + 1) * h
    eps = 10.0 ** (-3.0 + 0.5 * normal(seed, n))
    vx = np.pi * np.sin(np.pi * x) * np.cos(np.pi * y)        # d psi / dy
    vy = -np.pi * np.cos(np.pi * x) * np.sin(np.pi * y)       # -d psi / dx
    return eps, vx, vy


def config5(nside: int = 512, seed: int = 4, nrhs: int = 8):
    """512^2 variable-eps problem with 8 right-hand sides and a target u_t ~ U(-1,1)."""
    eps, vx, vy = config5_fields(nside, seed)
    A = advdiff_2d(nside, vx, vy, eps)
    n = A.n
    F = uniform_pm1(seed, n * nrhs, offset=2 * n).reshape(nrhs, n)
    Ut = uniform_pm1(seed, n * nrhs, offset=2 * n + n * nrhs).reshape(nrhs, n)
    return Problem(f"varcoef2d_{nside}", A, F, np.ones(n), "FC", 2,
                   {"nside": nside, "seed": seed, "eps_field": eps, "vx": vx, "vy": vy,
                    "u_target": Ut})
