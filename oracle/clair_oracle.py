"""Plain float64 oracle of CLAIR AMG: setup (Algorithm 1 per level) and V(1,1)-FGMRES solve.

TEST INFRASTRUCTURE ONLY (see the package docstring): the product path never imports it.

Readings of the paper taken here (the paper is silent or ambiguous on these points):

* Strength of connection is the classical measure on absolute values: entry ``a_ij``
  (``j != i``, ``a_ij != 0``) is strong iff ``|a_ij| >= theta * max_{k != i} |a_ik|``.
  The threshold product ``theta * max`` is formed in float64.
* "FC" coarsening (the paper's Ruge-Stueben first pass) is replaced by one deterministic
  parallel-MIS definition (``split_fc``), and greedy aggregation by a distance-two MIS
  definition (``aggregate``), both keyed by ``(lambda_i, lowbias32(i))``.
* The pattern expansion uses ``S + I`` in ``(S + I)^{m-1} T`` so that the degree-m
  pattern contains the degree-(m-1) one.
* The restriction is Algorithm 1 applied to ``A^T`` and transposed; its pattern uses the
  strength of ``A^T`` with the interpolation threshold.
* ``rho(D^-1 A)`` comes from 15 Arnoldi steps (modified Gram-Schmidt) started from a
  splitmix64 vector in [-1, 1) seeded with ``seed + level``; ``rho`` is the largest
  Ritz-value modulus.  The same weight serves the ``A^T`` side because ``D^-1 A^T`` is
  similar to ``D^-1 A``.
* The mode vector is smoothed separately for ``P`` (operator ``A``) and for ``R``
  (operator ``A^T``); each side injects its own smoothed vector to the next level.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

import workloads

C_PT = 1
F_PT = 0

__all__ = [
    "C_PT", "F_PT", "Params", "lowbias32", "strength", "split_fc", "aggregate",
    "arnoldi", "arnoldi_rho", "relax", "relax_cff", "relax_ffc", "smooth_modes", "base_pattern",
    "clair_pattern", "clair_algorithm1", "clair_transfer", "Level", "Hierarchy",
    "build_hierarchy", "vcycle", "fgmres", "pcg", "operator_complexity", "work_per_digit",
    "solve", "csr_of",
]


@dataclass
class Params:
    """Solver parameters (Section 4.2: theta_c = 0.25, theta_i = 0.05, m = 2, V(1,1),
    CFF pre / FFC post weighted Jacobi with the post weight removed, B = 1 smoothed by
    five CFF sweeps per level)."""
    theta_coarsen: float = 0.25
    theta_interp: float = 0.05
    degree: int = 2
    coarsen: str = "FC"            # "FC" or "AGG"
    b_smooth_iters: int = 5
    arnoldi_iters: int = 15
    post_weighted: bool = False    # nonsymmetric runs: post-smoothing weight 1
    coarse_max: int = 128
    max_levels: int = 25
    gmres_restart: int = 50
    gmres_maxit: int = 200
    rtol: float = 1e-8
    seed: int = 0x5EED
    inverse: str = "exact"         # block inverses: "exact" (Remark 3.2) or "diag"
    iterations: int = 1            # Algorithm 1 loop count k
    constrain: bool = True         # False reproduces lAIR (Remark 3.1)
    symmetric: bool = False        # R = P^T (the symmetric diffusion runs of Section 4.1)


def csr_of(A) -> sp.csr_matrix:
    """scipy CSR with sorted indices from a ``workloads.CSR`` or any scipy matrix."""
    if isinstance(A, workloads.CSR):
        M = sp.csr_matrix((A.val.astype(np.float64), A.col.astype(np.int64),
                           A.rowptr.astype(np.int64)), shape=(A.n, A.n))
    else:
        M = sp.csr_matrix(A, dtype=np.float64)
    M.sort_indices()
    return M


# --------------------------------------------------------------------------------------
# Strength of connection (Section 3.1.3: "classical strength measure"; parameters in
# Section 4.2: 0.25 for coarsening, 0.05 for interpolation)
# --------------------------------------------------------------------------------------
def strength(A: sp.csr_matrix, theta: float) -> sp.csr_matrix:
    """0/1 matrix ``S`` with ``S_ij = 1`` iff ``i`` strongly depends on ``j``."""
    A = csr_of(A)
    n = A.shape[0]
    rows = np.repeat(np.arange(n), np.diff(A.indptr))
    offd = A.indices != rows
    absv = np.abs(A.data) * offd
    rowmax = np.zeros(n)
    np.maximum.at(rowmax, rows, absv)
    strong = offd & (absv > 0.0) & (absv >= theta * rowmax[rows])
    S = sp.csr_matrix((strong.astype(np.float64), A.indices.copy(), A.indptr.copy()),
                      shape=A.shape)
    S.eliminate_zeros()
    S.sort_indices()
    return S


def lowbias32(i: np.ndarray) -> np.ndarray:
    """The 'lowbias32' integer hash (C. Wellons' hash-prospector): a bijection of uint32."""
    x = np.asarray(i, dtype=np.uint64) & np.uint64(0xFFFFFFFF)
    m32 = np.uint64(0xFFFFFFFF)
    x ^= x >> np.uint64(16)
    x = (x * np.uint64(0x7FEB352D)) & m32
    x ^= x >> np.uint64(15)
    x = (x * np.uint64(0x846CA68B)) & m32
    x ^= x >> np.uint64(16)
    return x


def _priority(S: sp.csr_matrix) -> tuple[np.ndarray, np.ndarray]:
    """``lambda_i`` = number of points strongly depending on ``i``; key = (lambda, hash)."""
    n = S.shape[0]
    lam = np.bincount(S.indices, minlength=n).astype(np.int64)
    key = (lam.astype(np.uint64) << np.uint64(32)) | lowbias32(np.arange(n))
    return lam, key


def _segment_max(G: sp.csr_matrix, vals: np.ndarray) -> np.ndarray:
    """Per row of the pattern ``G``: max of ``vals`` over the row's columns (0 if empty)."""
    n = G.shape[0]
    out = np.zeros(n, dtype=np.uint64)
    rows = np.repeat(np.arange(n), np.diff(G.indptr))
    np.maximum.at(out, rows, vals[G.indices])
    return out


def split_fc(A, theta: float) -> np.ndarray:
    """C/F splitting ("FC" coarsening, Section 3.1.3, Algorithm 1 input; Section 4.2).

    The paper uses the sequential Ruge-Stueben first pass.  This is its deterministic
    parallel reading (a PMIS-type independent set on the strength graph):

    1. ``S = strength(A, theta)``; ``lambda_i`` = #points strongly depending on ``i``;
       ``G`` = symmetrised ``S``; key_i = ``(lambda_i, lowbias32(i))`` (unique).
    2. Points with ``lambda_i = 0`` influence nobody and start as F; all others undecided.
    3. Rounds: every undecided point whose key exceeds the keys of all undecided
       G-neighbours becomes C; then every still-undecided point that strongly depends
       on one of the new C-points becomes F.  Repeat until nothing is undecided.
    4. An F-point that strongly depends on some point but on no C-point becomes C (as in
       the first pass, where F-points arise from a C dependence).  Such points all had
       ``lambda = 0``, so no two of them are G-neighbours and one step suffices.

    Returns int8 ``cf`` with 1 for C and 0 for F.
    """
    A = csr_of(A)
    S = strength(A, theta)
    n = S.shape[0]
    St = S.T.tocsr()
    G = (S + St).tocsr()
    G.sort_indices()
    lam, key = _priority(S)
    UND, CP, FP = 0, 1, 2
    state = np.zeros(n, dtype=np.int8)
    state[lam == 0] = FP
    while np.any(state == UND):
        und = state == UND
        nbr_max = _segment_max(G, np.where(und, key, np.uint64(0)))
        new_c = und & (key > nbr_max)
        state[new_c] = CP
        dep = (S @ new_c.astype(np.float64)) > 0
        state[und & ~new_c & dep] = FP
    has_dep = np.diff(S.indptr) > 0
    dep_c = (S @ (state == CP).astype(np.float64)) > 0
    state[(state == FP) & has_dep & ~dep_c] = CP
    return (state == CP).astype(np.int8)


def aggregate(A, theta: float) -> tuple[np.ndarray, np.ndarray]:
    """Aggregation ("Agg" coarsening; the footnote to Section 3.1.3 describing the
    greedy aggregation of Vanek-Mandel-Brezina).

    Deterministic parallel reading of "root with all-unmarked neighbours, then clean-up":

    1. ``S = strength(A, theta)``, ``G`` its symmetrisation, key as in ``split_fc``.
       Points with no G-neighbour are left out (F, no aggregate).
    2. Roots form a distance-two independent set: in rounds, every undecided point whose
       key is the largest among undecided points within graph distance two becomes a
       root, and every point within distance two of a new root is decided.
    3. Each point adjacent to a root joins it (roots are three or more apart, so the
       root is unique); each remaining point joins the adjacent aggregate of lowest index.

    Returns ``(cf, agg)``: roots are C-points; ``agg[j]`` is the aggregate (= coarse index
    of its root, roots numbered in increasing point index) or -1.
    """
    A = csr_of(A)
    S = strength(A, theta)
    n = S.shape[0]
    G = (S + S.T).tocsr()
    G.sort_indices()
    _, key = _priority(S)
    isolated = np.diff(G.indptr) == 0
    undecided = ~isolated
    root = np.zeros(n, dtype=bool)
    Gb = (G != 0).astype(np.float64)
    while np.any(undecided):
        k = np.where(undecided, key, np.uint64(0))
        m1 = np.maximum(k, _segment_max(G, k))
        m2 = np.maximum(m1, _segment_max(G, m1))
        new_root = undecided & (key == m2)
        root |= new_root
        near1 = (Gb @ new_root.astype(np.float64)) > 0
        near2 = (Gb @ near1.astype(np.float64)) > 0
        undecided &= ~(new_root | near1 | near2)
    coarse_index = np.cumsum(root) - 1
    agg = np.full(n, -1, dtype=np.int64)
    agg[root] = coarse_index[root]
    rows = np.repeat(np.arange(n), np.diff(G.indptr))
    for j in range(n):                      # distance one: the unique adjacent root
        if root[j] or isolated[j]:
            continue
        nb = G.indices[G.indptr[j]:G.indptr[j + 1]]
        r = nb[root[nb]]
        if r.size:
            assert r.size == 1
            agg[j] = coarse_index[r[0]]
    first = agg.copy()
    for j in range(n):                      # clean-up: lowest adjacent aggregate
        if agg[j] >= 0 or isolated[j]:
            continue
        nb = G.indices[G.indptr[j]:G.indptr[j + 1]]
        cand = first[nb]
        cand = cand[cand >= 0]
        assert cand.size > 0
        agg[j] = cand.min()
    del rows
    return root.astype(np.int8), agg


# --------------------------------------------------------------------------------------
# Relaxation weight and relaxation (Section 4: weight 1/rho(D^-1 A), rho from 15 Arnoldi
# iterations; CFF pre- and FFC post-smoothing; B smoothed by 5 CFF sweeps, Section 4.1)
# --------------------------------------------------------------------------------------
def arnoldi(A, iters: int, seed: int):
    """``iters`` Arnoldi steps on ``D^-1 A`` (Section 4) from the seeded start vector, each new
    vector orthogonalised against the basis by classical Gram-Schmidt applied twice, so the
    basis stays orthonormal to working precision (a single Gram-Schmidt pass loses that on
    the small, strongly non-normal coarse operators).  A step whose new vector has norm at
    most 1e-10 of its norm before orthogonalisation ends the run (invariant subspace).
    Returns (H, V, steps): H is (m + 1) x m upper Hessenberg, V holds the basis in rows."""
    A = csr_of(A)
    n = A.shape[0]
    dinv = 1.0 / A.diagonal()
    m = min(iters, n)
    V = np.zeros((m + 1, n))
    H = np.zeros((m + 1, m))
    v0 = workloads.uniform_pm1(seed, n)
    V[0] = v0 / np.linalg.norm(v0)
    steps = m
    for j in range(m):
        w = dinv * (A @ V[j])
        wnorm0 = np.linalg.norm(w)
        Vj = V[: j + 1]
        h1 = Vj @ w
        w = w - Vj.T @ h1
        h2 = Vj @ w
        w = w - Vj.T @ h2
        H[: j + 1, j] = h1 + h2
        H[j + 1, j] = np.linalg.norm(w)
        if H[j + 1, j] <= 1e-10 * wnorm0:
            steps = j + 1
            break
        V[j + 1] = w / H[j + 1, j]
    return H, V, steps


def arnoldi_rho(A, iters: int, seed: int) -> float:
    """Spectral radius estimate of ``D^-1 A``: the largest Ritz value modulus of ``iters``
    Arnoldi steps (Section 4)."""
    H, _, steps = arnoldi(A, iters, seed)
    ritz = np.linalg.eigvals(H[:steps, :steps])
    return float(np.max(np.abs(ritz)))


def relax(A, x: np.ndarray, b: np.ndarray, mask: np.ndarray, omega: float) -> np.ndarray:
    """One weighted-Jacobi sweep on the point subset ``mask``:
    ``x_X <- x_X + omega * D_XX^-1 (b - A x)_X`` with the residual of the incoming ``x``."""
    A = csr_of(A)
    d = A.diagonal()
    r = b - A @ x
    x = x.copy()
    if x.ndim == 1:
        x[mask] += omega * r[mask] / d[mask]
    else:
        x[mask] += omega * r[mask] / d[mask, None]
    return x


def relax_cff(A, x, b, cf, omega):
    """CFF: one Jacobi sweep on C-points, then two on F-points (Section 4)."""
    c = cf == C_PT
    x = relax(A, x, b, c, omega)
    x = relax(A, x, b, ~c, omega)
    return relax(A, x, b, ~c, omega)


def relax_ffc(A, x, b, cf, omega):
    """FFC: two Jacobi sweeps on F-points, then one on C-points (Section 4)."""
    c = cf == C_PT
    x = relax(A, x, b, ~c, omega)
    x = relax(A, x, b, ~c, omega)
    return relax(A, x, b, c, omega)


def smooth_modes(A, B: np.ndarray, cf: np.ndarray, omega: float, sweeps: int) -> np.ndarray:
    """``B <- CFF^sweeps (B)`` with a zero right-hand side (Section 4.1 parameters)."""
    zero = np.zeros_like(B)
    for _ in range(sweeps):
        B = relax_cff(A, B, zero, cf, omega)
    return B


# --------------------------------------------------------------------------------------
# Algorithm 1 (Section 3.1.3)
# --------------------------------------------------------------------------------------
def base_pattern(S: sp.csr_matrix, cf: np.ndarray, coarsen: str, agg=None) -> sp.csr_matrix:
    """Base pattern ``T`` of Algorithm 1: ``[S_fc, I]`` (FC) or the aggregation operator
    (Agg), as an ``n x n_c`` 0/1 matrix."""
    n = cf.size
    cpts = np.flatnonzero(cf == C_PT)
    nc = cpts.size
    if coarsen == "FC":
        Scols = S[:, cpts].tocsr()                      # n x n_c
        fmask = sp.diags((cf == F_PT).astype(np.float64))
        ident = sp.csr_matrix((np.ones(nc), (cpts, np.arange(nc))), shape=(n, nc))
        T = (fmask @ Scols + ident).tocsr()
    elif coarsen == "AGG":
        members = np.flatnonzero(agg >= 0)
        T = sp.csr_matrix((np.ones(members.size), (members, agg[members])), shape=(n, nc))
    else:
        raise ValueError(coarsen)
    T.data[:] = 1.0
    return T


def clair_pattern(S: sp.csr_matrix, T: sp.csr_matrix, cf: np.ndarray, degree: int) -> sp.csc_matrix:
    """``W = pattern((S^{m-1} T)|_F)`` (Algorithm 1, pattern expansion), with ``S + I``."""
    n = cf.size
    SI = (S + sp.identity(n, format="csr")).tocsr()
    SI.data[:] = 1.0
    E = T.tocsr().copy()
    for _ in range(degree - 1):
        E = (SI @ E).tocsr()
        E.data[:] = 1.0
    fmask = sp.diags((cf == F_PT).astype(np.float64))
    W = (fmask @ E).tocsc()
    W.eliminate_zeros()
    W.sort_indices()
    W.data[:] = 1.0
    return W


def _row_constraint_update(w: np.ndarray, Bc_J: np.ndarray, target: np.ndarray) -> np.ndarray:
    """Minimal-norm change of the row vector ``w`` so that ``w @ Bc_J = target``
    (least squares via the pseudo-inverse when it cannot be met exactly)."""
    G = Bc_J.T @ Bc_J
    resid = w @ Bc_J - target
    return w - (resid @ np.linalg.pinv(G)) @ Bc_J.T


def _row_least_squares(Bc_J: np.ndarray, target: np.ndarray) -> np.ndarray:
    """Least-squares (minimum-norm) solution of the row system ``w @ Bc_J = target``."""
    return (target @ np.linalg.pinv(Bc_J.T @ Bc_J)) @ Bc_J.T


def clair_algorithm1(Ahat, cf: np.ndarray, B: np.ndarray, Wpat: sp.csc_matrix,
                     params: Params, cpts: np.ndarray | None = None) -> sp.csc_matrix:
    """Algorithm 1 of the paper on operator ``Ahat``: returns the F-rows ``W`` (n x n_c,
    zero on C rows) of ``P = [W; I]`` obeying the pattern ``Wpat``.

    ``cpts`` (default: all C-points of ``cf`` in increasing order) names the C-point of each
    column of ``Wpat``; passing a subset of columns runs the algorithm on those columns
    only, which is exact for every F row whose pattern row lies inside the subset (every
    step of the algorithm is local to a column block or to an F row).

    Steps, in the paper's order:
      * tentative ``w_t`` from ``[-A_fc, I]`` on the pattern;
      * enforce ``Q w_t = B|_F`` row by row: each F row of ``w_t`` becomes the least-squares
        (minimum-norm) solution of ``w B_c = B`` on its pattern;
      * block inverses of ``A_ff^{(i)}`` (``A_ff`` restricted to ``W_i`` in rows and
        columns), exact or diagonal;
      * k times: ``wbar = Ahat_ff^-1 (-a_fc - A_ff w_t)`` per column block, project
        ``wbar <- (I - Q^T (Q Q^T)^+ Q) wbar`` row by row, ``w_t += wbar``.
    With ``params.constrain = False`` the two constraint steps are skipped (Remark 3.1).
    """
    Ahat = csr_of(Ahat)
    n = Ahat.shape[0]
    if cpts is None:
        cpts = np.flatnonzero(cf == C_PT)
    nc = cpts.size
    B = B.reshape(n, -1)
    Bc = B[cpts]
    Wpat = Wpat.tocsc()
    Wpat.sort_indices()
    assert Wpat.shape[1] == nc

    def block(rows, cols):
        """Dense ``Ahat[rows, cols]`` (``cols`` sorted ascending)."""
        cols = np.asarray(cols)
        out = np.zeros((len(rows), cols.size))
        for p, r in enumerate(rows):
            c = Ahat.indices[Ahat.indptr[r]:Ahat.indptr[r + 1]]
            v = Ahat.data[Ahat.indptr[r]:Ahat.indptr[r + 1]]
            q = np.searchsorted(cols, c)
            hit = (q < cols.size) & (cols[np.minimum(q, cols.size - 1)] == c)
            out[p, q[hit]] = v[hit]
        return out

    # tentative interpolation: -A_fc restricted to the pattern
    cols_of = [Wpat.indices[Wpat.indptr[i]:Wpat.indptr[i + 1]] for i in range(nc)]
    w_t = [-block(cols_of[i], [cpts[i]])[:, 0] if cols_of[i].size else np.zeros(0)
           for i in range(nc)]

    # row view of the pattern: for F row j, the (column i, position in column i) pairs
    Wr = Wpat.tocsr()
    Wr.sort_indices()
    pos_in_col = {}
    for i in range(nc):
        for p, j in enumerate(cols_of[i]):
            pos_in_col[(int(j), i)] = p
    rows_nz = np.flatnonzero(np.diff(Wr.indptr))

    def gather_row(w, j):
        J = Wr.indices[Wr.indptr[j]:Wr.indptr[j + 1]]
        return J, np.array([w[i][pos_in_col[(int(j), int(i))]] for i in J])

    def scatter_row(w, j, J, vals):
        for i, v in zip(J, vals):
            w[i][pos_in_col[(int(j), int(i))]] = v

    if params.constrain:
        # "least squares solution to w B_c = B" per F row: the minimum-norm solution (the
        # pattern of [-A_fc, I] fixes where w_t may be nonzero; its values are replaced)
        for j in rows_nz:
            J, _ = gather_row(w_t, j)
            scatter_row(w_t, j, J, _row_least_squares(Bc[J], B[j]))

    blocks = [block(cols_of[i], cols_of[i]) for i in range(nc)]
    rhs = [-block(cols_of[i], [cpts[i]])[:, 0] for i in range(nc)]
    if params.inverse == "exact":
        inv = [(lambda M: (lambda r: np.linalg.solve(M, r) if M.size else r))(M) for M in blocks]
    elif params.inverse == "diag":
        inv = [(lambda d: (lambda r: r / d))(np.diag(M).copy()) for M in blocks]
    else:
        raise ValueError(params.inverse)

    for _ in range(params.iterations):
        wbar = [inv[i](rhs[i] - blocks[i] @ w_t[i]) if cols_of[i].size else np.zeros(0)
                for i in range(nc)]
        if params.constrain:
            for j in rows_nz:
                J, vj = gather_row(wbar, j)
                scatter_row(wbar, j, J, _row_constraint_update(vj, Bc[J], np.zeros(B.shape[1])))
        w_t = [w_t[i] + wbar[i] for i in range(nc)]

    data = np.concatenate([w_t[i] for i in range(nc)]) if nc else np.zeros(0)
    return sp.csc_matrix((data, Wpat.indices.copy(), Wpat.indptr.copy()), shape=(n, nc))


def clair_transfer(Ahat, cf: np.ndarray, B: np.ndarray, params: Params, agg=None,
                   theta: float | None = None):
    """``P = [W; I]`` from Algorithm 1 on ``Ahat`` (use ``Ahat = A^T`` and transpose for R).

    Pattern from ``S = strength(Ahat, theta_interp)``.  Returns ``(P csr n x n_c, Wpat)``.
    """
    Ahat = csr_of(Ahat)
    n = Ahat.shape[0]
    S = strength(Ahat, params.theta_interp if theta is None else theta)
    T = base_pattern(S, cf, params.coarsen, agg)
    Wpat = clair_pattern(S, T, cf, params.degree)
    W = clair_algorithm1(Ahat, cf, B, Wpat, params)
    cpts = np.flatnonzero(cf == C_PT)
    ident = sp.csc_matrix((np.ones(cpts.size), (cpts, np.arange(cpts.size))), shape=W.shape)
    P = (W + ident).tocsr()
    P.sort_indices()
    return P, Wpat


# --------------------------------------------------------------------------------------
# Hierarchy (Section 1: A_c = R A P, recursive; Section 2.3: B_c = [0 I] B)
# --------------------------------------------------------------------------------------
@dataclass
class Level:
    A: sp.csr_matrix
    cf: np.ndarray | None = None
    agg: np.ndarray | None = None
    omega: float = 1.0
    B_P: np.ndarray | None = None     # mode vector after smoothing with A
    B_R: np.ndarray | None = None     # mode vector after smoothing with A^T
    P: sp.csr_matrix | None = None
    R: sp.csr_matrix | None = None


@dataclass
class Hierarchy:
    levels: list
    params: Params
    coarse_dense: np.ndarray | None = None
    info: dict = field(default_factory=dict)


def build_hierarchy(A, B: np.ndarray, params: Params, cf_override=None) -> Hierarchy:
    """CLAIR setup: per level split, weight, smoothed modes, P and R by Algorithm 1,
    Galerkin coarse operator; stop at ``coarse_max`` unknowns or ``max_levels``."""
    A = csr_of(A)
    B_P = np.asarray(B, dtype=np.float64).reshape(A.shape[0], -1).copy()
    B_R = B_P.copy()
    levels = []
    while True:
        n = A.shape[0]
        lev = Level(A=A)
        levels.append(lev)
        if n <= params.coarse_max or len(levels) >= params.max_levels:
            break
        if cf_override is not None and len(levels) == 1:
            cf, agg = np.asarray(cf_override, dtype=np.int8), None
        elif params.coarsen == "FC":
            cf, agg = split_fc(A, params.theta_coarsen), None
        else:
            cf, agg = aggregate(A, params.theta_coarsen)
        nc = int(cf.sum())
        if nc == 0 or nc == n:
            break
        lev.cf, lev.agg = cf, agg
        lev.omega = 1.0 / arnoldi_rho(A, params.arnoldi_iters, params.seed + len(levels) - 1)
        At = A.T.tocsr()
        At.sort_indices()
        lev.B_P = smooth_modes(A, B_P, cf, lev.omega, params.b_smooth_iters)
        lev.P, _ = clair_transfer(A, cf, lev.B_P, params, agg)
        if params.symmetric:
            # R = P^T (Section 4.1: the symmetric runs use the transpose of interpolation)
            lev.B_R = lev.B_P.copy()
            lev.R = lev.P.T.tocsr()
        else:
            lev.B_R = smooth_modes(At, B_R, cf, lev.omega, params.b_smooth_iters)
            Pt, _ = clair_transfer(At, cf, lev.B_R, params, agg)
            lev.R = Pt.T.tocsr()
        lev.R.sort_indices()
        Ac = (lev.R @ A) @ lev.P
        Ac = Ac.tocsr()
        Ac.sort_indices()
        cpts = np.flatnonzero(cf == C_PT)
        B_P, B_R = lev.B_P[cpts], lev.B_R[cpts]
        A = Ac
    H = Hierarchy(levels, params)
    H.coarse_dense = levels[-1].A.toarray()
    return H


def vcycle(H: Hierarchy, b: np.ndarray, k: int = 0) -> np.ndarray:
    """V(1,1) with x0 = 0: CFF pre, residual, restrict, recurse, interpolate, FFC post
    (Section 4; post weight 1 for nonsymmetric runs, Section 4.2)."""
    lev = H.levels[k]
    if k == len(H.levels) - 1:
        return np.linalg.solve(H.coarse_dense, b)
    A = lev.A
    x = np.zeros_like(b)
    x = relax_cff(A, x, b, lev.cf, lev.omega)
    r = b - A @ x
    xc = vcycle(H, lev.R @ r, k + 1)
    x = x + lev.P @ xc
    post = lev.omega if H.params.post_weighted else 1.0
    return relax_ffc(A, x, b, lev.cf, post)


def fgmres(A, f: np.ndarray, precond, restart: int, rtol: float, maxit: int,
           x0: np.ndarray | None = None):
    """Right-preconditioned flexible GMRES(restart) in float64 (Saad 1993), modified
    Gram-Schmidt, Givens rotations; stops when the true residual ||f - A x|| <= rtol ||f||.

    Returns ``(x, iterations, history of true/estimated residual norms)``."""
    A = csr_of(A)
    n = f.size
    x = np.zeros(n) if x0 is None else x0.astype(np.float64).copy()
    fnorm = np.linalg.norm(f)
    if fnorm == 0.0:
        return np.zeros(n), 0, [0.0]
    tol = rtol * fnorm
    r = f - A @ x
    beta = np.linalg.norm(r)
    hist = [beta]
    its = 0
    while beta > tol and its < maxit:
        m = restart
        V = np.zeros((m + 1, n))
        Z = np.zeros((m, n))
        Hm = np.zeros((m + 1, m))
        cs, sn = np.zeros(m), np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        j_end = 0
        for j in range(m):
            Z[j] = precond(V[j])
            w = A @ Z[j]
            for i in range(j + 1):
                Hm[i, j] = V[i] @ w
                w = w - Hm[i, j] * V[i]
            Hm[j + 1, j] = np.linalg.norm(w)
            if Hm[j + 1, j] > 0:
                V[j + 1] = w / Hm[j + 1, j]
            for i in range(j):
                t = cs[i] * Hm[i, j] + sn[i] * Hm[i + 1, j]
                Hm[i + 1, j] = -sn[i] * Hm[i, j] + cs[i] * Hm[i + 1, j]
                Hm[i, j] = t
            den = math.hypot(Hm[j, j], Hm[j + 1, j])
            cs[j], sn[j] = Hm[j, j] / den, Hm[j + 1, j] / den
            Hm[j, j] = den
            Hm[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            its += 1
            j_end = j + 1
            hist.append(abs(g[j + 1]))
            if abs(g[j + 1]) <= tol or its >= maxit:
                break
        y = np.zeros(j_end)
        for i in range(j_end - 1, -1, -1):
            y[i] = (g[i] - Hm[i, i + 1:j_end] @ y[i + 1:]) / Hm[i, i]
        x = x + Z[:j_end].T @ y
        r = f - A @ x
        beta = np.linalg.norm(r)
        hist[-1] = beta
    return x, its, hist


def pcg(A, f: np.ndarray, precond, rtol: float, maxit: int, x0: np.ndarray | None = None):
    """Preconditioned conjugate gradients in float64 (Hestenes-Stiefel with a symmetric
    positive definite preconditioner; Section 4.1 accelerates the symmetric runs with CG).
    Stops when the recursive residual meets ``rtol ||f||``; returns ``(x, iterations,
    history of residual norms)``, the last entry the true residual norm."""
    A = csr_of(A)
    x = np.zeros(f.size) if x0 is None else x0.astype(np.float64).copy()
    fnorm = np.linalg.norm(f)
    if fnorm == 0.0:
        return np.zeros(f.size), 0, [0.0]
    tol = rtol * fnorm
    r = f - A @ x
    hist = [np.linalg.norm(r)]
    its = 0
    z = precond(r)
    p = z.copy()
    rho = r @ z
    while hist[-1] > tol and its < maxit:
        q = A @ p
        alpha = rho / (p @ q)
        x = x + alpha * p
        r = r - alpha * q
        its += 1
        hist.append(np.linalg.norm(r))
        if hist[-1] <= tol:
            break
        z = precond(r)
        rho_new = r @ z
        p = z + (rho_new / rho) * p
        rho = rho_new
    hist[-1] = np.linalg.norm(f - A @ x)
    return x, its, hist


def operator_complexity(H: Hierarchy) -> float:
    """OC = sum_k nnz(A_k) / nnz(A_0) (Section 4)."""
    return sum(l.A.nnz for l in H.levels) / H.levels[0].A.nnz


def work_per_digit(oc: float, hist: list, its: int) -> tuple[float, float]:
    """gamma = (||r_k|| / ||r_0||)^(1/k) and wpd = 3.5 OC / (-log10 gamma) (Section 4)."""
    gamma = (hist[-1] / hist[0]) ** (1.0 / max(its, 1))
    return gamma, 3.5 * oc / (-math.log10(gamma)) if 0 < gamma < 1 else float("inf")


def solve(A, f: np.ndarray, B: np.ndarray, params: Params):
    """Setup then V(1,1)-preconditioned FGMRES to ``rtol`` relative true residual."""
    H = build_hierarchy(A, B, params)
    x, its, hist = fgmres(A, f, lambda v: vcycle(H, v), params.gmres_restart, params.rtol,
                          params.gmres_maxit)
    return H, x, its, hist
