"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a hand-derived worked
example, a closed form (ideal restriction, Schur complement, exact two-grid), a
brute-force restatement on tiny inputs, or a textbook special case.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def frac_array(rows):
    return np.array([[float(Fraction(x)) for x in r] for r in rows])


def small_problem(nside=6, angle=math.pi / 6, eps=1e-2):
    return O.csr_of(workloads.advdiff_2d(nside, math.cos(angle), math.sin(angle), eps))


def random_sparse(n, density, seed, diag=4.0):
    rng = np.random.default_rng(seed)
    M = sp.random(n, n, density=density, random_state=rng, format="csr")
    M.data = -np.abs(M.data) - 0.01
    M = M + sp.identity(n) * diag
    return O.csr_of(M)


# ---------------------------------------------------------------------------------------
# Worked example (tests/golden/hand_1d_4pt.json)
# ---------------------------------------------------------------------------------------
def test_hand_worked_example():
    g = json.load(open(os.path.join(GOLDEN, "hand_1d_4pt.json")))
    A = O.csr_of(sp.csr_matrix(frac_array(g["A_dense"])))
    cf = np.array(g["cf"], dtype=np.int8)
    B = np.array([float(Fraction(x)) for x in g["B"]])
    p = O.Params(theta_interp=g["theta_interp"], degree=g["degree"])
    P, _ = O.clair_transfer(A, cf, B, p)
    Pt, _ = O.clair_transfer(A.T.tocsr(), cf, B, p)
    R = Pt.T.toarray()
    np.testing.assert_allclose(R, frac_array(g["R"]), rtol=0, atol=1e-15)
    np.testing.assert_allclose(P.toarray(), frac_array(g["P"]), rtol=0, atol=1e-15)
    Ac = R @ A.toarray() @ P.toarray()
    np.testing.assert_allclose(Ac, frac_array(g["A_c"]), rtol=0, atol=1e-14)


# ---------------------------------------------------------------------------------------
# Strength, splitting, aggregation, pattern: brute force on tiny inputs
# ---------------------------------------------------------------------------------------
def strength_bruteforce(Ad, theta):
    n = Ad.shape[0]
    S = np.zeros((n, n), dtype=bool)
    for i in range(n):
        mx = max([abs(Ad[i, k]) for k in range(n) if k != i] + [0.0])
        for j in range(n):
            if j != i and Ad[i, j] != 0 and abs(Ad[i, j]) >= theta * mx:
                S[i, j] = True
    return S


def lowbias32_py(x):
    x &= 0xFFFFFFFF
    x ^= x >> 16
    x = (x * 0x7FEB352D) & 0xFFFFFFFF
    x ^= x >> 15
    x = (x * 0x846CA68B) & 0xFFFFFFFF
    x ^= x >> 16
    return x


def split_bruteforce(Ad, theta):
    S = strength_bruteforce(Ad, theta)
    n = S.shape[0]
    lam = [int(S[:, i].sum()) for i in range(n)]
    key = [(lam[i], lowbias32_py(i)) for i in range(n)]
    nbrs = [[j for j in range(n) if j != i and (S[i, j] or S[j, i])] for i in range(n)]
    state = ["F" if lam[i] == 0 else "U" for i in range(n)]
    while "U" in state:
        new_c = [i for i in range(n) if state[i] == "U"
                 and all(key[i] > key[j] for j in nbrs[i] if state[j] == "U")]
        for i in new_c:
            state[i] = "C"
        for j in range(n):
            if state[j] == "U" and any(S[j, i] for i in new_c):
                state[j] = "F"
    for j in range(n):
        if state[j] == "F" and S[j].any() and not any(S[j, i] and state[i] == "C" for i in range(n)):
            state[j] = "C"
    return np.array([1 if s == "C" else 0 for s in state], dtype=np.int8), S


@pytest.mark.parametrize("seed", range(4))
def test_strength_matches_bruteforce(seed):
    A = random_sparse(30, 0.15, seed)
    for theta in (0.0, 0.25, 0.5, 0.9):
        S = O.strength(A, theta).toarray() != 0
        np.testing.assert_array_equal(S, strength_bruteforce(A.toarray(), theta))


def test_lowbias32_is_the_published_hash():
    xs = np.array([0, 1, 2, 12345, 0xFFFFFFFF, 4096, 2**31 + 7], dtype=np.uint64)
    got = O.lowbias32(xs)
    assert [int(v) for v in got] == [lowbias32_py(int(x)) for x in xs]
    # bijection on a window: no collisions among 2^16 consecutive inputs
    assert np.unique(O.lowbias32(np.arange(70000))).size == 70000


@pytest.mark.parametrize("case", [("rand", 0), ("rand", 1), ("rand", 2), ("adv", 0.0),
                                  ("adv", 1e-2), ("adv", 1.0)])
def test_split_fc_matches_bruteforce(case):
    if case[0] == "rand":
        A = random_sparse(40, 0.1, case[1])
    else:
        A = small_problem(7, eps=case[1])
    cf = O.split_fc(A, 0.25)
    cf_bf, S = split_bruteforce(A.toarray(), 0.25)
    np.testing.assert_array_equal(cf, cf_bf)
    # invariant: every F point with a strong dependence depends on a C point
    for j in np.flatnonzero(cf == 0):
        if S[j].any():
            assert np.any(S[j] & (cf == 1))


def graph_dist(G, src):
    n = G.shape[0]
    d = np.full(n, 10**9)
    d[src] = 0
    frontier = [src]
    while frontier:
        nxt = []
        for u in frontier:
            for v in np.flatnonzero(G[u]):
                if d[v] > d[u] + 1:
                    d[v] = d[u] + 1
                    nxt.append(v)
        frontier = nxt
    return d


@pytest.mark.parametrize("which", [0, 1, 2])
def test_aggregate_properties(which):
    A = [small_problem(8, eps=1.0), small_problem(8, eps=1e-3),
         random_sparse(50, 0.08, 5)][which]
    cf, agg = O.aggregate(A, 0.25)
    S = strength_bruteforce(A.toarray(), 0.25)
    G = S | S.T
    roots = np.flatnonzero(cf == 1)
    # roots are at distance >= 3 from each other (distance-two independent set)
    for r in roots:
        d = graph_dist(G, r)
        assert np.all(d[roots[roots != r]] >= 3)
    # maximality: every non-isolated point is within distance 2 of a root
    dmin = np.min(np.stack([graph_dist(G, r) for r in roots]), axis=0)
    iso = ~G.any(axis=1)
    assert np.all(dmin[~iso] <= 2)
    assert np.all(agg[iso] == -1)
    # aggregate numbering: root r has aggregate = its rank among roots
    np.testing.assert_array_equal(agg[roots], np.arange(roots.size))
    # distance-one points join their unique adjacent root; others an adjacent aggregate
    for j in np.flatnonzero((cf == 0) & ~iso):
        nb = np.flatnonzero(G[j])
        adj_roots = [r for r in nb if cf[r] == 1]
        if adj_roots:
            assert len(adj_roots) == 1 and agg[j] == agg[adj_roots[0]]
        else:
            first = [agg[k] for k in nb if any(cf[r] == 1 for r in np.flatnonzero(G[k]))]
            assert agg[j] == min(first)


def pattern_bruteforce(Ahat, cf, theta, degree):
    """Column i: F-points j reachable from base T by up to degree-1 hops of S+I."""
    S = strength_bruteforce(Ahat.toarray(), theta)
    n = cf.size
    cpts = np.flatnonzero(cf == 1)
    cols = []
    for i in cpts:
        base = {i} | {j for j in range(n) if cf[j] == 0 and S[j, i]}
        reach = set(base)
        for _ in range(degree - 1):
            reach = reach | {j for j in range(n) for k in reach if S[j, k]}
        cols.append(sorted(j for j in reach if cf[j] == 0))
    return cols


@pytest.mark.parametrize("degree", [1, 2, 3])
@pytest.mark.parametrize("eps", [0.0, 1e-2, 1.0])
def test_pattern_matches_bruteforce(degree, eps):
    A = small_problem(7, eps=eps)
    cf = O.split_fc(A, 0.25)
    for Ahat in (A, A.T.tocsr()):
        S = O.strength(Ahat, 0.05)
        T = O.base_pattern(S, cf, "FC")
        W = O.clair_pattern(S, T, cf, degree)
        got = [list(W.indices[W.indptr[i]:W.indptr[i + 1]]) for i in range(W.shape[1])]
        assert got == pattern_bruteforce(Ahat, cf, 0.05, degree)


def agg_pattern_bruteforce(Ahat, agg, cf, theta, degree):
    """Column i of the aggregation-based pattern, written out from its definition
    (Algorithm 1 with T = the aggregation operator of the footnote to Section 3.1.3):
    start from every member of aggregate i (its root included), add j whenever j
    strongly depends on a point already reached, degree-1 times, keep the F-points."""
    S = strength_bruteforce(Ahat.toarray(), theta)
    n = cf.size
    nagg = int(cf.sum())
    cols = []
    for a in range(nagg):
        reach = {j for j in range(n) if agg[j] == a}
        for _ in range(degree - 1):
            reach = reach | {j for j in range(n) if any(S[j, k] for k in reach)}
        cols.append(sorted(j for j in reach if cf[j] == 0))
    return cols


def tiny_3d(nside=4, eps=1e-2):
    vel = lambda x, y, z: (2 * y * (1 - x * x), -2 * x * (1 - y * y), 0.5 + 0 * z)
    return O.csr_of(workloads.advdiff_3d(nside, vel, eps))


@pytest.mark.parametrize("degree", [1, 2, 3])
@pytest.mark.parametrize("which", ["2d_eps1", "2d_eps1e-3", "3d"])
def test_agg_pattern_matches_bruteforce(degree, which):
    """Agg base pattern + expansion (Algorithm 1, T = aggregation operator) against a
    brute-force walk that starts from every aggregate member, for R (A^T) and P (A)."""
    A = {"2d_eps1": lambda: small_problem(8, eps=1.0),
         "2d_eps1e-3": lambda: small_problem(8, eps=1e-3),
         "3d": lambda: tiny_3d(4, 1e-2)}[which]()
    cf, agg = O.aggregate(A, 0.25)
    assert cf.sum() >= 2
    for Ahat in (A, A.T.tocsr()):
        S = O.strength(Ahat, 0.05)
        T = O.base_pattern(S, cf, "AGG", agg)
        # T is the 0/1 aggregation operator itself: column i = members of aggregate i
        Td = T.toarray()
        for a in range(int(cf.sum())):
            np.testing.assert_array_equal(np.flatnonzero(Td[:, a]), np.flatnonzero(agg == a))
        W = O.clair_pattern(S, T, cf, degree)
        got = [list(W.indices[W.indptr[i]:W.indptr[i + 1]]) for i in range(W.shape[1])]
        assert got == agg_pattern_bruteforce(Ahat, agg, cf, 0.05, degree)


def cff_propagator(Ad, cf, omega):
    """Dense error propagator of one CFF sweep with zero right-hand side: a Jacobi sweep
    on the point set X maps x to (I - omega E_X D^-1 A) x, with E_X the 0/1 selector of X;
    CFF applies the C set once, then the F set twice (Section 4)."""
    n = Ad.shape[0]
    Dinv = np.diag(1.0 / np.diag(Ad))
    EC = np.diag((cf == 1).astype(float))
    EF = np.diag((cf == 0).astype(float))
    MC = np.eye(n) - omega * EC @ Dinv @ Ad
    MF = np.eye(n) - omega * EF @ Dinv @ Ad
    return MF @ MF @ MC


@pytest.mark.parametrize("eps", [0.0, 1e-2, 1.0])
def test_smooth_modes_closed_form(eps):
    """B_P = (CFF propagator of A)^5 B and B_R = (CFF propagator of A^T)^5 B on the fine
    level, and the same on level 1 from the injected vectors (Section 4.1 parameters:
    five CFF sweeps per level; A for interpolation, A^T for restriction)."""
    A = small_problem(6, eps=eps)                   # n = 36
    n = A.shape[0]
    B = np.ones(n)
    p = O.Params(coarse_max=4)
    H = O.build_hierarchy(A, B, p)
    assert len(H.levels) >= 3
    Bp, Br = B.copy(), B.copy()
    for k in range(2):
        lev = H.levels[k]
        Ad = lev.A.toarray()
        Mp = np.linalg.matrix_power(cff_propagator(Ad, lev.cf, lev.omega), 5)
        Mr = np.linalg.matrix_power(cff_propagator(Ad.T, lev.cf, lev.omega), 5)
        Bp, Br = Mp @ Bp, Mr @ Br
        scale = max(np.abs(Bp).max(), 1e-300)
        np.testing.assert_allclose(lev.B_P.ravel(), Bp, rtol=0, atol=1e-13 * scale)
        scale = max(np.abs(Br).max(), 1e-300)
        np.testing.assert_allclose(lev.B_R.ravel(), Br, rtol=0, atol=1e-13 * scale)
        if k == 0:  # A is nonsymmetric, so the two sides differ: a swap would fail
            assert np.abs(Bp - Br).max() > 1e-6 * np.abs(Bp).max()
        C = np.flatnonzero(lev.cf == 1)
        Bp, Br = Bp[C], Br[C]
    # with the sweep count taken from the parameters: 2 sweeps give a different vector
    lev = H.levels[0]
    B2 = O.smooth_modes(lev.A, B, lev.cf, lev.omega, 2)
    M2 = np.linalg.matrix_power(cff_propagator(lev.A.toarray(), lev.cf, lev.omega), 2)
    np.testing.assert_allclose(B2, M2 @ B, rtol=0, atol=1e-13)


# ---------------------------------------------------------------------------------------
# Local systems and constraint (Remarks 3.1, 3.2; Eqs. 2.5-2.8, 2.12, 3.3)
# ---------------------------------------------------------------------------------------
def restriction(A, cf, B, p, Wpat=None):
    At = A.T.tocsr()
    if Wpat is None:
        Pt, Wpat = O.clair_transfer(At, cf, B, p)
    else:
        W = O.clair_algorithm1(At, cf, B, Wpat, p)
        cp = np.flatnonzero(cf == 1)
        Pt = (W + sp.csc_matrix((np.ones(cp.size), (cp, np.arange(cp.size))), shape=W.shape)).tocsr()
    return Pt.T.tocsr(), Wpat


def full_f_pattern(cf):
    n = cf.size
    F = np.flatnonzero(cf == 0)
    nc = int(cf.sum())
    rows = np.tile(F, nc)
    cols = np.repeat(np.arange(nc), F.size)
    return sp.csc_matrix((np.ones(rows.size), (rows, cols)), shape=(n, nc))


@pytest.mark.parametrize("eps", [0.0, 1e-2, 1.0])
def test_remark31_lair_local_residual_zero(eps):
    """Constraints off, exact inverse: R A vanishes on each row's F pattern (Eq. 2.7)."""
    A = small_problem(9, eps=eps)
    cf = O.split_fc(A, 0.25)
    p = O.Params(constrain=False)
    R, Wpat = restriction(A, cf, np.ones(A.shape[0]), p)
    RA = (R @ A).toarray()
    scale = np.abs(A).max()
    for i in range(R.shape[0]):
        Zi = Wpat.indices[Wpat.indptr[i]:Wpat.indptr[i + 1]]
        assert np.all(np.abs(RA[i, Zi]) <= 1e-13 * scale)


@pytest.mark.parametrize("eps", [1e-2, 1.0])
def test_full_pattern_gives_ideal_restriction(eps):
    """Pattern = all of F, constraints off: R = R_ideal = [-A_cf A_ff^-1, I] (Eq. 2.5) and
    R A P = Schur complement for any P = [W; I] (Section 2)."""
    A = small_problem(5, eps=eps)
    cf = O.split_fc(A, 0.25)
    F, C = np.flatnonzero(cf == 0), np.flatnonzero(cf == 1)
    Ad = A.toarray()
    Aff, Afc, Acf, Acc = Ad[np.ix_(F, F)], Ad[np.ix_(F, C)], Ad[np.ix_(C, F)], Ad[np.ix_(C, C)]
    p = O.Params(constrain=False)
    R, _ = restriction(A, cf, np.ones(A.shape[0]), p, Wpat=full_f_pattern(cf))
    Rd = R.toarray()
    np.testing.assert_allclose(Rd[:, F], -Acf @ np.linalg.inv(Aff), rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(Rd[:, C], np.eye(C.size), atol=0)
    P, _ = O.clair_transfer(A, cf, np.ones(A.shape[0]), O.Params())
    schur = Acc - Acf @ np.linalg.solve(Aff, Afc)
    np.testing.assert_allclose(Rd @ Ad @ P.toarray(), schur, rtol=1e-11, atol=1e-10 * np.abs(schur).max())


def test_full_pattern_consistent_modes_give_ideal():
    """With B chosen so that R_ideal already meets the constraint, CLAIR = R_ideal."""
    A = small_problem(5, eps=1e-2)
    cf = O.split_fc(A, 0.25)
    F, C = np.flatnonzero(cf == 0), np.flatnonzero(cf == 1)
    Ad = A.toarray()
    rng = np.random.default_rng(3)
    B = np.zeros(A.shape[0])
    B[C] = rng.uniform(0.5, 1.5, C.size)
    # B_F := Z^T B_c with Z = -A_cf A_ff^-1, so sum_i z_ij B_c(i) = B_j holds
    Z = -Ad[np.ix_(C, F)] @ np.linalg.inv(Ad[np.ix_(F, F)])
    B[F] = Z.T @ B[C]
    R, _ = restriction(A, cf, B, O.Params(), Wpat=full_f_pattern(cf))
    np.testing.assert_allclose(R.toarray()[:, F], Z, rtol=1e-11, atol=1e-12)


@pytest.mark.parametrize("eps", [0.0, 1e-2, 1.0])
def test_constraint_is_min_norm_projection_of_lair(eps):
    """Algorithm 1 (exact inverse) = the Euclidean projection of the lAIR weights onto
    {w : Q w = B|_F}, checked with one dense global KKT solve built from an explicit Q
    (Eq. 3.3), plus the constraint itself."""
    A = small_problem(6, eps=eps)
    n = A.shape[0]
    cf = O.split_fc(A, 0.25)
    C = np.flatnonzero(cf == 1)
    B = 0.5 + workloads.uniform01(9, n)
    At = A.T.tocsr()
    S = O.strength(At, 0.05)
    Wpat = O.clair_pattern(S, O.base_pattern(S, cf, "FC"), cf, 2)
    w_lair = O.clair_algorithm1(At, cf, B, Wpat, O.Params(constrain=False)).tocsc()
    w_cl = O.clair_algorithm1(At, cf, B, Wpat, O.Params()).tocsc()
    # explicit Q: one row per F point with a nonempty pattern row, columns = CSC entries
    col_of_entry = np.repeat(np.arange(Wpat.shape[1]), np.diff(Wpat.indptr))
    row_of_entry = Wpat.indices
    Frows = np.unique(row_of_entry)
    Q = np.zeros((Frows.size, row_of_entry.size))
    for e in range(row_of_entry.size):
        Q[np.searchsorted(Frows, row_of_entry[e]), e] = B[C[col_of_entry[e]]]
    b = B[Frows]
    m = Q.shape[1]
    K = np.block([[np.eye(m), Q.T], [Q, np.zeros((Q.shape[0], Q.shape[0]))]])
    rhs = np.concatenate([w_lair.data, b])
    sol = np.linalg.lstsq(K, rhs, rcond=None)[0][:m]
    np.testing.assert_allclose(w_cl.data, sol, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(Q @ w_cl.data, b, rtol=1e-12, atol=1e-13)


def test_remark32_second_iteration_is_noop():
    A = small_problem(8, eps=1e-2)
    cf = O.split_fc(A, 0.25)
    B = 0.5 + workloads.uniform01(11, A.shape[0])
    R1, _ = restriction(A, cf, B, O.Params(iterations=1))
    R3, _ = restriction(A, cf, B, O.Params(iterations=3))
    np.testing.assert_allclose(R3.toarray(), R1.toarray(), rtol=1e-12, atol=1e-13)


def test_output_independent_of_tentative_for_exact_inverse():
    """With the exact inverse the result is the projection of lAIR regardless of w_t: the
    diagonal-inverse iteration converged far differs, the exact one does not move."""
    A = small_problem(6, eps=1.0)
    cf = O.split_fc(A, 0.25)
    B = np.ones(A.shape[0])
    Rd, _ = restriction(A, cf, B, O.Params(inverse="diag", iterations=1))
    Re, _ = restriction(A, cf, B, O.Params())
    assert np.abs((Rd - Re).toarray()).max() > 1e-3
    Wsum = np.asarray(Rd.sum(axis=0)).ravel()   # constraint still met with the diag inverse
    F = np.flatnonzero(cf == 0)
    has = np.diff(Rd.tocsc().indptr)[F] > 0
    np.testing.assert_allclose(Wsum[F][has], 1.0, rtol=1e-12)


# ---------------------------------------------------------------------------------------
# Relaxation, weight, two-grid cycle, Krylov
# ---------------------------------------------------------------------------------------
def test_relax_first_sweep_from_zero_closed_form():
    A = small_problem(5, eps=1e-2)
    n = A.shape[0]
    b = workloads.uniform_pm1(1, n)
    mask = np.arange(n) % 3 == 0
    x = O.relax(A, np.zeros(n), b, mask, 0.7)
    expect = np.where(mask, 0.7 * b / A.diagonal(), 0.0)
    np.testing.assert_allclose(x, expect, rtol=1e-15)


@pytest.mark.parametrize("nside", [3, 4])
def test_arnoldi_rho_symmetric_laplacian(nside):
    """D^-1 A for the 5-point Laplacian has eigenvalues 1 - (cos(k pi h) + cos(l pi h))/2;
    rho = 1 + cos(pi h).  With n <= 15 Arnoldi spans the whole space (exact Ritz values)."""
    A = O.csr_of(workloads.advdiff_2d(nside, 0.0, 0.0, 1.0))
    rho = O.arnoldi_rho(A, 15, 123)
    assert abs(rho - (1 + math.cos(math.pi / (nside + 1)))) < 1e-10


def test_arnoldi_rho_nonsymmetric_closed_form():
    """Constant-coefficient upwind advection-diffusion is a Kronecker sum of tridiagonal
    Toeplitz matrices T = tridiag(-a, d, -c) with eigenvalues d - 2 sqrt(ac) cos(k pi/(m+1));
    the diagonal is constant, so rho(D^-1 A) = (d_x + d_y + 2 (sqrt(a_x c_x) + sqrt(a_y c_y))
    cos(pi/(m+1))) / (d_x + d_y).  n = 9 <= 15 makes the Arnoldi Ritz values exact."""
    m, eps, ang = 3, 0.1, math.pi / 6
    vx, vy = math.cos(ang), math.sin(ang)
    h = 1.0 / (m + 1)
    A = O.csr_of(workloads.advdiff_2d(m, vx, vy, eps))
    e = eps / h**2
    ax, cx, ay, cy = e + vx / h, e, e + vy / h, e
    d = 4 * e + (vx + vy) / h
    rho = (d + 2 * (math.sqrt(ax * cx) + math.sqrt(ay * cy)) * math.cos(math.pi / (m + 1))) / d
    assert abs(O.arnoldi_rho(A, 15, 5) - rho) < 1e-10


def test_arnoldi_basis_orthonormal_and_relation_holds():
    """The Arnoldi pair of Section 4 on a small, strongly non-normal operator (5 x 5 upwind
    advection-diffusion, eps = 1e-3, 15 steps on 25 unknowns, so the Krylov space nearly
    closes): the basis is orthonormal to working precision and D^-1 A V_m = V_{m+1} H.  A
    single modified Gram-Schmidt pass leaves this basis non-orthogonal to about 3e-3, so
    the pin holds the two-pass orthogonalisation."""
    A = O.csr_of(workloads.advdiff_2d(5, math.cos(math.pi / 6), math.sin(math.pi / 6), 1e-3))
    H, V, steps = O.arnoldi(A, 15, 7)
    assert steps == 15
    Vm = V[:steps]
    assert np.abs(Vm @ Vm.T - np.eye(steps)).max() < 1e-13
    M = sp.diags(1.0 / A.diagonal()) @ A
    lhs = (M @ Vm.T).T
    rhs = H[: steps + 1, :steps].T @ V[: steps + 1]
    assert np.abs(lhs - rhs).max() < 1e-12 * np.abs(lhs).max()


def dense_two_grid(H):
    """E = S_post (I - P A_c^-1 R A) S_pre assembled from dense sweep propagators."""
    lev = H.levels[0]
    A = lev.A.toarray()
    n = A.shape[0]
    D = np.diag(A)
    I = np.eye(n)

    def sweep(mask, w):
        return I - w * np.diag(mask.astype(float) / D) @ A

    c = lev.cf == 1
    Spre = sweep(~c, lev.omega) @ sweep(~c, lev.omega) @ sweep(c, lev.omega)
    wp = lev.omega if H.params.post_weighted else 1.0
    Spost = sweep(c, wp) @ sweep(~c, wp) @ sweep(~c, wp)
    P, R = lev.P.toarray(), lev.R.toarray()
    cgc = I - P @ np.linalg.solve(R @ A @ P, R @ A)
    return Spost @ cgc @ Spre


@pytest.mark.parametrize("eps", [0.0, 1e-2, 1.0])
def test_two_grid_cycle_matches_dense_error_propagation(eps):
    """Eq. 1.2 with pre- and post-smoothing: u - V(A u) = E_TG u for unit vectors u."""
    A = small_problem(8, eps=eps)
    p = O.Params(max_levels=2, coarse_max=4)
    H = O.build_hierarchy(A, np.ones(A.shape[0]), p)
    assert len(H.levels) == 2
    E = dense_two_grid(H)
    n = A.shape[0]
    Ad = A.toarray()
    for j in range(0, n, 7):
        u = np.zeros(n)
        u[j] = 1.0
        got = u - O.vcycle(H, Ad @ u)
        np.testing.assert_allclose(got, E[:, j], atol=1e-11)


def test_ideal_restriction_exact_two_grid_for_triangular_advection():
    """eps = 0 with velocity angle pi/6: A is lower triangular (lexicographic order).  With
    R = R_ideal (full F pattern, no constraint), the coarse correction leaves e_c = 0 and
    n_f F-Jacobi sweeps with weight 1 (nilpotent on triangular A_ff) remove the rest:
    the two-grid error propagation is zero (R_ideal A = (0, S), Section 2.1)."""
    A = small_problem(5, eps=0.0)
    Ad = A.toarray()
    assert np.allclose(np.triu(Ad, 1), 0)
    n = A.shape[0]
    cf = O.split_fc(A, 0.25)
    R, _ = restriction(A, cf, np.ones(n), O.Params(constrain=False), Wpat=full_f_pattern(cf))
    P, _ = O.clair_transfer(A, cf, np.ones(n), O.Params())
    Rd, Pd = R.toarray(), P.toarray()
    F = cf == 0
    E = np.eye(n) - Pd @ np.linalg.solve(Rd @ Ad @ Pd, Rd @ Ad)
    for _ in range(int(F.sum())):
        E = (np.eye(n) - np.diag(F / np.diag(Ad)) @ Ad) @ E
    assert np.abs(E).max() < 1e-10


def test_fgmres_identity_preconditioner_solves_dense_system():
    rng = np.random.default_rng(0)
    M = np.eye(40) * 5 + rng.standard_normal((40, 40)) * 0.3
    f = rng.standard_normal(40)
    x, its, hist = O.fgmres(sp.csr_matrix(M), f, lambda v: v, 50, 1e-12, 100)
    np.testing.assert_allclose(x, np.linalg.solve(M, f), rtol=1e-10)
    assert hist[-1] <= 1e-12 * np.linalg.norm(f)


def test_fgmres_converges_in_number_of_distinct_eigenvalues():
    d = np.repeat([1.0, 2.0, 5.0], 20)
    f = workloads.uniform_pm1(4, d.size)
    x, its, _ = O.fgmres(sp.diags(d).tocsr(), f, lambda v: v, 50, 1e-10, 100)
    assert its == 3
    np.testing.assert_allclose(x, f / d, rtol=1e-9)


def test_fgmres_restart_acts_as_refinement():
    A = small_problem(12, eps=1e-2)
    f = workloads.uniform_pm1(2, A.shape[0])
    x, its, hist = O.fgmres(A, f, lambda v: v / A.diagonal(), 5, 1e-10, 400)
    assert np.linalg.norm(f - A @ x) <= 1e-10 * np.linalg.norm(f)


def test_operator_complexity_and_wpd():
    H = O.Hierarchy([], O.Params())
    H.levels = [type("X", (), {"A": sp.random(10, 10, density=d, random_state=1, format="csr")})()
                for d in (0.5, 0.3, 0.1)]
    oc = O.operator_complexity(H)
    assert oc == pytest.approx(sum(l.A.nnz for l in H.levels) / H.levels[0].A.nnz)
    gamma, wpd = O.work_per_digit(2.0, [1.0, 1e-2, 1e-4], 2)
    assert gamma == pytest.approx(1e-2)
    assert wpd == pytest.approx(3.5 * 2.0 / 2.0)


# ---------------------------------------------------------------------------------------
# Whole solver on the small workload
# ---------------------------------------------------------------------------------------
def test_solve_small_workload_reaches_tolerance():
    prob = workloads.config1()
    H, x, its, hist = O.solve(prob.A, prob.f, prob.B, O.Params())
    A = O.csr_of(prob.A)
    assert np.linalg.norm(prob.f - A @ x) <= 1e-8 * np.linalg.norm(prob.f)
    assert its <= 15
    # every P satisfies P B_c = B on F rows with a nonempty pattern (Eq. 2.12)
    for lev in H.levels[:-1]:
        C = np.flatnonzero(lev.cf == 1)
        PB = lev.P @ lev.B_P[C, 0]
        has = np.diff(lev.P.indptr) > 0
        np.testing.assert_allclose(PB[has], lev.B_P[has, 0], rtol=1e-12, atol=1e-14)
        RtB = lev.R.T @ lev.B_R[C, 0]
        hasr = np.diff(lev.R.tocsc().indptr) > 0
        np.testing.assert_allclose(RtB[hasr], lev.B_R[hasr, 0], rtol=1e-12, atol=1e-14)


def test_workload_generators():
    """Upwind FD: eps > 0, v = 0 gives the symmetric 5-point Laplacian / h^2; row sums of
    interior rows vanish for pure advection and diffusion alike."""
    A = O.csr_of(workloads.advdiff_2d(4, 0.0, 0.0, 1.0))
    T = sp.diags([-1.0, 2.0, -1.0], [-1, 0, 1], shape=(4, 4))
    L = (sp.kron(sp.identity(4), T) + sp.kron(T, sp.identity(4))) * 25.0
    np.testing.assert_allclose(A.toarray(), L.toarray())
    A = O.csr_of(workloads.advdiff_2d(6, 0.3, -0.8, 1e-2))
    rs = np.asarray(A.sum(axis=1)).ravel().reshape(6, 6)
    np.testing.assert_allclose(rs[1:-1, 1:-1], 0.0, atol=1e-10)
    u = workloads.uniform_pm1(7, 1000)
    assert u.min() >= -1 and u.max() < 1 and abs(u.mean()) < 0.1
    # splitmix64 reference values (sequential generator seeded with 0)
    z = workloads.splitmix64(0, 3)
    assert [hex(int(v)) for v in z] == ["0xe220a8397b1dcdaf", "0x6e789e6aa1b965f4", "0x6c45d188009454f"]


def test_algorithm1_on_column_subset_matches_full_run():
    """Running Algorithm 1 on the columns that touch a sample's F rows reproduces the full
    run on the sampled columns (used by the full-size GPU parity test)."""
    A = small_problem(10, eps=1e-2)
    At = A.T.tocsr()
    cf = O.split_fc(A, 0.25)
    B = 0.5 + workloads.uniform01(13, A.shape[0])
    S = O.strength(At, 0.05)
    Wpat = O.clair_pattern(S, O.base_pattern(S, cf, "FC"), cf, 2).tocsc()
    full = O.clair_algorithm1(At, cf, B, Wpat, O.Params()).tocsc()
    cpts = np.flatnonzero(cf)
    Wr = Wpat.tocsr()
    sample = np.array([1, 5, 9, 17])
    rows = np.unique(np.concatenate([Wpat.indices[Wpat.indptr[i]:Wpat.indptr[i + 1]] for i in sample]))
    cols = np.unique(np.concatenate([Wr.indices[Wr.indptr[j]:Wr.indptr[j + 1]] for j in rows]))
    sub = O.clair_algorithm1(At, cf, B, Wpat[:, cols], O.Params(), cpts=cpts[cols]).tocsc()
    for i in sample:
        k = int(np.searchsorted(cols, i))
        np.testing.assert_array_equal(sub.indices[sub.indptr[k]:sub.indptr[k + 1]],
                                      full.indices[full.indptr[i]:full.indptr[i + 1]])
        np.testing.assert_allclose(sub.data[sub.indptr[k]:sub.indptr[k + 1]],
                                   full.data[full.indptr[i]:full.indptr[i + 1]], rtol=1e-13, atol=1e-15)


# ---------------------------------------------------------------------------------------
# Several mode vectors (Eq. 3.3 with k > 1), diagonal block inverses (Section 3.1.2),
# the symmetric variant R = P^T with CG (Section 4.1)
# ---------------------------------------------------------------------------------------
def explicit_Q(Wpat, Bc, Bfull):
    """Dense Q of Eq. 3.3 for k modes: one row per (F row j with a nonempty pattern row,
    mode a); Q[(j, a), e] = B_c(i_e, a) for every pattern entry e = (j, i_e)."""
    col_of_entry = np.repeat(np.arange(Wpat.shape[1]), np.diff(Wpat.indptr))
    row_of_entry = Wpat.indices
    Frows = np.unique(row_of_entry)
    k = Bc.shape[1]
    Q = np.zeros((Frows.size * k, row_of_entry.size))
    for e in range(row_of_entry.size):
        r = np.searchsorted(Frows, row_of_entry[e])
        for a in range(k):
            Q[r * k + a, e] = Bc[col_of_entry[e], a]
    b = np.concatenate([Bfull[j, :] for j in Frows])
    return Q, b


@pytest.mark.parametrize("eps", [0.0, 1e-2, 1.0])
def test_two_modes_constraint_is_min_norm_projection_of_lair(eps):
    """k = 2 (constants and the x coordinate): Algorithm 1 with the exact inverse = the
    Euclidean projection of the lAIR weights onto {Q w = B|_F} (dense global least-norm
    solve), where |J_j| may be 1 < k (the pseudo-inverse case of the least-squares step)."""
    A = small_problem(7, eps=eps)
    n = A.shape[0]
    cf = O.split_fc(A, 0.25)
    C = np.flatnonzero(cf == 1)
    x = (np.arange(n) % 7 + 1) / 8.0
    B = np.stack([np.ones(n), x], axis=1)
    At = A.T.tocsr()
    S = O.strength(At, 0.05)
    Wpat = O.clair_pattern(S, O.base_pattern(S, cf, "FC"), cf, 2)
    w_lair = O.clair_algorithm1(At, cf, B, Wpat, O.Params(constrain=False)).tocsc()
    w_cl = O.clair_algorithm1(At, cf, B, Wpat, O.Params()).tocsc()
    Q, b = explicit_Q(Wpat, B[C], B)
    # min ||w - w_lair|| s.t. Q w = b, least squares where Q w = b has no solution
    sol = w_lair.data - np.linalg.pinv(Q) @ (Q @ w_lair.data - b)
    np.testing.assert_allclose(w_cl.data, sol, rtol=1e-10, atol=1e-12)
    # rows whose pattern holds two or more C-points with independent modes meet both
    rank_full = np.array([np.linalg.matrix_rank(Q[2 * r:2 * r + 2]) == 2 for r in range(Q.shape[0] // 2)])
    res = (Q @ w_cl.data - b).reshape(-1, 2)
    assert rank_full.sum() > 0
    np.testing.assert_allclose(res[rank_full], 0.0, atol=1e-12)


@pytest.mark.parametrize("eps", [0.0, 1e-2, 1.0])
@pytest.mark.parametrize("iters", [1, 3])
def test_diag_inverse_equals_exact_on_diagonal_blocks(eps, iters):
    """Degree-1 patterns on the 5-point operator hold F-points that are not neighbours of
    one another, so every local block is diagonal: the diagonal inverse is then the exact
    inverse and Algorithm 1 gives the exact-inverse result for any loop count."""
    A = small_problem(8, eps=eps)
    n = A.shape[0]
    cf = O.split_fc(A, 0.25)
    B = 0.5 + workloads.uniform01(9, n)
    for Ahat in (A, A.T.tocsr()):
        S = O.strength(Ahat, 0.05)
        Wpat = O.clair_pattern(S, O.base_pattern(S, cf, "FC"), cf, 1)
        Ad = Ahat.toarray()
        for i in range(Wpat.shape[1]):
            Z = Wpat.indices[Wpat.indptr[i]:Wpat.indptr[i + 1]]
            M = Ad[np.ix_(Z, Z)]
            assert np.all(M == np.diag(np.diag(M)))
        we = O.clair_algorithm1(Ahat, cf, B, Wpat, O.Params(degree=1)).toarray()
        wd = O.clair_algorithm1(Ahat, cf, B, Wpat, O.Params(degree=1, inverse="diag",
                                                            iterations=iters)).toarray()
        np.testing.assert_allclose(wd, we, rtol=0, atol=1e-14 * np.abs(we).max())


@pytest.mark.parametrize("eps", [1e-2, 1.0])
def test_diag_inverse_iteration_reaches_its_fixed_point(eps):
    """The diagonal-inverse loop converges to the w with Q w = B|_F whose block residual,
    scaled by D^-1, lies in the range of Q^T: A_ff* w + D* Q^T lam = -a_fc*, Q w = B|_F,
    solved here as one dense system; one pass is not yet there."""
    A = small_problem(6, eps=eps)
    n = A.shape[0]
    cf = O.split_fc(A, 0.25)
    C = np.flatnonzero(cf == 1)
    B = 0.5 + workloads.uniform01(9, n)
    At = A.T.tocsr()
    Ad = At.toarray()
    S = O.strength(At, 0.05)
    Wpat = O.clair_pattern(S, O.base_pattern(S, cf, "FC"), cf, 2)
    ne = Wpat.nnz
    Ablk = np.zeros((ne, ne))
    a = np.zeros(ne)
    d = np.zeros(ne)
    for i in range(Wpat.shape[1]):
        lo, hi = Wpat.indptr[i], Wpat.indptr[i + 1]
        Z = Wpat.indices[lo:hi]
        Ablk[lo:hi, lo:hi] = Ad[np.ix_(Z, Z)]
        a[lo:hi] = Ad[Z, C[i]]
        d[lo:hi] = np.diag(Ad)[Z]
    Q, b = explicit_Q(Wpat, B[C].reshape(-1, 1), B.reshape(-1, 1))
    m = Q.shape[0]
    K = np.block([[Ablk, np.diag(d) @ Q.T], [Q, np.zeros((m, m))]])
    fixed = np.linalg.lstsq(K, np.concatenate([-a, b]), rcond=None)[0][:ne]
    w_many = O.clair_algorithm1(At, cf, B, Wpat, O.Params(inverse="diag", iterations=300)).tocsc()
    np.testing.assert_allclose(w_many.data, fixed, rtol=1e-9, atol=1e-11)
    w_one = O.clair_algorithm1(At, cf, B, Wpat, O.Params(inverse="diag", iterations=1)).tocsc()
    assert np.abs(w_one.data - fixed).max() > 1e-6
    np.testing.assert_allclose(Q @ w_one.data, b, atol=1e-12)


def test_pcg_textbook_cases():
    """CG with the identity preconditioner on an SPD matrix with three distinct eigenvalues
    converges in three steps; with the exact inverse as preconditioner in one."""
    rng = np.random.default_rng(4)
    Qm, _ = np.linalg.qr(rng.standard_normal((12, 12)))
    lam = np.array([1.0] * 4 + [3.0] * 4 + [10.0] * 4)
    M = sp.csr_matrix(Qm @ np.diag(lam) @ Qm.T)
    f = rng.standard_normal(12)
    x, its, hist = O.pcg(M, f, lambda v: v, 1e-12, 50)
    assert its == 3
    np.testing.assert_allclose(M @ x, f, atol=1e-10)
    Minv = np.linalg.inv(M.toarray())
    x, its, _ = O.pcg(M, f, lambda v: Minv @ v, 1e-12, 50)
    assert its == 1


def poisson_2d(nside):
    return O.csr_of(workloads.advdiff_2d(nside, 0.0, 0.0, 1.0))


def diffusion_params(**kw):
    """Section 4.1's symmetric CLAIR parameters: strength 0.5 / 0.5, degree 2, B = 1 with
    5 CFF sweeps, R = P^T, aggregation; symmetric smoothing weights for CG."""
    d = dict(theta_coarsen=0.5, theta_interp=0.5, degree=2, coarsen="AGG", symmetric=True,
             post_weighted=True)
    d.update(kw)
    return O.Params(**d)


def test_symmetric_variant_gives_symmetric_preconditioner():
    """R = P^T and weighted FFC post-smoothing make the V(1,1) cycle a symmetric operator
    for symmetric A (the adjoint of CFF pre-smoothing), which CG needs: the dense matrix of
    the cycle is symmetric and positive definite, and every A_c is symmetric."""
    A = poisson_2d(8)
    n = A.shape[0]
    H = O.build_hierarchy(A, np.ones(n), diffusion_params(coarse_max=10))
    assert len(H.levels) >= 2
    for lev in H.levels[:-1]:
        np.testing.assert_array_equal(lev.R.toarray(), lev.P.T.toarray())
    for lev in H.levels:
        Ad = lev.A.toarray()
        np.testing.assert_allclose(Ad, Ad.T, atol=1e-13 * np.abs(Ad).max())
    Mi = np.stack([O.vcycle(H, e) for e in np.eye(n)], axis=1)
    np.testing.assert_allclose(Mi, Mi.T, atol=1e-12 * np.abs(Mi).max())
    assert np.linalg.eigvalsh(0.5 * (Mi + Mi.T)).min() > 0
    f = workloads.uniform_pm1(3, n)
    x, its, hist = O.pcg(A, f, lambda v: O.vcycle(H, v), 1e-10, 100)
    assert hist[-1] <= 1e-10 * np.linalg.norm(f) and its < 20
