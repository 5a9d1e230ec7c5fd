"""GPU parity at the full 1024^2 size of the bench workload, in the bench's configuration.

* Bench workload (eps 1e-2, m 2), FP64 and MIXED setups: the level-0 splitting is
  compared in full (bit-exact), the relaxation weight and both smoothed mode vectors in
  full, and the R and P weights on a seeded sample of coarse points.  The oracle computes
  the sampled weights exactly by running Algorithm 1 on the columns that touch the
  sample's F rows (every step of the algorithm is local to a column block or an F row).
* The other eps and m variants of the workload: properties that hold at any size (the
  mode constraint on every F column / row, the splitting invariant, every coarse operator
  equal to the Galerkin product of its level's R, A and P) and, where the method reaches
  it, convergence to the 1e-8 true residual with iteration counts within one.
Tolerances as in test_gpu_parity.py.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
import workloads

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
FP32_TOL = 2e-5
OMEGA_TOL = 1e-8
NSAMPLE = 160


@pytest.fixture(scope="module")
def cl():
    import torch
    from paper_2307_00229_gb300 import clair
    clair.load()
    torch.cuda.init()
    return clair


def dev(a, dtype):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def setup_gpu(cl, prob, precision, degree=2, sweeps=5, maxit=None):
    import torch
    p = cl.clair_params_default()
    p.precision = precision
    p.degree = degree
    p.b_smooth_iters = sweeps
    if maxit:
        p.gmres_maxit = maxit
    A = prob.A
    h = cl.clair_setup(dev(A.rowptr, torch.int32), dev(A.col, torch.int32),
                       dev(A.val, torch.float64), dev(prob.B, torch.float64), p)
    return h


def level0(cl, h, k=0):
    import torch
    torch.cuda.synchronize()
    v = cl.clair_level_view(h, k)
    out = {k: (x.cpu().numpy() if hasattr(x, "cpu") else x) for k, x in v.items()}
    n, nc = out["n"], out["nc"]
    out["A"] = sp.csr_matrix((out["A_val"], out["A_col"], out["A_rowptr"]), shape=(n, n))
    if nc:
        out["R"] = sp.csr_matrix((out["R_val"], out["R_col"], out["R_rowptr"]), shape=(nc, n))
        out["P"] = sp.csr_matrix((out["P_val"], out["P_col"], out["P_rowptr"]), shape=(n, nc))
    return out


def check_galerkin(cl, h):
    """Every coarse operator is the Galerkin product of its level (Section 2): (R A) P
    entry by entry to rounding, relative to the row's largest entry.  An entry whose
    products cancel may sum to an exact zero (dropped) in one summation order and to a
    rounding-size value in another, so the comparison runs over the union of both
    sparsity patterns and the patterns may differ only in such entries (pure advection
    with m = 1 leaves ~0.3% of the level-1 entries at rounding size).  At full size the
    coarse rows are long enough to reach every tier of the sparse product."""
    nlev = cl.clair_stats(h).levels
    prev = level0(cl, h, 0)
    for k in range(1, nlev):
        cur = level0(cl, h, k)
        ref = ((prev["R"] @ prev["A"]) @ prev["P"]).tocsr()
        ref.eliminate_zeros()
        Ac = cur["A"]
        assert Ac.shape == ref.shape, k
        D = (Ac - ref).tocoo()
        scale = np.abs(ref).max(axis=1).toarray().ravel()
        assert np.all(np.abs(D.data) <= 1e-12 * scale[D.row]), k
        prev = cur


@pytest.fixture(scope="module")
def bench_oracle():
    """Level-0 oracle quantities of the bench workload (1024^2, eps 1e-2, m 2)."""
    prob = workloads.config2()
    A = O.csr_of(prob.A)
    At = A.T.tocsr()
    At.sort_indices()
    p = O.Params()
    cf = O.split_fc(A, p.theta_coarsen)
    omega = 1.0 / O.arnoldi_rho(A, p.arnoldi_iters, p.seed)
    B = prob.B.reshape(-1, 1)
    B_P = O.smooth_modes(A, B, cf, omega, p.b_smooth_iters)[:, 0]
    B_R = O.smooth_modes(At, B, cf, omega, p.b_smooth_iters)[:, 0]
    pats = {}
    for side, Ahat in (("R", At), ("P", A)):
        S = O.strength(Ahat, p.theta_interp)
        pats[side] = O.clair_pattern(S, O.base_pattern(S, cf, "FC"), cf, p.degree)
    rng = np.random.default_rng(2024)
    nc = int(cf.sum())
    sample = np.sort(rng.choice(nc, NSAMPLE, replace=False))
    return {"prob": prob, "A": A, "At": At, "cf": cf, "omega": omega, "B_P": B_P, "B_R": B_R,
            "pats": pats, "sample": sample}


def sampled_columns(Ahat, cf, B, Wpat, sample):
    """Exact Algorithm 1 weights of the sampled columns: {column: (rows, values)}."""
    cpts = np.flatnonzero(cf)
    Wc = Wpat.tocsc()
    Wr = Wpat.tocsr()
    rows = np.unique(np.concatenate([Wc.indices[Wc.indptr[i]:Wc.indptr[i + 1]] for i in sample]))
    cols = np.unique(np.concatenate([Wr.indices[Wr.indptr[j]:Wr.indptr[j + 1]] for j in rows]))
    W = O.clair_algorithm1(Ahat, cf, B, Wc[:, cols], O.Params(), cpts=cpts[cols]).tocsc()
    pos = {c: k for k, c in enumerate(cols)}
    out = {}
    for i in sample:
        k = pos[i]
        out[i] = (W.indices[W.indptr[k]:W.indptr[k + 1]], W.data[W.indptr[k]:W.indptr[k + 1]])
    return out


@pytest.mark.parametrize("precision", [0, 1])
def test_bench_workload_level0_matches_oracle(cl, bench_oracle, precision):
    o = bench_oracle
    h = setup_gpu(cl, o["prob"], precision)
    try:
        g = level0(cl, h)
    finally:
        cl.clair_free(h)
    assert np.array_equal(g["cf"], o["cf"]), "splitting differs at full size"
    dom = abs(g["omega"] - o["omega"]) / o["omega"]
    assert dom <= OMEGA_TOL, dom
    tol = FP64_TOL + 100 * dom
    for key in ("B_P", "B_R"):
        assert np.abs(g[key] - o[key]).max() <= tol * np.abs(o[key]).max(), key
    wtol = tol if precision == 0 else FP32_TOL
    cpts = np.flatnonzero(o["cf"])
    Pt = g["P"].T.tocsr()
    for side, Ahat, Bv, Z in (("R", o["At"], o["B_R"], g["R"]), ("P", o["A"], o["B_P"], Pt)):
        ref = sampled_columns(Ahat, o["cf"], Bv, o["pats"][side], o["sample"])
        worst = 0.0
        for i, (rows, vals) in ref.items():
            s, e = Z.indptr[i], Z.indptr[i + 1]
            cols, gv = Z.indices[s:e], Z.data[s:e]
            keep = cols != cpts[i]
            assert np.array_equal(cols[keep], rows), (side, i)
            assert gv[~keep].tolist() == [1.0]
            if vals.size:
                worst = max(worst, np.abs(gv[keep] - vals).max() / np.abs(vals).max())
        assert worst <= wtol, (side, worst)


# (eps, m, B smoothing sweeps, precisions asserted to reach the 1e-8 true residual).
# With the five CFF sweeps per level of Section 4, pure or nearly pure advection drives
# the smoothed mode vector toward zero by about (1 - omega)^5 per level (the inflow
# boundary holds u = 0), so coarse-level B spans ~20 decades and the projected weights
# reach ~1e13 (oracle, 256^2, eps 0: min B 1e-21 on level 5).  An FP32 V-cycle cannot
# carry that range: MIXED solves there switch to the FP64 cycle when the FP32 cycle
# stalls (clair_stats_t.fp64_cycle_from), and FP64 itself does not reach 1e-8 within
# gmres_maxit for eps = 0, m = 2.  With B = 1 unsmoothed the same hierarchies converge in
# both precisions.
VARIANTS = [
    (1e-2, 1, 5, (0, 1)),
    (1.0, 2, 5, (0, 1)),
    (1e-4, 2, 5, (0, 1)),
    (0.0, 1, 5, (0, 1)),
    (0.0, 2, 5, (1,)),
    (0.0, 2, 0, (0, 1)),
    (0.0, 1, 0, (0, 1)),
]


@pytest.mark.parametrize("eps,degree,sweeps,converge", VARIANTS)
def test_full_size_properties(cl, eps, degree, sweeps, converge):
    import torch
    prob = workloads.config2(eps=eps, degree=degree)
    A = O.csr_of(prob.A)
    its, fell_back = {}, {}
    for precision in (0, 1):
        # pure advection: D^-1 A is I plus a nilpotent part, the coarse levels' Arnoldi
        # weights are set by rounding (see omega_spread) and the FP64 iteration count moves
        # with them (150 to 230 seen), so that case gets a larger iteration budget
        h = setup_gpu(cl, prob, precision, degree, sweeps, maxit=400 if eps == 0.0 else None)
        try:
            g = level0(cl, h)
            check_galerkin(cl, h)
            if precision in converge:
                f = dev(prob.f, torch.float64)
                u = torch.zeros_like(f)
                st, it, rel = cl.clair_solve(h, f, u)
                uh = u.cpu().numpy()
                assert np.linalg.norm(prob.f - A @ uh) <= 1e-8 * np.linalg.norm(prob.f)
                its[precision] = it
                fell_back[precision] = cl.clair_stats(h).fp64_cycle_from >= 0
        finally:
            cl.clair_free(h)
        cf = g["cf"].astype(bool)
        cpts = np.flatnonzero(cf)
        # the mode constraint sum_i R_ij B_c(i) = B(j), sum_i P_ji B_c(i) = B(j) on F, to
        # rounding relative to sum_i |w| |B_c(i)|
        for key, M in (("B_R", g["R"].T.tocsr()), ("B_P", g["P"])):
            Bv = g[key]
            lhs = M @ Bv[cpts]
            mag = np.asarray(abs(M) @ np.abs(Bv[cpts])).ravel()
            sel = ~cf & (np.diff(M.indptr) > 0) & (mag > 0)
            assert np.all(np.abs(lhs[sel] - Bv[sel]) <= 1e-12 * mag[sel]), key
        # splitting invariant: every F-point with a strong dependence depends on a C-point
        S = O.strength(A, 0.25)
        has = np.diff(S.indptr) > 0
        dep_c = (S @ cf.astype(np.float64)) > 0
        assert not np.any(~cf & has & ~dep_c)
    if len(its) == 2 and not fell_back[1]:
        assert abs(its[0] - its[1]) <= 1, its


def omega_spread(A, iters, seed, trials=2):
    """Largest relative change of the oracle's weight when A's values are scaled entry by
    entry by 1 + 1e-15 r (r uniform in [-1, 1], seeded): the part of omega that FP64
    arithmetic does not determine.  Nearly pure advection makes D^-1 A close to I plus a
    nilpotent part, whose Ritz values move like the k-th root of a perturbation; on such
    a level no two summation orders need agree."""
    ref = 1.0 / O.arnoldi_rho(A, iters, seed)
    rng = np.random.default_rng(17)
    out = 0.0
    for _ in range(trials):
        Ap = A.copy()
        Ap.data = Ap.data * (1.0 + 1e-15 * rng.uniform(-1.0, 1.0, Ap.nnz))
        out = max(out, abs(1.0 / O.arnoldi_rho(Ap, iters, seed) - ref) / ref)
    return ref, out


@pytest.mark.parametrize("eps,degree,sweeps", [(1e-2, 2, 5), (0.0, 1, 5)])
def test_weights_of_every_level_match_oracle(cl, eps, degree, sweeps):
    """Section 4's relaxation weight on every level of a full-size hierarchy: the GPU's
    omega against the oracle's Arnoldi (same steps, same seeded start vector, seed + level)
    on that level's own operator, as the GPU built it.  The large levels take the
    multi-launch Arnoldi, the small ones the one-launch cluster run.  The bar is the
    Ritz-value bar of the small parity cases plus 100 x what rounding-size changes of the
    operator move the oracle's own weight (omega_spread); on the advection-diffusion
    workload every level is held to the plain bar."""
    prob = workloads.config2(eps=eps, degree=degree)
    p = O.Params()
    for precision in (0, 1):
        h = setup_gpu(cl, prob, precision, degree, sweeps)
        try:
            nlev = cl.clair_stats(h).levels
            for k in range(nlev - 1):
                g = level0(cl, h, k)
                if not g["nc"]:
                    continue
                ref, spread = omega_spread(g["A"], p.arnoldi_iters, p.seed + k)
                if eps > 0:
                    assert spread <= 1e-9, (k, spread)
                dom = abs(g["omega"] - ref) / ref
                assert dom <= OMEGA_TOL + 100.0 * spread, (precision, k, g["n"], g["omega"], ref,
                                                            spread)
        finally:
            cl.clair_free(h)


@pytest.mark.parametrize("eps", [0.0, 1e-4])
def test_advection_dominated_iterations_match_oracle_256(cl, eps):
    """The variants whose 1024^2 MIXED solve hands over to the FP64 cycle, at 256^2 where
    the oracle's own iteration count is available (degree 2, five CFF sweeps on B): the
    FP64 path within one iteration of the oracle.  The MIXED cycle is a different
    preconditioner (FP32 rounding on its finer levels); it must not need more than one
    iteration beyond the oracle, or, where its FP32 cycle stalled (fp64_cycle_from >= 0),
    more than that plus the stall window (10 iterations) and the restart that hands over.
    (At eps = 0 it needs fewer: 9 against the oracle's 14.)"""
    import torch
    prob = workloads.constdir_2d(256, math.pi / 6, eps, seed=1, degree=2)
    A = O.csr_of(prob.A)
    H = O.build_hierarchy(prob.A, prob.B, O.Params())
    _, its_o, hist = O.fgmres(A, prob.f, lambda v: O.vcycle(H, v), 50, 1e-8, 200)
    assert hist[-1] <= 1e-8 * np.linalg.norm(prob.f)
    for precision in (0, 1):
        h = setup_gpu(cl, prob, precision)
        try:
            f = dev(prob.f, torch.float64)
            u = torch.zeros_like(f)
            st, its, rel = cl.clair_solve(h, f, u)
            uh = u.cpu().numpy()
            assert np.linalg.norm(prob.f - A @ uh) <= 1e-8 * np.linalg.norm(prob.f)
            fb = cl.clair_stats(h).fp64_cycle_from
            if precision == 0:
                assert abs(its - its_o) <= 1, (its, its_o)
            else:
                slack = 1 if fb < 0 else 1 + 10 + 1
                assert its <= its_o + slack, (its, its_o, fb)
        finally:
            cl.clair_free(h)


def test_fc_coarsening_on_the_3d_recirculating_problem(cl):
    """The documented fallback for the 3D recirculating workload (its aggregation variant
    stalls at eps = 1e-3, as the paper's does): C/F splitting at 64^3. The coarse rows grow
    long (operator complexity about 31); the solve reaches the 1e-8 true residual and every
    coarse operator is the Galerkin product of its level's own R, A and P."""
    import torch
    prob = workloads.config3(64)
    A = O.csr_of(prob.A)
    p = cl.clair_params_default()
    p.precision = 1
    h = cl.clair_setup(dev(prob.A.rowptr, torch.int32), dev(prob.A.col, torch.int32),
                       dev(prob.A.val, torch.float64), dev(prob.B, torch.float64), p)
    try:
        f = dev(prob.f, torch.float64)
        u = torch.zeros_like(f)
        st, its, rel = cl.clair_solve(h, f, u)
        uh = u.cpu().numpy()
        assert np.linalg.norm(prob.f - A @ uh) <= 1e-8 * np.linalg.norm(prob.f)
        assert its <= 12
        check_galerkin(cl, h)
    finally:
        cl.clair_free(h)
