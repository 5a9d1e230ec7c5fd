"""GPU parity of the method's variants and of the boundary's multi-process solve, through
the C ABI, against the FP64 oracle:

* k = 2 mode vectors (constants and the x coordinate; Eq. 3.3 with k > 1);
* diagonal block inverses with three passes of Algorithm 1's loop (Section 3.1.2);
* the symmetric variant R = P^T solved with preconditioned CG (Section 4.1 parameters:
  strength 0.5 / 0.5, aggregation, B = 1 smoothed by five CFF sweeps);
* a caller-given fine-level splitting (cf_marker);
* several right-hand sides in one clair_solve, and one Krylov process per instance of a
  batch, each with its own iteration count.

Bars as in test_gpu_parity.py: integer work bit-exact, FP64 values to 1e-12 per row
(widened by 100x the relative drift of the Arnoldi weight), iterations within one of the
oracle's, true relative residual <= 1e-8.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
import workloads

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
OMEGA_TOL = 1e-8


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


def gpu_setup(cl, A, B, precision=0, cf_marker=None, **kw):
    import torch
    p = cl.clair_params_default()
    p.precision = precision
    for k, v in kw.items():
        setattr(p, k, v)
    Bt = dev(np.ascontiguousarray(np.asarray(B).T) if np.ndim(B) == 2 else B, torch.float64)
    cfm = None if cf_marker is None else dev(cf_marker, torch.int8)
    return cl.clair_setup(dev(A.rowptr, torch.int32), dev(A.col, torch.int32),
                          dev(A.val, torch.float64), Bt, p, cf_marker=cfm)


def host_levels(cl, h):
    import torch
    torch.cuda.synchronize()
    out = []
    for k in range(cl.clair_stats(h).levels):
        v = cl.clair_level_view(h, k)
        out.append({key: (val.cpu().numpy() if hasattr(val, "cpu") else val) for key, val in v.items()})
    return out


def csr_from(d, prefix, shape):
    return sp.csr_matrix((d[prefix + "_val"], d[prefix + "_col"], d[prefix + "_rowptr"]), shape=shape)


def rowwise_err(G, Oref):
    G, Oref = G.tocsr(), Oref.tocsr()
    assert np.array_equal(G.indptr, Oref.indptr) and np.array_equal(G.indices, Oref.indices)
    worst = 0.0
    d = np.abs(G.data - Oref.data)
    a = np.abs(Oref.data)
    for r in range(G.shape[0]):
        s, e = G.indptr[r], G.indptr[r + 1]
        if e > s:
            worst = max(worst, d[s:e].max() / max(a[s:e].max(), 1e-300))
    return worst


U_ROUND = np.finfo(np.float64).eps / 2


def gram_condition(H):
    """Per level: the largest condition number of the k x k Gram matrices
    G_j = B_c[J_j]^T B_c[J_j] of the projection over both sides (k > 1)."""
    out = []
    for lev in H.levels[:-1]:
        C = np.flatnonzero(lev.cf == 1)
        worst = 1.0
        for M, Bv in ((lev.R.T.tocsr(), lev.B_R), (lev.P, lev.B_P)):
            Bc = Bv.reshape(lev.A.shape[0], -1)[C]
            for j in np.flatnonzero(lev.cf == 0):
                J = M.indices[M.indptr[j]:M.indptr[j + 1]]
                if J.size >= Bc.shape[1]:
                    worst = max(worst, np.linalg.cond(Bc[J].T @ Bc[J]))
        out.append(worst)
    return out


def compare_hierarchy(G, H, kmodes=1, kappa=None):
    """Level by level: structure bit-exact, values to FP64_TOL + 100 x weight drift.  With
    several modes the projection solves a k x k Gram system per F-point, whose rounding is
    amplified by its condition number: that level's bar (and the drift carried to the
    coarser levels) adds 4 u kappa_max (kappa from ``gram_condition``)."""
    assert len(G) == len(H.levels)
    drift = 0.0
    for k, lev in enumerate(H.levels):
        g = G[k]
        n = lev.A.shape[0]
        tol = FP64_TOL + 100.0 * drift
        Ag = csr_from(g, "A", (n, n))
        assert np.array_equal(Ag.indptr, lev.A.indptr) and np.array_equal(Ag.indices, lev.A.indices)
        assert np.abs(Ag.data - lev.A.data).max() <= tol * np.abs(lev.A.data).max(), k
        if lev.cf is None:
            continue
        assert np.array_equal(g["cf"], lev.cf), f"level {k}: splitting differs"
        nc = int(lev.cf.sum())
        dom = abs(g["omega"] - lev.omega) / lev.omega
        assert dom <= OMEGA_TOL, (k, dom)
        drift = max(drift, dom)
        tol = FP64_TOL + 100.0 * drift
        if kappa is not None:
            tol += 4.0 * U_ROUND * kappa[k]
        for key, ref in (("B_P", lev.B_P), ("B_R", lev.B_R)):
            got = g[key].reshape(kmodes, n).T
            assert np.abs(got - ref.reshape(n, kmodes)).max() <= tol * np.abs(ref).max(), (k, key)
        eR = rowwise_err(csr_from(g, "R", (nc, n)), lev.R)
        eP = rowwise_err(csr_from(g, "P", (n, nc)), lev.P)
        assert eR <= tol and eP <= tol, (k, eR, eP, tol)
        if kappa is not None:
            drift = max(drift, 0.04 * U_ROUND * kappa[k])


def solve_and_check(cl, h, A, f, its_ref, precision):
    import torch
    u = torch.zeros(f.size, dtype=torch.float64, device="cuda")
    st, its, rel = cl.clair_solve(h, dev(f, torch.float64), u)
    uh = u.cpu().numpy()
    true_rel = np.linalg.norm(f - A @ uh) / np.linalg.norm(f)
    assert true_rel <= 1e-8 and rel <= 1e-8, (true_rel, rel)
    assert abs(its - its_ref) <= 1, (its, its_ref, precision)
    return uh


# ---------------------------------------------------------------------------------------
# k = 2 mode vectors
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("eps", [1e-2, 1.0])
def test_two_modes_hierarchy_and_solve_match_oracle(cl, eps):
    prob = workloads.constdir_2d(40, math.pi / 6, eps, seed=1, degree=2)
    n = prob.A.n
    x = (np.arange(n) % 40 + 1) / 41.0
    B = np.stack([np.ones(n), x], axis=1)
    H = O.build_hierarchy(prob.A, B, O.Params())
    A = O.csr_of(prob.A)
    _, its_o, _ = O.fgmres(A, prob.f, lambda v: O.vcycle(H, v), 50, 1e-8, 200)
    for precision in (0, 1):
        h = gpu_setup(cl, prob.A, B, precision)
        try:
            assert cl.clair_stats(h).k == 2
            if precision == 0:
                compare_hierarchy(host_levels(cl, h), H, kmodes=2, kappa=gram_condition(H))
            solve_and_check(cl, h, A, prob.f, its_o, precision)
        finally:
            cl.clair_free(h)


# ---------------------------------------------------------------------------------------
# Diagonal block inverses, three passes of Algorithm 1's loop
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("eps", [1e-2, 1.0])
def test_diag_inverse_three_passes_matches_oracle(cl, eps):
    prob = workloads.constdir_2d(40, math.pi / 6, eps, seed=1, degree=2)
    H = O.build_hierarchy(prob.A, prob.B, O.Params(inverse="diag", iterations=3))
    h = gpu_setup(cl, prob.A, prob.B, 0, inverse=cl.CLAIR_INVERSE_DIAG, iterations=3)
    try:
        compare_hierarchy(host_levels(cl, h), H)
    finally:
        cl.clair_free(h)


# ---------------------------------------------------------------------------------------
# Symmetric variant: R = P^T, preconditioned CG
# ---------------------------------------------------------------------------------------
def sym_problem(tag):
    if tag == "poisson2d":
        return workloads.advdiff_2d(40, 0.0, 0.0, 1.0)
    return workloads.advdiff_3d(12, lambda x, y, z: (0 * x, 0 * y, 0 * z), 1.0)


@pytest.mark.parametrize("tag", ["poisson2d", "poisson3d"])
def test_symmetric_pcg_matches_oracle(cl, tag):
    A0 = sym_problem(tag)
    A = O.csr_of(A0)
    n = A0.n
    B = np.ones(n)
    f = workloads.uniform_pm1(5, n)
    params = O.Params(theta_coarsen=0.5, theta_interp=0.5, coarsen="AGG", symmetric=True,
                      post_weighted=True)
    H = O.build_hierarchy(A0, B, params)
    _, its_o, _ = O.pcg(A, f, lambda v: O.vcycle(H, v), 1e-8, 200)
    kw = dict(theta_coarsen=0.5, theta_interp=0.5, coarsen=cl.CLAIR_COARSEN_AGG, symmetric=1,
              post_weighted=1, krylov=cl.CLAIR_KRYLOV_PCG)
    for precision in (0, 1):
        h = gpu_setup(cl, A0, B, precision, **kw)
        try:
            if precision == 0:
                G = host_levels(cl, h)
                compare_hierarchy(G, H)
                for g in G[:-1]:
                    nn, nc = g["n"], g["nc"]
                    R, P = csr_from(g, "R", (nc, nn)), csr_from(g, "P", (nn, nc))
                    assert (R != P.T).nnz == 0
            solve_and_check(cl, h, A, f, its_o, precision)
        finally:
            cl.clair_free(h)


# ---------------------------------------------------------------------------------------
# Caller splitting
# ---------------------------------------------------------------------------------------
def test_cf_marker_replaces_fine_splitting(cl):
    prob = workloads.constdir_2d(40, math.pi / 6, 1e-2, seed=1, degree=2)
    A = O.csr_of(prob.A)
    cf = O.split_fc(A, 0.5)            # a different (coarser) splitting than the default
    assert not np.array_equal(cf, O.split_fc(A, 0.25))
    H = O.build_hierarchy(prob.A, prob.B, O.Params(), cf_override=cf)
    _, its_o, _ = O.fgmres(A, prob.f, lambda v: O.vcycle(H, v), 50, 1e-8, 200)
    h = gpu_setup(cl, prob.A, prob.B, 0, cf_marker=cf)
    try:
        compare_hierarchy(host_levels(cl, h), H)
        solve_and_check(cl, h, A, prob.f, its_o, 0)
    finally:
        cl.clair_free(h)


def test_cf_marker_with_aggregation_is_unsupported(cl):
    prob = workloads.config1()
    with pytest.raises(cl.ClairError) as exc:
        gpu_setup(cl, prob.A, prob.B, 0, cf_marker=np.zeros(prob.A.n, dtype=np.int8),
                  coarsen=cl.CLAIR_COARSEN_AGG)
    assert exc.value.status == cl.CLAIR_ERR_UNSUPPORTED


# ---------------------------------------------------------------------------------------
# Several right-hand sides in one call
# ---------------------------------------------------------------------------------------
@pytest.mark.parametrize("precision", [0, 1])
def test_multi_rhs_solve_matches_single_solves(cl, precision):
    import torch
    prob = workloads.config1()
    A = O.csr_of(prob.A)
    n = prob.A.n
    F = np.stack([workloads.uniform_pm1(10 + r, n) for r in range(4)])
    F[2] *= 1e-6                       # scales differ: each stops at its own rtol ||f_r||
    H = O.build_hierarchy(prob.A, prob.B, O.Params())
    its_o = [O.fgmres(A, F[r], lambda v: O.vcycle(H, v), 50, 1e-8, 200)[1] for r in range(4)]
    h = gpu_setup(cl, prob.A, prob.B, precision)
    try:
        U = torch.zeros(4, n, dtype=torch.float64, device="cuda")
        st, its, rel = cl.clair_solve(h, dev(F, torch.float64), U)
        Uh = U.cpu().numpy()
        single = []
        for r in range(4):
            u = torch.zeros(n, dtype=torch.float64, device="cuda")
            _, it1, _ = cl.clair_solve(h, dev(F[r], torch.float64), u)
            single.append(it1)
            true_rel = np.linalg.norm(F[r] - A @ Uh[r]) / np.linalg.norm(F[r])
            assert true_rel <= 1e-8 and rel[r] <= 1e-8, (r, true_rel, rel[r])
            assert abs(its[r] - its_o[r]) <= 1, (r, its, its_o)
            np.testing.assert_allclose(Uh[r], u.cpu().numpy(), rtol=0,
                                       atol=1e-7 * np.abs(Uh[r]).max())
        assert its == single, (its, single)
        segs_its, segs_rel = cl.clair_solve_detail(h)
        assert len(segs_its) == 1 and segs_its[0] == single[-1]
    finally:
        cl.clair_free(h)


def test_zero_rhs_gives_zero_solution(cl):
    import torch
    prob = workloads.config1()
    n = prob.A.n
    h = gpu_setup(cl, prob.A, prob.B, 0)
    try:
        F = np.stack([np.zeros(n), prob.f])
        U = torch.ones(2, n, dtype=torch.float64, device="cuda")
        st, its, rel = cl.clair_solve(h, dev(F, torch.float64), U)
        assert torch.all(U[0] == 0).item() and its[0] == 0 and rel[0] == 0.0
        assert rel[1] <= 1e-8
    finally:
        cl.clair_free(h)


# ---------------------------------------------------------------------------------------
# One Krylov process per instance of a batch
# ---------------------------------------------------------------------------------------
SIDES = [10, 20, 28, 36, 44, 24, 16]


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_instances_iterate_like_their_own_solves(cl, precision):
    import torch
    params = workloads.config4_params(len(SIDES))
    mats = [workloads.advdiff_2d(side, math.cos(a), math.sin(a), e)
            for side, (_, a, e) in zip(SIDES, params)]
    Ab, offs = workloads.block_diagonal(mats)
    f = workloads.uniform_pm1(4, Ab.n)
    p = cl.clair_params_default()
    p.precision = precision
    h = cl.clair_setup_batched(offs.tolist(), dev(Ab.rowptr, torch.int32), dev(Ab.col, torch.int32),
                               dev(Ab.val, torch.float64), dev(np.ones(Ab.n), torch.float64), p)
    try:
        u = torch.zeros(Ab.n, dtype=torch.float64, device="cuda")
        st, its, rel = cl.clair_solve(h, dev(f, torch.float64), u)
        seg_its, seg_rel = cl.clair_solve_detail(h)
        assert len(seg_its) == len(mats)
        uh = u.cpu().numpy()
        for i, M in enumerate(mats):
            Ai = O.csr_of(M)
            fi = f[offs[i]:offs[i + 1]]
            ri = np.linalg.norm(fi - Ai @ uh[offs[i]:offs[i + 1]]) / np.linalg.norm(fi)
            assert ri <= 1e-8 and abs(seg_rel[i] - ri) <= 1e-3 * ri + 1e-16, (i, ri, seg_rel[i])
            H = O.build_hierarchy(M, np.ones(M.n), O.Params())
            _, its_o, _ = O.fgmres(Ai, fi, lambda v: O.vcycle(H, v), 50, 1e-8, 200)
            assert abs(seg_its[i] - its_o) <= 1, (i, seg_its[i], its_o)
        assert its == max(seg_its)
    finally:
        cl.clair_free(h)


# ---------------------------------------------------------------------------------------
# Approximation-property constants (Appendix A) of the GPU's restriction
# ---------------------------------------------------------------------------------------
def test_approximation_constants_of_gpu_restriction_match_oracle(cl):
    from paper_2307_00229_gb300 import diagnostics as D
    A0 = workloads.advdiff_2d(32, math.cos(math.pi / 6), math.sin(math.pi / 6), 10.0)
    A = O.csr_of(A0)
    n = A0.n
    H = O.build_hierarchy(A0, np.ones(n), O.Params())
    h = gpu_setup(cl, A0, np.ones(n), 0)
    try:
        g = host_levels(cl, h)[0]
        Rg = csr_from(g, "R", (g["nc"], n)).toarray()
    finally:
        cl.clair_free(h)
    Ro = H.levels[0].R.toarray()
    for fn in (D.wap, D.sap):
        kg, _ = fn(A.toarray(), Rg.T, "R")
        ko, _ = fn(A.toarray(), Ro.T, "R")
        assert abs(kg - ko) <= 1e-9 * ko, (kg, ko)
