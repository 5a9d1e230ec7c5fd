"""GPU parity of the adjoint path against the adjoint oracle (oracle/adjoint.py).

* clair_sddmm_grad and clair_advdiff2d_param_grad on given inputs: the oracle's formulas
  on the same seeded vectors, to float64 rounding.
* clair_setup_adjoint: the hierarchy of A^T solves A^T lam = g to the requested residual.
* End to end at the full size of the variable-coefficient workload (512^2, 8 right-hand
  sides): the autograd Function (forward CLAIR solves, adjoint hierarchy, adjoint solves,
  sampled outer product) and the field chain rule against the oracle's gradient, which
  uses exact sparse LU solves.  The solves run to a 1e-12 relative residual, so the
  gradients agree to ~1e-7 (the oracle's own gradient is pinned to finite differences
  by test_adjoint_oracle.py).
"""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads
from oracle import adjoint as J

pytestmark = pytest.mark.gpu

NSIDE = 512
NRHS = 8


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


@pytest.fixture(scope="module")
def problem():
    prob = workloads.config5(NSIDE, nrhs=NRHS)
    return prob


@pytest.fixture(scope="module")
def exact(problem):
    A = problem.A
    U, Lam, dA = J.adjoint_gradient(A, problem.f, problem.meta["u_target"])
    grads = J.advdiff2d_param_gradient(NSIDE, problem.meta["eps_field"], problem.meta["vx"],
                                       problem.meta["vy"], A, dA)
    return U, Lam, dA, grads


def test_sddmm_matches_oracle(cl, problem):
    import torch
    A = problem.A
    lam = workloads.uniform_pm1(21, NRHS * A.n).reshape(NRHS, A.n)
    u = workloads.uniform_pm1(22, NRHS * A.n).reshape(NRHS, A.n)
    dA = torch.empty(A.nnz, dtype=torch.float64, device="cuda")
    cl.clair_sddmm_grad(dev(A.rowptr, torch.int32), dev(A.col, torch.int32), dev(lam, torch.float64),
                        dev(u, torch.float64), dA)
    ref = J.operator_gradient(A, u, lam)
    mag = J.operator_gradient(A, np.abs(u), -np.abs(lam))   # sum_r |lam| |u| per entry
    assert np.all(np.abs(dA.cpu().numpy() - ref) <= 1e-15 * NRHS * mag)


def test_param_grad_matches_oracle(cl, problem):
    import torch
    A = problem.A
    m = problem.meta
    dA = workloads.uniform_pm1(23, A.nnz)
    out = cl.clair_advdiff2d_param_grad(NSIDE, 1.0 / (NSIDE + 1), dev(m["eps_field"], torch.float64),
                                        dev(m["vx"], torch.float64), dev(m["vy"], torch.float64),
                                        dev(A.rowptr, torch.int32), dev(A.col, torch.int32),
                                        dev(dA, torch.float64))
    ref = J.advdiff2d_param_gradient(NSIDE, m["eps_field"], m["vx"], m["vy"], A, dA)
    # rounding bound per node: the |dA| of the node's and its neighbours' rows times the
    # largest coefficient (2/h^2 for eps: harmonic-mean derivative <= 2; 2/h for v)
    h = 1.0 / (NSIDE + 1)
    S = A.to_scipy().tocsr()
    pattern = sp.csr_matrix((np.ones(S.nnz), S.indices, S.indptr), shape=S.shape)
    rowabs = np.asarray(abs(sp.csr_matrix((dA, S.indices, S.indptr), shape=S.shape)).sum(axis=1)).ravel()
    near = pattern @ rowabs
    for g, r, scale in zip(out, ref, (2.0 / h ** 2, 2.0 / h, 2.0 / h)):
        assert np.all(np.abs(g.cpu().numpy() - r) <= 1e-14 * scale * near)


def test_param_grad_rejects_non_stencil_pattern(cl):
    import torch
    A = workloads.advdiff_2d(8, 1.0, 0.5, 0.1).to_scipy().tolil()
    A[0, 20] = 1.0
    A = A.tocsr()
    A.sort_indices()
    z = torch.zeros(64, dtype=torch.float64, device="cuda")
    with pytest.raises(cl.ClairError):
        cl.clair_advdiff2d_param_grad(8, 1.0 / 9, z + 1, z, z, dev(A.indptr, torch.int32),
                                      dev(A.indices, torch.int32), dev(A.data, torch.float64))


@pytest.mark.parametrize("precision", [0, 1])
def test_adjoint_hierarchy_solves_transpose(cl, problem, precision):
    import torch
    A = problem.A
    p = cl.clair_params_default()
    p.precision = precision
    fwd = cl.Hierarchy(cl.clair_setup(dev(A.rowptr, torch.int32), dev(A.col, torch.int32),
                                      dev(A.val, torch.float64), dev(np.ones(A.n), torch.float64), p))
    adj = cl.Hierarchy(cl.clair_setup_adjoint(fwd.handle))
    g = workloads.uniform_pm1(24, A.n)
    lam = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    st, its, rel = cl.clair_solve(adj.handle, dev(g, torch.float64), lam)
    At = A.to_scipy().T.tocsr()
    res = np.linalg.norm(g - At @ lam.cpu().numpy()) / np.linalg.norm(g)
    assert res <= 1e-8, (res, its)
    # the adjoint hierarchy's fine operator is A^T
    v = cl.clair_level_view(adj.handle, 0)
    M = sp.csr_matrix((v["A_val"].cpu().numpy(), v["A_col"].cpu().numpy(), v["A_rowptr"].cpu().numpy()),
                      shape=(A.n, A.n))
    assert (M != At).nnz == 0


@pytest.mark.parametrize("precision", [0, 1])
def test_end_to_end_gradient_matches_oracle(cl, problem, exact, precision):
    import torch
    A = problem.A
    m = problem.meta
    Ue, Lame, dAe, grads_e = exact
    p = cl.clair_params_default()
    p.precision = precision
    p.rtol = 1e-12
    p.gmres_maxit = 400
    rowptr, col = dev(A.rowptr, torch.int32), dev(A.col, torch.int32)
    val = dev(A.val, torch.float64).requires_grad_(True)
    F = dev(problem.f, torch.float64).requires_grad_(True)
    T = dev(m["u_target"], torch.float64)
    U = cl.ClairSolve.apply(val, F, rowptr, col, dev(np.ones(A.n), torch.float64), p)
    loss = ((U - T) ** 2).sum()
    loss.backward()
    rel = lambda a, b: np.linalg.norm(a - b) / np.linalg.norm(b)
    assert rel(U.detach().cpu().numpy(), Ue) <= 1e-8
    assert rel(F.grad.cpu().numpy(), Lame) <= 1e-7
    dval = val.grad.cpu().numpy()
    assert rel(dval, dAe) <= 1e-7
    out = cl.clair_advdiff2d_param_grad(NSIDE, 1.0 / (NSIDE + 1), dev(m["eps_field"], torch.float64),
                                        dev(m["vx"], torch.float64), dev(m["vy"], torch.float64),
                                        rowptr, col, val.grad)
    for g, r in zip(out, grads_e):
        assert rel(g.cpu().numpy(), r) <= 1e-7
