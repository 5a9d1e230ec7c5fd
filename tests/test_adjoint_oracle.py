"""Pins of the adjoint-gradient oracle (oracle/adjoint.py) to things other than itself.

* Central finite differences (h = 1e-6) of the loss, computed by assembly plus exact
  sparse LU solves, along random directions in the eps, v_x and v_y fields of the
  variable-coefficient workload (velocity directions restricted to nodes with
  |v| > 1e-3, away from the upwind switch).  A dropped face term, a wrong sign or a
  swapped neighbour in the chain rule fails one of them.
* Finite differences of the loss in single stored entries of A (checks the row/column
  order of the sampled outer product: a transposed lam u^T fails).
* The closed form for a diagonal operator: u = f/a, dL/da = -2 (f/a - t) f / a^2.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads
from oracle import adjoint as J

NSIDE = 14
H = 1e-6


@pytest.fixture(scope="module")
def case():
    eps, vx, vy = workloads.config5_fields(NSIDE, seed=4)
    A = workloads.advdiff_2d(NSIDE, vx, vy, eps)
    F = workloads.uniform_pm1(11, 3 * A.n).reshape(3, -1)
    T = workloads.uniform_pm1(12, 3 * A.n).reshape(3, -1)
    U, Lam, dA = J.adjoint_gradient(A, F, T)
    grads = J.advdiff2d_param_gradient(NSIDE, eps, vx, vy, A, dA)
    return dict(eps=eps, vx=vx, vy=vy, A=A, F=F, T=T, U=U, Lam=Lam, dA=dA, grads=grads)


def test_adjoint_equations_hold(case):
    A = case["A"].to_scipy()
    assert np.allclose(A @ case["U"].T, case["F"].T, rtol=0, atol=1e-10)
    rhs = 2.0 * (case["U"] - case["T"])
    assert np.allclose(A.T @ case["Lam"].T, rhs.T, rtol=0, atol=1e-9)


@pytest.mark.parametrize("which", [0, 1, 2])
@pytest.mark.parametrize("seed", [0, 1])
def test_param_gradient_matches_central_differences(case, which, seed):
    fields = [case["eps"], case["vx"], case["vy"]]
    rng = np.random.default_rng(seed)
    d = rng.standard_normal(NSIDE * NSIDE)
    if which == 0:
        d = d * case["eps"]                                   # relative steps in eps
    else:
        d = d * (np.abs(fields[which]) > 1e-3)                # away from the upwind switch
    plus = [f.copy() for f in fields]
    minus = [f.copy() for f in fields]
    plus[which] = fields[which] + H * d
    minus[which] = fields[which] - H * d
    fd = (J.advdiff2d_loss(NSIDE, *plus, case["F"], case["T"]) -
          J.advdiff2d_loss(NSIDE, *minus, case["F"], case["T"])) / (2 * H)
    an = float(np.dot(case["grads"][which], d))
    assert abs(fd - an) <= 1e-6 * abs(fd) + 1e-12, (fd, an)


def test_operator_gradient_matches_entry_differences(case):
    A = case["A"].to_scipy().tocsr()
    rng = np.random.default_rng(3)
    for e in rng.choice(A.nnz, 8, replace=False):
        step = 1e-5 * abs(A.data[e])   # relative step: balances truncation and rounding
        Ap, Am = A.copy(), A.copy()
        Ap.data[e] += step
        Am.data[e] -= step
        fd = (J.loss(Ap, case["F"], case["T"]) - J.loss(Am, case["F"], case["T"])) / (2 * step)
        assert abs(fd - case["dA"][e]) <= 2e-6 * abs(fd) + 1e-9, (e, fd, case["dA"][e])


def test_diagonal_operator_closed_form():
    a = np.array([2.0, -3.0, 0.5, 4.0])
    f = np.array([1.0, 2.0, -1.0, 0.25])
    t = np.array([0.1, 0.0, -0.3, 1.0])
    A = sp.diags(a).tocsr()
    U, Lam, dA = J.adjoint_gradient(A, f[None], t[None])
    expect = -2.0 * (f / a - t) * f / (a * a)
    np.testing.assert_allclose(dA, expect, rtol=1e-14, atol=0)


def test_scalar_eps_is_the_sum_of_nodal_derivatives():
    """With a constant field the harmonic mean is the field itself, and the derivative in
    a single global eps is the sum of the per-node derivatives."""
    n = 10
    A = workloads.advdiff_2d(n, 0.6, -0.8, np.full(n * n, 0.03))
    F = workloads.uniform_pm1(5, n * n)[None]
    T = workloads.uniform_pm1(6, n * n)[None]
    _, _, dA = J.adjoint_gradient(A, F, T)
    de, _, _ = J.advdiff2d_param_gradient(n, np.full(n * n, 0.03), 0.6, -0.8, A, dA)
    fd = (J.advdiff2d_loss(n, 0.03 + H, 0.6, -0.8, F, T) -
          J.advdiff2d_loss(n, 0.03 - H, 0.6, -0.8, F, T)) / (2 * H)
    assert abs(de.sum() - fd) <= 1e-6 * abs(fd)
