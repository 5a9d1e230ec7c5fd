"""Pins of the approximation-property diagnostics (Appendix A) against closed forms, and
the constants of CLAIR's restriction on the 32 x 32 upwind advection-diffusion stand-in
for the paper's DG problem.

Closed form: with M = U diag(s) U^T (s ascending) and T spanning the first n_c columns of
U, the eta-projection is the orthogonal projection onto span U[:, :n_c] for every eta, so
(I - Pi) M^-beta = U_2 diag(s_2^-beta) U_2^T and K_max = s_max^(2 beta - eta) *
s_{n_c+1}^(eta - 2 beta): sigma_max / sigma_{n_c+1} for both WAP and SAP.  A vector in the
range of T has K = 0; the singular vector n_c + 1 attains K_max.
"""
import math

import numpy as np
import pytest

import oracle as O
import workloads
from paper_2307_00229_gb300 import diagnostics as D


def nonsym(n=40, seed=2):
    rng = np.random.default_rng(seed)
    return np.eye(n) * 4 + rng.uniform(-1, 1, (n, n)) / math.sqrt(n)


@pytest.mark.parametrize("side", ["P", "R"])
@pytest.mark.parametrize("nc", [1, 10, 25])
def test_closed_form_for_singular_vector_ranges(side, nc):
    A = nonsym()
    U, s = D.energy_matrix(A, side)
    T = U[:, :nc] @ np.random.default_rng(1).standard_normal((nc, nc))  # same range
    for fn in (D.wap, D.sap):
        kmax, kv = fn(A, T, side)
        assert abs(kmax - s[-1] / s[nc]) <= 1e-10 * kmax
        np.testing.assert_allclose(kv[:nc], 0.0, atol=1e-12)
        assert abs(kv[nc] - kmax) <= 1e-10 * kmax
        assert np.all(kv <= kmax * (1 + 1e-10))


def test_energy_matrices_are_the_polar_factors():
    A = nonsym(30)
    for side, M2 in (("P", A.T @ A), ("R", A @ A.T)):
        U, s = D.energy_matrix(A, side)
        M = (U * s) @ U.T
        np.testing.assert_allclose(M @ M, M2, rtol=0, atol=1e-11 * np.abs(M2).max())
        assert np.all(s > 0) and np.all(np.diff(s) >= 0)


def test_full_coarse_space_has_zero_constant():
    A = nonsym(20)
    for side in ("P", "R"):
        kmax, kv = D.sap(A, np.eye(20), side)
        assert kmax <= 1e-20 and np.all(np.abs(kv) <= 1e-20)


def test_clair_restriction_constants_on_32x32():
    """Appendix A's comparison on the 32^2 stand-in (alpha = 10 read as eps = 10 with unit
    velocity at angle pi/6): CLAIR's restriction has a far smaller SAP constant than lAIR's
    (Remark 3.1: the same local solves without the constraint), and 25 B-smoothing sweeps
    lower it further than 5 (the paper's DG problem: 2246 for lAIR, 184 -> 77 for CLAIR)."""
    A = O.csr_of(workloads.advdiff_2d(32, math.cos(math.pi / 6), math.sin(math.pi / 6), 10.0))
    n = A.shape[0]
    Ad = A.toarray()
    out = {}
    for name, p in (("clair5", O.Params(b_smooth_iters=5)), ("clair25", O.Params(b_smooth_iters=25)),
                    ("lair", O.Params(constrain=False))):
        R = O.build_hierarchy(A, np.ones(n), p).levels[0].R.toarray()
        kw, _ = D.wap(Ad, R.T, "R")
        ks, kv = D.sap(Ad, R.T, "R")
        assert np.isfinite(kw) and np.isfinite(ks) and kw > 0 and ks > 0
        assert kv.max() <= ks * (1 + 1e-9)
        out[name] = (kw, ks)
    assert out["clair5"][1] < out["lair"][1] / 5, out
    assert out["clair25"][1] < out["clair5"][1], out
    assert out["clair5"][0] < out["lair"][0], out
