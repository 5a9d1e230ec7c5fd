"""GPU parity of the batched setup and solve against the single-instance oracle.

A batch is one block-diagonal operator; each instance's hierarchy inside it must equal
the oracle's hierarchy of that instance alone (oracle.build_hierarchy per instance):
splitting bit-exact, relaxation weight to OMEGA_TOL, R, P and the coarse operator blocks
to FP64 rounding (widened by the weight drift as in test_gpu_parity.py), level by level
while the instance is active.  An instance is frozen from its own coarsest level on; the
batch V-cycle must then equal the instance's own V-cycle, whose coarsest step is that
level's dense solve.  The solve must bring every instance to the relative tolerance.

Instances mix the many-instance workload's angles and diffusion coefficients with small
sides (one at or below the coarsest size, frozen from level 0), so the oracle runs in
seconds.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
import workloads

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
# The segmented Arnoldi sums each instance's dot products over its own block partition,
# and from level 1 on the operator itself differs from the oracle's by rounding; the
# Ritz values of the non-normal Hessenberg matrix amplify both (1.3e-8 seen on level 2).
OMEGA_TOL = 1e-7
SIDES = [10, 20, 28, 36, 44, 24, 16]


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
def batch():
    params = workloads.config4_params(len(SIDES))
    mats, probs = [], []
    for side, (_, angle, eps) in zip(SIDES, params):
        A = workloads.advdiff_2d(side, math.cos(angle), math.sin(angle), eps)
        mats.append(A)
    A, offs = workloads.block_diagonal(mats)
    f = workloads.uniform_pm1(4, A.n)
    H = [O.build_hierarchy(M, np.ones(M.n), O.Params()) for M in mats]
    return {"mats": mats, "A": A, "offs": offs, "f": f, "H": H}


def setup(cl, b, precision):
    import torch
    A = b["A"]
    p = cl.clair_params_default()
    p.precision = precision
    return cl.clair_setup_batched(b["offs"].tolist(), dev(A.rowptr, torch.int32),
                                  dev(A.col, torch.int32), dev(A.val, torch.float64),
                                  dev(np.ones(A.n), torch.float64), p)


def levels(cl, h):
    import torch
    torch.cuda.synchronize()
    out = []
    for k in range(cl.clair_stats(h).levels):
        v = cl.clair_level_view(h, k)
        d = {key: (x.cpu().numpy() if hasattr(x, "cpu") else x) for key, x in v.items()}
        n, nc = d["n"], d["nc"]
        d["A"] = sp.csr_matrix((d["A_val"], d["A_col"], d["A_rowptr"]), shape=(n, n))
        if nc:
            d["R"] = sp.csr_matrix((d["R_val"], d["R_col"], d["R_rowptr"]), shape=(nc, n))
            d["P"] = sp.csr_matrix((d["P_val"], d["P_col"], d["P_rowptr"]), shape=(n, nc))
        d.update(cl.clair_batch_view(h, k))
        out.append(d)
    return out


def block_err(G, Oref):
    G, Oref = G.tocsr(), Oref.tocsr()
    G.sort_indices()
    Oref.sort_indices()
    assert np.array_equal(G.indptr, Oref.indptr) and np.array_equal(G.indices, Oref.indices)
    if Oref.nnz == 0:
        return 0.0
    return np.abs(G.data - Oref.data).max() / np.abs(Oref.data).max()


def test_batch_hierarchy_matches_instances(cl, batch):
    h = setup(cl, batch, 0)
    try:
        G = levels(cl, h)
        for i, H in enumerate(batch["H"]):
            drift = 0.0
            last = len(H.levels) - 1           # the instance's coarsest level
            for k in range(len(G)):
                g = G[k]
                lo, hi = g["offsets"][i], g["offsets"][i + 1]
                if k > last:
                    # frozen instances pass through unchanged
                    assert g["frozen"][i] == 1 and hi - lo == H.levels[last].A.shape[0]
                    continue
                lev = H.levels[k]
                assert hi - lo == lev.A.shape[0], (i, k)
                tol = FP64_TOL + 100.0 * drift
                assert block_err(g["A"][lo:hi, lo:hi], lev.A) <= tol, (i, k)
                if k == last:
                    assert k == len(G) - 1 or g["frozen"][i] == 1, (i, k)
                    continue
                assert g["frozen"][i] == 0, (i, k)
                assert np.array_equal(g["cf"][lo:hi], lev.cf), f"instance {i} level {k}: splitting"
                dom = abs(g["omega"][i] - lev.omega) / lev.omega
                assert dom <= OMEGA_TOL, (i, k, dom)
                drift = max(drift, dom)
                tol = FP64_TOL + 100.0 * drift
                nxt = G[k + 1]
                clo, chi = nxt["offsets"][i], nxt["offsets"][i + 1]
                assert block_err(g["R"][clo:chi, lo:hi], lev.R) <= tol, (i, k)
                assert block_err(g["P"][lo:hi, clo:chi], lev.P) <= tol, (i, k)
                # no entry of the instance's rows leaves its block
                assert g["R"][clo:chi, :].nnz == g["R"][clo:chi, lo:hi].nnz
    finally:
        cl.clair_free(h)


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_vcycle_matches_instances(cl, batch, precision):
    import torch
    h = setup(cl, batch, precision)
    try:
        b = workloads.uniform_pm1(78, batch["A"].n)
        x = torch.zeros(batch["A"].n, dtype=torch.float64, device="cuda")
        cl.clair_vcycle(h, 0, dev(b, torch.float64), x)
        x = x.cpu().numpy()
        offs = batch["offs"]
        views = [cl.clair_batch_view(h, k) for k in range(cl.clair_stats(h).levels)]
        for i, H in enumerate(batch["H"]):
            # the instance's largest relative weight difference to the oracle widens the bound
            drift = max([abs(views[k]["omega"][i] - lev.omega) / lev.omega
                         for k, lev in enumerate(H.levels[:-1])] or [0.0])
            xo = O.vcycle(H, b[offs[i]:offs[i + 1]])
            err = np.linalg.norm(x[offs[i]:offs[i + 1]] - xo) / np.linalg.norm(xo)
            assert err <= (1e-11 + 100.0 * drift if precision == 0 else 1e-4), (i, err, drift)
    finally:
        cl.clair_free(h)


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_solve_reaches_every_instance(cl, batch, precision):
    import torch
    h = setup(cl, batch, precision)
    try:
        f = dev(batch["f"], torch.float64)
        u = torch.zeros_like(f)
        st, its, rel = cl.clair_solve(h, f, u)
        uh = u.cpu().numpy()
        offs = batch["offs"]
        worst = 0.0
        for i, M in enumerate(batch["mats"]):
            fi = batch["f"][offs[i]:offs[i + 1]]
            ri = fi - M.to_scipy() @ uh[offs[i]:offs[i + 1]]
            worst = max(worst, np.linalg.norm(ri) / np.linalg.norm(fi))
        assert worst <= 1e-8, worst
        assert abs(rel - worst) <= 1e-3 * worst + 1e-16, (rel, worst)
    finally:
        cl.clair_free(h)


def test_single_instance_batch_equals_setup(cl, batch):
    """A batch of one is the ordinary setup."""
    import torch
    M = batch["mats"][3]
    args = (dev(M.rowptr, torch.int32), dev(M.col, torch.int32), dev(M.val, torch.float64),
            dev(np.ones(M.n), torch.float64))
    h1 = cl.clair_setup(*args)
    h2 = cl.clair_setup_batched([0, M.n], *args)
    try:
        G1, G2 = levels(cl, h1), levels(cl, h2)
        assert len(G1) == len(G2)
        for a, b in zip(G1, G2):
            assert (a["A"] != b["A"]).nnz == 0
    finally:
        cl.clair_free(h1)
        cl.clair_free(h2)


def test_batch_rejects_coupled_instances(cl, batch):
    import torch
    A = batch["A"].to_scipy().tolil()
    o = batch["offs"]
    A[int(o[1]) - 1, int(o[1])] = -0.5       # couples instances 0 and 1
    A = A.tocsr()
    A.sort_indices()
    with pytest.raises(cl.ClairError):
        cl.clair_setup_batched(o.tolist(), dev(A.indptr, torch.int32), dev(A.indices, torch.int32),
                               dev(A.data, torch.float64), dev(np.ones(A.shape[0]), torch.float64))
