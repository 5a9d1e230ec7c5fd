"""The sparse product of the Galerkin step (C = A B, clair_spgemm) against scipy, on
inputs that route rows through every tier: small and large shared-memory hash tables,
the CTA-per-row path for long products, and rows with more distinct columns (over 16384)
than any shared-memory table holds, which take the dense global-memory accumulator.
Sums are in float64 in A's row order with separate multiply and add; scipy's may fuse
them, so the bar is the backward error of a sum of products: |C - C_ref| <= 64 u (|A| |B|)
entrywise (u = 2^-53; the longest sums here have about 900 terms, whose worst case is
900 u but whose rounding errors add like a random walk); the structure (columns, sorted)
is exact."""
import numpy as np
import pytest
import scipy.sparse as sp

pytestmark = pytest.mark.gpu


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


def check(cl, A, B):
    import torch
    A, B = sp.csr_matrix(A), sp.csr_matrix(B)
    A.sort_indices()
    B.sort_indices()
    rp, col, val = cl.clair_spgemm(dev(A.indptr, torch.int32), dev(A.indices, torch.int32),
                                   dev(A.data, torch.float64), dev(B.indptr, torch.int32),
                                   dev(B.indices, torch.int32), dev(B.data, torch.float64), B.shape[1])
    torch.cuda.synchronize()
    ref = (A @ B).tocsr()
    ref.sort_indices()
    got = sp.csr_matrix((val.cpu().numpy(), col.cpu().numpy(), rp.cpu().numpy()), shape=ref.shape)
    # scipy drops nothing here (random values do not cancel): same structure
    assert np.array_equal(got.indptr, ref.indptr)
    assert np.array_equal(got.indices, ref.indices)
    mag = (abs(A) @ abs(B)).tocsr()
    mag.sort_indices()
    assert np.array_equal(mag.indices, ref.indices)
    u = np.finfo(np.float64).eps / 2
    assert np.all(np.abs(got.data - ref.data) <= 64 * u * mag.data)
    return got


def test_short_rows(cl):
    rng = np.random.default_rng(0)
    A = sp.random(3000, 2000, density=0.003, random_state=rng, format="csr")
    B = sp.random(2000, 2500, density=0.003, random_state=rng, format="csr")
    check(cl, A, B)


def test_long_products(cl):
    """Mean products per row above the CTA-per-row threshold."""
    rng = np.random.default_rng(1)
    A = sp.random(400, 3000, density=0.02, random_state=rng, format="csr")
    B = sp.random(3000, 5000, density=0.02, random_state=rng, format="csr")
    check(cl, A, B)


@pytest.mark.parametrize("long_rows", [False, True])
def test_rows_beyond_every_shared_table(cl, long_rows):
    """A few rows whose products cover more than 16384 distinct columns of B (40000
    columns): the dense tier, on the flat-tier path (few products per row on average) and
    on the CTA path (many)."""
    rng = np.random.default_rng(2)
    n, ncols = 4000, 40000
    dens = 0.01 if long_rows else 0.0005
    A = sp.random(n, n, density=dens, random_state=rng, format="lil")
    for r in (0, 17, 3999):
        A[r, rng.choice(n, 900, replace=False)] = rng.uniform(-1, 1, 900)
    B = sp.random(n, ncols, density=0.005, random_state=rng, format="csr")
    got = check(cl, A.tocsr(), B)
    assert np.diff(got.indptr)[[0, 17, 3999]].min() > 16384
