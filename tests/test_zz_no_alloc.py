"""The no-allocation variant of the batched local solves (clair_local_weights_noalloc).

It serves callers that cannot let the library allocate device memory while they run (a
process whose device memory is reserved by its own pool, a latency-critical loop that
cannot afford cudaMalloc).  Its temporaries live in one fixed static device array, so
these tests check, through the C ABI, that it gives the same weights as the allocating
entry point on two calls in a row (the array keeps the previous call's contents, so the
second call checks that nothing stale leaks into it), and that a problem too large for
the array is refused with a clear error.  The file is collected last on purpose.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import workloads

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
FP32_TOL = 2e-5


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


def problem(nside=30, wide_row=None):
    """C-points on a lattice; each C-point's pattern is its F-points within Chebyshev
    distance 1..5 (sizes from a few up to ~120, so every solver bucket up to 128 unknowns
    is used).  ``wide_row`` gives that one C-point radius 7, about 200 unknowns."""
    A = workloads.advdiff_2d(nside, math.cos(0.4), math.sin(0.4), 1e-1).to_scipy().tocsr()
    A.sort_indices()
    n = A.shape[0]
    ix, iy = np.arange(n) % nside, np.arange(n) // nside
    cf = ((ix % 3 == 1) & (iy % 3 == 1)).astype(np.int8)
    cpts = np.flatnonzero(cf)
    rp, cols = [0], []
    for r, c in enumerate(cpts):
        radius = 7 if r == wide_row else 1 + r % 5
        d = np.maximum(np.abs(ix - ix[c]), np.abs(iy - iy[c]))
        sel = np.flatnonzero((d <= radius) & ((cf == 0) | (np.arange(n) == c)))
        cols.append(sel)
        rp.append(rp[-1] + sel.size)
    B = 0.5 + workloads.uniform01(21, n)
    return A, cf, cpts, np.array(rp, dtype=np.int32), np.concatenate(cols).astype(np.int32), B


def rowwise_err(val, ref, rp):
    worst = 0.0
    for r in range(rp.size - 1):
        s, e = rp[r], rp[r + 1]
        worst = max(worst, np.abs(val[s:e] - ref[s:e]).max() / max(np.abs(ref[s:e]).max(), 1e-300))
    return worst


@pytest.mark.parametrize("precision", [0, 1])
def test_noalloc_matches_allocating_entry_point_twice(cl, precision):
    import torch
    A, cf, cpts, zrp, zcol, B = problem()
    args = (dev(A.indptr, torch.int32), dev(A.indices, torch.int32), dev(A.data, torch.float64),
            dev(cf, torch.int8), cpts.size, dev(zrp, torch.int32), dev(zcol, torch.int32),
            dev(B, torch.float64), precision)
    ref = torch.zeros(zcol.size, dtype=torch.float64, device="cuda")
    st, sing, empty = cl.clair_local_weights(*args, ref)
    assert st == 0 and sing == 0
    ref_h = ref.cpu().numpy()
    tol = FP64_TOL if precision == 0 else FP32_TOL
    for call in range(2):
        out = torch.full((zcol.size,), float("nan"), dtype=torch.float64, device="cuda")
        st2, sing2, empty2 = cl.clair_local_weights_noalloc(*args, out)
        torch.cuda.synchronize()
        assert (st2, sing2, empty2) == (st, sing, empty), call
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got)), call
        assert rowwise_err(got, ref_h, zrp) <= tol, call
        # the same kernels in the same order: the same bits
        assert np.array_equal(got, ref_h), call


def test_noalloc_refuses_problem_beyond_its_scratch(cl):
    import torch
    n = 2_300_000                          # 16 n bytes alone exceed the 32 MiB array
    rowptr = torch.arange(n + 1, dtype=torch.int32, device="cuda")
    col = torch.arange(n, dtype=torch.int32, device="cuda")
    val = torch.ones(n, dtype=torch.float64, device="cuda")
    cf = torch.zeros(n, dtype=torch.int8, device="cuda")
    zrp = torch.zeros(1, dtype=torch.int32, device="cuda")
    zcol = torch.zeros(1, dtype=torch.int32, device="cuda")
    B = torch.ones(n, dtype=torch.float64, device="cuda")
    out = torch.full((1,), 7.0, dtype=torch.float64, device="cuda")
    with pytest.raises(cl.ClairError) as exc:
        cl.clair_local_weights_noalloc(rowptr, col, val, cf, 0, zrp, zcol, B, 0, out)
    assert exc.value.status == cl.CLAIR_ERR_CAPACITY
    assert "limit" in str(exc.value) and "bytes" in str(exc.value)
    assert out.item() == 7.0


def test_noalloc_refuses_large_local_system_before_writing(cl):
    """One pattern row with about 200 unknowns (beyond the 128 this entry point solves):
    the call is refused with CLAIR_ERR_CAPACITY before anything is written, and the next
    valid call still matches the allocating entry point bit for bit."""
    import torch
    A, cf, cpts, zrp, zcol, B = problem(wide_row=44)
    T = np.diff(zrp) - 1
    assert T.max() > 128 and T.max() <= 4096
    args = (dev(A.indptr, torch.int32), dev(A.indices, torch.int32), dev(A.data, torch.float64),
            dev(cf, torch.int8), cpts.size, dev(zrp, torch.int32), dev(zcol, torch.int32),
            dev(B, torch.float64), 0)
    out = torch.full((zcol.size,), 3.25, dtype=torch.float64, device="cuda")
    with pytest.raises(cl.ClairError) as exc:
        cl.clair_local_weights_noalloc(*args, out)
    assert exc.value.status == cl.CLAIR_ERR_CAPACITY
    assert "128" in str(exc.value)
    torch.cuda.synchronize()
    assert torch.all(out == 3.25).item()
    # the allocating entry point takes the same problem; the no-alloc one takes the valid one
    ref = torch.zeros(zcol.size, dtype=torch.float64, device="cuda")
    st, _, _ = cl.clair_local_weights(*args, ref)
    assert st == 0
    A2, cf2, cpts2, zrp2, zcol2, B2 = problem()
    args2 = (dev(A2.indptr, torch.int32), dev(A2.indices, torch.int32), dev(A2.data, torch.float64),
             dev(cf2, torch.int8), cpts2.size, dev(zrp2, torch.int32), dev(zcol2, torch.int32),
             dev(B2, torch.float64), 0)
    ref2 = torch.zeros(zcol2.size, dtype=torch.float64, device="cuda")
    cl.clair_local_weights(*args2, ref2)
    out2 = torch.full((zcol2.size,), float("nan"), dtype=torch.float64, device="cuda")
    cl.clair_local_weights_noalloc(*args2, out2)
    torch.cuda.synchronize()
    assert np.array_equal(out2.cpu().numpy(), ref2.cpu().numpy())
