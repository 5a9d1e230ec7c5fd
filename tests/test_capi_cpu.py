"""CPU-side checks of the CUDA library boundary (no kernel launches):

* the library builds for sm_103a and loads, and exports every function include/clair.h
  declares;
* argument validation returns an error status (never aborts) for null pointers;
* the Francis QR routine that turns the Arnoldi Hessenberg matrix into rho(D^-1 A),
  compiled for the host from the same header the kernels use, matches numpy's eigenvalues.
"""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "clair.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2307_00229_gb300 import clair
    return clair.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(clair_[a-z_0-9]+)\s*\(", text)))


def test_library_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert "clair_setup" in names and "clair_solve" in names and "clair_local_weights" in names
    out = subprocess.run(["nm", "-D", "--defined-only", lib._name], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (clair_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing


def test_library_is_built_for_sm103a(lib):
    from paper_2307_00229_gb300 import _build, clair
    assert clair.clair_compiled_arch() == 1030
    assert _build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_null_arguments_return_status(lib):
    from paper_2307_00229_gb300 import clair
    h = ctypes.c_void_p()
    st = lib.clair_setup(4, 4, None, None, None, 1, None, None, None, None, ctypes.byref(h))
    assert st == clair.CLAIR_ERR_ARG and h.value is None
    assert "null" in clair.clair_last_error()
    assert lib.clair_params_default(None) == clair.CLAIR_ERR_ARG
    assert lib.clair_free(None) == clair.CLAIR_OK
    p = clair.clair_params_default()
    assert p.theta_coarsen == 0.25 and p.theta_interp == 0.05 and p.degree == 2
    assert p.b_smooth_iters == 5 and p.arnoldi_iters == 15 and p.post_weighted == 0
    assert p.inverse == clair.CLAIR_INVERSE_EXACT and p.iterations == 1
    assert p.symmetric == 0 and p.krylov == clair.CLAIR_KRYLOV_FGMRES
    nseg = ctypes.c_int()
    assert lib.clair_solve_detail(None, ctypes.byref(nseg), None, None) == clair.CLAIR_ERR_ARG
    assert lib.clair_solve(None, None, None, 1, None, None, None) == clair.CLAIR_ERR_ARG


@pytest.fixture(scope="module")
def hessenberg(tmp_path_factory):
    d = tmp_path_factory.mktemp("hqr")
    src = d / "hqr.cpp"
    src.write_text('#include "hessenberg.cuh"\n'
                   'extern "C" double rho(double* H, int ld, int m) '
                   '{ return clair::hessenberg_spectral_radius(H, ld, m); }\n')
    so = d / "libhqr.so"
    csrc = os.path.join(ROOT, "paper_2307_00229_gb300", "csrc")
    subprocess.run(["g++", "-O2", "-shared", "-fPIC", "-I", csrc, str(src), "-o", str(so)], check=True)
    h = ctypes.CDLL(str(so))
    h.rho.restype = ctypes.c_double
    h.rho.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_int]
    return h


@pytest.mark.parametrize("seed", range(12))
def test_hessenberg_spectral_radius_matches_numpy(hessenberg, seed):
    rng = np.random.default_rng(seed)
    m = [1, 2, 3, 5, 8, 15, 15, 15, 10, 4, 15, 7][seed]
    H = np.triu(rng.standard_normal((m, m)), -1)
    if seed % 3 == 0:
        H += np.diag(np.full(m, 3.0))
    expect = np.max(np.abs(np.linalg.eigvals(H)))
    Hf = np.asfortranarray(H).copy(order="F")
    got = hessenberg.rho(Hf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), m, m)
    assert abs(got - expect) <= 1e-10 * max(1.0, expect)


def test_hessenberg_on_arnoldi_matrix(hessenberg):
    """The Hessenberg matrix of 15 Arnoldi steps on D^-1 A for an upwind problem."""
    import math
    import oracle as O
    import workloads
    A = O.csr_of(workloads.advdiff_2d(12, math.cos(0.5), math.sin(0.5), 1e-2))
    n = A.shape[0]
    dinv = 1.0 / A.diagonal()
    V = np.zeros((16, n))
    H = np.zeros((16, 15))
    v = workloads.uniform_pm1(3, n)
    V[0] = v / np.linalg.norm(v)
    for j in range(15):
        w = dinv * (A @ V[j])
        for i in range(j + 1):
            H[i, j] = V[i] @ w
            w -= H[i, j] * V[i]
        H[j + 1, j] = np.linalg.norm(w)
        V[j + 1] = w / H[j + 1, j]
    Hs = H[:15, :15]
    expect = np.max(np.abs(np.linalg.eigvals(Hs)))
    Hf = np.asfortranarray(Hs).copy(order="F")
    got = hessenberg.rho(Hf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 15, 15)
    assert abs(got - expect) <= 1e-10 * expect
