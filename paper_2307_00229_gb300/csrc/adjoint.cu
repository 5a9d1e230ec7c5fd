// Adjoint gradient kernels: the operator gradient sampled on the sparsity of A and its
// chain rule to the fields of the 5-point upwind advection-diffusion discretization.
//
// Loss L = sum_r ||u_r - t_r||^2 with A u_r = f_r.  Differentiating A u_r = f_r gives
// A du_r = -dA u_r, so with the adjoint A^T lam_r = dL/du_r the gradient in a stored entry
// is dL/da_ij = -sum_r lam_r[i] u_r[j].  The entries of A are functions of per-node fields
// (the advection-diffusion problem of Section 4.2, Eq. 4.1, discretized by first-order
// upwind finite differences with harmonic-mean diffusion faces), so the field gradient
// is a gather over each node's stencil and its neighbours' stencils.
#include <cuda_runtime.h>

#include "common.cuh"

namespace clair {

// dA[e] = -sum_r lam[r][row(e)] * u[r][col(e)], one thread per row (FP64 arithmetic runs
// one row per thread: an FP64 warp instruction costs the same with 1 or 32 active lanes).
// Vectors are RHS-major: lam[r * n + i].  The sum over r runs in increasing r.
__global__ void sddmm_grad_kernel(const int* __restrict__ rowptr, const int* __restrict__ col,
                                  int n, int nrhs, const double* __restrict__ lam,
                                  const double* __restrict__ u, double* __restrict__ dA) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
    const int j = col[e];
    double acc = 0.0;
    for (int r = 0; r < nrhs; ++r)
      acc = fma(lam[(size_t)r * n + i], u[(size_t)r * n + j], acc);
    dA[e] = -acc;
  }
}

// Entry (k, k + off) of row k, or 0 when it is not stored.
__device__ __forceinline__ double stencil_entry(const int* __restrict__ rowptr,
                                                const int* __restrict__ col,
                                                const double* __restrict__ dA, int k, int j) {
  for (int e = rowptr[k]; e < rowptr[k + 1]; ++e)
    if (col[e] == j) return dA[e];
  return 0.0;
}

// Per node k of an nside x nside grid (x fastest):
//   deps[k] = sum over k's faces: interior face to Q, e_f = 2 e_k e_Q / (e_k + e_Q):
//             (g_kk - g_kQ + g_QQ - g_Qk) * 2 e_Q^2 / (e_k + e_Q)^2 / h^2;
//             boundary face (e_f = e_k): g_kk / h^2
//   dvx[k]  = g_kk sign(vx_k)/h - [vx_k > 0, west exists] g_kW/h + [vx_k < 0, east exists] g_kE/h
//   dvy[k]  likewise with south / north.
// bad counts rows that hold a column outside the 5-point stencil.
__global__ void advdiff2d_grad_kernel(int nside, double h, const double* __restrict__ eps,
                                      const double* __restrict__ vx,
                                      const double* __restrict__ vy,
                                      const int* __restrict__ rowptr,
                                      const int* __restrict__ col,
                                      const double* __restrict__ dA, double* __restrict__ deps,
                                      double* __restrict__ dvx, double* __restrict__ dvy,
                                      int* __restrict__ bad) {
  const int n = nside * nside;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int ix = k % nside, iy = k / nside;
  for (int e = rowptr[k]; e < rowptr[k + 1]; ++e) {
    const int d = col[e] - k;
    if (d != 0 && d != 1 && d != -1 && d != nside && d != -nside) atomicAdd(bad, 1);
  }
  const double inv_h = 1.0 / h;
  const double inv_h2 = inv_h * inv_h;
  const double gkk = stencil_entry(rowptr, col, dA, k, k);
  const double ek = eps[k];
  const int q[4] = {k - nside, k - 1, k + 1, k + nside};
  const bool valid[4] = {iy > 0, ix > 0, ix < nside - 1, iy < nside - 1};
  double de = 0.0;
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    if (valid[f]) {
      const int Q = q[f];
      const double eq = eps[Q];
      const double s = ek + eq;
      const double dface = 2.0 * eq * eq / (s * s);
      const double gface = gkk - stencil_entry(rowptr, col, dA, k, Q) +
                           stencil_entry(rowptr, col, dA, Q, Q) -
                           stencil_entry(rowptr, col, dA, Q, k);
      de += gface * dface * inv_h2;
    } else {
      de += gkk * inv_h2;
    }
  }
  deps[k] = de;
  const double vxk = vx[k], vyk = vy[k];
  double gx = gkk * (double)((vxk > 0.0) - (vxk < 0.0)) * inv_h;
  double gy = gkk * (double)((vyk > 0.0) - (vyk < 0.0)) * inv_h;
  if (vxk > 0.0 && ix > 0) gx -= stencil_entry(rowptr, col, dA, k, k - 1) * inv_h;
  if (vxk < 0.0 && ix < nside - 1) gx += stencil_entry(rowptr, col, dA, k, k + 1) * inv_h;
  if (vyk > 0.0 && iy > 0) gy -= stencil_entry(rowptr, col, dA, k, k - nside) * inv_h;
  if (vyk < 0.0 && iy < nside - 1) gy += stencil_entry(rowptr, col, dA, k, k + nside) * inv_h;
  dvx[k] = gx;
  dvy[k] = gy;
}

}  // namespace clair

using namespace clair;

extern "C" {

clair_status clair_sddmm_grad(int n, int nnz, const int* rowptr, const int* col, int nrhs,
                              const double* lambda, const double* u, double* dA,
                              void* stream) {
  CLAIR_API_BEGIN
  CLAIR_REQUIRE(rowptr && col && lambda && u && dA, CLAIR_ERR_ARG, "clair_sddmm_grad: null pointer");
  CLAIR_REQUIRE(n > 0 && nnz >= 0 && nrhs >= 1, CLAIR_ERR_ARG,
                "clair_sddmm_grad: bad sizes n=%d nnz=%d nrhs=%d", n, nnz, nrhs);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  validate_csr(rowptr, col, n, n, nnz, "A", s);
  sddmm_grad_kernel<<<ceil_div(n, 256), 256, 0, s>>>(rowptr, col, n, nrhs, lambda, u, dA);
  ::clair::count_launch();
  CLAIR_LAUNCHED();
  CLAIR_API_END
}

clair_status clair_advdiff2d_param_grad(int nside, double h, const double* eps, const double* vx,
                                        const double* vy, const int* rowptr, const int* col,
                                        int nnz, const double* dA, double* deps, double* dvx,
                                        double* dvy, void* stream) {
  CLAIR_API_BEGIN
  CLAIR_REQUIRE(eps && vx && vy && rowptr && col && dA && deps && dvx && dvy, CLAIR_ERR_ARG,
                "clair_advdiff2d_param_grad: null pointer");
  CLAIR_REQUIRE(nside > 0 && nside <= 46340 && h > 0.0, CLAIR_ERR_ARG,
                "clair_advdiff2d_param_grad: bad nside=%d or h", nside);
  const int n = nside * nside;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  validate_csr(rowptr, col, n, n, nnz, "A", s);
  int* bad = dalloc<int>(1, s);
  CLAIR_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
  advdiff2d_grad_kernel<<<ceil_div(n, 256), 256, 0, s>>>(nside, h, eps, vx, vy, rowptr, col, dA,
                                                          deps, dvx, dvy, bad);
  ::clair::count_launch();
  CLAIR_LAUNCHED();
  int hb = 0;
  CLAIR_CUDA(cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
  CLAIR_CUDA(cudaStreamSynchronize(s));
  dfree(bad, s);
  CLAIR_REQUIRE(hb == 0, CLAIR_ERR_ARG,
                "clair_advdiff2d_param_grad: %d entries outside the 5-point stencil", hb);
  CLAIR_API_END
}

}  // extern "C"
