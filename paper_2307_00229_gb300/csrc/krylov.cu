// Segmented Krylov building blocks: many independent Krylov processes in lockstep, one
// per segment of a long vector.  A segment is one right-hand side of one instance (rows
// r * n + off[i] .. r * n + off[i + 1] - 1 for right-hand side r and instance i of a
// block-diagonal batch), so nrhs solves of a batch of ninst instances are nrhs * ninst
// independent FGMRES (or CG) runs that share every vector kernel launch and every V-cycle
// launch, each with its own Hessenberg matrix, rotations, step lengths and stopping test.
//
// Rows are cut into chunks that never straddle a segment; every vector kernel runs one
// block per chunk, so a block knows its segment without a per-row lookup.  Dot products
// are summed per chunk and then per segment over its chunks in a fixed order, so results
// do not depend on scheduling.
#include <algorithm>
#include <vector>

#include "common.cuh"

namespace clair {

constexpr int KR_THREADS = 256;
constexpr int KR_ROWS_PER_THREAD = 8;
constexpr int KR_CHUNK = KR_THREADS * KR_ROWS_PER_THREAD;  // rows per chunk (at most)
constexpr int KR_GROUP = 8;                                  // dot products per pass

void Segments::build(int nrhs, const std::vector<int>& off, cudaStream_t s) {
  release(s);
  const int ninst = (int)off.size() - 1;
  const long long n = off.back();
  nseg = nrhs * ninst;
  len = n * nrhs;
  std::vector<int> cseg;
  std::vector<long long> clo;
  std::vector<int> s0;
  for (int r = 0; r < nrhs; ++r)
    for (int i = 0; i < ninst; ++i) {
      s0.push_back((int)cseg.size());
      const long long lo = r * n + off[i], hi = r * n + off[i + 1];
      for (long long a = lo; a < hi; a += KR_CHUNK) {
        cseg.push_back(r * ninst + i);
        clo.push_back(a);
      }
    }
  s0.push_back((int)cseg.size());
  nchunk = (int)cseg.size();
  // chunk c covers [clo[c], min(clo[c] + KR_CHUNK, end of its segment))
  std::vector<long long> chi(nchunk);
  for (int c = 0; c < nchunk; ++c) {
    const int sg = cseg[c];
    const int r = sg / ninst, i = sg % ninst;
    chi[c] = std::min(clo[c] + KR_CHUNK, r * n + (long long)off[i + 1]);
  }
  chunk_seg = dalloc<int>(std::max(nchunk, 1), s);
  chunk_lo = dalloc<long long>(std::max(nchunk, 1), s);
  chunk_hi = dalloc<long long>(std::max(nchunk, 1), s);
  seg_chunk0 = dalloc<int>(nseg + 1, s);
  CLAIR_CUDA(cudaMemcpyAsync(chunk_seg, cseg.data(), sizeof(int) * nchunk, cudaMemcpyHostToDevice, s));
  CLAIR_CUDA(cudaMemcpyAsync(chunk_lo, clo.data(), sizeof(long long) * nchunk, cudaMemcpyHostToDevice, s));
  CLAIR_CUDA(cudaMemcpyAsync(chunk_hi, chi.data(), sizeof(long long) * nchunk, cudaMemcpyHostToDevice, s));
  CLAIR_CUDA(cudaMemcpyAsync(seg_chunk0, s0.data(), sizeof(int) * (nseg + 1), cudaMemcpyHostToDevice, s));
  // the host copies are pageable: make sure they are consumed before the vectors die
  CLAIR_CUDA(cudaStreamSynchronize(s));
}

void Segments::release(cudaStream_t s) {
  dfree(chunk_seg, s);
  dfree(chunk_lo, s);
  dfree(chunk_hi, s);
  dfree(seg_chunk0, s);
  nseg = nchunk = 0;
  len = 0;
}

// MG dot products (compile-time count, so no FP64 work for absent vectors) of the chunk's
// rows, summed over the block: warp trees, then the warps in order.
template <int MG>
__device__ __forceinline__ void dot_group(const double* __restrict__ V, long long ldv, int q0,
                                          const double* __restrict__ w, long long lo, long long hi,
                                          int nchunk, double* __restrict__ partial,
                                          double (*sh)[KR_THREADS / 32]) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  double acc[MG];
#pragma unroll
  for (int g = 0; g < MG; ++g) acc[g] = 0.0;
  for (long long i = lo + threadIdx.x; i < hi; i += KR_THREADS) {
    const double wi = w[i];
#pragma unroll
    for (int g = 0; g < MG; ++g) acc[g] = fma(V[(long long)(q0 + g) * ldv + i], wi, acc[g]);
  }
#pragma unroll
  for (int g = 0; g < MG; ++g) {
    const double v = warp_sum(acc[g]);
    if (lane == 0) sh[g][wid] = v;
  }
  __syncthreads();
  if (threadIdx.x < MG) {
    double v = 0.0;
    for (int k = 0; k < KR_THREADS / 32; ++k) v += sh[threadIdx.x][k];
    partial[(long long)(q0 + threadIdx.x) * nchunk + blockIdx.x] = v;
  }
  __syncthreads();
}

// partial[q * nchunk + c] = sum over the rows of chunk c of V_q[i] * w[i], q < m
// (V_q at V + q * ldv); rows in increasing order per thread, threads in a fixed tree.
__global__ void __launch_bounds__(KR_THREADS)
seg_dot_partial(const double* __restrict__ V, long long ldv, int m, const double* __restrict__ w,
                const long long* __restrict__ clo, const long long* __restrict__ chi, int nchunk,
                double* __restrict__ partial) {
  __shared__ double sh[KR_GROUP][KR_THREADS / 32];
  const int c = blockIdx.x;
  const long long lo = clo[c], hi = chi[c];
  for (int q0 = 0; q0 < m; q0 += KR_GROUP) {
    switch (min(KR_GROUP, m - q0)) {  // block-uniform
      case 1: dot_group<1>(V, ldv, q0, w, lo, hi, nchunk, partial, sh); break;
      case 2: dot_group<2>(V, ldv, q0, w, lo, hi, nchunk, partial, sh); break;
      case 3: dot_group<3>(V, ldv, q0, w, lo, hi, nchunk, partial, sh); break;
      case 4: dot_group<4>(V, ldv, q0, w, lo, hi, nchunk, partial, sh); break;
      case 5: dot_group<5>(V, ldv, q0, w, lo, hi, nchunk, partial, sh); break;
      case 6: dot_group<6>(V, ldv, q0, w, lo, hi, nchunk, partial, sh); break;
      case 7: dot_group<7>(V, ldv, q0, w, lo, hi, nchunk, partial, sh); break;
      default: dot_group<8>(V, ldv, q0, w, lo, hi, nchunk, partial, sh); break;
    }
  }
}

// out[seg * ldo + q] = sum over the segment's chunks of partial[q][chunk] (one warp per
// (segment, q), lanes over chunks in a fixed order)
__global__ void seg_dot_final(const double* __restrict__ partial, int nchunk, int m,
                              const int* __restrict__ seg_chunk0, int nseg, double* __restrict__ out,
                              int ldo) {
  const int warp = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (warp >= nseg * m) return;
  const int sg = warp / m, q = warp % m;
  double v = 0.0;
  for (int c = seg_chunk0[sg] + lane; c < seg_chunk0[sg + 1]; c += 32)
    v += partial[(long long)q * nchunk + c];
  v = warp_sum(v);
  if (lane == 0) out[(long long)sg * ldo + q] = v;
}

void seg_dot(const Segments& S, const double* V, long long ldv, int m, const double* w,
             double* out, int ldo, double* partial, cudaStream_t s) {
  if (m <= 0 || S.nseg == 0) return;
  seg_dot_partial<<<S.nchunk, KR_THREADS, 0, s>>>(V, ldv, m, w, S.chunk_lo, S.chunk_hi, S.nchunk,
                                                  partial); ::clair::count_launch();
  const long long warps = (long long)S.nseg * m;
  seg_dot_final<<<ceil_div(warps * 32, 256), 256, 0, s>>>(partial, S.nchunk, m, S.seg_chunk0, S.nseg,
                                                          out, ldo); ::clair::count_launch();
  CLAIR_LAUNCHED();
}

// w[i] -= sum_{q < m} coef[seg * ldc + q] * V_q[i]
__global__ void __launch_bounds__(KR_THREADS)
seg_axpy_kernel(const double* __restrict__ V, long long ldv, int m, const double* __restrict__ coef,
                int ldc, double* __restrict__ w, const int* __restrict__ cseg,
                const long long* __restrict__ clo, const long long* __restrict__ chi) {
  const int c = blockIdx.x;
  const long long lo = clo[c], hi = chi[c];
  const double* h = coef + (long long)cseg[c] * ldc;
  for (long long i = lo + threadIdx.x; i < hi; i += KR_THREADS) {
    double acc = w[i];
    for (int q = 0; q < m; ++q) acc = fma(-h[q], V[(long long)q * ldv + i], acc);
    w[i] = acc;
  }
}

void seg_axpy(const Segments& S, const double* V, long long ldv, int m, const double* coef,
              int ldc, double* w, cudaStream_t s) {
  if (m <= 0 || S.nchunk == 0) return;
  seg_axpy_kernel<<<S.nchunk, KR_THREADS, 0, s>>>(V, ldv, m, coef, ldc, w, S.chunk_seg, S.chunk_lo,
                                                  S.chunk_hi); ::clair::count_launch();
  CLAIR_LAUNCHED();
}

// y[i] = x[i] * f[seg * ldf]  (f per segment, device)
__global__ void __launch_bounds__(KR_THREADS)
seg_scale_kernel(const double* __restrict__ x, const double* __restrict__ f, int ldf,
                 double* __restrict__ y, const int* __restrict__ cseg,
                 const long long* __restrict__ clo, const long long* __restrict__ chi) {
  const int c = blockIdx.x;
  const long long lo = clo[c], hi = chi[c];
  const double a = f[(long long)cseg[c] * ldf];
  for (long long i = lo + threadIdx.x; i < hi; i += KR_THREADS) y[i] = x[i] * a;
}

void seg_scale(const Segments& S, const double* x, const double* f, int ldf, double* y,
               cudaStream_t s) {
  if (S.nchunk == 0) return;
  seg_scale_kernel<<<S.nchunk, KR_THREADS, 0, s>>>(x, f, ldf, y, S.chunk_seg, S.chunk_lo,
                                                   S.chunk_hi); ::clair::count_launch();
  CLAIR_LAUNCHED();
}

// y[i] += a[seg] * x[i] and, with z, z[i] = x2[i] + b[seg] * z[i]  (CG updates)
__global__ void __launch_bounds__(KR_THREADS)
seg_axpby_kernel(const double* __restrict__ x, const double* __restrict__ a, double* __restrict__ y,
                 const int* __restrict__ cseg, const long long* __restrict__ clo,
                 const long long* __restrict__ chi) {
  const int c = blockIdx.x;
  const long long lo = clo[c], hi = chi[c];
  const double f = a[cseg[c]];
  for (long long i = lo + threadIdx.x; i < hi; i += KR_THREADS) y[i] = fma(f, x[i], y[i]);
}

void seg_axpy1(const Segments& S, const double* x, const double* a, double* y, cudaStream_t s) {
  if (S.nchunk == 0) return;
  seg_axpby_kernel<<<S.nchunk, KR_THREADS, 0, s>>>(x, a, y, S.chunk_seg, S.chunk_lo, S.chunk_hi); ::clair::count_launch();
  CLAIR_LAUNCHED();
}

__global__ void __launch_bounds__(KR_THREADS)
seg_xpby_kernel(const double* __restrict__ x, const double* __restrict__ b, double* __restrict__ z,
                const int* __restrict__ cseg, const long long* __restrict__ clo,
                const long long* __restrict__ chi) {
  const int c = blockIdx.x;
  const long long lo = clo[c], hi = chi[c];
  const double f = b[cseg[c]];
  for (long long i = lo + threadIdx.x; i < hi; i += KR_THREADS) z[i] = fma(f, z[i], x[i]);
}

void seg_xpby(const Segments& S, const double* x, const double* b, double* z, cudaStream_t s) {
  if (S.nchunk == 0) return;
  seg_xpby_kernel<<<S.nchunk, KR_THREADS, 0, s>>>(x, b, z, S.chunk_seg, S.chunk_lo, S.chunk_hi); ::clair::count_launch();
  CLAIR_LAUNCHED();
}

// ------------------------------------------------------------------------------------
// FGMRES scalar steps, one thread per segment.  Per segment: g[m+1], cs[m], sn[m],
// H[(m+1) x m] column-major, and the state fields of SegState.
// ------------------------------------------------------------------------------------
// Start of a restart cycle: beta = ||r_seg||; a segment whose true residual already meets
// its tolerance (or whose right-hand side is zero) is inactive for the whole cycle.
// summary[0] = active segments, summary[1] = largest beta / tolerance among them.
__global__ void seg_gmres_start(int nseg, int m, const double* __restrict__ beta2,
                                const double* __restrict__ tol, double* __restrict__ g,
                                double* __restrict__ inv, int* __restrict__ active,
                                int* __restrict__ jend, double* __restrict__ summary) {
  __shared__ int s_act;
  __shared__ unsigned long long s_ratio;
  if (threadIdx.x == 0) {
    s_act = 0;
    s_ratio = 0ull;
  }
  __syncthreads();
  for (int sg = threadIdx.x; sg < nseg; sg += blockDim.x) {
    const double beta = sqrt(beta2[sg]);
    double* gs = g + (long long)sg * (m + 1);
    for (int i = 0; i <= m; ++i) gs[i] = 0.0;
    const bool act = beta > tol[sg];
    gs[0] = beta;
    inv[sg] = act ? 1.0 / beta : 0.0;
    active[sg] = act ? 1 : 0;
    jend[sg] = 0;
    const double ratio = beta / tol[sg];
    if (act) atomicAdd(&s_act, 1);
    if (act || !isfinite(beta))
      atomicMax(&s_ratio, isfinite(ratio) ? (unsigned long long)__double_as_longlong(ratio)
                                          : (unsigned long long)__double_as_longlong(INFINITY));
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    summary[0] = (double)s_act;
    summary[1] = __longlong_as_double((long long)s_ratio);
  }
}

// Column j of each active segment's Hessenberg matrix from the two Gram-Schmidt passes
// (h1 + h2) and ||w||^2, the rotations, the new residual estimate; a segment whose
// estimate meets its tolerance stops (its later basis vectors are zero).  summary[0] =
// number of segments still active, summary[1] = largest estimate / tolerance among them.
__global__ void seg_gmres_givens(int nseg, int m, int j, const double* __restrict__ h1,
                                 const double* __restrict__ h2, int ldh12,
                                 const double* __restrict__ wn2, double* __restrict__ H,
                                 double* __restrict__ cs, double* __restrict__ sn,
                                 double* __restrict__ g, double* __restrict__ inv,
                                 int* __restrict__ active, int* __restrict__ jend,
                                 int* __restrict__ its, const double* __restrict__ tol,
                                 double* __restrict__ summary) {
  __shared__ int s_act;
  __shared__ unsigned long long s_ratio;
  if (threadIdx.x == 0) {
    s_act = 0;
    s_ratio = 0ull;
  }
  __syncthreads();
  for (int sg = threadIdx.x; sg < nseg; sg += blockDim.x) {
    if (!active[sg]) continue;
    double* col = H + ((long long)sg * m + j) * (m + 1);
    double* css = cs + (long long)sg * m;
    double* sns = sn + (long long)sg * m;
    double* gs = g + (long long)sg * (m + 1);
    const double* a1 = h1 + (long long)sg * ldh12;
    const double* a2 = h2 + (long long)sg * ldh12;
    for (int i = 0; i <= j; ++i) col[i] = a1[i] + a2[i];
    const double hn = sqrt(wn2[sg]);
    col[j + 1] = hn;
    inv[sg] = hn > 0.0 ? 1.0 / hn : 0.0;
    for (int i = 0; i < j; ++i) {
      const double t = css[i] * col[i] + sns[i] * col[i + 1];
      col[i + 1] = -sns[i] * col[i] + css[i] * col[i + 1];
      col[i] = t;
    }
    const double den = hypot(col[j], col[j + 1]);
    css[j] = den > 0.0 ? col[j] / den : 1.0;
    sns[j] = den > 0.0 ? col[j + 1] / den : 0.0;
    col[j] = den;
    col[j + 1] = 0.0;
    gs[j + 1] = -sns[j] * gs[j];
    gs[j] = css[j] * gs[j];
    const double est = fabs(gs[j + 1]);
    its[sg] += 1;
    jend[sg] = j + 1;
    const double ratio = est / tol[sg];
    if (!(est > tol[sg]) || hn == 0.0) {
      // converged (or a nonfinite estimate, which the host sees in the ratio) or an
      // invariant subspace: this segment's cycle ends here
      active[sg] = 0;
      inv[sg] = 0.0;
      if (!isfinite(ratio)) atomicMax(&s_ratio, __double_as_longlong(INFINITY));
    } else {
      atomicAdd(&s_act, 1);
      atomicMax(&s_ratio, (unsigned long long)__double_as_longlong(ratio));  // ratio >= 0
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    summary[0] = (double)s_act;
    summary[1] = __longlong_as_double((long long)s_ratio);
  }
}

// y = R^-1 g over each segment's own jend columns; stores -y (the update is w -= Z (-y)).
__global__ void seg_gmres_backsolve(int nseg, int m, const double* __restrict__ H,
                                    const double* __restrict__ g, const int* __restrict__ jend,
                                    double* __restrict__ ny) {
  const int sg = blockIdx.x * blockDim.x + threadIdx.x;
  if (sg >= nseg) return;
  const double* Hs = H + (long long)sg * m * (m + 1);
  const double* gs = g + (long long)sg * (m + 1);
  double* ys = ny + (long long)sg * m;
  const int je = jend[sg];
  for (int i = 0; i < m; ++i) ys[i] = 0.0;
  for (int i = je - 1; i >= 0; --i) {
    double acc = gs[i];
    for (int c = i + 1; c < je; ++c) acc -= Hs[(long long)c * (m + 1) + i] * (-ys[c]);
    const double d = Hs[(long long)i * (m + 1) + i];
    ys[i] = -(d != 0.0 ? acc / d : 0.0);
  }
}

void seg_gmres_start_launch(int nseg, int m, const double* beta2, const double* tol, double* g,
                            double* inv, int* active, int* jend, double* summary, cudaStream_t s) {
  seg_gmres_start<<<1, 256, 0, s>>>(nseg, m, beta2, tol, g, inv, active, jend, summary); ::clair::count_launch();
  CLAIR_LAUNCHED();
}

void seg_gmres_givens_launch(int nseg, int m, int j, const double* h1, const double* h2, int ldh12,
                             const double* wn2, double* H, double* cs, double* sn, double* g,
                             double* inv, int* active, int* jend, int* its, const double* tol,
                             double* summary, cudaStream_t s) {
  seg_gmres_givens<<<1, 256, 0, s>>>(nseg, m, j, h1, h2, ldh12, wn2, H, cs, sn, g, inv, active, jend,
                                     its, tol, summary); ::clair::count_launch();
  CLAIR_LAUNCHED();
}

void seg_gmres_backsolve_launch(int nseg, int m, const double* H, const double* g, const int* jend,
                                double* ny, cudaStream_t s) {
  seg_gmres_backsolve<<<ceil_div(nseg, 128), 128, 0, s>>>(nseg, m, H, g, jend, ny); ::clair::count_launch();
  CLAIR_LAUNCHED();
}

// ------------------------------------------------------------------------------------
// CG scalar steps (one thread per segment).
// ------------------------------------------------------------------------------------
// alpha = rho / (p, A p) for active segments, 0 for the others (their vectors freeze)
__global__ void seg_cg_alpha(int nseg, const double* __restrict__ rho, const double* __restrict__ pq,
                             const int* __restrict__ active, double* __restrict__ alpha,
                             double* __restrict__ malpha) {
  const int sg = blockIdx.x * blockDim.x + threadIdx.x;
  if (sg >= nseg) return;
  const double a = (active[sg] && pq[sg] != 0.0) ? rho[sg] / pq[sg] : 0.0;
  alpha[sg] = a;
  malpha[sg] = -a;
}

// after r -= alpha A p: test ||r||, then beta = rho_new / rho (0 when inactive)
__global__ void seg_cg_beta(int nseg, const double* __restrict__ rr, const double* __restrict__ tol,
                            const double* __restrict__ rho_new, double* __restrict__ rho,
                            int* __restrict__ active, int* __restrict__ its,
                            double* __restrict__ beta, double* __restrict__ summary) {
  __shared__ int s_act;
  __shared__ unsigned long long s_ratio;
  if (threadIdx.x == 0) {
    s_act = 0;
    s_ratio = 0ull;
  }
  __syncthreads();
  for (int sg = threadIdx.x; sg < nseg; sg += blockDim.x) {
    double b = 0.0;
    if (active[sg]) {
      its[sg] += 1;
      const double est = sqrt(rr[sg]);
      const double ratio = est / tol[sg];
      if (!(est > tol[sg])) {
        active[sg] = 0;
        if (!isfinite(ratio)) atomicMax(&s_ratio, __double_as_longlong(INFINITY));
      } else {
        b = rho[sg] != 0.0 ? rho_new[sg] / rho[sg] : 0.0;
        rho[sg] = rho_new[sg];
        atomicAdd(&s_act, 1);
        atomicMax(&s_ratio, (unsigned long long)__double_as_longlong(ratio));
      }
    }
    beta[sg] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    summary[0] = (double)s_act;
    summary[1] = __longlong_as_double((long long)s_ratio);
  }
}

__global__ void seg_cg_start(int nseg, const double* __restrict__ rr, const double* __restrict__ tol,
                             const double* __restrict__ rz, double* __restrict__ rho,
                             int* __restrict__ active, double* __restrict__ summary) {
  __shared__ int s_act;
  __shared__ unsigned long long s_ratio;
  if (threadIdx.x == 0) {
    s_act = 0;
    s_ratio = 0ull;
  }
  __syncthreads();
  for (int sg = threadIdx.x; sg < nseg; sg += blockDim.x) {
    const double beta = sqrt(rr[sg]);
    const bool act = beta > tol[sg];
    active[sg] = act ? 1 : 0;
    rho[sg] = rz[sg];
    const double ratio = beta / tol[sg];
    if (act) atomicAdd(&s_act, 1);
    if (act || !isfinite(beta))
      atomicMax(&s_ratio, isfinite(ratio) ? (unsigned long long)__double_as_longlong(ratio)
                                          : (unsigned long long)__double_as_longlong(INFINITY));
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    summary[0] = (double)s_act;
    summary[1] = __longlong_as_double((long long)s_ratio);
  }
}

void seg_cg_alpha_launch(int nseg, const double* rho, const double* pq, const int* active,
                         double* alpha, double* malpha, cudaStream_t s) {
  seg_cg_alpha<<<ceil_div(nseg, 128), 128, 0, s>>>(nseg, rho, pq, active, alpha, malpha); ::clair::count_launch();
  CLAIR_LAUNCHED();
}

void seg_cg_beta_launch(int nseg, const double* rr, const double* tol, const double* rho_new,
                        double* rho, int* active, int* its, double* beta, double* summary,
                        cudaStream_t s) {
  seg_cg_beta<<<1, 256, 0, s>>>(nseg, rr, tol, rho_new, rho, active, its, beta, summary); ::clair::count_launch();
  CLAIR_LAUNCHED();
}

void seg_cg_start_launch(int nseg, const double* rr, const double* tol, const double* rz,
                         double* rho, int* active, double* summary, cudaStream_t s) {
  seg_cg_start<<<1, 256, 0, s>>>(nseg, rr, tol, rz, rho, active, summary); ::clair::count_launch();
  CLAIR_LAUNCHED();
}

// tol[seg] = rtol * ||f_seg|| from fnorm2; zero right-hand sides: u_seg = 0 (below)
__global__ void seg_tolerance(int nseg, const double* __restrict__ fn2, double rtol,
                              double* __restrict__ tol, double* __restrict__ fnorm) {
  const int sg = blockIdx.x * blockDim.x + threadIdx.x;
  if (sg >= nseg) return;
  const double f = sqrt(fn2[sg]);
  fnorm[sg] = f;
  tol[sg] = rtol * f;
}

__global__ void __launch_bounds__(KR_THREADS)
seg_zero_where(const double* __restrict__ fnorm, double* __restrict__ u,
               const int* __restrict__ cseg, const long long* __restrict__ clo,
               const long long* __restrict__ chi) {
  const int c = blockIdx.x;
  if (fnorm[cseg[c]] != 0.0) return;
  for (long long i = clo[c] + threadIdx.x; i < chi[c]; i += KR_THREADS) u[i] = 0.0;
}

void seg_tolerance_launch(const Segments& S, const double* fn2, double rtol, double* tol,
                          double* fnorm, double* u, cudaStream_t s) {
  seg_tolerance<<<ceil_div(S.nseg, 128), 128, 0, s>>>(S.nseg, fn2, rtol, tol, fnorm); ::clair::count_launch();
  seg_zero_where<<<S.nchunk, KR_THREADS, 0, s>>>(fnorm, u, S.chunk_seg, S.chunk_lo, S.chunk_hi); ::clair::count_launch();
  CLAIR_LAUNCHED();
}

}  // namespace clair
