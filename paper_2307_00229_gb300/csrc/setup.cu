// Setup kernels of the CLAIR hierarchy (one level at a time):
//  * classical strength of connection (absolute values, Section 3.1.3) as masks over A
//    and A^T,
//  * the C/F splitting: a deterministic parallel independent-set reading of the
//    Ruge-Stueben first pass ("FC"), keyed by (lambda_i, lowbias32(i)),
//  * the sparsity pattern W = pattern(((S + I)^{m-1} T)|_F) of Algorithm 1 for m <= 2,
//  * the relaxation weight 1/rho(D^-1 A) from Arnoldi (Section 4), with a Francis
//    double-shift QR for the Ritz values,
//  * weighted Jacobi on the C or F subset (CFF / FFC, Section 4; also smooths B),
//  * the dense inverse of the coarsest operator.
#include <limits.h>
#include <math.h>

#include <algorithm>
#include <utility>
#include <new>
#include <vector>

#include <cooperative_groups.h>

#include "common.cuh"
#include "hessenberg.cuh"

namespace clair {

// ------------------------------------------------------------------------------------
// Strength masks.  mode 0: entry (r, c) of M is strong iff |m_rc| >= theta * thr[r]
// (row-relative, thr = row maxima of M); mode 1: iff |m_rc| >= theta * thr[c]
// (column-relative: thr = row maxima of M^T).  Diagonal and zero entries are never strong.
// ------------------------------------------------------------------------------------
// Two masks of the same matrix in one pass over its entries (the coarsening and the
// interpolation thresholds): mask1 with (thr1, theta1, mode1), mask2 with (thr2, theta2,
// mode2).  W lanes per row (entries e0 + lane, e0 + lane + W, ...): short rows one per
// thread, the long rows of coarse levels spread over lanes.
template <int W>
__global__ void strength_mask2(const int* __restrict__ rowptr, const int* __restrict__ col,
                               const double* __restrict__ val, int rows,
                               const double* __restrict__ thr1, double theta1, int mode1,
                               unsigned char* __restrict__ mask1,
                               const double* __restrict__ thr2, double theta2, int mode2,
                               unsigned char* __restrict__ mask2) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int r = (int)(t / W), lane = (int)(t % W);
  if (r >= rows) return;
  const double tr1 = mode1 == 0 ? theta1 * thr1[r] : 0.0;
  const double tr2 = mode2 == 0 ? theta2 * thr2[r] : 0.0;
  for (int e = rowptr[r] + lane; e < rowptr[r + 1]; e += W) {
    const int c = col[e];
    const double a = fabs(val[e]);
    const double th1 = mode1 == 0 ? tr1 : theta1 * thr1[c];
    const double th2 = mode2 == 0 ? tr2 : theta2 * thr2[c];
    const bool off = c != r && a > 0.0;
    mask1[e] = (off && a >= th1) ? 1 : 0;
    mask2[e] = (off && a >= th2) ? 1 : 0;
  }
}

void strength2(const Csr& M, const double* thr1, double theta1, int mode1, unsigned char* mask1,
               const double* thr2, double theta2, int mode2, unsigned char* mask2,
               cudaStream_t s) {
  if (!M.rows) return;
  const double avg = (double)M.nnz / M.rows;
  int W = 1;
  while (W < 32 && 4 * W < avg) W <<= 1;
  const int blocks = ceil_div((long long)M.rows * W, 256);
  switch (W) {
#define CLAIR_SM2_CASE(WW)                                                                   \
  case WW:                                                                                   \
    strength_mask2<WW><<<blocks, 256, 0, s>>>(M.rowptr, M.col, M.val, M.rows, thr1, theta1, \
                                              mode1, mask1, thr2, theta2, mode2, mask2);    \
    break;
    CLAIR_SM2_CASE(1)
    CLAIR_SM2_CASE(2)
    CLAIR_SM2_CASE(4)
    CLAIR_SM2_CASE(8)
    CLAIR_SM2_CASE(16)
    CLAIR_SM2_CASE(32)
#undef CLAIR_SM2_CASE
  }
  ::clair::count_launch();
  CLAIR_LAUNCHED();
}


// ------------------------------------------------------------------------------------
// C/F splitting.  sA: mask of S over A's entries (row i of A: S_ij, i depends on j);
// sAt: mask over A^T's entries (row i of A^T: S_ji, j depends on i).
// state: 0 undecided, 1 C, 2 F.
// ------------------------------------------------------------------------------------
enum : signed char { ST_U = 0, ST_C = 1, ST_F = 2 };

#define CLAIR_DISPATCH_W2(W, ...)                            \
  switch (W) {                                               \
    case 1: { constexpr int WW = 1; __VA_ARGS__; ::clair::count_launch(); } break;   \
    case 2: { constexpr int WW = 2; __VA_ARGS__; ::clair::count_launch(); } break;   \
    case 4: { constexpr int WW = 4; __VA_ARGS__; ::clair::count_launch(); } break;   \
    case 8: { constexpr int WW = 8; __VA_ARGS__; ::clair::count_launch(); } break;   \
    case 16: { constexpr int WW = 16; __VA_ARGS__; ::clair::count_launch(); } break; \
    default: { constexpr int WW = 32; __VA_ARGS__; ::clair::count_launch(); } break; \
  }

// The splitting kernels take W lanes per point (coarse operators have rows of a hundred
// entries; one lane per row would walk them one dependent load at a time).  Rows of a
// warp's groups are consecutive; every lane takes part in the group reductions.
template <int W>
__device__ __forceinline__ int group_or(int v) {
#pragma unroll
  for (int o = W / 2; o > 0; o >>= 1) v |= __shfl_xor_sync(0xffffffffu, v, o, W);
  return v;
}

template <int W>
__global__ void pmis_init(const int* __restrict__ Atrp, const unsigned char* __restrict__ sAt,
                          int n, const int* __restrict__ lbase, unsigned long long* __restrict__ key,
                          signed char* __restrict__ state, int* __restrict__ mark) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int i = (int)(t / W), sub = (int)(t % W);
  const bool ok = i < n;
  unsigned lam = 0;
  if (ok)
    for (int e = Atrp[i] + sub; e < Atrp[i + 1]; e += W) lam += sAt[e];
  lam = group_sum<W>(lam);
  if (!ok || sub != 0) return;
  // the hash takes the index within the point's instance (a batch is block-diagonal)
  key[i] = ((unsigned long long)lam << 32) | lowbias32((uint32_t)(i - (lbase ? lbase[i] : 0)));
  state[i] = lam == 0 ? ST_F : ST_U;
  mark[i] = -1;
}

// An undecided point whose key exceeds every undecided strong neighbour's becomes C.
template <int W>
__global__ void pmis_select(const int* __restrict__ Arp, const int* __restrict__ Acol,
                            const unsigned char* __restrict__ sA, const int* __restrict__ Atrp,
                            const int* __restrict__ Atcol, const unsigned char* __restrict__ sAt,
                            int n, const unsigned long long* __restrict__ key,
                            const signed char* __restrict__ state, int* __restrict__ mark,
                            int round) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int i = (int)(t / W), sub = (int)(t % W);
  const bool act = i < n && state[i] == ST_U;
  int beaten = 0;
  if (act) {
    const unsigned long long k = key[i];
    for (int e = Arp[i] + sub; e < Arp[i + 1] && !beaten; e += W)
      if (sA[e]) {
        const int j = Acol[e];
        beaten = state[j] == ST_U && key[j] > k;
      }
    for (int e = Atrp[i] + sub; e < Atrp[i + 1] && !beaten; e += W)
      if (sAt[e]) {
        const int j = Atcol[e];
        beaten = state[j] == ST_U && key[j] > k;
      }
  }
  beaten = group_or<W>(beaten);
  if (act && sub == 0 && !beaten) mark[i] = round;
}

// New C-points are fixed; undecided points strongly depending on one become F.
template <int W>
__global__ void pmis_update(const int* __restrict__ Arp, const int* __restrict__ Acol,
                            const unsigned char* __restrict__ sA, int n,
                            const int* __restrict__ mark, signed char* __restrict__ state,
                            int round, int* __restrict__ remaining) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int i = (int)(t / W), sub = (int)(t % W);
  const bool act = i < n && state[i] == ST_U;
  const bool newc = act && mark[i] == round;
  int dep = 0;
  if (act && !newc)
    for (int e = Arp[i] + sub; e < Arp[i + 1] && !dep; e += W)
      dep = sA[e] && mark[Acol[e]] == round;
  dep = group_or<W>(dep);
  if (!act || sub != 0) return;
  if (newc)
    state[i] = ST_C;
  else if (dep)
    state[i] = ST_F;
  else
    atomicAdd(remaining, 1);
}

// F-points with a strong dependence but none on a C-point.
template <int W>
__global__ void pmis_fixup_find(const int* __restrict__ Arp, const int* __restrict__ Acol,
                                const unsigned char* __restrict__ sA, int n,
                                const signed char* __restrict__ state, int* __restrict__ mark) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int i = (int)(t / W), sub = (int)(t % W);
  const bool act = i < n && state[i] == ST_F;
  int has = 0, hasc = 0;
  if (act)
    for (int e = Arp[i] + sub; e < Arp[i + 1]; e += W)
      if (sA[e]) {
        has = 1;
        if (state[Acol[e]] == ST_C) {
          hasc = 1;
          break;
        }
      }
  has = group_or<W>(has);
  hasc = group_or<W>(hasc);
  if (i < n && sub == 0) mark[i] = (act && has && !hasc) ? 1 : 0;
}

__global__ void pmis_finish(int n, const int* __restrict__ mark, const signed char* __restrict__ state,
                            signed char* __restrict__ cf) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  cf[i] = (state[i] == ST_C || mark[i] == 1) ? 1 : 0;
}

void split_fc(const Csr& A, const Csr& At, const unsigned char* sA, const unsigned char* sAt,
              const int* lbase, signed char* cf, cudaStream_t s) {
  const int n = A.rows;
  if (!n) return;
  unsigned long long* key = dalloc<unsigned long long>(n, s);
  signed char* state = dalloc<signed char>(n, s);
  int* mark = dalloc<int>(n, s);
  int* remaining = dalloc<int>(1, s);
  const int g = ceil_div(n, 256);
  // lanes per point from the mean row length of A (the longer of the two walks)
  const double avg = (double)A.nnz / n;
  int W = 1;
  while (W < 32 && 4 * W < avg) W <<= 1;
  const int gw = (int)ceil_div((long long)n * W, 256);
  CLAIR_DISPATCH_W2(W, (pmis_init<WW><<<gw, 256, 0, s>>>(At.rowptr, sAt, n, lbase, key, state, mark)));
  CLAIR_LAUNCHED();
  // Rounds go in groups between host checks (six, then three: the stencil hierarchies
  // here take six to nine): a round after the last undecided point is decided changes
  // nothing, and the check reads the last round's count.
  for (int round = 0;;) {
    CLAIR_REQUIRE(round < 10000, CLAIR_ERR_CAPACITY, "C/F splitting did not terminate");
    const int group = round == 0 ? 6 : 3;
    for (int q = 0; q < group; ++q, ++round) {
      CLAIR_CUDA(cudaMemsetAsync(remaining, 0, sizeof(int), s));
      CLAIR_DISPATCH_W2(W, (pmis_select<WW><<<gw, 256, 0, s>>>(A.rowptr, A.col, sA, At.rowptr, At.col,
                                                             sAt, n, key, state, mark, round)));
      CLAIR_DISPATCH_W2(W, (pmis_update<WW><<<gw, 256, 0, s>>>(A.rowptr, A.col, sA, n, mark, state,
                                                             round, remaining)));
    }
    CLAIR_LAUNCHED();
    int h = 0;
    CLAIR_CUDA(cudaMemcpyAsync(&h, remaining, sizeof(int), cudaMemcpyDeviceToHost, s));
    CLAIR_CUDA(cudaStreamSynchronize(s));
    if (h == 0) break;
  }
  CLAIR_DISPATCH_W2(W, (pmis_fixup_find<WW><<<gw, 256, 0, s>>>(A.rowptr, A.col, sA, n, state, mark)));
  pmis_finish<<<g, 256, 0, s>>>(n, mark, state, cf); ::clair::count_launch();
  CLAIR_LAUNCHED();
  dfree(key, s);
  dfree(state, s);
  dfree(mark, s);
  dfree(remaining, s);
}

// ------------------------------------------------------------------------------------
// Aggregation ("Agg" coarsening): roots form a distance-two independent set of the
// symmetrised strength graph G (neighbours of i: strong entries of row i of A and of row
// i of A^T), chosen in rounds by the largest key (lambda_i, lowbias32(i)) among the
// undecided points within distance two; every point within distance two of a new root
// is decided.  Points without G-neighbours stay out of every aggregate.  A point next
// to a root joins it (roots are at least three apart, so it is unique); every other
// point joins the adjacent aggregate of lowest index.  Roots become the C-points,
// numbered in increasing point index.
// ------------------------------------------------------------------------------------
int coarse_points(const signed char* cf, int n, int** cpts_out, cudaStream_t s);

struct GraphG {
  const int* Arp;
  const int* Acol;
  const unsigned char* sA;
  const int* Atrp;
  const int* Atcol;
  const unsigned char* sAt;
};

__global__ void agg_init(GraphG g, int n, const int* __restrict__ lbase,
                         unsigned long long* __restrict__ key, signed char* __restrict__ und,
                         signed char* __restrict__ iso, signed char* __restrict__ root) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  unsigned lam = 0;
  for (int e = g.Atrp[i]; e < g.Atrp[i + 1]; ++e) lam += g.sAt[e];
  bool has = lam > 0;
  for (int e = g.Arp[i]; e < g.Arp[i + 1] && !has; ++e) has = g.sA[e] != 0;
  key[i] = ((unsigned long long)lam << 32) | lowbias32((uint32_t)(i - (lbase ? lbase[i] : 0)));
  und[i] = has ? 1 : 0;
  iso[i] = has ? 0 : 1;
  root[i] = 0;
}

// m1_i = max over i and its G-neighbours of (undecided ? key : 0)
__global__ void agg_max1(GraphG g, int n, const unsigned long long* __restrict__ key,
                         const signed char* __restrict__ und, unsigned long long* __restrict__ m1) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  unsigned long long m = und[i] ? key[i] : 0ull;
  for (int e = g.Arp[i]; e < g.Arp[i + 1]; ++e)
    if (g.sA[e]) {
      const int j = g.Acol[e];
      if (und[j] && key[j] > m) m = key[j];
    }
  for (int e = g.Atrp[i]; e < g.Atrp[i + 1]; ++e)
    if (g.sAt[e]) {
      const int j = g.Atcol[e];
      if (und[j] && key[j] > m) m = key[j];
    }
  m1[i] = m;
}

// m2_i = max(m1 over i and its G-neighbours); an undecided point with key == m2 is a root
__global__ void agg_max2(GraphG g, int n, const unsigned long long* __restrict__ key,
                         const signed char* __restrict__ und,
                         const unsigned long long* __restrict__ m1,
                         signed char* __restrict__ newr, signed char* __restrict__ root) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  unsigned long long m = m1[i];
  for (int e = g.Arp[i]; e < g.Arp[i + 1]; ++e)
    if (g.sA[e] && m1[g.Acol[e]] > m) m = m1[g.Acol[e]];
  for (int e = g.Atrp[i]; e < g.Atrp[i + 1]; ++e)
    if (g.sAt[e] && m1[g.Atcol[e]] > m) m = m1[g.Atcol[e]];
  const bool r = und[i] && key[i] == m;
  newr[i] = r ? 1 : 0;
  if (r) root[i] = 1;
}

// out_i = 1 if some G-neighbour of i has in_j != 0
__global__ void agg_near(GraphG g, int n, const signed char* __restrict__ in,
                         signed char* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  bool hit = false;
  for (int e = g.Arp[i]; e < g.Arp[i + 1] && !hit; ++e) hit = g.sA[e] && in[g.Acol[e]];
  for (int e = g.Atrp[i]; e < g.Atrp[i + 1] && !hit; ++e) hit = g.sAt[e] && in[g.Atcol[e]];
  out[i] = hit ? 1 : 0;
}

// decides every point within distance two of a new root; counts the undecided rest
__global__ void agg_decide(GraphG g, int n, const signed char* __restrict__ newr,
                           const signed char* __restrict__ near1, signed char* __restrict__ und,
                           int* __restrict__ remaining) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || !und[i]) return;
  bool hit = newr[i] || near1[i];
  for (int e = g.Arp[i]; e < g.Arp[i + 1] && !hit; ++e) hit = g.sA[e] && near1[g.Acol[e]];
  for (int e = g.Atrp[i]; e < g.Atrp[i + 1] && !hit; ++e) hit = g.sAt[e] && near1[g.Atcol[e]];
  if (hit)
    und[i] = 0;
  else
    atomicAdd(remaining, 1);
}

__global__ void agg_root_index(const int* __restrict__ cpts, int nc, int* __restrict__ cidx) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < nc) cidx[cpts[r]] = r;
}

// first_j: the root's own index, the unique adjacent root's index, or -1
__global__ void agg_first(GraphG g, int n, const signed char* __restrict__ root,
                          const signed char* __restrict__ iso, const int* __restrict__ cidx,
                          int* __restrict__ first, int* __restrict__ err) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  if (root[j]) {
    first[j] = cidx[j];
    return;
  }
  int found = -1;
  if (!iso[j]) {
    for (int e = g.Arp[j]; e < g.Arp[j + 1]; ++e)
      if (g.sA[e] && root[g.Acol[e]]) {
        const int r = g.Acol[e];
        if (found >= 0 && found != r) atomicAdd(err, 1);
        found = r;
      }
    for (int e = g.Atrp[j]; e < g.Atrp[j + 1]; ++e)
      if (g.sAt[e] && root[g.Atcol[e]]) {
        const int r = g.Atcol[e];
        if (found >= 0 && found != r) atomicAdd(err, 1);
        found = r;
      }
  }
  first[j] = found >= 0 ? cidx[found] : -1;
}

// remaining points: the lowest aggregate index among their G-neighbours' first choices
__global__ void agg_final(GraphG g, int n, const signed char* __restrict__ iso,
                          const int* __restrict__ first, int* __restrict__ agg,
                          int* __restrict__ err) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  int a = first[j];
  if (a < 0 && !iso[j]) {
    int best = INT_MAX;
    for (int e = g.Arp[j]; e < g.Arp[j + 1]; ++e)
      if (g.sA[e] && first[g.Acol[e]] >= 0) best = min(best, first[g.Acol[e]]);
    for (int e = g.Atrp[j]; e < g.Atrp[j + 1]; ++e)
      if (g.sAt[e] && first[g.Atcol[e]] >= 0) best = min(best, first[g.Atcol[e]]);
    if (best == INT_MAX) atomicAdd(err, 1);
    a = best == INT_MAX ? -1 : best;
  }
  agg[j] = a;
}

__global__ void agg_to_cf(int n, const signed char* __restrict__ root, signed char* __restrict__ cf) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) cf[i] = root[i];
}

void aggregate(const Csr& A, const Csr& At, const unsigned char* sA, const unsigned char* sAt,
               const int* lbase, signed char* cf, int* agg, cudaStream_t s) {
  const int n = A.rows;
  if (!n) return;
  const GraphG g{A.rowptr, A.col, sA, At.rowptr, At.col, sAt};
  unsigned long long* key = dalloc<unsigned long long>(n, s);
  unsigned long long* m1 = dalloc<unsigned long long>(n, s);
  signed char* und = dalloc<signed char>(n, s);
  signed char* iso = dalloc<signed char>(n, s);
  signed char* root = dalloc<signed char>(n, s);
  signed char* newr = dalloc<signed char>(n, s);
  signed char* near1 = dalloc<signed char>(n, s);
  int* remaining = dalloc<int>(2, s);
  const int gr = ceil_div(n, 256);
  agg_init<<<gr, 256, 0, s>>>(g, n, lbase, key, und, iso, root); ::clair::count_launch();
  CLAIR_LAUNCHED();
  for (int round = 0;; ++round) {
    CLAIR_REQUIRE(round < 10000, CLAIR_ERR_CAPACITY, "aggregation did not terminate");
    CLAIR_CUDA(cudaMemsetAsync(remaining, 0, sizeof(int), s));
    agg_max1<<<gr, 256, 0, s>>>(g, n, key, und, m1); ::clair::count_launch();
    agg_max2<<<gr, 256, 0, s>>>(g, n, key, und, m1, newr, root); ::clair::count_launch();
    agg_near<<<gr, 256, 0, s>>>(g, n, newr, near1); ::clair::count_launch();
    agg_decide<<<gr, 256, 0, s>>>(g, n, newr, near1, und, remaining); ::clair::count_launch();
    CLAIR_LAUNCHED();
    int h = 0;
    CLAIR_CUDA(cudaMemcpyAsync(&h, remaining, sizeof(int), cudaMemcpyDeviceToHost, s));
    CLAIR_CUDA(cudaStreamSynchronize(s));
    if (h == 0) break;
  }
  agg_to_cf<<<gr, 256, 0, s>>>(n, root, cf); ::clair::count_launch();
  CLAIR_LAUNCHED();
  int* cpts = nullptr;
  const int nc = coarse_points(cf, n, &cpts, s);
  int* cidx = dalloc<int>(n, s);
  int* first = dalloc<int>(n, s);
  int* err = remaining + 1;
  CLAIR_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
  if (nc) {
    agg_root_index<<<ceil_div(nc, 256), 256, 0, s>>>(cpts, nc, cidx); ::clair::count_launch();
  }
  agg_first<<<gr, 256, 0, s>>>(g, n, root, iso, cidx, first, err); ::clair::count_launch();
  agg_final<<<gr, 256, 0, s>>>(g, n, iso, first, agg, err); ::clair::count_launch();
  CLAIR_LAUNCHED();
  int h = 0;
  CLAIR_CUDA(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s));
  CLAIR_CUDA(cudaStreamSynchronize(s));
  dfree(key, s);
  dfree(m1, s);
  dfree(und, s);
  dfree(iso, s);
  dfree(root, s);
  dfree(newr, s);
  dfree(near1, s);
  dfree(remaining, s);
  dfree(cpts, s);
  dfree(cidx, s);
  dfree(first, s);
  CLAIR_REQUIRE(h == 0, CLAIR_ERR_ARG, "aggregation: %d points without a unique root or aggregate", h);
}

// Members of every aggregate as a CSR (nc rows; order within a row is irrelevant: the
// pattern is a set).
__global__ void agg_count(const int* __restrict__ agg, int n, int* __restrict__ cnt) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n && agg[j] >= 0) atomicAdd(&cnt[agg[j]], 1);
}

__global__ void agg_fill(const int* __restrict__ agg, int n, const int* __restrict__ rp,
                         int* __restrict__ cursor, int* __restrict__ members) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n && agg[j] >= 0) members[rp[agg[j]] + atomicAdd(&cursor[agg[j]], 1)] = j;
}

void aggregate_members(const int* agg, int n, int nc, int** rp_out, int** members_out,
                       cudaStream_t s) {
  int* cnt = dalloc<int>(nc + 1, s);
  CLAIR_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * (nc + 1), s));
  if (n) agg_count<<<ceil_div(n, 256), 256, 0, s>>>(agg, n, cnt); ::clair::count_launch();
  CLAIR_LAUNCHED();
  int* rp = dalloc<int>(nc + 1, s);
  const int total = (int)exclusive_scan(cnt, rp, nc, s, true);
  int* members = dalloc<int>(std::max(total, 1), s);
  CLAIR_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * (nc + 1), s));
  if (n) agg_fill<<<ceil_div(n, 256), 256, 0, s>>>(agg, n, rp, cnt, members); ::clair::count_launch();
  CLAIR_LAUNCHED();
  dfree(cnt, s);
  *rp_out = rp;
  *members_out = members;
}

// ------------------------------------------------------------------------------------
// Pattern of Algorithm 1 for the operator Ahat, walked on Ahat^T (= Wm): the column of
// coarse point i collects the F-points j with S_ji (row i of Wm, strong in the column-
// relative sense) and, for m = 2, the F-points j with S_jk for such an F-point k.  The C
// column itself is added so every row carries its identity entry.  One warp per coarse
// point with a shared-memory hash set; COUNT = true writes the row length, otherwise
// the sorted row.
// ------------------------------------------------------------------------------------
constexpr int PT_CAP = 1024;
constexpr int PT_WARPS = 4;

__device__ __forceinline__ int pt_hash(int key, int cap) {
  return (int)(((unsigned)key * 2654435761u) & (unsigned)(cap - 1));
}

// cap: the row's table size, a power of two (32 .. PT_CAP) at least twice an upper bound
// of the row's pattern size, so clearing and compacting cost what the row needs
__device__ __forceinline__ void pt_insert(int* keys, int cap, int key, int* fresh, int* err) {
  int h = pt_hash(key, cap);
  for (int probe = 0; probe < cap; ++probe) {
    int prev = atomicCAS(&keys[h], -1, key);
    if (prev == -1) {
      ++*fresh;
      return;
    }
    if (prev == key) return;
    h = (h + 1) & (cap - 1);
  }
  atomicExch(err, 1);
}

__device__ __forceinline__ int pt_cap_for(int bound) {
  int cap = 32;
  while (cap < PT_CAP && cap < 2 * bound) cap <<= 1;
  return cap;
}

// Second hop for up to 32 first-hop rows at once: lane q holds row q's start and length
// (length 0 for no row); the rows' entries are flattened over the lanes (a warp scan of
// the lengths, then each lane finds its entry's row by binary search), so the loads of
// different rows are independent.  Called by all 32 lanes.
__device__ __forceinline__ void pt_second_hop(int start, int len, int lane, int* P, int* S,
                                              const int* __restrict__ Wcol,
                                              const unsigned char* __restrict__ sW,
                                              const signed char* __restrict__ cf, int* K, int cap,
                                              int* fresh, int* err) {
  int incl = len;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  P[lane + 1] = incl;
  if (lane == 0) P[0] = 0;
  S[lane] = start;
  __syncwarp();
  const int tot = P[32];
  for (int f = lane; f < tot; f += 32) {
    int lo = 0, hi = 32;  // row with P[lo] <= f < P[lo + 1]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (P[mid] <= f) lo = mid; else hi = mid;
    }
    const int e = S[lo] + (f - P[lo]);
    if (sW[e] && !cf[Wcol[e]]) pt_insert(K, cap, Wcol[e], fresh, err);
  }
  __syncwarp();  // P and S are rewritten by the next call
}

// Stash of the first pass: rows that fit are written, sorted, at a position taken from a
// bump counter, so the second pass copies them instead of building them again.
struct PatternStash {
  int* start;                // per row: position in `buf`, -1 if the row did not fit
  int* buf;
  long long cap;             // entries of buf
  unsigned long long* bump;  // next free entry
};

template <bool COUNT, bool AGG>
__global__ void __launch_bounds__(32 * PT_WARPS)
pattern_kernel(const int* __restrict__ Wrp, const int* __restrict__ Wcol,
               const unsigned char* __restrict__ sW, const signed char* __restrict__ cf,
               const int* __restrict__ cpts, int nc, int degree, const int* __restrict__ Mrp,
               const int* __restrict__ Mcol, int* __restrict__ count,
               const int* __restrict__ Zrp, int* __restrict__ Zcol, int* __restrict__ err,
               PatternStash st, const unsigned char* __restrict__ done) {
  __shared__ int keys[PT_WARPS][PT_CAP];
  __shared__ int hop_pre[PT_WARPS][33];
  __shared__ int hop_start[PT_WARPS][32];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int r = blockIdx.x * PT_WARPS + w;
  if (r >= nc) return;  // warp-uniform
  if (COUNT && done && done[r]) return;  // counted (and stashed) by the group pass
  if (!COUNT && st.buf) {
    const int p0 = st.start[r];
    if (p0 >= 0) {  // built by the first pass
      const int base = Zrp[r], len = Zrp[r + 1] - base;
      for (int t = lane; t < len; t += 32) Zcol[base + t] = st.buf[p0 + t];
      return;
    }
  }
  int* K = keys[w];
  const int i = cpts[r];
  // upper bound of the row's pattern: the base points plus every second-hop candidate
  int bound = 0;
  if (!AGG) {
    for (int e = Wrp[i] + lane; e < Wrp[i + 1]; e += 32) {
      bound += 1;
      if (degree >= 2) {
        const int k = Wcol[e];
        if (sW[e] && !cf[k]) bound += Wrp[k + 1] - Wrp[k];
      }
    }
  } else {
    for (int m = Mrp[r] + lane; m < Mrp[r + 1]; m += 32) {
      bound += 1;
      if (degree >= 2) bound += Wrp[Mcol[m] + 1] - Wrp[Mcol[m]];
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) bound += __shfl_xor_sync(0xffffffffu, bound, o);
  const int cap = pt_cap_for(bound + 1);
  for (int t = lane; t < cap; t += 32) K[t] = -1;
  __syncwarp();
  int fresh = 0;
  if (lane == 0) pt_insert(K, cap, i, &fresh, err);
  if (!AGG) {
    // T column i = i and the F-points j with S_ji
    for (int e = Wrp[i] + lane; e < Wrp[i + 1]; e += 32)
      if (sW[e] && !cf[Wcol[e]]) pt_insert(K, cap, Wcol[e], &fresh, err);
    if (degree >= 2) {
      // second hop from every first-hop F-point, 32 first-hop points at a time
      const int e_end = Wrp[i + 1];
      for (int c0 = Wrp[i]; c0 < e_end; c0 += 32) {
        const int e1 = c0 + lane;
        int start = 0, len = 0;
        if (e1 < e_end) {
          const int k = Wcol[e1];
          if (sW[e1] && !cf[k]) {
            start = Wrp[k];
            len = Wrp[k + 1] - start;
          }
        }
        pt_second_hop(start, len, lane, hop_pre[w], hop_start[w], Wcol, sW, cf, K, cap, &fresh, err);
      }
    }
  } else {
    // T column i = the members of aggregate r (its root i included)
    for (int m = Mrp[r] + lane; m < Mrp[r + 1]; m += 32)
      if (!cf[Mcol[m]]) pt_insert(K, cap, Mcol[m], &fresh, err);
    if (degree >= 2) {
      // second hop: F-points j with S_jk for every member k, 32 members at a time
      const int m_end = Mrp[r + 1];
      for (int c0 = Mrp[r]; c0 < m_end; c0 += 32) {
        const int m = c0 + lane;
        int start = 0, len = 0;
        if (m < m_end) {
          const int k = Mcol[m];
          start = Wrp[k];
          len = Wrp[k + 1] - start;
        }
        pt_second_hop(start, len, lane, hop_pre[w], hop_start[w], Wcol, sW, cf, K, cap, &fresh, err);
      }
    }
  }
  __syncwarp();
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) fresh += __shfl_xor_sync(0xffffffffu, fresh, o);
  int* out = nullptr;
  if (COUNT) {
    if (lane == 0) count[r] = fresh;
    if (!st.buf) return;
    // take room for the row in the stash; a row that does not fit is built again later
    unsigned long long p0 = 0;
    if (lane == 0) p0 = atomicAdd(st.bump, (unsigned long long)fresh);
    p0 = __shfl_sync(0xffffffffu, p0, 0);
    const bool fits = p0 + (unsigned long long)fresh <= (unsigned long long)st.cap;
    if (lane == 0) st.start[r] = fits ? (int)p0 : -1;
    if (!fits) return;
    out = st.buf + p0;
  } else {
    out = Zcol + Zrp[r];
  }
  // compact occupied slots in place (reads of a chunk precede its writes), then rank-sort
  int total = 0;
  for (int c = 0; c < cap; c += 32) {
    const int v = K[c + lane];
    const unsigned occ = __ballot_sync(0xffffffffu, v >= 0);
    __syncwarp();
    if (v >= 0) K[total + __popc(occ & ((1u << lane) - 1u))] = v;
    total += __popc(occ);
    __syncwarp();
  }
  for (int t = lane; t < total; t += 32) {
    const int v = K[t];
    int rank = 0;
    for (int u = 0; u < total; ++u) rank += K[u] < v;
    out[rank] = v;
  }
}

// Builds the pattern CSR Z (nc rows) for Algorithm 1 on Ahat, walking Wm = Ahat^T with
// its strength mask sW.
// Counting pass for short rows: PS_G lanes per coarse point, 32 / PS_G points per warp,
// each with a hash set of PS_CAP slots; the steps are pattern_kernel's, every warp
// primitive restricted to the point's lane group (the groups of a warp run independent
// trip counts).  A point whose bound does not fit is left to pattern_kernel (done = 0).
constexpr int PS_G = 8;
constexpr int PS_RPW = 32 / PS_G;
constexpr int PS_CAP = 256;
constexpr int PS_WARPS = 4;

template <bool AGG>
__global__ void __launch_bounds__(32 * PS_WARPS)
pattern_small(const int* __restrict__ Wrp, const int* __restrict__ Wcol,
              const unsigned char* __restrict__ sW, const signed char* __restrict__ cf,
              const int* __restrict__ cpts, int nc, int degree, const int* __restrict__ Mrp,
              const int* __restrict__ Mcol, int* __restrict__ count, int* __restrict__ err,
              PatternStash st, unsigned char* __restrict__ done) {
  __shared__ int keys[PS_WARPS][PS_RPW][PS_CAP];
  __shared__ int hop_pre[PS_WARPS][PS_RPW][PS_G + 1];
  __shared__ int hop_start[PS_WARPS][PS_RPW][PS_G];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane / PS_G, sub = lane % PS_G;
  const unsigned gmask = ((1u << PS_G) - 1u) << (g * PS_G);
  const int r = (blockIdx.x * PS_WARPS + w) * PS_RPW + g;
  if (r >= nc) return;  // group-uniform; the group primitives below name only live lanes
  int* K = keys[w][g];
  int* P = hop_pre[w][g];
  int* S = hop_start[w][g];
  const int i = cpts[r];
  int bound = 0;
  if (!AGG) {
    for (int e = Wrp[i] + sub; e < Wrp[i + 1]; e += PS_G) {
      bound += 1;
      if (degree >= 2) {
        const int k = Wcol[e];
        if (sW[e] && !cf[k]) bound += Wrp[k + 1] - Wrp[k];
      }
    }
  } else {
    for (int m = Mrp[r] + sub; m < Mrp[r + 1]; m += PS_G) {
      bound += 1;
      if (degree >= 2) bound += Wrp[Mcol[m] + 1] - Wrp[Mcol[m]];
    }
  }
#pragma unroll
  for (int o = PS_G / 2; o > 0; o >>= 1) bound += __shfl_xor_sync(gmask, bound, o, PS_G);
  if (2 * (bound + 1) > PS_CAP) {  // group-uniform: the warp-per-point pass takes it
    if (sub == 0) done[r] = 0;
    return;
  }
  const int cap = pt_cap_for(bound + 1);  // <= PS_CAP
  for (int t = sub; t < cap; t += PS_G) K[t] = -1;
  __syncwarp(gmask);
  int fresh = 0;
  if (sub == 0) pt_insert(K, cap, i, &fresh, err);
  // candidates of a batch of up to PS_G first-hop rows, flattened over the group's lanes
  auto second_hop = [&](int start, int len) {
    int incl = len;
#pragma unroll
    for (int o = 1; o < PS_G; o <<= 1) {
      const int v = __shfl_up_sync(gmask, incl, o, PS_G);
      if (sub >= o) incl += v;
    }
    P[sub + 1] = incl;
    if (sub == 0) P[0] = 0;
    S[sub] = start;
    __syncwarp(gmask);
    const int tot = P[PS_G];
    for (int f = sub; f < tot; f += PS_G) {
      int lo = 0, hi = PS_G;
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (P[mid] <= f) lo = mid; else hi = mid;
      }
      const int e = S[lo] + (f - P[lo]);
      if (sW[e] && !cf[Wcol[e]]) pt_insert(K, cap, Wcol[e], &fresh, err);
    }
    __syncwarp(gmask);
  };
  if (!AGG) {
    for (int e = Wrp[i] + sub; e < Wrp[i + 1]; e += PS_G)
      if (sW[e] && !cf[Wcol[e]]) pt_insert(K, cap, Wcol[e], &fresh, err);
    if (degree >= 2) {
      const int e_end = Wrp[i + 1];
      for (int c0 = Wrp[i]; c0 < e_end; c0 += PS_G) {
        const int e1 = c0 + sub;
        int start = 0, len = 0;
        if (e1 < e_end) {
          const int k = Wcol[e1];
          if (sW[e1] && !cf[k]) {
            start = Wrp[k];
            len = Wrp[k + 1] - start;
          }
        }
        second_hop(start, len);
      }
    }
  } else {
    for (int m = Mrp[r] + sub; m < Mrp[r + 1]; m += PS_G)
      if (!cf[Mcol[m]]) pt_insert(K, cap, Mcol[m], &fresh, err);
    if (degree >= 2) {
      const int m_end = Mrp[r + 1];
      for (int c0 = Mrp[r]; c0 < m_end; c0 += PS_G) {
        const int m = c0 + sub;
        int start = 0, len = 0;
        if (m < m_end) {
          const int k = Mcol[m];
          start = Wrp[k];
          len = Wrp[k + 1] - start;
        }
        second_hop(start, len);
      }
    }
  }
  __syncwarp(gmask);
#pragma unroll
  for (int o = PS_G / 2; o > 0; o >>= 1) fresh += __shfl_xor_sync(gmask, fresh, o, PS_G);
  if (sub == 0) {
    count[r] = fresh;
    done[r] = 1;
  }
  if (!st.buf) return;
  unsigned long long p0 = 0;
  if (sub == 0) p0 = atomicAdd(st.bump, (unsigned long long)fresh);
  p0 = __shfl_sync(gmask, p0, 0, PS_G);
  const bool fits = p0 + (unsigned long long)fresh <= (unsigned long long)st.cap;
  if (sub == 0) st.start[r] = fits ? (int)p0 : -1;
  if (!fits) return;
  int* out = st.buf + p0;
  int total = 0;
  for (int c = 0; c < cap; c += PS_G) {
    const int v = K[c + sub];
    const unsigned occ = (__ballot_sync(gmask, v >= 0) >> (g * PS_G)) & ((1u << PS_G) - 1u);
    __syncwarp(gmask);
    if (v >= 0) K[total + __popc(occ & ((1u << sub) - 1u))] = v;
    total += __popc(occ);
    __syncwarp(gmask);
  }
  for (int t = sub; t < total; t += PS_G) {
    const int v = K[t];
    int rank = 0;
    for (int u = 0; u < total; ++u) rank += K[u] < v;
    out[rank] = v;
  }
}

// First stage of the pattern: the counting pass (with the stash), launched only.
PatternJob pattern_count(const Csr& Wm, const unsigned char* sW, const signed char* cf,
                         const int* cpts, int nc, int n, int degree, const int* Mrp,
                         const int* Mcol, cudaStream_t s) {
  CLAIR_REQUIRE(degree == 1 || degree == 2, CLAIR_ERR_UNSUPPORTED,
                "pattern degree %d not supported (1 or 2)", degree);
  PatternJob j;
  j.Wm = Wm;
  j.sW = sW;
  j.cf = cf;
  j.cpts = cpts;
  j.nc = nc;
  j.n = n;
  j.degree = degree;
  j.Mrp = Mrp;
  j.Mcol = Mcol;
  j.count = dalloc<int>(nc + 1, s);
  j.err = dalloc<int>(1, s);
  CLAIR_CUDA(cudaMemsetAsync(j.err, 0, sizeof(int), s));
  const int g = ceil_div(nc, PT_WARPS);
  const bool agg = Mrp != nullptr;
  // the stash: room for about twice the entries of Wm (rows beyond it are built twice)
  if (nc) {
    j.cap = std::min<long long>(2LL * Wm.nnz + 8LL * nc + 1024, 64LL << 20);
    j.start = dalloc<int>(nc, s);
    j.buf = dalloc<int>((size_t)j.cap, s);
    j.bump = dalloc<unsigned long long>(1, s);
    CLAIR_CUDA(cudaMemsetAsync(j.bump, 0, sizeof(unsigned long long), s));
    const PatternStash st{j.start, j.buf, j.cap, j.bump};
    // short rows (a fine stencil level): the group pass counts every point whose bound
    // fits its table, the warp-per-point pass the rest; with longer rows eight lanes walk
    // too many candidates per point and the warp per point is faster
    const bool short_rows = Wm.rows && (double)Wm.nnz / Wm.rows <= 8.0;
    if (short_rows) {
      j.done = dalloc<unsigned char>(nc, s);
      const int gs = ceil_div(nc, PS_WARPS * PS_RPW);
      if (agg)
        pattern_small<true><<<gs, 32 * PS_WARPS, 0, s>>>(Wm.rowptr, Wm.col, sW, cf, cpts, nc, degree,
                                                          Mrp, Mcol, j.count, j.err, st, j.done);
      else
        pattern_small<false><<<gs, 32 * PS_WARPS, 0, s>>>(Wm.rowptr, Wm.col, sW, cf, cpts, nc,
                                                           degree, nullptr, nullptr, j.count,
                                                           j.err, st, j.done);
      ::clair::count_launch();
    }
    if (agg)
      pattern_kernel<true, true><<<g, 32 * PT_WARPS, 0, s>>>(Wm.rowptr, Wm.col, sW, cf, cpts, nc,
                                                             degree, Mrp, Mcol, j.count, nullptr,
                                                             nullptr, j.err, st, j.done);
    else
      pattern_kernel<true, false><<<g, 32 * PT_WARPS, 0, s>>>(Wm.rowptr, Wm.col, sW, cf, cpts, nc,
                                                              degree, nullptr, nullptr, j.count,
                                                              nullptr, nullptr, j.err, st, j.done);
    ::clair::count_launch();
  }
  CLAIR_LAUNCHED();
  return j;
}

static void pattern_release(PatternJob& j, cudaStream_t s) {
  dfree(j.done, s);
  dfree(j.count, s);
  dfree(j.err, s);
  dfree(j.start, s);
  dfree(j.buf, s);
  dfree(j.bump, s);
  dfree(j.ovf, s);
}

// Row pointers of the pattern from the counting pass (device only).
void pattern_scan(PatternJob& j, Csr& Z, cudaStream_t s) {
  Z.rows = j.nc;
  Z.cols = j.n;
  Z.rowptr = dalloc<int>(j.nc + 1, s);
  j.ovf = dalloc<int>(1, s);
  exclusive_scan_into(j.count, Z.rowptr, j.nc, j.ovf, s);
}

// One host read for k scanned patterns: entry counts, scan overflow, table overflow of the
// counting pass (a row that overflows its table does so there: the filling pass inserts the
// same keys).  On an error every job's buffers are released.
void pattern_read(PatternJob* const* jobs, Csr* const* Z, int k, cudaStream_t s) {
  int h[3 * 2] = {0, 0, 0, 0, 0, 0};
  CLAIR_REQUIRE(k >= 1 && k <= 2, CLAIR_ERR_ARG, "pattern_read: %d jobs", k);
  for (int q = 0; q < k; ++q) {
    CLAIR_CUDA(cudaMemcpyAsync(&h[3 * q], Z[q]->rowptr + jobs[q]->nc, sizeof(int),
                               cudaMemcpyDeviceToHost, s));
    CLAIR_CUDA(cudaMemcpyAsync(&h[3 * q + 1], jobs[q]->ovf, sizeof(int), cudaMemcpyDeviceToHost, s));
    CLAIR_CUDA(cudaMemcpyAsync(&h[3 * q + 2], jobs[q]->err, sizeof(int), cudaMemcpyDeviceToHost, s));
  }
  CLAIR_CUDA(cudaStreamSynchronize(s));
  bool bad_ovf = false, bad_cap = false;
  for (int q = 0; q < k; ++q) {
    Z[q]->nnz = h[3 * q];
    bad_ovf = bad_ovf || h[3 * q + 1];
    bad_cap = bad_cap || h[3 * q + 2];
  }
  if (bad_ovf || bad_cap) {
    for (int q = 0; q < k; ++q) {
      pattern_release(*jobs[q], s);
      dfree(Z[q]->rowptr, s);
      Z[q]->rowptr = nullptr;
    }
    CLAIR_REQUIRE(!bad_ovf, CLAIR_ERR_CAPACITY, "scan total exceeds int32");
    CLAIR_REQUIRE(false, CLAIR_ERR_CAPACITY, "pattern row exceeds %d entries", PT_CAP);
  }
}

// The rows: stashed rows copied, the others built again; releases the job's buffers.
void pattern_build(PatternJob& j, Csr& Z, cudaStream_t s) {
  const int nc = j.nc;
  const int g = ceil_div(nc, PT_WARPS);
  const bool agg = j.Mrp != nullptr;
  const PatternStash st{j.start, j.buf, j.cap, j.bump};
  Z.col = dalloc<int>(Z.nnz, s);
  if (nc) {
    const Csr& Wm = j.Wm;
    if (agg)
      pattern_kernel<false, true><<<g, 32 * PT_WARPS, 0, s>>>(Wm.rowptr, Wm.col, j.sW, j.cf, j.cpts,
                                                              nc, j.degree, j.Mrp, j.Mcol, nullptr,
                                                              Z.rowptr, Z.col, j.err, st, nullptr);
    else
      pattern_kernel<false, false><<<g, 32 * PT_WARPS, 0, s>>>(Wm.rowptr, Wm.col, j.sW, j.cf,
                                                               j.cpts, nc, j.degree, nullptr,
                                                               nullptr, nullptr, Z.rowptr, Z.col,
                                                               j.err, st, nullptr);
    ::clair::count_launch();
  }
  CLAIR_LAUNCHED();
  pattern_release(j, s);
}

// Second stage of the pattern: scan, the host read, the rows.
void pattern_fill(PatternJob& j, Csr& Z, cudaStream_t s) {
  pattern_scan(j, Z, s);
  PatternJob* jp = &j;
  Csr* zp = &Z;
  pattern_read(&jp, &zp, 1, s);
  pattern_build(j, Z, s);
}

// Builds the pattern CSR Z (nc rows) for Algorithm 1 on Ahat, walking Wm = Ahat^T with
// its strength mask sW.
void build_pattern(const Csr& Wm, const unsigned char* sW, const signed char* cf, const int* cpts,
                   int nc, int n, int degree, const int* Mrp, const int* Mcol, Csr& Z,
                   cudaStream_t s) {
  PatternJob j = pattern_count(Wm, sW, cf, cpts, nc, n, degree, Mrp, Mcol, s);
  pattern_fill(j, Z, s);
}

// ------------------------------------------------------------------------------------
// Weighted Jacobi on the subset {cf == which}: x_out = x_in + omega D^-1 (b - A x_in) on
// the subset, x_out = x_in elsewhere (b = NULL means a zero right-hand side).
// ------------------------------------------------------------------------------------
template <int W, class T>
__global__ void jacobi_kernel(const int* __restrict__ rowptr, const int* __restrict__ col,
                              const T* __restrict__ val, const T* __restrict__ dinv, int rows,
                              const signed char* __restrict__ cf, int which, T omega,
                              const T* __restrict__ b, const T* __restrict__ xin,
                              T* __restrict__ xout, const T* __restrict__ omega_dev) {
  pdl_prologue();
  if (omega_dev) omega = *omega_dev;  // weight produced on the device by the Arnoldi step
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int r = (int)(t / W), lane = (int)(t % W);
  const bool ok = r < rows;
  const bool act = ok && cf[r] == which;
  T acc = 0;
  if (act)
    acc = csr_row_dot<W>(col, val, xin, rowptr[r], rowptr[r + 1], lane);
  acc = group_sum<W>(acc);
  if (ok && lane == 0) {
    const T xr = xin[r];
    xout[r] = act ? xr + omega * dinv[r] * ((b ? b[r] : T(0)) - acc) : xr;
  }
}

// First sweep of a cycle from x = 0: x = omega D^-1 b on the subset, 0 elsewhere.
template <class T>
__global__ void jacobi_first(const T* __restrict__ dinv, int rows, const signed char* __restrict__ cf,
                             int which, T omega, const T* __restrict__ b, T* __restrict__ x) {
  pdl_prologue();
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < rows;
       r += (long long)gridDim.x * blockDim.x)
    x[r] = cf[r] == which ? omega * dinv[r] * b[r] : T(0);
}

// FP64 short rows one per thread (an FP64 warp instruction costs ~16 SM cycles whatever
// the number of active lanes), long rows about four entries per lane (else one thread's
// chain of dependent index and value loads); FP32: W lanes per row, W >= the mean row
// length.
static int lanes_of(const Csr& A, bool fp64) {
  double avg = A.rows ? (double)A.nnz / A.rows : 1.0;
  if (fp64 || cycle_short_lanes() == 1) {
    if (avg <= 8.0) return 1;
    int w = 2;
    while (w < 32 && 4 * w < avg) w <<= 1;
    return w;
  }
  if (cycle_short_lanes() == 2) {  // FP32, about eight entries per lane (one thread up to 16 entries)
    if (avg <= 16.0) return 1;
    int w = 2;
    while (w < 32 && 8 * w < avg) w <<= 1;
    return w;
  }
  int w = 2;
  while (w < 32 && w < avg) w <<= 1;
  return w;
}


template <class T>
void jacobi(const Csr& A, const T* vals, const T* dinv, const signed char* cf, int which, T omega,
            const T* b, const T* xin, T* xout, cudaStream_t s, const T* omega_dev = nullptr) {
  if (!A.rows) return;
  const int W = lanes_of(A, sizeof(T) == 8);
  const int blocks = ceil_div((long long)A.rows * W, 256);
  CLAIR_DISPATCH_W2(W, launch_k(jacobi_kernel<WW, T>, blocks, 256, 0, s, A.rowptr, A.col, vals,
                                 dinv, A.rows, cf, which, omega, b, xin, xout, omega_dev));
  CLAIR_LAUNCHED();
}

// Mode-vector smoothing B <- CFF^sweeps(B) with a zero right-hand side and the weight
// read from device memory (so it can follow the Arnoldi step without a host round trip).
// The sweeps alternate between Bv and tmp (every sweep writes all rows); one copy at the
// end when the result sits in tmp.
void smooth_modes(const Csr& M, const double* dinv, const signed char* cf, const double* omega_dev,
                  int sweeps, double* Bv, double* tmp, cudaStream_t s) {
  double* x = Bv;
  double* y = tmp;
  for (int it = 0; it < sweeps; ++it) {
    jacobi<double>(M, M.val, dinv, cf, 1, 1.0, nullptr, x, y, s, omega_dev);
    jacobi<double>(M, M.val, dinv, cf, 0, 1.0, nullptr, y, x, s, omega_dev);
    jacobi<double>(M, M.val, dinv, cf, 0, 1.0, nullptr, x, y, s, omega_dev);
    std::swap(x, y);
  }
  if (x != Bv) CLAIR_CUDA(cudaMemcpyAsync(Bv, x, sizeof(double) * M.rows, cudaMemcpyDeviceToDevice, s));
}
// Mode smoothing of several vectors in one launch per relaxation (SmoothSides): the
// per-row arithmetic is jacobi_kernel's.
template <int W>
__global__ void jacobi_sides(SmoothSides p, const double* __restrict__ dinv, int rows,
                             const signed char* __restrict__ cf, int which, double omega,
                             const double* __restrict__ omega_dev, int flip) {
  if (omega_dev) omega = *omega_dev;
  const int g = blockIdx.y;
  const double* __restrict__ xin = flip ? p.y[g] : p.x[g];
  double* __restrict__ xout = flip ? p.x[g] : p.y[g];
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int r = (int)(t / W), lane = (int)(t % W);
  const bool ok = r < rows;
  const bool act = ok && cf[r] == which;
  double acc = 0;
  if (act)
    acc = csr_row_dot<W>(p.col[g], p.val[g], xin, p.rowptr[g][r], p.rowptr[g][r + 1], lane);
  acc = group_sum<W>(acc);
  if (ok && lane == 0) {
    const double xr = xin[r];
    xout[r] = act ? xr + omega * dinv[r] * (0.0 - acc) : xr;
  }
}

// B <- (CFF sweep)^sweeps B for every side at once (zero right-hand side); each side's
// vector ends in its x buffer.  Same kernels' arithmetic as smooth_modes.
void smooth_modes_sides(const SmoothSides& sides, int rows, double avg_row, const double* dinv,
                        const signed char* cf, const double* omega_dev, double omega, int sweeps,
                        cudaStream_t s) {
  if (!rows || !sides.count) return;
  // one lane per row up to 16 entries (two batches of eight), then one lane per 16: the
  // FP64 pipe, not the rows' dependent loads, then sets the pace
  int W = 1;
  while (W < 32 && 16 * W < avg_row) W <<= 1;
  const dim3 grid((unsigned)ceil_div((long long)rows * W, 256), (unsigned)sides.count);
  for (int it = 0; it < sweeps; ++it) {
    // x -> y (C), y -> x (F), x -> y (F), then the roles swap: in place of std::swap the
    // flip flag alternates, and after an odd count the result is in y
    const int f0 = it & 1;
    CLAIR_DISPATCH_W2(W, (jacobi_sides<WW><<<grid, 256, 0, s>>>(sides, dinv, rows, cf, 1, omega,
                                                                  omega_dev, f0)));
    CLAIR_DISPATCH_W2(W, (jacobi_sides<WW><<<grid, 256, 0, s>>>(sides, dinv, rows, cf, 0, omega,
                                                                  omega_dev, f0 ^ 1)));
    CLAIR_DISPATCH_W2(W, (jacobi_sides<WW><<<grid, 256, 0, s>>>(sides, dinv, rows, cf, 0, omega,
                                                                  omega_dev, f0)));
  }
  CLAIR_LAUNCHED();
  if (sweeps & 1)
    for (int g = 0; g < sides.count; ++g)
      CLAIR_CUDA(cudaMemcpyAsync(sides.x[g], sides.y[g], sizeof(double) * rows,
                                 cudaMemcpyDeviceToDevice, s));
}

template void jacobi<double>(const Csr&, const double*, const double*, const signed char*, int,
                             double, const double*, const double*, double*, cudaStream_t,
                             const double*);
template void jacobi<float>(const Csr&, const float*, const float*, const signed char*, int, float,
                            const float*, const float*, float*, cudaStream_t, const float*);

template <class T>
void jacobi_from_zero(int rows, const T* dinv, const signed char* cf, int which, T omega,
                      const T* b, T* x, cudaStream_t s) {
  if (!rows) return;
  launch_k(jacobi_first<T>, std::min(ceil_div(rows, 256), 32 * sm_count()), 256, 0, s, dinv, rows,
           cf, which, omega, b, x); ::clair::count_launch();
  CLAIR_LAUNCHED();
}
template void jacobi_from_zero<double>(int, const double*, const signed char*, int, double,
                                       const double*, double*, cudaStream_t);
template void jacobi_from_zero<float>(int, const float*, const signed char*, int, float, const float*,
                                      float*, cudaStream_t);

// ------------------------------------------------------------------------------------
// Relaxation weight: Arnoldi on D^-1 A (classical Gram-Schmidt applied twice), start
// vector splitmix64 in [-1, 1) seeded with `seed`; rho = max |Ritz value|.
// ------------------------------------------------------------------------------------
__global__ void arnoldi_start(double* __restrict__ v, int n, uint64_t seed) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    v[i] = splitmix_pm1(seed, (uint64_t)i);
}

__global__ void scale_by_inv_sqrt(double* __restrict__ v, int n, const double* __restrict__ nrm2) {
  const double s = 1.0 / sqrt(*nrm2);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    v[i] *= s;
}

__global__ void dinv_scale(double* __restrict__ w, const double* __restrict__ dinv, int n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    w[i] *= dinv[i];
}

// After the two projection passes: H[:, j] = h1 + h2, H[j+1, j] = ||w||, breakdown test,
// v_{j+1} scale.  state[0] = active steps (m until breakdown), state scalars in dev.
__global__ void arnoldi_column(double* __restrict__ H, int ldh, int j, const double* __restrict__ h1,
                               const double* __restrict__ h2, const double* __restrict__ wn2,
                               const double* __restrict__ w0n2, int* __restrict__ steps,
                               double* __restrict__ inv_norm) {
  if (threadIdx.x != 0) return;
  const bool active = *steps < 0;  // -1 while no breakdown
  for (int i = 0; i <= j; ++i) H[i + (long long)j * ldh] = active ? h1[i] + h2[i] : 0.0;
  const double hn = sqrt(*wn2);
  H[j + 1 + (long long)j * ldh] = active ? hn : 0.0;
  if (active && hn <= 1e-10 * sqrt(*w0n2)) *steps = j + 1;
  *inv_norm = (active && hn > 0.0) ? 1.0 / hn : 0.0;
}

__global__ void scale_vec(const double* __restrict__ w, double* __restrict__ v, int n,
                          const double* __restrict__ s) {
  const double f = *s;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    v[i] = w[i] * f;
}

struct WarpSync {
  __device__ void operator()() const { __syncwarp(); }
};

// One warp: the leading k x k block of H (k <= 60) is copied to shared memory and the
// Francis iteration runs there with the reflector updates split among the lanes.
__global__ void __launch_bounds__(32) ritz_kernel(const double* __restrict__ H, int ldh, int m,
                                                  const int* __restrict__ steps,
                                                  double* __restrict__ omega) {
  __shared__ double Hs[60 * 60];
  const int lane = threadIdx.x;
  const int k = *steps < 0 ? m : *steps;
  for (int idx = lane; idx < k * k; idx += 32) Hs[idx] = H[(idx % k) + (long long)(idx / k) * ldh];
  __syncwarp();
  const double rho = hessenberg_spectral_radius_lanes(Hs, k, k, lane, 32, WarpSync{});
  if (lane == 0) *omega = rho > 0.0 ? 1.0 / rho : 1.0;
}

// ---- fused Arnoldi step (m <= AR_MAXV): three launches per step -------------------------
// K1  v_j = w_prev * scale (stored), w = D^-1 A v_j, dots of w with v_0..v_j and with
//     itself                                   -> h1, ||w||^2 before CGS
// K2  w -= V h1, dots of the new w with v_0..v_j  -> h2
// K3  w -= V h2, ||w||^2                        -> H column, breakdown, scale of v_{j+1}
// Block b owns the rows [b R, (b + 1) R).  FP64 is the scarce pipe on this part (an FP64
// warp instruction holds it for tens of cycles), so nothing beyond v_j is touched: after
// the row updates, warp q of the block takes the dot products q, q + 8, ... over the
// block's rows (two running sums per lane, one warp tree), and writes the block's partial
// of each.  The kernels hold no shared-memory table, so they fit beside the other
// stream's blocks.  The last block to arrive (atomic ticket) adds the partials in block
// order and publishes the step's scalars, so the next kernel reads finished values, no
// finalize launch sits between the kernels, and the result does not depend on
// scheduling.  steps_hist[t] is the breakdown state after step t-1 (-1: none).
constexpr int AR_MAXV = 15;
constexpr int AR_THREADS = 256;
constexpr int AR_WARPS = AR_THREADS / 32;
constexpr int AR_SLOTS = AR_MAXV + 2;  // 0..AR_MAXV-1: projections, AR_MAXV+1: squared norm

struct ArnoldiState {
  double* H;            // ldh x m, column-major
  int ldh;
  double* h1;           // h1 of the current step (AR_MAXV)
  double* h2;           // h2 of the current step (AR_MAXV)
  double* w0n2;         // ||w||^2 before orthogonalisation, current step
  double* scale;        // scale of the next basis vector
  int* steps_hist;      // m + 1 entries, [0] = -1
  unsigned* ticket;     // arrival counter (0 between kernels)
};

// Row dot with four entries per lane in flight (indices and values first, then the four
// gathers) and two partial sums; the order is fixed, so the result is reproducible.
template <int W>
__device__ __forceinline__ double csr_row_dot_cl(const int* __restrict__ col,
                                                 const double* __restrict__ val,
                                                 const double* x, int e0, int e1, int lane) {
  double a0 = 0.0, a1 = 0.0;
  int e = e0 + lane;
  for (; e + 3 * W < e1; e += 4 * W) {
    const int c0 = col[e], c1 = col[e + W], c2 = col[e + 2 * W], c3 = col[e + 3 * W];
    const double v0 = val[e], v1 = val[e + W], v2 = val[e + 2 * W], v3 = val[e + 3 * W];
    const double x0 = x[c0], x1 = x[c1], x2 = x[c2], x3 = x[c3];
    a0 = fma(v0, x0, a0);
    a1 = fma(v1, x1, a1);
    a0 = fma(v2, x2, a0);
    a1 = fma(v3, x3, a1);
  }
  for (; e < e1; e += W) a0 = fma(val[e], x[col[e]], a0);
  return a0 + a1;
}

// Sum over i in [lo, hi) of a[i] * b[i], by one warp (all lanes get the result): eight
// entries per lane in flight (sixteen independent loads) into four running sums, so the
// loop waits on one memory round trip per 256 entries, not per entry.
__device__ __forceinline__ double warp_dot(const double* a, const double* b, int lo, int hi,
                                           int lane) {
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  int i = lo + lane;
  for (; i + 224 < hi; i += 256) {
    double x[8], y[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      x[u] = a[i + 32 * u];
      y[u] = b[i + 32 * u];
    }
    s0 = fma(x[0], y[0], s0);
    s1 = fma(x[1], y[1], s1);
    s2 = fma(x[2], y[2], s2);
    s3 = fma(x[3], y[3], s3);
    s0 = fma(x[4], y[4], s0);
    s1 = fma(x[5], y[5], s1);
    s2 = fma(x[6], y[6], s2);
    s3 = fma(x[7], y[7], s3);
  }
  for (; i < hi; i += 32) s0 = fma(a[i], b[i], s0);
  return warp_sum((s0 + s1) + (s2 + s3));
}

// Block partials of the dots <a_q, w> (a_q = v_q for q <= nproj - 1) and, with `norm`,
// <w, w> into partial[slot][block]; the rows are the block's own, w complete (synced).
__device__ __forceinline__ void block_dots(const double* V, long long n, int nproj, bool norm,
                                           const double* w, int lo, int hi,
                                           double* __restrict__ partial) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nq = nproj + (norm ? 1 : 0);
  for (int q = wid; q < nq; q += AR_WARPS) {
    const bool is_norm = q >= nproj;
    const double v = warp_dot(is_norm ? w : V + (long long)q * n, w, lo, hi, lane);
    if (lane == 0) partial[(long long)(is_norm ? AR_SLOTS - 1 : q) * gridDim.x + blockIdx.x] = v;
  }
}

// After the block's partials are written: true in the block that arrives last, which then
// holds the grand sums of the live slots in red[] (slot order, block order within).
__device__ __forceinline__ bool finish_slots(const double* partial, int nproj, bool norm,
                                             unsigned* ticket, double* red) {
  __shared__ bool is_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!is_last) return false;
  __threadfence();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nb = gridDim.x;
  const int nq = nproj + (norm ? 1 : 0);
  for (int q = wid; q < nq; q += AR_WARPS) {
    const int k = q < nproj ? q : AR_SLOTS - 1;
    double t = 0.0;
    for (int b = lane; b < nb; b += 32) t += __ldcg(&partial[(long long)k * nb + b]);
    t = warp_sum(t);
    if (lane == 0) red[k] = t;
  }
  __syncthreads();
  return true;
}

template <int W>
__global__ void __launch_bounds__(AR_THREADS, 6)
arnoldi_k1(const int* __restrict__ rp, const int* __restrict__ ci, const double* __restrict__ av,
           const double* __restrict__ dinv, int n, double* __restrict__ V, int j,
           const double* __restrict__ wprev, ArnoldiState st, double* __restrict__ w,
           double* __restrict__ partial) {
  __shared__ double red[AR_SLOTS];
  const double sc = j > 0 ? *st.scale : 1.0;  // v_0 is normalised already
  const long long R = (n + (long long)gridDim.x - 1) / gridDim.x;
  const int lo = (int)min((long long)n, R * blockIdx.x), hi = (int)min((long long)n, lo + R);
  constexpr int GPW = 32 / W;
  const int lane = threadIdx.x & 31, sub = lane % W, grp = lane / W, warp = threadIdx.x >> 5;
  double* __restrict__ Vj = V + (long long)j * n;
  for (int base = lo + warp * GPW; base < hi; base += AR_WARPS * GPW) {
    const int i = base + grp;
    double s = 0.0;
    if (i < hi) s = csr_row_dot_cl<W>(ci, av, wprev, rp[i], rp[i + 1], sub);
    s = group_sum<W>(s);
    if (sub == 0 && i < hi) {
      w[i] = dinv[i] * (sc * s);
      if (j > 0) Vj[i] = wprev[i] * sc;
    }
  }
  __syncthreads();  // w and v_j of the block's rows, written above
  block_dots(V, n, j + 1, true, w, lo, hi, partial);
  if (!finish_slots(partial, j + 1, true, st.ticket, red)) return;
  if (threadIdx.x <= j) st.h1[threadIdx.x] = red[threadIdx.x];
  if (threadIdx.x == 0) {
    *st.w0n2 = red[AR_SLOTS - 1];
    *st.ticket = 0u;
  }
}

// FIRST: w -= V h1, dots of the new w with v_0..v_j -> h2.  Otherwise: w -= V h2,
// ||w||^2 -> the step's H column, breakdown state and the scale of v_{j+1}.
template <bool FIRST>
__global__ void __launch_bounds__(AR_THREADS, 6)
arnoldi_cgs(const double* __restrict__ V, int j, int n, ArnoldiState st, double* __restrict__ w,
            double* __restrict__ partial) {
  __shared__ double red[AR_SLOTS];
  __shared__ double hk[AR_MAXV];
  const double* h = FIRST ? st.h1 : st.h2;
  if (threadIdx.x <= j) hk[threadIdx.x] = h[threadIdx.x];
  __syncthreads();
  const long long R = (n + (long long)gridDim.x - 1) / gridDim.x;
  const int lo = (int)min((long long)n, R * blockIdx.x), hi = (int)min((long long)n, lo + R);
  for (int i = lo + threadIdx.x; i < hi; i += AR_THREADS) {
    double wi = w[i];
    for (int k = 0; k <= j; ++k) wi = fma(-hk[k], V[(long long)k * n + i], wi);
    w[i] = wi;
  }
  __syncthreads();  // the block's rows of w
  block_dots(V, n, FIRST ? j + 1 : 0, !FIRST, w, lo, hi, partial);
  if (!finish_slots(partial, FIRST ? j + 1 : 0, !FIRST, st.ticket, red)) return;
  if (FIRST) {
    if (threadIdx.x <= j) st.h2[threadIdx.x] = red[threadIdx.x];
    if (threadIdx.x == 0) *st.ticket = 0u;
    return;
  }
  if (threadIdx.x != 0) return;
  // close step j: H column, breakdown test, scale of the next basis vector
  const bool active = st.steps_hist[j] < 0;
  const double hn = sqrt(red[AR_SLOTS - 1]);
  for (int i = 0; i <= j; ++i) st.H[i + (long long)j * st.ldh] = active ? st.h1[i] + st.h2[i] : 0.0;
  st.H[j + 1 + (long long)j * st.ldh] = active ? hn : 0.0;
  st.steps_hist[j + 1] = (active && hn <= 1e-10 * sqrt(*st.w0n2)) ? j + 1 : st.steps_hist[j];
  *st.scale = (active && hn > 0.0) ? 1.0 / hn : 0.0;
  *st.ticket = 0u;
}

// w of step j lives in wbuf[j & 1] while K1 gathers v_j from the previous step's w in the
// other buffer.  nb blocks: one or two per SM, fewer on small levels.
static void arnoldi_fused_steps(const Csr& A, const double* dinv, int m, double* V,
                                double* const wbuf[2], const ArnoldiState& st, double* partial,
                                int nb, cudaStream_t s) {
  const int n = A.rows;
  // at most four lanes per row: eight or more rows per warp in flight
  const int W = std::min(lanes_of(A, true), 4);
  for (int j = 0; j < m; ++j) {
    double* w = wbuf[j & 1];
    const double* wprev = j == 0 ? V : wbuf[(j + 1) & 1];
    if (W == 1)
      arnoldi_k1<1><<<nb, AR_THREADS, 0, s>>>(A.rowptr, A.col, A.val, dinv, n, V, j, wprev, st, w,
                                             partial);
    else if (W == 2)
      arnoldi_k1<2><<<nb, AR_THREADS, 0, s>>>(A.rowptr, A.col, A.val, dinv, n, V, j, wprev, st, w,
                                             partial);
    else
      arnoldi_k1<4><<<nb, AR_THREADS, 0, s>>>(A.rowptr, A.col, A.val, dinv, n, V, j, wprev, st, w,
                                             partial);
    ::clair::count_launch();
    arnoldi_cgs<true><<<nb, AR_THREADS, 0, s>>>(V, j, n, st, w, partial); ::clair::count_launch();
    arnoldi_cgs<false><<<nb, AR_THREADS, 0, s>>>(V, j, n, st, w, partial); ::clair::count_launch();
    CLAIR_LAUNCHED();
  }
}

// Register-accumulator reductions of the segmented (batch) Arnoldi below: the block's
// warp sums of the live values (v < nv), one partial per value and block.
template <int NV>
__device__ __forceinline__ void block_reduce_to_partial(double (&acc)[NV], int nv,
                                                        double* __restrict__ partial) {
  __shared__ double sh[NV][AR_THREADS / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    if (v < nv) {  // warp-uniform: no FP64 shuffle-adds for dead values
      const double t = warp_sum(acc[v]);
      if (lane == 0) sh[v][wid] = t;
    }
  }
  __syncthreads();
  if (threadIdx.x < nv) {
    double t = 0.0;
    for (int k = 0; k < AR_THREADS / 32; ++k) t += sh[threadIdx.x][k];
    partial[(long long)threadIdx.x * gridDim.x + blockIdx.x] = t;
  }
}

// After the block's partials are written: true in the block that arrives last.
__device__ __forceinline__ bool last_block(unsigned* ticket) {
  __shared__ bool is_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  return is_last;
}

// In the last block: out[v] = sum over blocks of partial v, lanes over blocks then the
// warp tree (reads bypass L1: the other blocks wrote them in this kernel).
__device__ __forceinline__ void sum_partials(const double* partial, int nv, double* out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nb = gridDim.x;
  for (int v = wid; v < nv; v += AR_THREADS / 32) {
    double t = 0.0;
    for (int b = lane; b < nb; b += 32) t += __ldcg(&partial[(long long)v * nb + b]);
    t = warp_sum(t);
    if (lane == 0) out[v] = t;
  }
  __syncthreads();
}

// ---- one-launch Arnoldi on a thread-block cluster (levels of a few thousand rows) ----
// The whole run (start vector, m steps of CGS2, the H columns) is one launch of one
// cluster of C CTAs; CTA r owns rows [r n / C, (r + 1) n / C).  Every reduction is: warp
// sums, the CTA's partial in its shared memory, a hardware cluster barrier, then every
// CTA adds the C partials in rank order through distributed shared memory, so all CTAs
// hold the same sums and take the same breakdown decisions, and there is no spin-wait.
// Partials alternate between two buffers: a CTA rewrites a buffer two reductions later,
// after a barrier that every reader of its previous contents has passed.  The next basis
// vector is kept unscaled (w) and its scale applied when the SpMV reads it, as in the
// multi-launch path.  Other CTAs' rows of w are read with ordinary (coherent, L1-cached)
// loads: the barrier's release by the writers and an acquire fence after it make them
// visible; the read-only path (ld.global.nc) is never used for w.
constexpr int AC_THREADS = 256;
constexpr int AC_WARPS = AC_THREADS / 32;

struct ClusterSums {
  double part[2][AR_SLOTS];
  double out[AR_SLOTS];
};

// The CTA's partials of <v_q, w> (q < nproj) and, with `norm`, <w, w> over its rows (warp q
// takes dots q, q + 8, ...), then out[slot] = the cluster-wide sums; called by every
// thread of every CTA once the CTA's rows of w are written.
__device__ __forceinline__ void cluster_dots(const double* V, long long n, int nproj, bool norm,
                                             const double* w, int lo, int hi, ClusterSums& cs,
                                             int& buf) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nq = nproj + (norm ? 1 : 0);
  for (int q = wid; q < nq; q += AC_WARPS) {
    const bool is_norm = q >= nproj;
    const double v = warp_dot(is_norm ? w : V + (long long)q * n, w, lo, hi, lane);
    if (lane == 0) cs.part[buf][is_norm ? AR_SLOTS - 1 : q] = v;
  }
  __threadfence();  // this CTA's global writes before the barrier, for the other CTAs
  cl.sync();
  __threadfence();  // acquire: the other CTAs' writes before the barrier, for this CTA
  if ((int)threadIdx.x < nq) {
    const int k = (int)threadIdx.x < nproj ? (int)threadIdx.x : AR_SLOTS - 1;
    double v = 0.0;
    const int C = (int)cl.num_blocks();
    for (int c = 0; c < C; ++c) v += *cl.map_shared_rank(&cs.part[buf][k], c);
    cs.out[k] = v;
  }
  __syncthreads();
  buf ^= 1;
}

template <int W>
__global__ void __launch_bounds__(AC_THREADS, 2)
arnoldi_cluster(const int* __restrict__ rp, const int* __restrict__ ci,
                const double* __restrict__ av, const double* __restrict__ dinv, int n, int m,
                uint64_t seed, double* __restrict__ V, double* wb0, double* wb1,
                double* __restrict__ H, int ldh, int* __restrict__ steps_out) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  __shared__ ClusterSums cs;
  __shared__ double h1s[AR_MAXV], h2s[AR_MAXV];
  const int C = (int)cl.num_blocks(), r = (int)cl.block_rank();
  const int lo = (int)((long long)n * r / C), hi = (int)((long long)n * (r + 1) / C);
  const int tid = threadIdx.x;
  int buf = 0;
  // start vector, unscaled, in wb1 (the "previous w" of step 0); its squared norm
  for (int i = lo + tid; i < hi; i += AC_THREADS) wb1[i] = splitmix_pm1(seed, (uint64_t)i);
  cluster_dots(V, n, 0, true, wb1, lo, hi, cs, buf);
  double sc = 1.0 / sqrt(cs.out[AR_SLOTS - 1]);
  int steps = -1;  // breakdown step, -1 while none
  constexpr int GPW = 32 / W;
  const int lane = tid & 31, sub = lane % W, grp = lane / W, warp = tid >> 5;
  for (int j = 0; j < m; ++j) {
    const double* wprev = (j & 1) ? wb0 : wb1;
    double* w = (j & 1) ? wb1 : wb0;
    double* Vj = V + (long long)j * n;
    // P1: v_j = sc * w_prev (own rows), w = D^-1 A v_j, then <v_k, w> and <w, w>
    for (int base = lo + warp * GPW; base < hi; base += AC_WARPS * GPW) {
      const int i = base + grp;
      double s = 0.0;
      if (i < hi) s = csr_row_dot_cl<W>(ci, av, wprev, rp[i], rp[i + 1], sub);
      s = group_sum<W>(s);
      if (sub == 0 && i < hi) {
        w[i] = dinv[i] * (sc * s);
        Vj[i] = wprev[i] * sc;
      }
    }
    cluster_dots(V, n, j + 1, true, w, lo, hi, cs, buf);
    const double w0n2 = cs.out[AR_SLOTS - 1];
    if (tid <= j) h1s[tid] = cs.out[tid];
    __syncthreads();
    // P2: w -= V h1, then the projections again
    for (int i = lo + tid; i < hi; i += AC_THREADS) {
      double wi = w[i];
      for (int k = 0; k <= j; ++k) wi = fma(-h1s[k], V[(long long)k * n + i], wi);
      w[i] = wi;
    }
    cluster_dots(V, n, j + 1, false, w, lo, hi, cs, buf);
    if (tid <= j) h2s[tid] = cs.out[tid];
    __syncthreads();
    // P3: w -= V h2, ||w||^2 -> the H column, the breakdown test, the next scale
    for (int i = lo + tid; i < hi; i += AC_THREADS) {
      double wi = w[i];
      for (int k = 0; k <= j; ++k) wi = fma(-h2s[k], V[(long long)k * n + i], wi);
      w[i] = wi;
    }
    cluster_dots(V, n, 0, true, w, lo, hi, cs, buf);
    const bool active = steps < 0;
    const double hn = sqrt(cs.out[AR_SLOTS - 1]);
    if (r == 0 && tid <= j) H[tid + (long long)j * ldh] = active ? h1s[tid] + h2s[tid] : 0.0;
    if (r == 0 && tid == 0) H[j + 1 + (long long)j * ldh] = active ? hn : 0.0;
    if (active && hn <= 1e-10 * sqrt(w0n2)) steps = j + 1;
    sc = (active && hn > 0.0) ? 1.0 / hn : 0.0;
  }
  if (r == 0 && tid == 0) *steps_out = steps;
  cl.sync();  // no CTA leaves while another may still read its partials
}

template <int W>
static void allow_cluster16() {
  CLAIR_CUDA(cudaFuncSetAttribute(arnoldi_cluster<W>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
}

// Largest cluster (16 or 8) the device schedules for this kernel, per device.
static int ac_cluster_max() {
  static int cmax[256] = {};
  int dev = 0;
  CLAIR_CUDA(cudaGetDevice(&dev));
  once_per_device((const void*)&ac_cluster_max, [] {
    int d = 0;
    CLAIR_CUDA(cudaGetDevice(&d));
    allow_cluster16<1>();
    allow_cluster16<2>();
    allow_cluster16<4>();
    int best = 8;
    for (int c : {16, 12}) {
      cudaLaunchConfig_t cfg = {};
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = c;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.gridDim = dim3(c);
      cfg.blockDim = dim3(AC_THREADS);
      cfg.attrs = at;
      cfg.numAttrs = 1;
      int nclusters = 0;
      if (cudaOccupancyMaxActiveClusters(&nclusters, arnoldi_cluster<4>, &cfg) == cudaSuccess &&
          nclusters >= 1) {
        best = c;
        break;
      }
      cudaGetLastError();
    }
    if (d >= 0 && d < 256) cmax[d] = best;
  });
  return (dev >= 0 && dev < 256 && cmax[dev]) ? cmax[dev] : 8;
}

// Levels this small take the one-launch path: its cluster's FP64 pipes do the level's
// work in less time than the multi-launch path spends on its 3 m launches.
static bool arnoldi_on_cluster(const Csr& A, int m) {
  return m <= AR_MAXV && A.rows >= 1 && A.nnz <= (1 << 20);
}

static void arnoldi_cluster_run(const Csr& A, const double* dinv, int m, uint64_t seed,
                                double* V, double* w0, double* w1, double* H, int ldh,
                                int* steps, cudaStream_t s) {
  // every SM of the cluster adds FP64 throughput; at least 64 rows per CTA
  int C = std::max(1, std::min(ac_cluster_max(), (A.rows + 63) / 64));
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(C);
  cfg.blockDim = dim3(AC_THREADS);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  // at most four lanes per row: a CTA then keeps eight rows per warp in flight, and its
  // FP64 pipe, not the latency of one row, sets the pace
  const int W = std::min(lanes_of(A, true), 4);
  if (W == 1)
    CLAIR_CUDA(cudaLaunchKernelEx(&cfg, arnoldi_cluster<1>, A.rowptr, A.col, A.val, dinv, A.rows,
                                  m, seed, V, w0, w1, H, ldh, steps));
  else if (W == 2)
    CLAIR_CUDA(cudaLaunchKernelEx(&cfg, arnoldi_cluster<2>, A.rowptr, A.col, A.val, dinv, A.rows,
                                  m, seed, V, w0, w1, H, ldh, steps));
  else
    CLAIR_CUDA(cudaLaunchKernelEx(&cfg, arnoldi_cluster<4>, A.rowptr, A.col, A.val, dinv, A.rows,
                                  m, seed, V, w0, w1, H, ldh, steps));
  ::clair::count_launch();
  CLAIR_LAUNCHED();
}

// ---- Ritz values on the host --------------------------------------------------------
// The 15 x 15 Hessenberg QR is a chain of dependent FP64 operations (about 0.5 ms on one
// warp at 64-cycle FP64 latency, tens of microseconds on a host core).  The Hessenberg
// matrices are copied to pinned host memory, a stream callback computes the weights and
// the next copy puts them back on the device, all in stream order.
struct RitzHost {
  int ldh = 0, m = 0, ninst = 0;
  size_t bytes = 0;         // the pinned block holding this header and the arrays
  double* H = nullptr;      // ninst x ldh x m, pinned
  int* steps = nullptr;     // ninst, pinned
  double* omega = nullptr;  // ninst, pinned
};

static void CUDART_CB ritz_on_host(void* data) {
  RitzHost* r = static_cast<RitzHost*>(data);
  double Hs[AR_MAXV * AR_MAXV];
  for (int i = 0; i < r->ninst; ++i) {
    const double* Hi = r->H + (size_t)i * r->ldh * r->m;
    const int k = r->steps[i] < 0 ? r->m : r->steps[i];
    for (int c = 0; c < k; ++c)
      for (int q = 0; q < k; ++q) Hs[q + c * k] = Hi[q + (size_t)c * r->ldh];
    const double rho = hessenberg_spectral_radius(Hs, k, k);
    r->omega[i] = rho > 0.0 ? 1.0 / rho : 1.0;
  }
}

// Pinned buffers for one Arnoldi run's Ritz step, one recycled block (released by the
// caller after the stream has passed the run).
RitzHost* ritz_host_alloc(int ninst) {
  const int ldh = AR_MAXV + 1;
  const size_t head = 64;
  const size_t hbytes = sizeof(double) * (size_t)ninst * ldh * AR_MAXV;
  const size_t obytes = sizeof(double) * (size_t)ninst;
  const size_t sbytes = sizeof(int) * (size_t)ninst;
  const size_t bytes = head + hbytes + obytes + sbytes;
  static_assert(sizeof(RitzHost) <= 64, "RitzHost header must fit its slot");
  char* base = static_cast<char*>(pinned_get(bytes));
  RitzHost* r = new (base) RitzHost();
  r->bytes = bytes;
  r->ninst = ninst;
  r->H = reinterpret_cast<double*>(base + head);
  r->omega = reinterpret_cast<double*>(base + head + hbytes);
  r->steps = reinterpret_cast<int*>(base + head + hbytes + obytes);
  return r;
}

void ritz_host_free(RitzHost* r) {
  if (!r) return;
  const size_t bytes = r->bytes;
  r->~RitzHost();
  pinned_put(r, bytes);
}

// Enqueues: H, steps -> host; the callback; weights -> omega_dev.
static void ritz_via_host(const double* H, int ldh, int m, const int* steps, int ninst,
                          double* omega_dev, RitzHost* r, cudaStream_t s) {
  CLAIR_REQUIRE(m <= AR_MAXV && r && r->ninst >= ninst, CLAIR_ERR_ARG, "host Ritz step misuse");
  r->ldh = ldh;
  r->m = m;
  r->ninst = ninst;
  CLAIR_CUDA(cudaMemcpyAsync(r->H, H, sizeof(double) * ninst * ldh * m, cudaMemcpyDeviceToHost, s));
  CLAIR_CUDA(cudaMemcpyAsync(r->steps, steps, sizeof(int) * ninst, cudaMemcpyDeviceToHost, s));
  CLAIR_CUDA(cudaLaunchHostFunc(s, ritz_on_host, r));
  CLAIR_CUDA(cudaMemcpyAsync(omega_dev, r->omega, sizeof(double) * ninst, cudaMemcpyHostToDevice, s));
}

// ---- segmented Arnoldi: one independent run per instance of a block-diagonal batch ----
// Block b of every launch owns rows [lo[b], hi[b]) of instance inst[b]; an instance's
// blocks are consecutive (first bfirst[i], count bcount[i]) and its finalize adds their
// partial sums in block order, so every instance's weight is deterministic and equals a
// run on that instance alone up to the summation order.  The start vector of instance i
// is draw (row - off[i]) of the stream seeded with `seed`, as in a run on the instance.
struct SegBlocks {
  const int* lo;
  const int* hi;
  const int* inst;
};
constexpr int SEG_HS = AR_MAXV + 1;  // per-instance stride of h1 / h2

__global__ void seg_start(double* __restrict__ v, SegBlocks sb, const int* __restrict__ off,
                          uint64_t seed, double* __restrict__ partial) {
  const int b = blockIdx.x;
  const int lo = sb.lo[b], hi = sb.hi[b], base = off[sb.inst[b]];
  double acc[1] = {0.0};
  for (int i = lo + threadIdx.x; i < hi; i += AR_THREADS) {
    const double x = splitmix_pm1(seed, (uint64_t)(i - base));
    v[i] = x;
    acc[0] += x * x;
  }
  block_reduce_to_partial<1>(acc, 1, partial);
}

template <int W>
__global__ void __launch_bounds__(AR_THREADS)
seg_k1(const int* __restrict__ rp, const int* __restrict__ ci, const double* __restrict__ av,
       const double* __restrict__ dinv, int n, double* __restrict__ V, int j,
       const double* __restrict__ wprev, const double* __restrict__ sc, int use_scale,
       double* __restrict__ w, double* __restrict__ partial, SegBlocks sb) {
  constexpr int GPW = 32 / W;
  const int b = blockIdx.x;
  const int lo = sb.lo[b], hi = sb.hi[b];
  const double scl = use_scale ? sc[2 * sb.inst[b] + 1] : 1.0;
  double acc[AR_MAXV + 2];
#pragma unroll
  for (int v = 0; v < AR_MAXV + 2; ++v) acc[v] = 0.0;
  const int lane = threadIdx.x & 31, sub = lane % W, grp = lane / W;
  const int warp = threadIdx.x >> 5;
  for (int base = lo + warp * GPW; base < hi; base += (AR_THREADS / 32) * GPW) {  // warp-uniform
    const int i = base + grp;
    double s = 0.0;
    if (i < hi)
      s = csr_row_dot<W>(ci, av, wprev, rp[i], rp[i + 1], sub);
    s = group_sum<W>(s);
    if (sub == 0 && i < hi) {
      const double wi = dinv[i] * (scl * s);
      const double vj = wprev[i] * scl;
      w[i] = wi;
      if (j > 0) V[(long long)j * n + i] = vj;
#pragma unroll
      for (int k = 0; k < AR_MAXV; ++k)
        if (k <= j) acc[k] += (k < j ? V[(long long)k * n + i] : vj) * wi;
      acc[AR_MAXV + 1] += wi * wi;
    }
  }
  block_reduce_to_partial<AR_MAXV + 2>(acc, AR_MAXV + 2, partial);
}

template <bool DOTS>
__global__ void __launch_bounds__(AR_THREADS)
seg_cgs(const double* __restrict__ V, int j, int n, const double* __restrict__ h,
        double* __restrict__ w, double* __restrict__ partial, SegBlocks sb) {
  const int b = blockIdx.x;
  const int lo = sb.lo[b], hi = sb.hi[b];
  const double* hi_ = h + (long long)SEG_HS * sb.inst[b];
  double acc[AR_MAXV + 1];
#pragma unroll
  for (int v = 0; v < AR_MAXV + 1; ++v) acc[v] = 0.0;
  double hk[AR_MAXV];
#pragma unroll
  for (int k = 0; k < AR_MAXV; ++k) hk[k] = k <= j ? hi_[k] : 0.0;
  for (int i = lo + threadIdx.x; i < hi; i += AR_THREADS) {
    double vk[AR_MAXV];
    double wi = w[i];
#pragma unroll
    for (int k = 0; k < AR_MAXV; ++k) {
      vk[k] = k <= j ? V[(long long)k * n + i] : 0.0;
      if (k <= j) wi = fma(-hk[k], vk[k], wi);
    }
    w[i] = wi;
    if (DOTS) {
#pragma unroll
      for (int k = 0; k < AR_MAXV; ++k)
        if (k <= j) acc[k] += vk[k] * wi;
    } else {
      acc[0] += wi * wi;
    }
  }
  block_reduce_to_partial<AR_MAXV + 1>(acc, DOTS ? j + 1 : 1, partial);
}

// One block per instance: adds its blocks' partials in block order.  mode 0: h1, ||w||^2
// before orthogonalisation; 1: h2; 2: H column, breakdown test, next scale; 3: scale of
// the start vector (1/||v_0||), stored as the next scale.
__global__ void __launch_bounds__(512)
seg_finalize(const double* __restrict__ partial, int nb, int nv, int mode, int j,
             const int* __restrict__ bfirst, const int* __restrict__ bcount,
             double* __restrict__ h1, double* __restrict__ h2, double* __restrict__ sc,
             double* __restrict__ H, int ldh, int m, int* __restrict__ steps) {
  __shared__ double out[AR_MAXV + 2];
  const int inst = blockIdx.x;
  const int b0 = bfirst[inst], b1 = b0 + bcount[inst];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int v = wid; v < nv; v += 16) {
    double t = 0.0;
    for (int b = b0 + lane; b < b1; b += 32) t += partial[(long long)v * nb + b];
    t = warp_sum(t);
    if (lane == 0) out[v] = t;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  double* h1i = h1 + (long long)SEG_HS * inst;
  double* h2i = h2 + (long long)SEG_HS * inst;
  double* sci = sc + 2 * inst;
  double* Hi = H + (long long)inst * ldh * m;
  if (mode == 0) {
    for (int k = 0; k <= j; ++k) h1i[k] = out[k];
    sci[0] = out[AR_MAXV + 1];
  } else if (mode == 1) {
    for (int k = 0; k <= j; ++k) h2i[k] = out[k];
  } else if (mode == 2) {
    const bool active = steps[inst] < 0;
    for (int i = 0; i <= j; ++i) Hi[i + (long long)j * ldh] = active ? h1i[i] + h2i[i] : 0.0;
    const double hn = sqrt(out[0]);
    Hi[j + 1 + (long long)j * ldh] = active ? hn : 0.0;
    if (active && hn <= 1e-10 * sqrt(sci[0])) steps[inst] = j + 1;
    sci[1] = (active && hn > 0.0) ? 1.0 / hn : 0.0;
  } else {
    sci[1] = out[0] > 0.0 ? 1.0 / sqrt(out[0]) : 0.0;
  }
}

__global__ void seg_scale_start(double* __restrict__ v, SegBlocks sb, const double* __restrict__ sc) {
  const int b = blockIdx.x;
  const double f = sc[2 * sb.inst[b] + 1];
  for (int i = sb.lo[b] + threadIdx.x; i < sb.hi[b]; i += blockDim.x) v[i] *= f;
}

__global__ void __launch_bounds__(32) seg_ritz(const double* __restrict__ H, int ldh, int m,
                                               const int* __restrict__ steps,
                                               double* __restrict__ omega) {
  __shared__ double Hs[AR_MAXV * AR_MAXV];
  const int inst = blockIdx.x, lane = threadIdx.x;
  const double* Hi = H + (long long)inst * ldh * m;
  const int k = steps[inst] < 0 ? m : steps[inst];
  for (int idx = lane; idx < k * k; idx += 32) Hs[idx] = Hi[(idx % k) + (long long)(idx / k) * ldh];
  __syncwarp();
  const double rho = hessenberg_spectral_radius_lanes(Hs, k, k, lane, 32, WarpSync{});
  if (lane == 0) omega[inst] = rho > 0.0 ? 1.0 / rho : 1.0;
}

// Enqueues omega_i = 1 / rho(D_i^-1 A_i) for every diagonal block i of A (rows off[i] ..
// off[i+1]-1, host offsets) into omega_dev[i].  iters <= 15.
void arnoldi_weight_batched(const Csr& A, const double* dinv, int iters, uint64_t seed,
                            const std::vector<int>& off, double* omega_dev, RitzHost* rh,
                            cudaStream_t s) {
  const int n = A.rows;
  const int ninst = (int)off.size() - 1;
  const int m = std::max(1, std::min(iters, AR_MAXV));
  const int ldh = m + 1;
  // blocks per instance in proportion to its rows (at least one)
  const int target = partial_blocks();
  std::vector<int> lo, hi, inst, bfirst(ninst), bcount(ninst);
  for (int i = 0; i < ninst; ++i) {
    const int ni = off[i + 1] - off[i];
    const int nb = std::max(1, std::min(ceil_div(ni, AR_THREADS),
                                        (int)((long long)target * ni / std::max(n, 1))));
    bfirst[i] = (int)lo.size();
    bcount[i] = nb;
    for (int b = 0; b < nb; ++b) {
      lo.push_back(off[i] + (int)((long long)ni * b / nb));
      hi.push_back(off[i] + (int)((long long)ni * (b + 1) / nb));
      inst.push_back(i);
    }
  }
  const int nb = (int)lo.size();
  std::vector<int> pack;
  for (const std::vector<int>* v : {(const std::vector<int>*)&lo, (const std::vector<int>*)&hi,
                                    (const std::vector<int>*)&inst, (const std::vector<int>*)&bfirst,
                                    (const std::vector<int>*)&bcount, &off})
    pack.insert(pack.end(), v->begin(), v->end());
  int* dpack = dalloc<int>(pack.size(), s);
  CLAIR_CUDA(cudaMemcpyAsync(dpack, pack.data(), sizeof(int) * pack.size(), cudaMemcpyHostToDevice, s));
  const SegBlocks sb{dpack, dpack + nb, dpack + 2 * nb};
  const int* d_bfirst = dpack + 3 * nb;
  const int* d_bcount = d_bfirst + ninst;
  const int* d_off = d_bcount + ninst;
  double* V = dalloc<double>((size_t)(m + 1) * n, s);
  double* w0 = dalloc<double>(n, s);
  double* w1 = dalloc<double>(n, s);
  double* H = dalloc<double>((size_t)ninst * ldh * m, s);
  double* h1 = dalloc<double>((size_t)ninst * SEG_HS, s);
  double* h2 = dalloc<double>((size_t)ninst * SEG_HS, s);
  double* sc = dalloc<double>((size_t)ninst * 2, s);
  int* steps = dalloc<int>(ninst, s);
  double* partial = dalloc<double>((size_t)nb * (AR_MAXV + 2), s);
  CLAIR_CUDA(cudaMemsetAsync(H, 0, sizeof(double) * ninst * ldh * m, s));
  CLAIR_CUDA(cudaMemsetAsync(steps, 0xff, sizeof(int) * ninst, s));  // -1: no breakdown
  seg_start<<<nb, AR_THREADS, 0, s>>>(V, sb, d_off, seed, partial); ::clair::count_launch();
  seg_finalize<<<ninst, 512, 0, s>>>(partial, nb, 1, 3, 0, d_bfirst, d_bcount, h1, h2, sc, H, ldh,
                                     m, steps); ::clair::count_launch();
  seg_scale_start<<<nb, AR_THREADS, 0, s>>>(V, sb, sc); ::clair::count_launch();
  CLAIR_LAUNCHED();
  double* const wbuf[2] = {w0, w1};
  for (int j = 0; j < m; ++j) {
    double* w = wbuf[j & 1];
    const double* wprev = j == 0 ? V : wbuf[(j + 1) & 1];
    seg_k1<1><<<nb, AR_THREADS, 0, s>>>(A.rowptr, A.col, A.val, dinv, n, V, j, wprev, sc, j > 0, w,
                                        partial, sb); ::clair::count_launch();
    seg_finalize<<<ninst, 512, 0, s>>>(partial, nb, AR_MAXV + 2, 0, j, d_bfirst, d_bcount, h1, h2,
                                       sc, H, ldh, m, steps); ::clair::count_launch();
    seg_cgs<true><<<nb, AR_THREADS, 0, s>>>(V, j, n, h1, w, partial, sb); ::clair::count_launch();
    seg_finalize<<<ninst, 512, 0, s>>>(partial, nb, j + 1, 1, j, d_bfirst, d_bcount, h1, h2, sc, H,
                                       ldh, m, steps); ::clair::count_launch();
    seg_cgs<false><<<nb, AR_THREADS, 0, s>>>(V, j, n, h2, w, partial, sb); ::clair::count_launch();
    seg_finalize<<<ninst, 512, 0, s>>>(partial, nb, 1, 2, j, d_bfirst, d_bcount, h1, h2, sc, H, ldh,
                                       m, steps); ::clair::count_launch();
    CLAIR_LAUNCHED();
  }
  if (rh) {
    ritz_via_host(H, ldh, m, steps, ninst, omega_dev, rh, s);
  } else {
    seg_ritz<<<ninst, 32, 0, s>>>(H, ldh, m, steps, omega_dev); ::clair::count_launch();
    CLAIR_LAUNCHED();
  }
  dfree(V, s);
  dfree(w0, s);
  dfree(w1, s);
  dfree(H, s);
  dfree(h1, s);
  dfree(h2, s);
  dfree(sc, s);
  dfree(partial, s);
  dfree(steps, s);
  dfree(dpack, s);
}

// Enqueues omega = 1 / rho(D^-1 A) into the device scalar *omega_dev (no host sync).
double arnoldi_weight(const Csr& A, const double* dinv, int iters, uint64_t seed,
                      double* omega_dev, RitzHost* rh, cudaStream_t s) {
  const int n = A.rows;
  const int m = std::max(1, std::min(iters, n));
  const int ldh = m + 1;
  if (arnoldi_on_cluster(A, m)) {
    double* V = dalloc<double>((size_t)m * n, s);
    double* w = dalloc<double>((size_t)2 * n, s);
    double* H = dalloc<double>((size_t)ldh * m, s);
    int* steps = dalloc<int>(1, s);
    CLAIR_CUDA(cudaMemsetAsync(H, 0, sizeof(double) * ldh * m, s));
    arnoldi_cluster_run(A, dinv, m, seed, V, w, w + n, H, ldh, steps, s);
    if (rh) {
      ritz_via_host(H, ldh, m, steps, 1, omega_dev, rh, s);
    } else {
      ritz_kernel<<<1, 32, 0, s>>>(H, ldh, m, steps, omega_dev); ::clair::count_launch();
      CLAIR_LAUNCHED();
    }
    dfree(V, s);
    dfree(w, s);
    dfree(H, s);
    dfree(steps, s);
    return 0.0;
  }
  double* V = dalloc<double>((size_t)(m + 1) * n, s);
  double* w = dalloc<double>(n, s);
  double* H = dalloc<double>((size_t)ldh * m, s);
  double* sc = dalloc<double>(2 * 64 + 8, s);  // h1[64], h2[64], wn2, w0n2, inv
  double* h1 = sc;
  double* h2 = sc + 64;
  double* wn2 = sc + 128;
  double* w0n2 = sc + 129;
  double* inv = sc + 130;
  int* steps = dalloc<int>(1, s);
  double* partial = dalloc<double>((size_t)partial_blocks() * (std::max(m, AR_MAXV) + 2), s);
  const int grid = std::min(ceil_div(n, 256), 32 * sm_count());
  CLAIR_CUDA(cudaMemsetAsync(H, 0, sizeof(double) * ldh * m, s));
  const int minus1 = -1;
  CLAIR_CUDA(cudaMemcpyAsync(steps, &minus1, sizeof(int), cudaMemcpyHostToDevice, s));
  arnoldi_start<<<grid, 256, 0, s>>>(V, n, seed); ::clair::count_launch();
  multi_dot(V, 1, V, n, wn2, partial, s);
  scale_by_inv_sqrt<<<grid, 256, 0, s>>>(V, n, wn2); ::clair::count_launch();
  CLAIR_LAUNCHED();
  int* steps_hist = nullptr;
  if (m <= AR_MAXV) {
    // up to six blocks per SM (the kernels' registers allow it), at least 32 rows a block
    const int nb = std::max(1, std::min(6 * sm_count(), ceil_div(n, 32)));
    double* w2 = dalloc<double>(n, s);
    double* p2 = dalloc<double>((size_t)nb * (AR_MAXV + 2), s);
    steps_hist = dalloc<int>(m + 1, s);
    unsigned* ticket = dalloc<unsigned>(1, s);
    CLAIR_CUDA(cudaMemsetAsync(steps_hist, 0xff, sizeof(int) * (m + 1), s));  // -1
    CLAIR_CUDA(cudaMemsetAsync(ticket, 0, sizeof(unsigned), s));
    double* const wbuf[2] = {w, w2};
    const ArnoldiState st{H, ldh, h1, h2, sc + 129, sc + 131, steps_hist, ticket};
    arnoldi_fused_steps(A, dinv, m, V, wbuf, st, p2, nb, s);
    CLAIR_CUDA(cudaMemcpyAsync(steps, steps_hist + m, sizeof(int), cudaMemcpyDeviceToDevice, s));
    dfree(w2, s);
    dfree(p2, s);
    dfree(ticket, s);
  }
  for (int j = 0; j < m && m > AR_MAXV; ++j) {
    double* vj = V + (size_t)j * n;
    spmv(A, vj, w, 1.0, 0.0, s);
    dinv_scale<<<grid, 256, 0, s>>>(w, dinv, n); ::clair::count_launch();
    CLAIR_LAUNCHED();
    multi_dot(w, 1, w, n, w0n2, partial, s);
    multi_dot(V, j + 1, w, n, h1, partial, s);
    multi_axpy(V, j + 1, h1, w, n, s);
    multi_dot(V, j + 1, w, n, h2, partial, s);
    multi_axpy(V, j + 1, h2, w, n, s);
    multi_dot(w, 1, w, n, wn2, partial, s);
    arnoldi_column<<<1, 32, 0, s>>>(H, ldh, j, h1, h2, wn2, w0n2, steps, inv); ::clair::count_launch();
    scale_vec<<<grid, 256, 0, s>>>(w, V + (size_t)(j + 1) * n, n, inv); ::clair::count_launch();
    CLAIR_LAUNCHED();
  }
  if (rh && m <= AR_MAXV) {
    ritz_via_host(H, ldh, m, steps, 1, omega_dev, rh, s);
  } else {
    ritz_kernel<<<1, 32, 0, s>>>(H, ldh, m, steps, omega_dev); ::clair::count_launch();
    CLAIR_LAUNCHED();
  }
  dfree(V, s);
  dfree(w, s);
  dfree(H, s);
  dfree(sc, s);
  dfree(steps, s);
  dfree(steps_hist, s);
  dfree(partial, s);
  return 0.0;  // the weight is in *omega_dev once the stream reaches this point
}

// ------------------------------------------------------------------------------------
// Coarsest level: dense inverse by Gauss-Jordan elimination with partial pivoting (one
// block; n <= a few hundred).  M is n x n column-major in global memory, overwritten.
// ------------------------------------------------------------------------------------
// Dense inverses of the diagonal blocks of the coarsest operator: block i holds rows and
// columns off[i] .. off[i+1]-1 (one block when the hierarchy is not a batch) and is stored
// column-major at Inv + ioff[i], ioff[i] = sum_{j<i} n_j^2.  One CUDA block per diagonal
// block: Gauss-Jordan with partial pivoting.
__global__ void csr_to_dense_blocks(const int* __restrict__ rowptr, const int* __restrict__ col,
                                    const double* __restrict__ val, const int* __restrict__ off,
                                    const long long* __restrict__ ioff, double* __restrict__ M) {
  const int i = blockIdx.x;
  const int r0 = off[i], nb = off[i + 1] - r0;
  double* Mi = M + ioff[i];
  for (long long idx = threadIdx.x; idx < (long long)nb * nb; idx += blockDim.x) Mi[idx] = 0.0;
  __syncthreads();
  for (int r = threadIdx.x; r < nb; r += blockDim.x)
    for (int e = rowptr[r0 + r]; e < rowptr[r0 + r + 1]; ++e)
      Mi[r + (long long)(col[e] - r0) * nb] = val[e];
}

__global__ void gauss_jordan_blocks(double* __restrict__ M, double* __restrict__ Inv,
                                    const int* __restrict__ off, const long long* __restrict__ ioff,
                                    int* __restrict__ singular) {
  // Inv starts as identity; row operations on [M | Inv].
  __shared__ int s_piv;
  __shared__ double s_pv;
  const int blk = blockIdx.x;
  const int n = off[blk + 1] - off[blk];
  double* Mb = M + ioff[blk];
  double* Ib = Inv + ioff[blk];
  const int t = threadIdx.x, nt = blockDim.x;
  for (int idx = t; idx < n * n; idx += nt) Ib[idx] = (idx % n == idx / n) ? 1.0 : 0.0;
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (t == 0) {
      int p = k;
      double best = fabs(Mb[k + (long long)k * n]);
      for (int r = k + 1; r < n; ++r) {
        const double v = fabs(Mb[r + (long long)k * n]);
        if (v > best) {
          best = v;
          p = r;
        }
      }
      s_piv = p;
      s_pv = Mb[p + (long long)k * n];
      if (best == 0.0) *singular = 1;
    }
    __syncthreads();
    const int p = s_piv;
    if (p != k)
      for (int c = t; c < n; c += nt) {
        double a = Mb[k + (long long)c * n];
        Mb[k + (long long)c * n] = Mb[p + (long long)c * n];
        Mb[p + (long long)c * n] = a;
        double b = Ib[k + (long long)c * n];
        Ib[k + (long long)c * n] = Ib[p + (long long)c * n];
        Ib[p + (long long)c * n] = b;
      }
    __syncthreads();
    const double pv = s_pv;
    for (int c = t; c < n; c += nt) {
      if (pv != 0.0) {
        Mb[k + (long long)c * n] /= pv;
        Ib[k + (long long)c * n] /= pv;
      }
    }
    __syncthreads();
    // eliminate column k from every other row (rows split over threads)
    for (int r = t; r < n; r += nt) {
      if (r == k) continue;
      const double f = Mb[r + (long long)k * n];
      if (f == 0.0) continue;
      for (int c = 0; c < n; ++c) {
        Mb[r + (long long)c * n] -= f * Mb[k + (long long)c * n];
        Ib[r + (long long)c * n] -= f * Ib[k + (long long)c * n];
      }
    }
    __syncthreads();
  }
}

// d_off / d_ioff receive device copies of the block offsets (caller frees them).
void dense_inverse(const Csr& A, const std::vector<int>& off, double* Inv, int** d_off,
                   long long** d_ioff, cudaStream_t s) {
  const int nblk = (int)off.size() - 1;
  std::vector<long long> ioff(nblk + 1, 0);
  for (int i = 0; i < nblk; ++i) {
    const long long ni = off[i + 1] - off[i];
    ioff[i + 1] = ioff[i] + ni * ni;
  }
  *d_off = dalloc<int>(nblk + 1, s);
  *d_ioff = dalloc<long long>(nblk + 1, s);
  CLAIR_CUDA(cudaMemcpyAsync(*d_off, off.data(), sizeof(int) * (nblk + 1), cudaMemcpyHostToDevice, s));
  CLAIR_CUDA(cudaMemcpyAsync(*d_ioff, ioff.data(), sizeof(long long) * (nblk + 1),
                             cudaMemcpyHostToDevice, s));
  double* M = dalloc<double>(std::max<long long>(ioff[nblk], 1), s);
  int* sing = dalloc<int>(1, s);
  CLAIR_CUDA(cudaMemsetAsync(sing, 0, sizeof(int), s));
  if (A.rows) {
    csr_to_dense_blocks<<<nblk, 256, 0, s>>>(A.rowptr, A.col, A.val, *d_off, *d_ioff, M); ::clair::count_launch();
    gauss_jordan_blocks<<<nblk, 256, 0, s>>>(M, Inv, *d_off, *d_ioff, sing); ::clair::count_launch();
  }
  CLAIR_LAUNCHED();
  int h = 0;
  CLAIR_CUDA(cudaMemcpyAsync(&h, sing, sizeof(int), cudaMemcpyDeviceToHost, s));
  CLAIR_CUDA(cudaStreamSynchronize(s));
  dfree(M, s);
  dfree(sing, s);
  CLAIR_REQUIRE(h == 0, CLAIR_ERR_SINGULAR_BLOCK, "coarsest operator is singular");
}

// x = Inv b blockwise (row r of block i: sum over the block's columns).
template <class T>
__global__ void dense_gemv_blocks(const T* __restrict__ Inv, const int* __restrict__ off,
                                  const long long* __restrict__ ioff, int nblk, int n,
                                  const T* __restrict__ b, T* __restrict__ x) {
  pdl_prologue();
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
    int lo = 0, hi = nblk;  // block holding row r: largest i with off[i] <= r
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (off[mid] <= r) lo = mid; else hi = mid;
    }
    const int r0 = off[lo], nb = off[lo + 1] - r0;
    const T* Ib = Inv + ioff[lo];
    T acc = 0;
    for (int c = 0; c < nb; ++c) acc += Ib[(r - r0) + (long long)c * nb] * b[r0 + c];
    x[r] = acc;
  }
}
template <class T>
void coarse_apply(const T* Inv, const int* d_off, const long long* d_ioff, int nblk, int n,
                  const T* b, T* x, cudaStream_t s) {
  if (!n) return;
  launch_k(dense_gemv_blocks<T>, ceil_div(n, 128), 128, 0, s, Inv, d_off, d_ioff, nblk, n, b, x); ::clair::count_launch();
  CLAIR_LAUNCHED();
}
template void coarse_apply<double>(const double*, const int*, const long long*, int, int,
                                   const double*, double*, cudaStream_t);
template void coarse_apply<float>(const float*, const int*, const long long*, int, int,
                                  const float*, float*, cudaStream_t);

}  // namespace clair
