// Batched constrained local solves (the CLAIR hot loop).
//
// For every coarse point i with pattern W_i = {l_1 < ... < l_T} (F-points), Algorithm 1
// with exact block inverses and one iteration (Remark 3.2) needs the local lAIR system
// (Eq. 3.1; Eq. 2.8 for the restriction, which is the same system on A^T):
//     Ahat[W_i, W_i] w_i = -Ahat[W_i, i],
// followed by the projection onto the mode constraint W B_c = B|_F (Eq. 3.3), which for
// one mode vector and exact inverses reduces to, per F-point j with J_j = {i : j in W_i},
//     w_ji <- w_ji - mu_j B_c(i),  mu_j = (sum_i w_ji B_c(i) - B_j) / sum_i B_c(i)^2.
// (With the exact inverse, Algorithm 1 returns the Euclidean projection of the lAIR
// weights onto {Q w = B|_F}; the tentative weights cancel.)
//
// Layout: the pattern is a CSR with one row per coarse point (the transposed P_hat), each
// row holding the coarse point's own column (identity weight 1) and its F-points sorted.
// Systems are bucketed by T: T <= 8, 16 use G lanes of a warp per system (row p of the
// local matrix lives in the registers of lane p; the pivot row is broadcast with
// shuffles); 16 < T <= 128 uses one CTA of 32, 64 or 128 threads per system with the
// matrix in shared memory.
// Pivoting is partial (largest |entry| among rows not yet used, lowest row on ties),
// done implicitly by marking rows instead of swapping them.
#include <algorithm>
#include <mutex>
#include <type_traits>
#include <vector>

#include "common.cuh"

namespace clair {

// Solvable buckets: T in [0,8], (8,16], (16,32], (32,64], (64,128], (128,tmed] and
// (tmed,4096] (global tiles, eliminated in panels where a panel fits shared memory, else
// step by step; bucket 5 in one launch of tiles of pitch tmed, 128 threads per system, so
// that several of its many systems share an SM: tmed = LS_TMED32 in FP32, LS_TMED64 in
// FP64); bucket 7 counts systems larger than LS_TBIG (refused).
constexpr int LS_BUCKETS = 7;
constexpr int LS_TBIG = 4096;
constexpr int LS_TMED32 = 224;
constexpr int LS_TMED64 = 160;
__host__ __device__ inline int ls_bucket(int T, int tmed) {
  return T <= 8 ? 0 : T <= 16 ? 1 : T <= 32 ? 2 : T <= 64 ? 3 : T <= 128 ? 4
       : T <= tmed ? 5 : T <= LS_TBIG ? 6 : 7;
}

// Position of column c in the sorted list z[0..T-1], or -1.
__device__ __forceinline__ int find_sorted(const int* z, int T, int c) {
  int lo = 0, hi = T - 1;
  while (lo <= hi) {
    int mid = (lo + hi) >> 1;
    int v = z[mid];
    if (v == c) return mid;
    if (v < c)
      lo = mid + 1;
    else
      hi = mid - 1;
  }
  return -1;
}

// ------------------------------------------------------------------------------------
// Sub-warp path: G lanes per system, G in {8, 16}, T <= G.
// ------------------------------------------------------------------------------------
constexpr int LS_WARPS = 4;  // warps per block in the sub-warp path
// Row updates of the shared- and global-tile solves read LS_CHUNK entries of the pivot
// row and of the own row before writing any: both rows live in one array, so without
// that the compiler must order every load after the previous store.
constexpr int LS_CHUNK = 8;

// Shared memory of one warp's groups (32 / G systems).
template <class Real, int G>
struct GroupSmem {
  static constexpr int GPW = 32 / G;
  Real tile[GPW][G][G + 1];
  Real rhs_s[GPW][G];
  int zl[GPW][G];
  int pre[GPW][G + 1];
  int rs[GPW][G];          // start of each pattern row in Ahat
  int pivlane[GPW][G];     // lane that pivoted each elimination step
};

// One warp solves 32 / G systems: `item` is this lane's group's position in `work`
// (live when < nwork); row p of the local matrix lives in the registers of lane p, the
// pivot row is broadcast with shuffles.  Every lane of the warp must call it.
template <class Real, class VT, int G>
__device__ __forceinline__ void group_body(const int* __restrict__ Arp, const int* __restrict__ Acol,
                                           const VT* __restrict__ Aval, const int* __restrict__ Zrp,
                                           const int* __restrict__ Zcol, const int* __restrict__ cpts,
                                           const int* __restrict__ work, long long item, long long nwork,
                                           double* __restrict__ Zval,
                                           unsigned long long* __restrict__ nsingular,
                                           GroupSmem<Real, G>& sm) {
  const int lane = threadIdx.x & 31;
  const int gsub = lane / G;          // group within warp
  const int p = lane % G;             // row owned by this lane
  const bool live = item < nwork;

  int r = 0, i = 0, base = 0, len = 1;
  if (live) {
    r = work[item];
    i = cpts[r];
    base = Zrp[r];
    len = Zrp[r + 1] - base;
  }
  const int T = len - 1;
  // position d of the identity column within the row
  int zc = (live && p < len) ? Zcol[base + p] : -1;
  unsigned m = __ballot_sync(0xffffffffu, live && p < len && zc == i);
  const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (gsub * G));
  m &= gmask;
  // the identity sits at position G (unseen by the G lanes) only when T == G
  const int d = m ? (__ffs(m) - 1 - gsub * G) : T;
  // F-only column list
  int fcol = -1;
  if (live && p < T) fcol = Zcol[base + p + (p >= d ? 1 : 0)];
  sm.zl[gsub][p] = fcol;
  __syncwarp();

  // Gather the local matrix (row p = row l_p of Ahat restricted to the pattern) and the
  // right-hand side -Ahat[l_p, i].  The rows' entries are flattened (a group scan of the
  // row lengths) and spread over all G lanes so their loads are independent.
#pragma unroll
  for (int q = 0; q < G; ++q) sm.tile[gsub][p][q] = Real(0);
  sm.rhs_s[gsub][p] = Real(0);
  const int row0 = (live && p < T) ? Arp[fcol] : 0;
  int rlen = (live && p < T) ? Arp[fcol + 1] - row0 : 0;
  sm.rs[gsub][p] = row0;
#pragma unroll
  for (int o = 1; o < G; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, rlen, o, G);
    if (p >= o) rlen += t;
  }
  sm.pre[gsub][p + 1] = rlen;  // inclusive prefix
  if (p == 0) sm.pre[gsub][0] = 0;
  __syncwarp();
  const int total = sm.pre[gsub][G];
  // entry indices come from shared memory, so the loads of different entries are
  // independent (no global row-pointer load in front of each); entries go in batches of
  // GB per lane, all loads and column searches of a batch before its stores
  constexpr int GB = 4;
  for (int t0 = p; t0 < total; t0 += GB * G) {
    int row_of[GB], col_of[GB];
    Real val_of[GB];
#pragma unroll
    for (int u = 0; u < GB; ++u) {
      const int t = t0 + u * G;
      row_of[u] = -1;
      if (t < total) {
        int lo = 0, hi = G;  // row r with pre[r] <= t < pre[r + 1]
        while (hi - lo > 1) {
          const int mid = (lo + hi) >> 1;
          if (sm.pre[gsub][mid] <= t) lo = mid; else hi = mid;
        }
        const int e = sm.rs[gsub][lo] + (t - sm.pre[gsub][lo]);
        row_of[u] = lo;
        col_of[u] = Acol[e];
        val_of[u] = Real(Aval[e]);
      }
    }
    int q_of[GB];
#pragma unroll
    for (int u = 0; u < GB; ++u)
      q_of[u] = row_of[u] < 0 ? -1 : (col_of[u] == i ? T : find_sorted(sm.zl[gsub], T, col_of[u]));
#pragma unroll
    for (int u = 0; u < GB; ++u) {
      if (q_of[u] == T) sm.rhs_s[gsub][row_of[u]] = -val_of[u];
      else if (q_of[u] >= 0) sm.tile[gsub][row_of[u]][q_of[u]] = val_of[u];
    }
  }
  __syncwarp();
  Real a[G];
#pragma unroll
  for (int q = 0; q < G; ++q) a[q] = sm.tile[gsub][p][q];
  Real b = sm.rhs_s[gsub][p];

  // elimination with implicit partial pivoting; steps and columns beyond the largest
  // system of the warp are no-ops for every group, so the loops stop there (warp-uniform)
  const int Tw = __reduce_max_sync(0xffffffffu, live ? T : 0);
  bool done = !(live && p < T);
  int mystep = -1;
  bool singular = false;
#pragma unroll
  for (int k = 0; k < G; ++k) {
    if (k >= Tw) break;
    Real v = done ? Real(-1) : (a[k] < 0 ? -a[k] : a[k]);
    int who = p;
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
      Real v2 = __shfl_xor_sync(0xffffffffu, v, o, G);
      int w2 = __shfl_xor_sync(0xffffffffu, who, o, G);
      if (v2 > v || (v2 == v && w2 < who)) {
        v = v2;
        who = w2;
      }
    }
    if (p == 0) sm.pivlane[gsub][k] = who;
    const bool step = k < T;
    if (step && !(v > Real(0))) singular = true;
    const Real pk = __shfl_sync(0xffffffffu, a[k], who, G);
    const Real pb = __shfl_sync(0xffffffffu, b, who, G);
    const bool upd = step && !done && p != who && pk != Real(0);
    const Real l = upd ? a[k] / pk : Real(0);
    if (step && p == who) {
      done = true;
      mystep = k;
    }
#pragma unroll
    for (int j = k + 1; j < G; ++j) {
      if (j >= Tw) break;
      const Real pj = __shfl_sync(0xffffffffu, a[j], who, G);
      a[j] -= l * pj;
    }
    b -= l * pb;
  }
  __syncwarp();  // the pivot lanes lane 0 stored are read by every lane below
  // back substitution (right-looking): x_k from the lane that pivoted step k
  Real myx = 0;
#pragma unroll
  for (int k = G - 1; k >= 0; --k) {
    if (k >= Tw) continue;
    const int own = sm.pivlane[gsub][k];
    Real xk = (p == own && a[k] != Real(0)) ? b / a[k] : Real(0);
    xk = __shfl_sync(0xffffffffu, xk, own, G);
    if (k < T) {
      if (p == k) myx = xk;
      if (mystep >= 0 && mystep < k) b -= a[k] * xk;
    }
  }
  // any lane of the group may have flagged a zero pivot (ballot before any exit)
  const bool sing = (__ballot_sync(0xffffffffu, singular) & gmask) != 0;
  if (live) {
    if (p < T) Zval[base + p + (p >= d ? 1 : 0)] = sing ? 0.0 : (double)myx;
    if (p == 0) {
      Zval[base + d] = 1.0;
      if (sing) atomicAdd(nsingular, 1ull);
    }
  }
  __syncwarp();  // the shared arrays are reused by the warp's next systems
}

// register budget: 8 blocks per SM (6 for the FP64 16-lane variant), which shared
// memory and the rows held in registers allow without spills
template <class Real, class VT, int G>
__global__ void __launch_bounds__(32 * LS_WARPS, (sizeof(Real) == 8 && G >= 16) ? 6 : 8)
lsolve_group(const int* __restrict__ Arp, const int* __restrict__ Acol,
             const VT* __restrict__ Aval, const int* __restrict__ Zrp,
             const int* __restrict__ Zcol, const int* __restrict__ cpts,
             const int* __restrict__ work, int nwork, double* __restrict__ Zval,
             unsigned long long* __restrict__ nsingular) {
  constexpr int GPW = 32 / G;
  __shared__ GroupSmem<Real, G> sm[LS_WARPS];
  const int wib = threadIdx.x >> 5;
  const int gsub = (threadIdx.x & 31) / G;
  const long long item = ((long long)blockIdx.x * LS_WARPS + wib) * GPW + gsub;
  group_body<Real, VT, G>(Arp, Acol, Aval, Zrp, Zcol, cpts, work, item, nwork, Zval, nsingular,
                          sm[wib]);
}

// ------------------------------------------------------------------------------------
// Team path: one system per team of TMAX threads (a warp, a pair of warps with a named
// barrier, or a whole block), T <= TMAX; the matrix lives in shared memory, thread r owns
// row r.  Rows are padded to a multiple of 16 bytes so that a row update moves 16-byte
// vectors; it starts at the vector holding column k+1, which also rewrites columns <= k
// of the row: those are never read again (a row's entries left of its own pivot step
// take no part in back substitution).
// ------------------------------------------------------------------------------------
template <class Real>
struct Vec16;
template <>
struct Vec16<float> {
  using type = float4;
};
template <>
struct Vec16<double> {
  using type = double2;
};
__device__ __forceinline__ void sub_scaled(float4& r, float l, const float4& p) {
  r.x = r.x - l * p.x;
  r.y = r.y - l * p.y;
  r.z = r.z - l * p.z;
  r.w = r.w - l * p.w;
}
__device__ __forceinline__ void sub_scaled(double2& r, double l, const double2& p) {
  r.x = r.x - l * p.x;
  r.y = r.y - l * p.y;
}

template <class Real, int TMAX>
__host__ __device__ constexpr int cta_pitch() {
  return TMAX + 16 / (int)sizeof(Real);  // 16-byte rows, row starts 4 banks apart
}

// Shared memory of one team (the tile first: 16-byte aligned rows).
template <class Real, int TMAX>
struct alignas(16) TeamSmem {
  static constexpr int NW = TMAX / 32;
  Real tile[TMAX * cta_pitch<Real, TMAX>()];
  Real rhs[TMAX];
  Real xs[TMAX];
  Real red_v[2][NW];      // FP64: largest |value| of each warp (by step parity)
  int zl[TMAX];
  int steprow[TMAX];
  int pre[TMAX + 1];
  int rs[TMAX];           // start of each pattern row in Ahat
  int wsum[NW];
  unsigned red_k[2][NW];  // FP32: largest pivot key of each warp (by step parity)
  int red_w[2][NW];       // and its row
  int s_d, s_sing;
};

// Barrier of a team: the warp itself, a named barrier of TMAX threads, or the block.
enum { TEAM_WARP = 0, TEAM_NAMED = 1, TEAM_BLOCK = 2 };
template <int KIND, int TMAX>
__device__ __forceinline__ void team_sync(int bar_id) {
  if constexpr (KIND == TEAM_WARP) {
    __syncwarp();
  } else if constexpr (KIND == TEAM_NAMED) {
    asm volatile("bar.sync %0, %1;" ::"r"(bar_id), "r"(TMAX) : "memory");
  } else {
    __syncthreads();
  }
}

// Team thread t (0 <= t < TMAX) of the team that solves system r (a row of the pattern).
template <class Real, class VT, int TMAX, int KIND>
__device__ __forceinline__ void team_body(const int* __restrict__ Arp, const int* __restrict__ Acol,
                                          const VT* __restrict__ Aval, const int* __restrict__ Zrp,
                                          const int* __restrict__ Zcol, const int* __restrict__ cpts,
                                          int r, double* __restrict__ Zval,
                                          unsigned long long* __restrict__ nsingular,
                                          TeamSmem<Real, TMAX>& sm, int t, int bar_id) {
  using V = typename Vec16<Real>::type;
  constexpr int VN = 16 / (int)sizeof(Real);
  constexpr int PITCH = cta_pitch<Real, TMAX>();
  constexpr int NW = TMAX / 32;
  Real* tile = sm.tile;
  Real* rhs = sm.rhs;
  const int lane = t & 31, wid = t >> 5;
  const int i = cpts[r];
  const int base = Zrp[r];
  const int len = Zrp[r + 1] - base;
  const int T = len - 1;
  if (t == 0) {
    sm.s_d = T;  // position TMAX (unseen by the threads) only when T == TMAX
    sm.s_sing = 0;
  }
  team_sync<KIND, TMAX>(bar_id);
  if (t < len && Zcol[base + t] == i) sm.s_d = t;
  team_sync<KIND, TMAX>(bar_id);
  const int d = sm.s_d;
  if (t < T) sm.zl[t] = Zcol[base + t + (t >= d ? 1 : 0)];
  Real* row = tile + t * PITCH;
  for (int q = 0; q < TMAX; q += VN) *reinterpret_cast<V*>(row + q) = V{};
  rhs[t] = Real(0);
  team_sync<KIND, TMAX>(bar_id);
  // flattened gather: team scan of the row lengths, then all threads over the entries
  const int rstart = t < T ? Arp[sm.zl[t]] : 0;
  sm.rs[t] = rstart;
  int rlen = t < T ? Arp[sm.zl[t] + 1] - rstart : 0;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, rlen, o);
    if (lane >= o) rlen += v;
  }
  if (lane == 31) sm.wsum[wid] = rlen;
  team_sync<KIND, TMAX>(bar_id);
  for (int w = 0; w < wid; ++w) rlen += sm.wsum[w];
  sm.pre[t + 1] = rlen;
  if (t == 0) sm.pre[0] = 0;
  team_sync<KIND, TMAX>(bar_id);
  const int total = sm.pre[TMAX];
  // entries in batches of GB per thread: all loads of a batch, then its column searches,
  // then its stores (zl shares the shared block with the tile, so a store would order
  // every later load after it)
  constexpr int GB = 4;
  for (int f0 = t; f0 < total; f0 += GB * TMAX) {
    int row_of[GB], col_of[GB];
    Real val_of[GB];
#pragma unroll
    for (int u = 0; u < GB; ++u) {
      const int f = f0 + u * TMAX;
      row_of[u] = -1;
      if (f < total) {
        int lo = 0, hi = TMAX;  // row r with pre[r] <= f < pre[r + 1]
        while (hi - lo > 1) {
          const int mid = (lo + hi) >> 1;
          if (sm.pre[mid] <= f) lo = mid; else hi = mid;
        }
        const int e = sm.rs[lo] + (f - sm.pre[lo]);
        row_of[u] = lo;
        col_of[u] = Acol[e];
        val_of[u] = Real(Aval[e]);
      }
    }
    int q_of[GB];
#pragma unroll
    for (int u = 0; u < GB; ++u)
      q_of[u] = row_of[u] < 0 ? -1 : (col_of[u] == i ? T : find_sorted(sm.zl, T, col_of[u]));
#pragma unroll
    for (int u = 0; u < GB; ++u) {
      if (q_of[u] == T) rhs[row_of[u]] = -val_of[u];
      else if (q_of[u] >= 0) tile[row_of[u] * PITCH + q_of[u]] = val_of[u];
    }
  }
  bool done = t >= T;
  int mystep = -1;
  team_sync<KIND, TMAX>(bar_id);
  // One barrier per step: each thread updates only its own row and right-hand side, and
  // the barrier after the next step's candidate posts orders the pivot owner's last update
  // before anyone reads the pivot row; the candidate arrays alternate by step parity, so
  // a fast thread's next post cannot overwrite what a slow one is still reading.
  for (int k = 0; k < T; ++k) {
    const int par = k & 1;
    // pivot: largest |a| of column k among the rows not yet eliminated, lowest row on
    // ties; each warp posts its candidate, every thread then reads the team's
    const Real rk = row[k];
    if constexpr (sizeof(Real) == 4) {
      // non-negative floats order as their bit patterns; key 0 marks eliminated rows
      const unsigned key = done ? 0u : __float_as_uint(fabsf(rk)) + 1u;
      const unsigned wmax = __reduce_max_sync(0xffffffffu, key);
      const unsigned bal = __ballot_sync(0xffffffffu, key == wmax);
      if (lane == 0) {
        sm.red_k[par][wid] = wmax;
        sm.red_w[par][wid] = wid * 32 + __ffs(bal) - 1;
      }
    } else {
      Real v = done ? Real(-1) : (rk < 0 ? -rk : rk);
      int who = t;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const Real v2 = __shfl_xor_sync(0xffffffffu, v, o);
        const int w2 = __shfl_xor_sync(0xffffffffu, who, o);
        if (v2 > v || (v2 == v && w2 < who)) {
          v = v2;
          who = w2;
        }
      }
      if (lane == 0) {
        sm.red_v[par][wid] = v;
        sm.red_w[par][wid] = who;
      }
    }
    team_sync<KIND, TMAX>(bar_id);
    int piv = sm.red_w[par][0];
    if constexpr (sizeof(Real) == 4) {
      unsigned bk = sm.red_k[par][0];
#pragma unroll
      for (int w = 1; w < NW; ++w)
        if (sm.red_k[par][w] > bk) {  // warps hold increasing rows: strict keeps the lowest
          bk = sm.red_k[par][w];
          piv = sm.red_w[par][w];
        }
    } else {
      Real bv = sm.red_v[par][0];
#pragma unroll
      for (int w = 1; w < NW; ++w)
        if (sm.red_v[par][w] > bv) {
          bv = sm.red_v[par][w];
          piv = sm.red_w[par][w];
        }
    }
    const Real* prow = tile + piv * PITCH;
    const Real pk = prow[k];
    if (t == 0) {
      sm.steprow[k] = piv;
      if (!((pk < 0 ? -pk : pk) > Real(0))) sm.s_sing = 1;
    }
    if (t == piv) {
      done = true;
      mystep = k;
    } else if (!done && pk != Real(0)) {
      const Real l = rk / pk;
      for (int j0 = (k + 1) & ~(VN - 1); j0 < T; j0 += 2 * VN) {
        const bool two = j0 + VN < T;
        const V p0 = *reinterpret_cast<const V*>(prow + j0);
        V r0 = *reinterpret_cast<const V*>(row + j0);
        V p1 = p0, r1 = r0;
        if (two) {
          p1 = *reinterpret_cast<const V*>(prow + j0 + VN);
          r1 = *reinterpret_cast<const V*>(row + j0 + VN);
        }
        sub_scaled(r0, l, p0);
        *reinterpret_cast<V*>(row + j0) = r0;
        if (two) {
          sub_scaled(r1, l, p1);
          *reinterpret_cast<V*>(row + j0 + VN) = r1;
        }
      }
      rhs[t] -= l * rhs[piv];
    }
  }
  team_sync<KIND, TMAX>(bar_id);  // the last updates and steprow before back substitution
  // back substitution: one barrier per step suffices, each thread updates only its own
  // right-hand side and every x_k has its own slot
  for (int k = T - 1; k >= 0; --k) {
    const int own = sm.steprow[k];
    if (t == own) sm.xs[k] = row[k] != Real(0) ? rhs[t] / row[k] : Real(0);
    team_sync<KIND, TMAX>(bar_id);
    const Real xk = sm.xs[k];
    if (mystep >= 0 && mystep < k) rhs[t] -= row[k] * xk;
  }
  team_sync<KIND, TMAX>(bar_id);
  const bool sing = sm.s_sing != 0;
  if (t < T) Zval[base + t + (t >= d ? 1 : 0)] = sing ? 0.0 : (double)sm.xs[t];
  if (t == 0) {
    Zval[base + d] = 1.0;
    if (sing) atomicAdd(nsingular, 1ull);
  }
  team_sync<KIND, TMAX>(bar_id);  // the team's shared block is reused by its next system
}

// One warp solves a system of up to 32 * RPT unknowns: lane l owns rows l, l + 32, ...
// The same arithmetic as team_body (same pivots, same operations per row, hence the same
// bits), but the pivot search is two warp reductions and no step needs a block barrier.
template <class Real, class VT, int RPT>
__device__ __forceinline__ void warp_body(const int* __restrict__ Arp, const int* __restrict__ Acol,
                                          const VT* __restrict__ Aval, const int* __restrict__ Zrp,
                                          const int* __restrict__ Zcol, const int* __restrict__ cpts,
                                          int r, double* __restrict__ Zval,
                                          unsigned long long* __restrict__ nsingular,
                                          TeamSmem<Real, 32 * RPT>& sm, int lane) {
  using V = typename Vec16<Real>::type;
  constexpr int VN = 16 / (int)sizeof(Real);
  constexpr int TMAX = 32 * RPT;
  constexpr int PITCH = cta_pitch<Real, TMAX>();
  constexpr unsigned FULL = 0xffffffffu;
  Real* tile = sm.tile;
  Real* rhs = sm.rhs;
  const int i = cpts[r];
  const int base = Zrp[r];
  const int len = Zrp[r + 1] - base;
  const int T = len - 1;
  // position of the identity column (TMAX, unseen, only when T == TMAX)
  int d = T;
#pragma unroll
  for (int q = RPT - 1; q >= 0; --q) {
    const int tq = lane + 32 * q;
    const unsigned m = __ballot_sync(FULL, tq < len && Zcol[base + tq] == i);
    if (m) d = 32 * q + __ffs(m) - 1;
  }
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    const int tq = lane + 32 * q;
    if (tq < T) sm.zl[tq] = Zcol[base + tq + (tq >= d ? 1 : 0)];
    Real* row = tile + tq * PITCH;
    for (int c = 0; c < TMAX; c += VN) *reinterpret_cast<V*>(row + c) = V{};
    rhs[tq] = Real(0);
  }
  __syncwarp();
  // row starts and the prefix of the row lengths in row order
  int off = 0;
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    const int tq = lane + 32 * q;
    const int rstart = tq < T ? Arp[sm.zl[tq]] : 0;
    int rlen = tq < T ? Arp[sm.zl[tq] + 1] - rstart : 0;
    sm.rs[tq] = rstart;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(FULL, rlen, o);
      if (lane >= o) rlen += v;
    }
    sm.pre[tq + 1] = off + rlen;
    off += __shfl_sync(FULL, rlen, 31);
  }
  if (lane == 0) sm.pre[0] = 0;
  __syncwarp();
  const int total = sm.pre[TMAX];
  constexpr int GB = 4;
  for (int f0 = lane; f0 < total; f0 += GB * 32) {
    int row_of[GB], col_of[GB];
    Real val_of[GB];
#pragma unroll
    for (int u = 0; u < GB; ++u) {
      const int f = f0 + u * 32;
      row_of[u] = -1;
      if (f < total) {
        int lo = 0, hi = TMAX;  // row with pre[row] <= f < pre[row + 1]
        while (hi - lo > 1) {
          const int mid = (lo + hi) >> 1;
          if (sm.pre[mid] <= f) lo = mid; else hi = mid;
        }
        const int e = sm.rs[lo] + (f - sm.pre[lo]);
        row_of[u] = lo;
        col_of[u] = Acol[e];
        val_of[u] = Real(Aval[e]);
      }
    }
    int q_of[GB];
#pragma unroll
    for (int u = 0; u < GB; ++u)
      q_of[u] = row_of[u] < 0 ? -1 : (col_of[u] == i ? T : find_sorted(sm.zl, T, col_of[u]));
#pragma unroll
    for (int u = 0; u < GB; ++u) {
      if (q_of[u] == T) rhs[row_of[u]] = -val_of[u];
      else if (q_of[u] >= 0) tile[row_of[u] * PITCH + q_of[u]] = val_of[u];
    }
  }
  __syncwarp();
  bool done[RPT];
  int mystep[RPT];
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    done[q] = lane + 32 * q >= T;
    mystep[q] = -1;
  }
  bool sing = false;
  for (int k = 0; k < T; ++k) {
    // pivot: largest |a| of column k among the rows not yet eliminated, lowest row on ties
    int piv;
    if constexpr (sizeof(Real) == 4) {
      unsigned key = 0u;
      int row = 0x7fffffff;
#pragma unroll
      for (int q = 0; q < RPT; ++q)
        if (!done[q]) {
          const unsigned kq = __float_as_uint(fabsf(tile[(lane + 32 * q) * PITCH + k])) + 1u;
          if (kq > key) {
            key = kq;
            row = lane + 32 * q;
          }
        }
      const unsigned wmax = __reduce_max_sync(FULL, key);
      piv = __reduce_min_sync(FULL, key == wmax ? row : 0x7fffffff);
    } else {
      Real v = Real(-1);
      int who = 0x7fffffff;
#pragma unroll
      for (int q = 0; q < RPT; ++q)
        if (!done[q]) {
          const Real a = tile[(lane + 32 * q) * PITCH + k];
          const Real m = a < 0 ? -a : a;
          if (m > v) {
            v = m;
            who = lane + 32 * q;
          }
        }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const Real v2 = __shfl_xor_sync(FULL, v, o);
        const int w2 = __shfl_xor_sync(FULL, who, o);
        if (v2 > v || (v2 == v && w2 < who)) {
          v = v2;
          who = w2;
        }
      }
      piv = who;
    }
    const Real* prow = tile + piv * PITCH;
    const Real pk = prow[k];
    if (!((pk < 0 ? -pk : pk) > Real(0))) sing = true;
    if (lane == 0) sm.steprow[k] = piv;
    const Real rpiv = rhs[piv];
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      const int tq = lane + 32 * q;
      if (tq == piv) {
        done[q] = true;
        mystep[q] = k;
      } else if (!done[q] && pk != Real(0)) {
        Real* row = tile + tq * PITCH;
        const Real l = row[k] / pk;
        for (int j0 = (k + 1) & ~(VN - 1); j0 < T; j0 += 2 * VN) {
          const bool two = j0 + VN < T;
          const V p0 = *reinterpret_cast<const V*>(prow + j0);
          V r0 = *reinterpret_cast<const V*>(row + j0);
          V p1 = p0, r1 = r0;
          if (two) {
            p1 = *reinterpret_cast<const V*>(prow + j0 + VN);
            r1 = *reinterpret_cast<const V*>(row + j0 + VN);
          }
          sub_scaled(r0, l, p0);
          *reinterpret_cast<V*>(row + j0) = r0;
          if (two) {
            sub_scaled(r1, l, p1);
            *reinterpret_cast<V*>(row + j0 + VN) = r1;
          }
        }
        rhs[tq] -= l * rpiv;
      }
    }
    __syncwarp();
  }
  // back substitution
  for (int k = T - 1; k >= 0; --k) {
    const int own = sm.steprow[k];
    if (lane == (own & 31)) {
      const Real dk = tile[own * PITCH + k];
      sm.xs[k] = dk != Real(0) ? rhs[own] / dk : Real(0);
    }
    __syncwarp();
    const Real xk = sm.xs[k];
#pragma unroll
    for (int q = 0; q < RPT; ++q)
      if (mystep[q] >= 0 && mystep[q] < k) {
        const int tq = lane + 32 * q;
        rhs[tq] -= tile[tq * PITCH + k] * xk;
      }
  }
  __syncwarp();
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    const int tq = lane + 32 * q;
    if (tq < T) Zval[base + tq + (tq >= d ? 1 : 0)] = sing ? 0.0 : (double)sm.xs[tq];
  }
  if (lane == 0) {
    Zval[base + d] = 1.0;
    if (sing) atomicAdd(nsingular, 1ull);
  }
  __syncwarp();  // the warp's shared block is reused by its next system
}

// shared memory holds these to about 1024 resident threads per SM, so the register
// budget is set for that many (64 each) rather than for full occupancy
template <class Real, class VT, int TMAX>
__global__ void __launch_bounds__(TMAX, 1024 / TMAX)
lsolve_cta(const int* __restrict__ Arp, const int* __restrict__ Acol,
           const VT* __restrict__ Aval, const int* __restrict__ Zrp,
           const int* __restrict__ Zcol, const int* __restrict__ cpts,
           const int* __restrict__ work, double* __restrict__ Zval,
           unsigned long long* __restrict__ nsingular) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  auto& sm = *reinterpret_cast<TeamSmem<Real, TMAX>*>(smem_raw);
  team_body<Real, VT, TMAX, TEAM_BLOCK>(Arp, Acol, Aval, Zrp, Zcol, cpts, work[blockIdx.x], Zval,
                                        nsingular, sm, threadIdx.x, 0);
}

template <class Real, int TMAX>
static size_t cta_smem() {
  return sizeof(TeamSmem<Real, TMAX>);
}

// ------------------------------------------------------------------------------------
// Persistent launch: the systems of up to 64 unknowns of both sides of a level (R on
// A^T, P on A) in one launch of a fixed grid.  Blocks of four warps take tasks from a
// device ticket; the task list is derived on the device from the bucket counts, largest
// systems first.  A task is 16 systems of T <= 8 (4 groups of 8 lanes per warp), 8 of
// T <= 16 (2 groups of 16), 4 of T <= 32 (a warp each) or 2 of T <= 64 (a pair of warps
// each, synchronised by a named barrier).  Systems with 8 < T <= 16 go to the 16-lane
// groups or to single warps, as the autotuner chose.
// ------------------------------------------------------------------------------------
constexpr int LP_THREADS = 128;
enum { LK_G8 = 0, LK_G16 = 1, LK_W32 = 2, LK_P64 = 3, LK_W64 = 4 };
__host__ __device__ constexpr int lk_systems(int kind) {
  return kind == LK_G8 ? 16 : kind == LK_G16 ? 8 : kind == LK_W32 ? 4 : kind == LK_P64 ? 2 : 4;
}

template <class VT>
struct SideArgs {
  const int *Arp, *Acol;
  const VT* Aval;
  const int *Zrp, *Zcol, *cpts, *lists;  // lists: bucket b at lists + b * nc
  const int* counts;                      // device bucket counts
  double* Zval;
  int nc;
};

template <class Real>
union PersistSmem {
  GroupSmem<Real, 8> g8[4];
  GroupSmem<Real, 16> g16[4];
  TeamSmem<Real, 32> w32[4];
  TeamSmem<Real, 64> p64[2];
  TeamSmem<Real, 64> w64[4];
};

template <class Real>
static size_t persist_smem(const bool* has) {
  size_t b = 16;
  if (has[LK_G8]) b = std::max(b, 4 * sizeof(GroupSmem<Real, 8>));
  if (has[LK_G16]) b = std::max(b, 4 * sizeof(GroupSmem<Real, 16>));
  if (has[LK_W32]) b = std::max(b, 4 * sizeof(TeamSmem<Real, 32>));
  if (has[LK_P64]) b = std::max(b, 2 * sizeof(TeamSmem<Real, 64>));
  if (has[LK_W64]) b = std::max(b, 4 * sizeof(TeamSmem<Real, 64>));
  return b;
}

constexpr int LP_WAVES = 4;  // blocks launched per resident block of the persistent launch

template <class Real, class VT>
__global__ void __launch_bounds__(LP_THREADS)
lsolve_persist(SideArgs<VT> S0, SideArgs<VT> S1, int nsides, int kind_b1, int kind_b3,
               int* __restrict__ ticket, unsigned long long* __restrict__ nsingular, int budget) {
  extern __shared__ __align__(16) unsigned char lp_smem[];
  auto& sm = *reinterpret_cast<PersistSmem<Real>*>(lp_smem);
  __shared__ int seg_end[8], seg_kind[8];
  __shared__ int s_task;
  // segment q: bucket 3 - q / 2 (largest first), side q % 2
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int q = 0; q < 8; ++q) {
      const int b = 3 - (q >> 1), side = q & 1;
      const int cnt = side < nsides ? (side ? S1.counts[b] : S0.counts[b]) : 0;
      const int kind = b == 3 ? kind_b3 : b == 2 ? LK_W32 : b == 1 ? kind_b1 : LK_G8;
      acc += (cnt + lk_systems(kind) - 1) / lk_systems(kind);
      seg_end[q] = acc;
      seg_kind[q] = kind;
    }
  }
  __syncthreads();
  const int total = seg_end[7];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int taken = 0; taken < budget; ++taken) {
    if (threadIdx.x == 0) s_task = atomicAdd(ticket, 1);
    __syncthreads();
    const int task = s_task;
    __syncthreads();  // every thread has read s_task before thread 0 rewrites it
    if (task >= total) break;
    int q = 0;
    while (task >= seg_end[q]) ++q;
    const int b = 3 - (q >> 1);
    const SideArgs<VT>& S = (q & 1) ? S1 : S0;
    const int kind = seg_kind[q];
    const long long first = (long long)(task - (q ? seg_end[q - 1] : 0)) * lk_systems(kind);
    const long long cnt = S.counts[b];
    const int* list = S.lists + (long long)b * S.nc;
    if (kind == LK_G8) {
      group_body<Real, VT, 8>(S.Arp, S.Acol, S.Aval, S.Zrp, S.Zcol, S.cpts, list,
                              first + wib * 4 + lane / 8, cnt, S.Zval, nsingular, sm.g8[wib]);
    } else if (kind == LK_G16) {
      group_body<Real, VT, 16>(S.Arp, S.Acol, S.Aval, S.Zrp, S.Zcol, S.cpts, list,
                               first + wib * 2 + lane / 16, cnt, S.Zval, nsingular, sm.g16[wib]);
    } else if (kind == LK_W32) {
      const long long item = first + wib;
      if (item < cnt)
        team_body<Real, VT, 32, TEAM_WARP>(S.Arp, S.Acol, S.Aval, S.Zrp, S.Zcol, S.cpts, list[item],
                                           S.Zval, nsingular, sm.w32[wib], lane, 0);
    } else if (kind == LK_P64) {
      const int team = wib >> 1;
      const long long item = first + team;
      if (item < cnt)
        team_body<Real, VT, 64, TEAM_NAMED>(S.Arp, S.Acol, S.Aval, S.Zrp, S.Zcol, S.cpts,
                                            list[item], S.Zval, nsingular, sm.p64[team],
                                            threadIdx.x & 63, 1 + team);
    } else {
      const long long item = first + wib;
      if (item < cnt)
        warp_body<Real, VT, 2>(S.Arp, S.Acol, S.Aval, S.Zrp, S.Zcol, S.cpts, list[item], S.Zval,
                               nsingular, sm.w64[wib], lane);
    }
  }
}

// ------------------------------------------------------------------------------------
// Large systems (128 < T <= LS_TBIG, rare: long rows on coarse levels): one block of 256
// threads per system, the matrix in a global scratch tile stored column-major (leading
// dimension `pitch`) so that the threads, which own rows t, t+256, ..., touch consecutive
// addresses in every column; same implicit partial pivoting as above.  The per-system
// index and vector arrays live in dynamic shared memory sized for `pitch` unknowns.
// ------------------------------------------------------------------------------------
constexpr int LB_THREADS = 256;

template <class Real>
__host__ __device__ constexpr size_t big_smem(int pitch) {
  return (size_t)pitch * (3 * sizeof(int) + 3 * sizeof(Real)) + 2 * sizeof(Real);
}

template <class Real, class VT>
__global__ void __launch_bounds__(LB_THREADS)
lsolve_big(const int* __restrict__ Arp, const int* __restrict__ Acol,
           const VT* __restrict__ Aval, const int* __restrict__ Zrp,
           const int* __restrict__ Zcol, const int* __restrict__ cpts,
           const int* __restrict__ work, double* __restrict__ Zval,
           unsigned long long* __restrict__ nsingular, Real* __restrict__ scratch, int pitch) {
  extern __shared__ __align__(16) unsigned char lb_smem[];
  Real* rhs = reinterpret_cast<Real*>(lb_smem);
  Real* xs = rhs + pitch;
  Real* prow = xs + pitch;  // the step's pivot row, columns k+1 .. T-1
  int* zl = reinterpret_cast<int*>(prow + pitch);
  int* stepof = zl + pitch;
  int* steprow = stepof + pitch;
  __shared__ Real red_v[LB_THREADS / 32];
  __shared__ int red_w[LB_THREADS / 32];
  __shared__ int s_piv, s_d, s_sing;
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  const int r = work[blockIdx.x];
  const int i = cpts[r];
  const int base = Zrp[r];
  const int len = Zrp[r + 1] - base;
  const int T = len - 1;  // T <= pitch (pitch = the largest T of the launch)
  Real* M = scratch + (size_t)blockIdx.x * pitch * pitch;  // M(p, q) at M[q * pitch + p]
  if (t == 0) {
    s_d = T;
    s_sing = 0;
  }
  __syncthreads();
  for (int q = t; q < len; q += LB_THREADS)
    if (Zcol[base + q] == i) s_d = q;
  __syncthreads();
  const int d = s_d;
  for (int p = t; p < T; p += LB_THREADS) {
    zl[p] = Zcol[base + p + (p >= d ? 1 : 0)];
    rhs[p] = Real(0);
    stepof[p] = -1;
  }
  for (int q = 0; q < T; ++q)
    for (int p = t; p < T; p += LB_THREADS) M[(size_t)q * pitch + p] = Real(0);
  __syncthreads();
  // row p's entries in batches of 4: loads and column searches before the stores
  for (int p = t; p < T; p += LB_THREADS) {
    const int l = zl[p];
    const int e_end = Arp[l + 1];
    for (int e0 = Arp[l]; e0 < e_end; e0 += 4) {
      int col_of[4], q_of[4];
      Real val_of[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const bool in = e0 + u < e_end;
        col_of[u] = in ? Acol[e0 + u] : -1;
        val_of[u] = in ? Real(Aval[e0 + u]) : Real(0);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        q_of[u] = col_of[u] < 0 ? -1 : (col_of[u] == i ? T : find_sorted(zl, T, col_of[u]));
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (q_of[u] == T) rhs[p] = -val_of[u];
        else if (q_of[u] >= 0) M[(size_t)q_of[u] * pitch + p] = val_of[u];
      }
    }
  }
  __syncthreads();
  for (int k = 0; k < T; ++k) {
    const Real* colk = M + (size_t)k * pitch;
    Real v = Real(-1);
    int who = T;
    for (int p = t; p < T; p += LB_THREADS)
      if (stepof[p] < 0) {
        const Real a = colk[p];
        const Real m = a < 0 ? -a : a;
        if (m > v) {  // rows visited in increasing order: ties keep the lowest row
          v = m;
          who = p;
        }
      }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const Real v2 = __shfl_xor_sync(0xffffffffu, v, o);
      const int w2 = __shfl_xor_sync(0xffffffffu, who, o);
      if (v2 > v || (v2 == v && w2 < who)) {
        v = v2;
        who = w2;
      }
    }
    if (lane == 0) {
      red_v[wid] = v;
      red_w[wid] = who;
    }
    __syncthreads();
    if (t == 0) {
      Real bv = red_v[0];
      int bw = red_w[0];
      for (int w = 1; w < LB_THREADS / 32; ++w)
        if (red_v[w] > bv || (red_v[w] == bv && red_w[w] < bw)) {
          bv = red_v[w];
          bw = red_w[w];
        }
      s_piv = bw;
      steprow[k] = bw;
      stepof[bw] = k;
      if (!(bv > Real(0))) s_sing = 1;
    }
    __syncthreads();
    const int piv = s_piv;
    const Real pk = colk[piv];
    for (int j = k + 1 + t; j < T; j += LB_THREADS) prow[j] = M[(size_t)j * pitch + piv];
    __syncthreads();
    for (int p = t; p < T; p += LB_THREADS)
      if (stepof[p] < 0 && pk != Real(0)) {
        const Real l = colk[p] / pk;
        for (int j0 = k + 1; j0 < T; j0 += LS_CHUNK) {
          Real pv[LS_CHUNK], rv[LS_CHUNK];
#pragma unroll
          for (int u = 0; u < LS_CHUNK; ++u)
            if (j0 + u < T) {
              pv[u] = prow[j0 + u];
              rv[u] = M[(size_t)(j0 + u) * pitch + p];
            }
#pragma unroll
          for (int u = 0; u < LS_CHUNK; ++u)
            if (j0 + u < T) M[(size_t)(j0 + u) * pitch + p] = rv[u] - l * pv[u];
        }
        rhs[p] -= l * rhs[piv];
      }
    __syncthreads();
  }
  for (int k = T - 1; k >= 0; --k) {
    const int own = steprow[k];
    const Real* colk = M + (size_t)k * pitch;
    if (t == 0) {
      const Real dk = colk[own];
      xs[k] = dk != Real(0) ? rhs[own] / dk : Real(0);
    }
    __syncthreads();
    const Real xk = xs[k];
    for (int p = t; p < T; p += LB_THREADS)
      if (stepof[p] < k) rhs[p] -= colk[p] * xk;
    __syncthreads();
  }
  const bool sing = s_sing != 0;
  for (int p = t; p < T; p += LB_THREADS) Zval[base + p + (p >= d ? 1 : 0)] = sing ? 0.0 : (double)xs[p];
  if (t == 0) {
    Zval[base + d] = 1.0;
    if (sing) atomicAdd(nsingular, 1ull);
  }
}

// ------------------------------------------------------------------------------------
// Large systems, blocked (128 < T up to a few thousand): one block of NT threads per
// system at a time (128 for tiles of pitch <= 256, so that several systems share an SM;
// else 256), the matrix in a global scratch tile stored row-major (row p at
// M + p * pitch), eliminated in panels of NB columns.  Each panel's columns are loaded
// into shared memory and factored there step by step (the same implicit partial pivoting,
// one barrier per step); the pivot rows' entries right of the panel (the rows of U) and
// then the remaining rows are updated once per panel, by a thread per column holding the
// panel's NB entries of U in registers.  Every entry receives the same updates, in the
// same order and with the same operands, as in the unblocked elimination; the trailing
// matrix is read and written once per panel instead of once per step.  Back substitution
// runs in blocks of 32 steps: the dot products with the solved tail by warps (coalesced
// row reads), then the 32 x 32 triangle by one warp from shared memory.
// Blocks take systems from a device ticket, the largest size class first.
// ------------------------------------------------------------------------------------
constexpr int LK_SMALL_PITCH = 256;

template <class Real>
__host__ __device__ constexpr int blk_ps(int nb) {
  return nb + 16 / (int)sizeof(Real);  // panel row stride: 16-byte aligned rows
}

template <class Real>
static size_t blk_smem(int pitch, int nb) {
  return (size_t)pitch * blk_ps<Real>(nb) * sizeof(Real) + 2 * (size_t)pitch * sizeof(Real) +
         32 * 33 * sizeof(Real) + 3 * (size_t)pitch * sizeof(int);
}

template <class Real, class VT, int NB, int NT>
__global__ void __launch_bounds__(NT, (sizeof(Real) == 4 ? 512 : 256) / NT)
lsolve_blk(const int* __restrict__ Arp, const int* __restrict__ Acol,
           const VT* __restrict__ Aval, const int* __restrict__ Zrp,
           const int* __restrict__ Zcol, const int* __restrict__ cpts,
           const int* __restrict__ cls, const int* __restrict__ ccount, int cls_stride, int ncls,
           int* __restrict__ ticket, double* __restrict__ Zval,
           unsigned long long* __restrict__ nsingular, Real* __restrict__ scratch, int pitch) {
  using V = typename Vec16<Real>::type;
  constexpr int VN = 16 / (int)sizeof(Real);
  constexpr int PS = NB + VN;
  extern __shared__ __align__(16) unsigned char kb_smem[];
  Real* Pn = reinterpret_cast<Real*>(kb_smem);  // panel: row p at Pn + p * PS
  Real* rhs = Pn + (size_t)pitch * PS;
  Real* xs = rhs + pitch;
  Real* tri = xs + pitch;  // 32 x 33: a block of back substitution
  int* zl = reinterpret_cast<int*>(tri + 32 * 33);
  int* steprow = zl + pitch;
  int* ulist = steprow + pitch;
  __shared__ Real red_v[2][NT / 32];
  __shared__ int red_w[2][NT / 32];
  __shared__ int s_task, s_d, s_sing, s_nu;
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  Real* M = scratch + (size_t)blockIdx.x * pitch * pitch;
  for (;;) {
    if (t == 0) s_task = atomicAdd(ticket, 1);
    __syncthreads();
    int task = s_task, r = -1;
    for (int c = ncls - 1; c >= 0; --c) {  // largest class first
      const int n = ccount[c];
      if (task < n) {
        r = cls[(size_t)c * cls_stride + task];
        break;
      }
      task -= n;
    }
    if (r < 0) break;  // the same for every thread of the block
    const int i = cpts[r];
    const int base = Zrp[r];
    const int len = Zrp[r + 1] - base;
    const int T = len - 1;  // T <= pitch (the host sized the tiles for the largest class)
    if (t == 0) {
      s_d = T;
      s_sing = 0;
    }
    __syncthreads();
    for (int q = t; q < len; q += NT)
      if (Zcol[base + q] == i) s_d = q;
    __syncthreads();
    const int d = s_d;
    for (int p = t; p < T; p += NT) {
      zl[p] = Zcol[base + p + (p >= d ? 1 : 0)];
      rhs[p] = Real(0);
    }
    for (int p = wid; p < T; p += NT / 32)
      for (int q = lane; q < T; q += 32) M[(size_t)p * pitch + q] = Real(0);
    __syncthreads();
    // row p's entries in batches of 4: loads and column searches before the stores
    for (int p = t; p < T; p += NT) {
      const int l = zl[p];
      const int e_end = Arp[l + 1];
      for (int e0 = Arp[l]; e0 < e_end; e0 += 4) {
        int col_of[4], q_of[4];
        Real val_of[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const bool in = e0 + u < e_end;
          col_of[u] = in ? Acol[e0 + u] : -1;
          val_of[u] = in ? Real(Aval[e0 + u]) : Real(0);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
          q_of[u] = col_of[u] < 0 ? -1 : (col_of[u] == i ? T : find_sorted(zl, T, col_of[u]));
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (q_of[u] == T) rhs[p] = -val_of[u];
          else if (q_of[u] >= 0) M[(size_t)p * pitch + q_of[u]] = val_of[u];
        }
      }
    }
    // thread t owns rows t + 256 rr; bit rr of `done`: that row is eliminated (or absent)
    const int nr = (T + NT - 1) / NT;
    unsigned done = 0;
    for (int rr = 0; rr < nr; ++rr)
      if (t + NT * rr >= T) done |= 1u << rr;
    __syncthreads();
    for (int k0 = 0; k0 < T; k0 += NB) {
      const int nb = min(NB, T - k0);
      for (int e = t; e < T * NB; e += NT) {
        const int p = e / NB, kk = e % NB;
        if (kk < nb) Pn[p * PS + kk] = M[(size_t)p * pitch + k0 + kk];
      }
      if (t == 0) s_nu = 0;
      __syncthreads();
      // the panel's steps: one barrier each (each thread updates only its own rows; the
      // candidate arrays alternate by step parity, as in the shared-memory CTA solve)
      for (int kk = 0; kk < nb; ++kk) {
        const int k = k0 + kk, par = k & 1;
        Real v = Real(-1);
        int who = 0x7fffffff;
        for (int rr = 0; rr < nr; ++rr)
          if (!((done >> rr) & 1u)) {
            const int p = t + NT * rr;
            const Real a = Pn[p * PS + kk];
            Real m = a < 0 ? -a : a;
            if (!(m >= Real(0))) m = Real(-0.5);  // NaN: still a row to take, after any number
            if (m > v) {  // rows visited in increasing order: ties keep the lowest
              v = m;
              who = p;
            }
          }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const Real v2 = __shfl_xor_sync(0xffffffffu, v, o);
          const int w2 = __shfl_xor_sync(0xffffffffu, who, o);
          if (v2 > v || (v2 == v && w2 < who)) {
            v = v2;
            who = w2;
          }
        }
        if (lane == 0) {
          red_v[par][wid] = v;
          red_w[par][wid] = who;
        }
        __syncthreads();
        Real bv = red_v[par][0];
        int piv = red_w[par][0];
#pragma unroll
        for (int w = 1; w < NT / 32; ++w)
          if (red_v[par][w] > bv || (red_v[par][w] == bv && red_w[par][w] < piv)) {
            bv = red_v[par][w];
            piv = red_w[par][w];
          }
        // piv is a row not yet eliminated: T - k of them are left at step k < T
        const Real* prow = Pn + piv * PS;
        const Real pk = prow[kk];
        if (t == 0) {
          steprow[k] = piv;
          if (!((pk < 0 ? -pk : pk) > Real(0))) s_sing = 1;
        }
        const Real rpiv = rhs[piv];
        for (int rr = 0; rr < nr; ++rr) {
          if ((done >> rr) & 1u) continue;
          const int p = t + NT * rr;
          if (p == piv) {
            done |= 1u << rr;
            continue;
          }
          if (pk == Real(0)) continue;
          Real* row = Pn + p * PS;
          const Real l = row[kk] / pk;
          row[kk] = l;  // the multiplier, read by the updates right of the panel
          for (int k2 = kk + 1; k2 < nb; ++k2) row[k2] = row[k2] - l * prow[k2];
          rhs[p] -= l * rpiv;
        }
      }
      __syncthreads();  // the panel's last updates and its pivot rows
      for (int e = t; e < T * NB; e += NT) {
        const int p = e / NB, kk = e % NB;
        if (kk < nb) M[(size_t)p * pitch + k0 + kk] = Pn[p * PS + kk];
      }
      for (int rr = 0; rr < nr; ++rr)
        if (!((done >> rr) & 1u)) ulist[atomicAdd(&s_nu, 1)] = t + NT * rr;
      __syncthreads();
      const int jt0 = k0 + NB;  // columns right of a full panel (a partial one ends at T)
      if (jt0 < T) {
        const int nu = s_nu;
        const int width = T - jt0;
        const int cw = width > 128 && NT > 128 ? 256 : width > 64 ? 128 : width > 32 ? 64 : 32;
        const int G = NT / cw, g = t / cw, cl = t % cw;
        for (int jc = jt0; jc < T; jc += cw) {
          const int j = jc + cl;
          const bool act = j < T;
          Real u[NB];
#pragma unroll
          for (int kk = 0; kk < NB; ++kk)
            u[kk] = act ? M[(size_t)steprow[k0 + kk] * pitch + j] : Real(0);
          // the pivot rows' updates by the earlier pivots of the panel, in step order
#pragma unroll
          for (int kk = 1; kk < NB; ++kk) {
            const Real* lrow = Pn + steprow[k0 + kk] * PS;
#pragma unroll
            for (int k2 = 0; k2 < kk; ++k2) u[kk] = u[kk] - lrow[k2] * u[k2];
          }
          if (act && g == 0) {
#pragma unroll
            for (int kk = 0; kk < NB; ++kk) M[(size_t)steprow[k0 + kk] * pitch + j] = u[kk];
          }
          for (int i0 = g; i0 < nu; i0 += 4 * G) {
            int pr[4];
            Real c[4];
#pragma unroll
            for (int m = 0; m < 4; ++m) {
              const int ii = i0 + m * G;
              pr[m] = ii < nu ? ulist[ii] : -1;
              c[m] = (act && pr[m] >= 0) ? M[(size_t)pr[m] * pitch + j] : Real(0);
            }
#pragma unroll
            for (int kk = 0; kk < NB; kk += VN) {
#pragma unroll
              for (int m = 0; m < 4; ++m) {
                const V l4 = *reinterpret_cast<const V*>(Pn + (pr[m] < 0 ? 0 : pr[m]) * PS + kk);
                if constexpr (VN == 4) {
                  c[m] = c[m] - l4.x * u[kk];
                  c[m] = c[m] - l4.y * u[kk + 1];
                  c[m] = c[m] - l4.z * u[kk + 2];
                  c[m] = c[m] - l4.w * u[kk + 3];
                } else {
                  c[m] = c[m] - l4.x * u[kk];
                  c[m] = c[m] - l4.y * u[kk + 1];
                }
              }
            }
#pragma unroll
            for (int m = 0; m < 4; ++m)
              if (act && pr[m] >= 0) M[(size_t)pr[m] * pitch + j] = c[m];
          }
        }
      }
      __syncthreads();  // the tile's updates before the next panel is loaded
    }
    // back substitution, 32 steps at a time from the last
    for (int ke = T; ke > 0; ke -= 32) {
      const int kb = ke > 32 ? ke - 32 : 0, nbk = ke - kb;
      for (int kq = wid; kq < nbk; kq += NT / 32) {
        const Real* urow = M + (size_t)steprow[kb + kq] * pitch;
        Real acc = Real(0);
        for (int q = ke + lane; q < T; q += 32) acc += urow[q] * xs[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) xs[kb + kq] = rhs[steprow[kb + kq]] - acc;
        if (lane < nbk) tri[kq * 33 + lane] = urow[kb + lane];
      }
      __syncthreads();
      if (wid == 0) {
        Real rr = lane < nbk ? xs[kb + lane] : Real(0);
        for (int c = nbk - 1; c >= 0; --c) {
          Real xc = Real(0);
          if (lane == c) {
            const Real dk = tri[c * 33 + c];
            xc = dk != Real(0) ? rr / dk : Real(0);
            xs[kb + c] = xc;
          }
          xc = __shfl_sync(0xffffffffu, xc, c);
          if (lane < c) rr -= tri[lane * 33 + c] * xc;
        }
      }
      __syncthreads();
    }
    const bool sing = s_sing != 0;
    for (int p = t; p < T; p += NT)
      Zval[base + p + (p >= d ? 1 : 0)] = sing ? 0.0 : (double)xs[p];
    if (t == 0) {
      Zval[base + d] = 1.0;
      if (sing) atomicAdd(nsingular, 1ull);
    }
    __syncthreads();  // the shared arrays are reused by the block's next system
  }
}

// ------------------------------------------------------------------------------------
// Bucketing and the projection.
// ------------------------------------------------------------------------------------
// work[0..2] = sum T^3, T^2, T; work[3] = A entries gathered (row lengths of the pattern's
// F-points in Ahat)
// Writes nothing but the lists and counters, so a caller may still refuse the call after
// reading the counts (a row with T = 0, the identity entry alone, goes to bucket 0, whose
// kernel writes that entry).
__global__ void bucket_rows(const int* __restrict__ Zrp, int nc, int tmed, int* __restrict__ lists,
                            int* __restrict__ counts, const int* __restrict__ Zcol,
                            const int* __restrict__ cpts, const int* __restrict__ Arp,
                            int* __restrict__ too_big, unsigned long long* __restrict__ work) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  const int T = r < nc ? Zrp[r + 1] - Zrp[r] - 1 : -1;
  const int b = T >= 0 ? ls_bucket(T, tmed) : -1;
  if (b >= LS_BUCKETS) atomicAdd(too_big, 1);
  if (b == LS_BUCKETS - 1) atomicMax(too_big + 1, T);  // largest T of the big bucket
  unsigned long long t3 = 0, t2 = 0, t1 = 0, g = 0;
  // one atomic per bucket and warp: lanes of the same bucket share a block of positions
  const int key = (b >= 0 && b < LS_BUCKETS) ? b : -1;
  const unsigned grp = __match_any_sync(0xffffffffu, key);
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(grp) - 1;
  int base = 0;
  if (lane == leader && key >= 0) base = atomicAdd(&counts[key], __popc(grp));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (key >= 0) {
    const int pos = base + __popc(grp & ((1u << lane) - 1u));
    lists[(long long)b * nc + pos] = r;
    for (int e = Zrp[r]; e < Zrp[r + 1]; ++e) {
      const int l = Zcol[e];
      if (l != cpts[r]) g += (unsigned long long)(Arp[l + 1] - Arp[l]);
    }
    t1 = (unsigned long long)T;
    t2 = t1 * t1;
    t3 = t2 * t1;
  }
  // one atomic per warp for the work counters
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    t3 += __shfl_xor_sync(0xffffffffu, t3, o);
    t2 += __shfl_xor_sync(0xffffffffu, t2, o);
    t1 += __shfl_xor_sync(0xffffffffu, t1, o);
    g += __shfl_xor_sync(0xffffffffu, g, o);
  }
  if (lane == 0 && (t1 | g)) {
    atomicAdd(&work[0], t3);
    atomicAdd(&work[1], t2);
    atomicAdd(&work[2], t1);
    atomicAdd(&work[3], g);
  }
}

// Projection on the transposed weights: rows are fine points j, entries (j, coarse i).
template <int W>
__global__ void project_rows(const int* __restrict__ Wrp, const int* __restrict__ Wcol,
                             double* __restrict__ Wval, int n, const signed char* __restrict__ cf,
                             const double* __restrict__ Bc, const double* __restrict__ B,
                             unsigned long long* __restrict__ nempty) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int j = (int)(t / W), lane = (int)(t % W);
  // C rows hold the identity entry only; no early exit before the shuffles
  const bool ok = j < n && !cf[j];
  const int b = ok ? Wrp[j] : 0, e = ok ? Wrp[j + 1] : 0;
  double g = 0.0, s = 0.0;
  for (int k = b + lane; k < e; k += W) {
    const double bc = Bc[Wcol[k]];
    g += bc * bc;
    s += Wval[k] * bc;
  }
  g = group_sum<W>(g);
  s = group_sum<W>(s);
  if (!ok) return;
  if (g > 0.0) {
    const double mu = (s - B[j]) / g;
    for (int k = b + lane; k < e; k += W) Wval[k] -= mu * Bc[Wcol[k]];
  } else if (lane == 0) {
    atomicAdd(nempty, 1ull);
  }
}

// Pseudo-inverse solve of the symmetric positive semidefinite k x k system G mu = r (cyclic
// Jacobi eigenvalue iteration, then mu = V diag(1/lambda) V^T r over the eigenvalues above
// 1e-15 of the largest, the cutoff numpy's pinv uses); k <= CLAIR_KMAX.
template <int K>
__device__ void psd_pinv_solve(double (&G)[K][K], const double (&r)[K], double (&mu)[K], int k) {
  double V[K][K];
#pragma unroll
  for (int a = 0; a < K; ++a)
#pragma unroll
    for (int b = 0; b < K; ++b) V[a][b] = a == b ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 30; ++sweep) {
    double off = 0.0, diag = 0.0;
    for (int a = 0; a < k; ++a) {
      diag += G[a][a] * G[a][a];
      for (int b = a + 1; b < k; ++b) off += G[a][b] * G[a][b];
    }
    if (off <= 1e-34 * diag) break;
    for (int p = 0; p < k; ++p)
      for (int q = p + 1; q < k; ++q) {
        if (G[p][q] == 0.0) continue;
        // rotation that zeroes G[p][q] (Golub & Van Loan, symmetric Schur decomposition)
        const double tau = (G[q][q] - G[p][p]) / (2.0 * G[p][q]);
        const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        const double c = 1.0 / sqrt(1.0 + t * t), sn = t * c;
        for (int j = 0; j < k; ++j) {  // G <- J^T G J
          const double gp = G[j][p], gq = G[j][q];
          G[j][p] = c * gp - sn * gq;
          G[j][q] = sn * gp + c * gq;
        }
        for (int j = 0; j < k; ++j) {
          const double gp = G[p][j], gq = G[q][j];
          G[p][j] = c * gp - sn * gq;
          G[q][j] = sn * gp + c * gq;
        }
        for (int j = 0; j < k; ++j) {
          const double vp = V[j][p], vq = V[j][q];
          V[j][p] = c * vp - sn * vq;
          V[j][q] = sn * vp + c * vq;
        }
      }
  }
  double lmax = 0.0;
  for (int a = 0; a < k; ++a) lmax = fmax(lmax, fabs(G[a][a]));
  for (int a = 0; a < k; ++a) mu[a] = 0.0;
  for (int e = 0; e < k; ++e) {
    const double lam = G[e][e];
    if (!(lam > 1e-15 * lmax)) continue;
    double c = 0.0;
    for (int a = 0; a < k; ++a) c += V[a][e] * r[a];
    c /= lam;
    for (int a = 0; a < k; ++a) mu[a] += V[a][e] * c;
  }
}

// Projection with k mode vectors (Eq. 3.3): per F row j with coarse points J_j,
// G = sum_i Bc(i,:)^T Bc(i,:), s = sum_i w_ji Bc(i,:), mu = G^+ (s - B(j,:)),
// w_ji <- w_ji - Bc(i,:) mu.  Bc is nc x k and B n x k, column-major; B may be null
// (target 0: the projection of an update, Algorithm 1's second constraint step).
__global__ void project_rows_k(const int* __restrict__ Wrp, const int* __restrict__ Wcol,
                               double* __restrict__ Wval, int n, const signed char* __restrict__ cf,
                               const double* __restrict__ Bc, int nc, const double* __restrict__ B,
                               int k, unsigned long long* __restrict__ nempty) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n || cf[j]) return;
  const int b = Wrp[j], e = Wrp[j + 1];
  double G[CLAIR_KMAX][CLAIR_KMAX], sv[CLAIR_KMAX], mu[CLAIR_KMAX];
  for (int a = 0; a < CLAIR_KMAX; ++a) {
    sv[a] = 0.0;
    for (int c = 0; c < CLAIR_KMAX; ++c) G[a][c] = 0.0;
  }
  for (int q = b; q < e; ++q) {
    const int i = Wcol[q];
    const double w = Wval[q];
    for (int a = 0; a < k; ++a) {
      const double ba = Bc[(long long)a * nc + i];
      sv[a] += w * ba;
      for (int c = 0; c <= a; ++c) G[a][c] += ba * Bc[(long long)c * nc + i];
    }
  }
  double gmax = 0.0;
  for (int a = 0; a < k; ++a) {
    for (int c = a + 1; c < k; ++c) G[a][c] = G[c][a];
    gmax = fmax(gmax, G[a][a]);
    sv[a] -= B ? B[(long long)a * n + j] : 0.0;
  }
  if (!(gmax > 0.0)) {
    if (nempty) atomicAdd(nempty, 1ull);
    return;
  }
  psd_pinv_solve<CLAIR_KMAX>(G, sv, mu, k);
  for (int q = b; q < e; ++q) {
    const int i = Wcol[q];
    double d = 0.0;
    for (int a = 0; a < k; ++a) d += Bc[(long long)a * nc + i] * mu[a];
    Wval[q] -= d;
  }
}

// The residual step of Algorithm 1's loop with the diagonal block inverse: for each coarse
// point i (row r of Z) and F-point l of its pattern,
//   wbar_l = (-Ahat[l, i] - sum_{c in W_i} Ahat[l, c] w_c) / Ahat[l, l],
// written at l's entry of the row (0 at the identity entry).  One warp per coarse row.
__global__ void diag_update(const int* __restrict__ Arp, const int* __restrict__ Acol,
                            const double* __restrict__ Aval, const int* __restrict__ Zrp,
                            const int* __restrict__ Zcol, const double* __restrict__ Zval,
                            const int* __restrict__ cpts, int nc, double* __restrict__ out) {
  const int r = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (r >= nc) return;
  const int i = cpts[r];
  const int z0 = Zrp[r], z1 = Zrp[r + 1];
  for (int q = z0 + lane; q < z1; q += 32) {
    const int l = Zcol[q];
    if (l == i) {
      out[q] = 0.0;
      continue;
    }
    double acc = 0.0, d = 0.0;
    for (int e = Arp[l]; e < Arp[l + 1]; ++e) {
      const int c = Acol[e];
      const double a = Aval[e];
      if (c == l) d = a;
      if (c == i) {
        acc -= a;
      } else {
        const int pos = find_sorted(Zcol + z0, z1 - z0, c);
        if (pos >= 0) acc -= a * Zval[z0 + pos];
      }
    }
    out[q] = d != 0.0 ? acc / d : 0.0;
  }
}

__global__ void add_into(const double* __restrict__ x, double* __restrict__ y, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) y[i] += x[i];
}

__global__ void unit_on_c_rows(const int* __restrict__ rp, const signed char* __restrict__ cf,
                               int n, double* __restrict__ val) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  for (int e = rp[j]; e < rp[j + 1]; ++e) val[e] = cf[j] ? 1.0 : 0.0;
}

__global__ void coarse_of(const signed char* __restrict__ cf, const int* __restrict__ cidx_incl,
                          int n, int* __restrict__ cpts) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n && cf[j]) cpts[cidx_incl[j]] = j;
}

__global__ void cf_to_int(const signed char* __restrict__ cf, int n, int* __restrict__ out) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) out[j] = cf[j] ? 1 : 0;
}

// cpts[k] = fine index of the k-th C-point; returns nc.
int coarse_points(const signed char* cf, int n, int** cpts_out, cudaStream_t s) {
  int* flag = dalloc<int>(n, s);
  int* pre = dalloc<int>(n + 1, s);
  if (n) cf_to_int<<<ceil_div(n, 256), 256, 0, s>>>(cf, n, flag); ::clair::count_launch();
  CLAIR_LAUNCHED();
  int nc = (int)exclusive_scan(flag, pre, n, s, true);
  int* cpts = dalloc<int>(nc, s);
  if (n) coarse_of<<<ceil_div(n, 256), 256, 0, s>>>(cf, pre, n, cpts); ::clair::count_launch();
  CLAIR_LAUNCHED();
  dfree(flag, s);
  dfree(pre, s);
  *cpts_out = cpts;
  return nc;
}

// vals: Ahat's values in the gather's type (a float copy in MIXED mode, so each value is
// converted once instead of once per local system it appears in; converting the copy
// gives the same floats).
// Size classes of the global-tile systems and the tile memory one launch may take (more
// concurrent tiles than this spill out of L2 and the launch slows down; measured on the
// 3D aggregation hierarchies).
constexpr int LB_CLASSES = 5;
constexpr size_t LB_BUDGET = 256ull << 20;

// cls[c * nb + k]: the systems of list[0 .. nb) with T <= 256 << c and above the previous
// class's limit, in list order per class (one atomic per system: these are rare)
__global__ void class_big(const int* __restrict__ list, int nb, const int* __restrict__ Zrp,
                          int* __restrict__ cls, int* __restrict__ ccount) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nb) return;
  const int r = list[k];
  const int T = Zrp[r + 1] - Zrp[r] - 1;
  int c = 0;
  while (c < LB_CLASSES - 1 && T > (256 << c)) ++c;
  cls[(size_t)c * nb + atomicAdd(&ccount[c], 1)] = r;
}

// Panel width of the blocked kernel for a tile pitch: 32 columns where its shared memory
// allows, else 16, else 0 (those systems take the unblocked global-tile kernel).
constexpr size_t LK_SMEM_MAX = 225u << 10;
template <class Real>
static int blk_nb(int pitch) {
  return blk_smem<Real>(pitch, 32) <= LK_SMEM_MAX ? 32 : blk_smem<Real>(pitch, 16) <= LK_SMEM_MAX ? 16 : 0;
}

// One launch of the blocked kernel over the classes [0, ncls) of cls (sizes in ccount on
// the device), tiles of `pitch`; returns the tile buffer (freed by the caller after the
// launch on the same stream).
template <class Real, class VT>
static Real* launch_blocked(const Csr& Ahat, const VT* vals, const int* Zrp, const int* Zcol,
                            const int* cpts, const int* cls, const int* ccount, int cls_stride,
                            int ncls, int* ticket, double* Zval, unsigned long long* nsing,
                            int pitch, int nsys, cudaStream_t s) {
  const int nbw = blk_nb<Real>(pitch);
  const bool small = pitch <= LK_SMALL_PITCH && nbw == 32;
  const int nt = small ? 128 : 256;
  const size_t smem = blk_smem<Real>(pitch, nbw);
  auto kernel = small ? lsolve_blk<Real, VT, 32, 128>
                      : nbw == 32 ? lsolve_blk<Real, VT, 32, 256> : lsolve_blk<Real, VT, 16, 256>;
  once_per_device((const void*)lsolve_blk<Real, VT, 32, 256>, [] {
    CLAIR_CUDA(cudaFuncSetAttribute(lsolve_blk<Real, VT, 32, 128>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LK_SMEM_MAX));
    CLAIR_CUDA(cudaFuncSetAttribute(lsolve_blk<Real, VT, 32, 256>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LK_SMEM_MAX));
    CLAIR_CUDA(cudaFuncSetAttribute(lsolve_blk<Real, VT, 16, 256>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LK_SMEM_MAX));
  });
  int dev = 0, sms = 0, per_sm = 0;
  CLAIR_CUDA(cudaGetDevice(&dev));
  CLAIR_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  CLAIR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, nt, smem));
  const size_t tile = (size_t)pitch * pitch * sizeof(Real);
  const int grid = (int)std::max<long long>(
      1, std::min<long long>({(long long)nsys, (long long)std::max(per_sm, 1) * sms,
                              (long long)(LB_BUDGET / tile)}));
  Real* tiles = dalloc<Real>((size_t)grid * pitch * pitch, s);
  kernel<<<grid, nt, smem, s>>>(Ahat.rowptr, Ahat.col, vals, Zrp, Zcol, cpts, cls, ccount,
                                cls_stride, ncls, ticket, Zval, nsing, tiles, pitch); ::clair::count_launch();
  CLAIR_LAUNCHED();
  return tiles;
}

// The classes [c0, LB_CLASSES) of cls with the unblocked global-tile kernel (systems too
// large for the blocked kernel's shared memory; rare), each class on a stream of its own.
template <class Real, class VT>
static void big_classes(const Csr& Ahat, const VT* vals, const int* Zrp, const int* Zcol,
                        const int* cpts, const int* cls, const int* ccount, int nb, int c0,
                        double* Zval, unsigned long long* nsing, cudaStream_t s) {
  int ch[LB_CLASSES];
  CLAIR_CUDA(cudaMemcpyAsync(ch, ccount, sizeof(ch), cudaMemcpyDeviceToHost, s));
  CLAIR_CUDA(cudaStreamSynchronize(s));
  // the classes run side by side, one stream each (forked from and joined back to s):
  // a launch lasts as long as its slowest system, so classes in sequence would add up
  struct Fork {
    cudaStream_t st[LB_CLASSES] = {};
    cudaEvent_t ev[LB_CLASSES + 1] = {};
    ~Fork() {
      for (cudaStream_t x : st)
        if (x) cudaStreamDestroy(x);
      for (cudaEvent_t e : ev)
        if (e) cudaEventDestroy(e);
    }
  } fk;
  Real* tiles[LB_CLASSES] = {};
  int chunk[LB_CLASSES] = {}, pitch[LB_CLASSES] = {};
  for (int c = c0; c < LB_CLASSES; ++c) {
    if (!ch[c]) continue;
    pitch[c] = std::min(LS_TBIG, 256 << c);
    const size_t tile = (size_t)pitch[c] * pitch[c] * sizeof(Real);
    chunk[c] = (int)std::max<size_t>(1, std::min<size_t>(ch[c], LB_BUDGET / tile));
    tiles[c] = dalloc<Real>((size_t)chunk[c] * pitch[c] * pitch[c], s);
  }
  CLAIR_CUDA(cudaEventCreateWithFlags(&fk.ev[LB_CLASSES], cudaEventDisableTiming));
  CLAIR_CUDA(cudaEventRecord(fk.ev[LB_CLASSES], s));
  for (int c = c0; c < LB_CLASSES; ++c) {
    if (!ch[c]) continue;
    CLAIR_CUDA(cudaStreamCreateWithFlags(&fk.st[c], cudaStreamNonBlocking));
    CLAIR_CUDA(cudaEventCreateWithFlags(&fk.ev[c], cudaEventDisableTiming));
    CLAIR_CUDA(cudaStreamWaitEvent(fk.st[c], fk.ev[LB_CLASSES], 0));
    for (int off = 0; off < ch[c]; off += chunk[c]) {
      const int cnt = std::min(chunk[c], ch[c] - off);
      lsolve_big<Real, VT><<<cnt, LB_THREADS, big_smem<Real>(pitch[c]), fk.st[c]>>>(
          Ahat.rowptr, Ahat.col, vals, Zrp, Zcol, cpts, cls + (size_t)c * nb + off, Zval, nsing,
          tiles[c], pitch[c]); ::clair::count_launch();
    }
    CLAIR_CUDA(cudaEventRecord(fk.ev[c], fk.st[c]));
    CLAIR_CUDA(cudaStreamWaitEvent(s, fk.ev[c], 0));
  }
  CLAIR_LAUNCHED();
  for (int c = c0; c < LB_CLASSES; ++c) dfree(tiles[c], s);
}

template <class Real, class VT>
static void launch_solves(const Csr& Ahat, const VT* vals, const int* Zrp, const int* Zcol,
                          const int* cpts, const int* lists, const int* counts_h, int nc,
                          double* Zval, unsigned long long* nsing, cudaStream_t s,
                          bool big_scratch_forbidden = false, int first_bucket = 0,
                          const int* counts_dev = nullptr) {
  // the shared-memory limits above 48 KB are per-device function attributes
  constexpr int TMED = sizeof(Real) == 8 ? LS_TMED64 : LS_TMED32;
  once_per_device((const void*)lsolve_cta<Real, VT, 128>, [] {
    CLAIR_CUDA(cudaFuncSetAttribute(lsolve_cta<Real, VT, 64>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)cta_smem<Real, 64>()));
    CLAIR_CUDA(cudaFuncSetAttribute(lsolve_cta<Real, VT, 128>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)cta_smem<Real, 128>()));
    CLAIR_CUDA(cudaFuncSetAttribute(lsolve_big<Real, VT>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)big_smem<Real>(LS_TBIG)));
  });
  const int per_block[2] = {LS_WARPS * 4, LS_WARPS * 2};
  if (counts_h[0] && first_bucket <= 0)
    lsolve_group<Real, VT, 8><<<ceil_div(counts_h[0], per_block[0]), 32 * LS_WARPS, 0, s>>>(
        Ahat.rowptr, Ahat.col, vals, Zrp, Zcol, cpts, lists + 0LL * nc, counts_h[0], Zval, nsing); ::clair::count_launch();
  if (counts_h[1] && first_bucket <= 1)
    lsolve_group<Real, VT, 16><<<ceil_div(counts_h[1], per_block[1]), 32 * LS_WARPS, 0, s>>>(
        Ahat.rowptr, Ahat.col, vals, Zrp, Zcol, cpts, lists + 1LL * nc, counts_h[1], Zval, nsing); ::clair::count_launch();
  // 16 < T <= 32: the CTA kernel with one warp per block (rolled loops; a 32-lane register
  // elimination unrolls into more code than the instruction cache holds)
  if (counts_h[2] && first_bucket <= 2)
    lsolve_cta<Real, VT, 32><<<counts_h[2], 32, cta_smem<Real, 32>(), s>>>(
        Ahat.rowptr, Ahat.col, vals, Zrp, Zcol, cpts, lists + 2LL * nc, Zval, nsing); ::clair::count_launch();
  if (counts_h[3] && first_bucket <= 3)
    lsolve_cta<Real, VT, 64><<<counts_h[3], 64, cta_smem<Real, 64>(), s>>>(
        Ahat.rowptr, Ahat.col, vals, Zrp, Zcol, cpts, lists + 3LL * nc, Zval, nsing); ::clair::count_launch();
  if (counts_h[4])
    lsolve_cta<Real, VT, 128><<<counts_h[4], 128, cta_smem<Real, 128>(), s>>>(
        Ahat.rowptr, Ahat.col, vals, Zrp, Zcol, cpts, lists + 4LL * nc, Zval, nsing); ::clair::count_launch();
  Real* b5_tiles = nullptr;
  int* b5_ticket = nullptr;
  if (counts_h[5] && first_bucket <= 5) {
    CLAIR_REQUIRE(!big_scratch_forbidden && counts_dev, CLAIR_ERR_CAPACITY,
                  "%d local systems larger than 128 unknowns need a tile buffer", counts_h[5]);
    b5_ticket = dalloc<int>(1, s);
    CLAIR_CUDA(cudaMemsetAsync(b5_ticket, 0, sizeof(int), s));
    b5_tiles = launch_blocked<Real, VT>(Ahat, vals, Zrp, Zcol, cpts, lists + 5LL * nc,
                                        counts_dev + 5, 0, 1, b5_ticket, Zval, nsing,
                                        ceil_div(TMED, 32) * 32, counts_h[5], s);
  }
  if (counts_h[6]) {
    CLAIR_REQUIRE(!big_scratch_forbidden, CLAIR_ERR_CAPACITY,
                  "%d local systems larger than %d unknowns need a tile buffer", counts_h[6], TMED);
    const int nb = counts_h[6];
    const int tmax = counts_h[LS_BUCKETS + 1];  // the bucket's largest T
    int* cls = dalloc<int>((size_t)LB_CLASSES * nb, s);
    int* ccount = dalloc<int>(LB_CLASSES + 1, s);  // class sizes, then the blocked ticket
    CLAIR_CUDA(cudaMemsetAsync(ccount, 0, sizeof(int) * (LB_CLASSES + 1), s));
    class_big<<<ceil_div(nb, 256), 256, 0, s>>>(lists + 6LL * nc, nb, Zrp, cls, ccount); ::clair::count_launch();
    CLAIR_LAUNCHED();
    // the blocked kernel takes the classes whose tile pitch fits its shared memory
    int cblk = 0;
    while (cblk < LB_CLASSES && blk_nb<Real>(256 << cblk) > 0) ++cblk;
    Real* blk_tiles = nullptr;
    if (cblk > 0) {
      const int pitch = std::min(256 << (cblk - 1), ceil_div(tmax, 32) * 32);
      blk_tiles = launch_blocked<Real, VT>(Ahat, vals, Zrp, Zcol, cpts, cls, ccount, nb, cblk,
                                           ccount + LB_CLASSES, Zval, nsing, pitch, nb, s);
    }
    if (tmax > (256 << (cblk - 1))) big_classes<Real, VT>(Ahat, vals, Zrp, Zcol, cpts, cls, ccount,
                                                        nb, cblk, Zval, nsing, s);
    dfree(blk_tiles, s);
    dfree(cls, s);
    dfree(ccount, s);
  }
  dfree(b5_tiles, s);
  dfree(b5_ticket, s);
  CLAIR_LAUNCHED();
}


// Streams of the highest priority per device for the large local systems (the ones whose
// single-system latency sets a level's time), one per side, created once.
static cudaStream_t large_stream(int side) {
  static std::mutex mu;
  static cudaStream_t st[256][2] = {};
  int dev = 0;
  CLAIR_CUDA(cudaGetDevice(&dev));
  CLAIR_REQUIRE(dev >= 0 && dev < 256, CLAIR_ERR_ARG, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lock(mu);
  if (!st[dev][side]) {
    int lo = 0, hi = 0;
    CLAIR_CUDA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    CLAIR_CUDA(cudaStreamCreateWithPriority(&st[dev][side], cudaStreamNonBlocking, hi));
  }
  return st[dev][side];
}

// ---- execution configuration of the persistent launch, per device and precision -------
struct LsolveConfig {
  int kind_b1 = LK_G16;   // systems with 8 < T <= 16: 16-lane groups or single warps
  int kind_b3 = LK_P64;   // systems with 32 < T <= 64: warp pairs or single warps
  int blocks_per_sm = 0;  // 0: as many as fit
  int tuned = 0;          // 1: chosen by timing, 2: set by the caller
};
static std::mutex g_cfg_mu;
static LsolveConfig g_cfg[256][2];

static LsolveConfig& config_slot(int precision) {
  int dev = 0;
  CLAIR_CUDA(cudaGetDevice(&dev));
  CLAIR_REQUIRE(dev >= 0 && dev < 256, CLAIR_ERR_ARG, "device ordinal %d out of range", dev);
  return g_cfg[dev][precision == CLAIR_MIXED ? 1 : 0];
}

// Levels with fewer systems of T <= 64 than this are not used for timing candidates.
constexpr long long LS_TUNE_MIN = 20000;

struct SideIn {
  const Csr* Ahat;
  const int* Zrp;
  const int* Zcol;
  double* Zval;
  int nc;
};

template <class Real, class VT>
static void persistent_launch(const SideArgs<VT>* sa, int nsides, const int (*counts_h)[LS_BUCKETS + 2],
                              const LsolveConfig& cfg, int* ticket, unsigned long long* nsing,
                              cudaStream_t s) {
  bool has[5] = {false, false, false, false, false};
  long long tasks = 0;
  for (int q = 0; q < nsides; ++q) {
    has[LK_G8] |= counts_h[q][0] > 0;
    has[cfg.kind_b1] |= counts_h[q][1] > 0;
    has[LK_W32] |= counts_h[q][2] > 0;
    has[cfg.kind_b3] |= counts_h[q][3] > 0;
    tasks += ceil_div(counts_h[q][0], lk_systems(LK_G8)) +
             ceil_div(counts_h[q][1], lk_systems(cfg.kind_b1)) +
             ceil_div(counts_h[q][2], lk_systems(LK_W32)) +
             ceil_div(counts_h[q][3], lk_systems(cfg.kind_b3));
  }
  if (tasks == 0) return;
  once_per_device((const void*)lsolve_persist<Real, VT>, [] {
    CLAIR_CUDA(cudaFuncSetAttribute(lsolve_persist<Real, VT>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)sizeof(PersistSmem<Real>)));
  });
  const size_t smem = persist_smem<Real>(has);
  int fit = 0;
  CLAIR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, lsolve_persist<Real, VT>, LP_THREADS,
                                                           smem));
  const int per_sm = std::max(1, cfg.blocks_per_sm > 0 ? std::min(fit, cfg.blocks_per_sm) : fit);
  // LP_WAVES times the resident blocks, each taking at most an even share of the tasks
  // from the ticket and then leaving: the budgets add up to every task, and a leaving
  // block frees its slot for the other stream's waiting blocks (the mode smoothing, of
  // higher priority), which a block that stays to the end would hold off
  const long long resident = (long long)sm_count() * per_sm;
  const int grid = (int)std::min<long long>(tasks, resident * LP_WAVES);
  const int budget = (int)((tasks + grid - 1) / grid);
  CLAIR_CUDA(cudaMemsetAsync(ticket, 0, sizeof(int), s));
  lsolve_persist<Real, VT><<<grid, LP_THREADS, smem, s>>>(sa[0], nsides > 1 ? sa[1] : sa[0], nsides,
                                                          cfg.kind_b1, cfg.kind_b3, ticket, nsing,
                                                          budget); ::clair::count_launch();
  CLAIR_LAUNCHED();
}

// Times the candidate configurations on this level (the launches are idempotent: they
// rewrite the same weights) and keeps the fastest for the process.
template <class Real, class VT>
static void autotune(const SideArgs<VT>* sa, int nsides, const int (*counts_h)[LS_BUCKETS + 2],
                     LsolveConfig& cfg, int* ticket, cudaStream_t s) {
  unsigned long long* scratch = dalloc<unsigned long long>(1, s);
  constexpr int NC = 5;
  LsolveConfig cands[NC];
  cands[1].kind_b1 = LK_W32;
  cands[2].blocks_per_sm = 4;
  cands[3].kind_b3 = LK_W64;
  cands[4].kind_b1 = LK_W32;
  cands[4].kind_b3 = LK_W64;
  cudaEvent_t e0, e1;
  CLAIR_CUDA(cudaEventCreate(&e0));
  CLAIR_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  int pick = 0;
  for (int c = 0; c < NC; ++c) {
    for (int rep = 0; rep < 2; ++rep) {  // the first run warms the caches and the code
      CLAIR_CUDA(cudaEventRecord(e0, s));
      persistent_launch<Real, VT>(sa, nsides, counts_h, cands[c], ticket, scratch, s);
      CLAIR_CUDA(cudaEventRecord(e1, s));
    }
    CLAIR_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    CLAIR_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    if (ms < best) {
      best = ms;
      pick = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  dfree(scratch, s);
  cfg = cands[pick];
  cfg.tuned = 1;
}

// Local lAIR solves for all coarse rows of one or two patterns (the two sides of a level:
// R on A^T and P on A), values into each side's Zval.  Systems of up to 64 unknowns of
// every side go to one persistent launch; larger ones to the CTA and large-tile kernels.
void local_solves_multi(const SideIn* sides, int nsides, const int* cpts, int precision,
                        LocalStats& st, cudaStream_t s) {
  int* lists[2] = {nullptr, nullptr};
  int* counts = dalloc<int>(2 * (LS_BUCKETS + 2), s);
  // [0] singular, [1..4] work: the owner's device counters when it has them (layout
  // [singular, empty, work...]: the work counters follow at +2), else read back here
  unsigned long long* own = nullptr;
  unsigned long long* nsing = nullptr;
  unsigned long long* work = nullptr;
  if (st.dev) {
    nsing = st.dev;
    work = st.dev + 2;
  } else {
    own = dalloc<unsigned long long>(5, s);
    CLAIR_CUDA(cudaMemsetAsync(own, 0, 5 * sizeof(unsigned long long), s));
    nsing = own;
    work = own + 1;
  }
  int* ticket = dalloc<int>(1, s);
  CLAIR_CUDA(cudaMemsetAsync(counts, 0, sizeof(int) * 2 * (LS_BUCKETS + 2), s));
  for (int q = 0; q < nsides; ++q) {
    const SideIn& S = sides[q];
    lists[q] = dalloc<int>((long long)LS_BUCKETS * std::max(S.nc, 1), s);
    int* cq = counts + q * (LS_BUCKETS + 2);
    const int tmed = precision == CLAIR_MIXED ? LS_TMED32 : LS_TMED64;
    if (S.nc) bucket_rows<<<ceil_div(S.nc, 256), 256, 0, s>>>(S.Zrp, S.nc, tmed, lists[q], cq, S.Zcol, cpts,
                                                             S.Ahat->rowptr, cq + LS_BUCKETS,
                                                             work); ::clair::count_launch();
  }
  CLAIR_LAUNCHED();
  int counts_h[2][LS_BUCKETS + 2] = {};
  CLAIR_CUDA(cudaMemcpyAsync(counts_h, counts, sizeof(int) * nsides * (LS_BUCKETS + 2),
                             cudaMemcpyDeviceToHost, s));
  CLAIR_CUDA(cudaStreamSynchronize(s));
  for (int q = 0; q < nsides; ++q)
    CLAIR_REQUIRE(counts_h[q][LS_BUCKETS] == 0, CLAIR_ERR_CAPACITY,
                  "%d local systems larger than %d unknowns", counts_h[q][LS_BUCKETS], LS_TBIG);
  {
    ClockScope clk(PH_LSOLVE, s);
    auto run = [&](auto real_tag, auto& vals) {
      using Real = decltype(real_tag);
      using VT = typename std::remove_cv<typename std::remove_pointer<
          typename std::remove_reference<decltype(vals[0])>::type>::type>::type;
      SideArgs<VT> sa[2];
      for (int q = 0; q < nsides; ++q) {
        const SideIn& S = sides[q];
        sa[q] = SideArgs<VT>{S.Ahat->rowptr, S.Ahat->col, vals[q], S.Zrp, S.Zcol, cpts, lists[q],
                             counts + q * (LS_BUCKETS + 2), S.Zval, S.nc};
      }
      LsolveConfig cfg;
      {
        std::lock_guard<std::mutex> lock(g_cfg_mu);
        LsolveConfig& slot = config_slot(precision);
        long long small = 0, b3 = 0;
        for (int q = 0; q < nsides; ++q) {
          for (int b = 0; b < 4; ++b) small += counts_h[q][b];
          b3 += counts_h[q][3];
        }
        // timed on the first level with enough systems, among them enough of 32 < T <= 64
        if (!slot.tuned && small >= LS_TUNE_MIN && b3 >= LS_TUNE_MIN / 10)
          autotune<Real, VT>(sa, nsides, counts_h, slot, ticket, s);
        cfg = slot;
      }
      st.config_kind_b1 = cfg.kind_b1;
      st.config_kind_b3 = cfg.kind_b3;
      st.config_blocks_per_sm = cfg.blocks_per_sm;
      st.config_tuned = cfg.tuned;
      // the systems with T > 64 (one CTA each, or a global tile) beside the persistent
      // launch, each side on a stream of its own: a coarse level's time is then the
      // longest of the three
      bool large = false;
      for (int q = 0; q < nsides; ++q)
        large = large || counts_h[q][4] + counts_h[q][5] + counts_h[q][6] > 0;
      cudaStream_t ls[2] = {s, s};
      cudaEvent_t fork = nullptr, join[2] = {nullptr, nullptr};
      auto join_all = [&]() {
        for (int q = 0; q < nsides; ++q)
          if (join[q]) {
            cudaEventRecord(join[q], ls[q]);
            cudaStreamWaitEvent(s, join[q], 0);
            cudaEventDestroy(join[q]);
            join[q] = nullptr;
          }
        if (fork) cudaEventDestroy(fork);
        fork = nullptr;
      };
      if (large) {
        CLAIR_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
        CLAIR_CUDA(cudaEventRecord(fork, s));
        for (int q = 0; q < nsides; ++q) {
          ls[q] = large_stream(q);
          CLAIR_CUDA(cudaEventCreateWithFlags(&join[q], cudaEventDisableTiming));
          CLAIR_CUDA(cudaStreamWaitEvent(ls[q], fork, 0));
        }
      }
      persistent_launch<Real, VT>(sa, nsides, counts_h, cfg, ticket, nsing, s);
      try {
        for (int q = 0; q < nsides; ++q) {
          const SideIn& S = sides[q];
          launch_solves<Real, VT>(*S.Ahat, vals[q], S.Zrp, S.Zcol, cpts, lists[q], counts_h[q],
                                  S.nc, S.Zval, nsing, ls[q], false, /*first_bucket=*/4,
                                  counts + q * (LS_BUCKETS + 2));
        }
      } catch (...) {
        join_all();
        throw;
      }
      join_all();
    };
    if (precision == CLAIR_MIXED) {
      // values converted once per side instead of once per local system they appear in
      float* vals32[2] = {nullptr, nullptr};
      for (int q = 0; q < nsides; ++q) {
        vals32[q] = dalloc<float>(std::max(sides[q].Ahat->nnz, 1), s);
        to_float(sides[q].Ahat->val, vals32[q], sides[q].Ahat->nnz, s);
      }
      const float* v[2] = {vals32[0], vals32[1]};
      run(float(0), v);
      for (int q = 0; q < nsides; ++q) dfree(vals32[q], s);
    } else {
      const double* v[2] = {sides[0].Ahat->val, nsides > 1 ? sides[1].Ahat->val : nullptr};
      run(double(0), v);
    }
  }
  if (own) {
    unsigned long long h[5] = {0, 0, 0, 0, 0};
    CLAIR_CUDA(cudaMemcpyAsync(h, own, sizeof(h), cudaMemcpyDeviceToHost, s));
    CLAIR_CUDA(cudaStreamSynchronize(s));
    st.singular += (long long)h[0];
    st.sum_t3 += (double)h[1];
    st.sum_t2 += (double)h[2];
    st.sum_t += (double)h[3];
    st.gathered += (long long)h[4];
  }
  for (int q = 0; q < nsides; ++q)
    for (int b = 0; b < LS_BUCKETS; ++b) st.hist[b] += counts_h[q][b];
  for (int q = 0; q < nsides; ++q) dfree(lists[q], s);
  dfree(counts, s);
  dfree(own, s);
  dfree(ticket, s);
}

void LocalStats::absorb_device(cudaStream_t s) {
  if (!dev) return;
  unsigned long long h[6] = {0, 0, 0, 0, 0, 0};
  CLAIR_CUDA(cudaMemcpyAsync(h, dev, sizeof(h), cudaMemcpyDeviceToHost, s));
  CLAIR_CUDA(cudaMemsetAsync(dev, 0, sizeof(h), s));
  CLAIR_CUDA(cudaStreamSynchronize(s));
  singular += (long long)h[0];
  empty += (long long)h[1];
  sum_t3 += (double)h[2];
  sum_t2 += (double)h[3];
  sum_t += (double)h[4];
  gathered += (long long)h[5];
}

void local_solves(const Csr& Ahat, const int* Zrp, const int* Zcol, const int* cpts, int nc,
                  int precision, double* Zval, LocalStats& st, cudaStream_t s) {
  SideIn side{&Ahat, Zrp, Zcol, Zval, nc};
  local_solves_multi(&side, 1, cpts, precision, st, s);
}

// Sets (kind_b1 >= 0) or reads the execution configuration of the persistent local-solve
// launch on the current device for one precision.
void lsolve_config(int precision, int* kind_b1, int* kind_b3, int* blocks_per_sm, int* tuned,
                   bool set) {
  std::lock_guard<std::mutex> lock(g_cfg_mu);
  LsolveConfig& slot = config_slot(precision);
  if (set) {
    slot.kind_b1 = *kind_b1;
    slot.kind_b3 = *kind_b3;
    slot.blocks_per_sm = *blocks_per_sm;
    slot.tuned = *tuned;
  } else {
    *kind_b1 = slot.kind_b1;
    *kind_b3 = slot.kind_b3;
    *blocks_per_sm = slot.blocks_per_sm;
    *tuned = slot.tuned;
  }
}

// Projection of the transposed weights Wt (rows = fine points) onto the constraint; Bc is
// nc x k and B n x k (column-major); B null projects onto Q w = 0 (an update).
void project_constraint(Csr& Wt, const signed char* cf, const double* Bc, int nc, const double* B,
                        int k, LocalStats& st, cudaStream_t s) {
  unsigned long long* nempty = st.dev ? st.dev + 1 : dalloc<unsigned long long>(1, s);
  if (!st.dev) CLAIR_CUDA(cudaMemsetAsync(nempty, 0, sizeof(unsigned long long), s));
  if (Wt.rows && k == 1 && B) {
    constexpr int W = 1;  // FP64: one thread per row
    project_rows<W><<<ceil_div((long long)Wt.rows * W, 256), 256, 0, s>>>(
        Wt.rowptr, Wt.col, Wt.val, Wt.rows, cf, Bc, B, nempty); ::clair::count_launch();
  } else if (Wt.rows) {
    project_rows_k<<<ceil_div(Wt.rows, 128), 128, 0, s>>>(Wt.rowptr, Wt.col, Wt.val, Wt.rows, cf, Bc,
                                                           nc, B, k, nempty); ::clair::count_launch();
  }
  CLAIR_LAUNCHED();
  if (st.dev) return;
  unsigned long long h = 0;
  CLAIR_CUDA(cudaMemcpyAsync(&h, nempty, sizeof(h), cudaMemcpyDeviceToHost, s));
  CLAIR_CUDA(cudaStreamSynchronize(s));
  st.empty += (long long)h;
  dfree(nempty, s);
}

// Full transfer-weight computation: local solves on Ahat over pattern Z (nc x n), then the
// projection.  On return Z.val holds the projected weights (row = coarse point) and, if
// keep_t is set, Zt receives the transposed operator (rows = fine points) with the same
// projected values.
void transfer_project(const signed char* cf, const int* cpts, Csr& Z, const double* B, int k,
                      LocalStats& st, Csr* keep_t, cudaStream_t s);

// First half: the local lAIR solves into Z.val (no mode vector needed).
void transfer_solve(const Csr& Ahat, const int* cpts, Csr& Z, int precision, LocalStats& st,
                    cudaStream_t s) {
  if (!Z.val) Z.val = dalloc<double>(Z.nnz, s);
  local_solves(Ahat, Z.rowptr, Z.col, cpts, Z.rows, precision, Z.val, st, s);
}

// Both sides of a level in one go: R's pattern on A^T and P's (transposed) pattern on A.
void transfer_solve_pair(const Csr& At, Csr& R, const Csr& A, Csr& Pt, const int* cpts,
                         int precision, LocalStats& st, cudaStream_t s) {
  if (!R.val) R.val = dalloc<double>(R.nnz, s);
  if (!Pt.val) Pt.val = dalloc<double>(Pt.nnz, s);
  SideIn sides[2] = {{&At, R.rowptr, R.col, R.val, R.rows}, {&A, Pt.rowptr, Pt.col, Pt.val, Pt.rows}};
  local_solves_multi(sides, 2, cpts, precision, st, s);
}

void transfer_weights(const Csr& Ahat, const signed char* cf, const int* cpts, Csr& Z,
                      const double* B, int precision, LocalStats& st, Csr* keep_t,
                      cudaStream_t s) {
  transfer_solve(Ahat, cpts, Z, precision, st, s);
  transfer_project(cf, cpts, Z, B, 1, st, keep_t, s);
}

// Second half: projection onto the mode constraint (needs the smoothed mode vector B).
void transfer_project(const signed char* cf, const int* cpts, Csr& Z, const double* B, int k,
                      LocalStats& st, Csr* keep_t, cudaStream_t s) {
  const int nc = Z.rows, n = Z.cols;
  ClockScope clk(PH_PROJECT, s);
  Csr Zt;
  int* perm = nullptr;
  csr_transpose(Z, Zt, &perm, s);
  double* Bc = dalloc<double>((size_t)nc * k, s);
  for (int a = 0; a < k; ++a) gather(B + (size_t)a * n, cpts, Bc + (size_t)a * nc, nc, s);
  project_constraint(Zt, cf, Bc, nc, B, k, st, s);
  scatter_vals(Zt.val, perm, Z.val, Z.nnz, s);
  dfree(Bc, s);
  dfree(perm, s);
  if (keep_t)
    *keep_t = Zt;
  else
    Zt.release(s);
}

// Algorithm 1 with the diagonal block inverses (Section 3.1.2) and `iterations` passes of
// its loop, in float64:
//   w_t: per F row the minimum-norm solution of w B_c = B (the projection of zero onto the
//        constraint set);
//   each pass: wbar = D^-1 (-a_fc - A_ff w_t) per coarse point's block, wbar projected onto
//        Q wbar = 0, w_t += wbar.
// On return Z.val holds the weights (row = coarse point); keep_t as in transfer_project.
void transfer_diag(const Csr& Ahat, const signed char* cf, const int* cpts, Csr& Z,
                   const double* B, int k, int iterations, LocalStats& st, Csr* keep_t,
                   cudaStream_t s) {
  const int nc = Z.rows, n = Z.cols;
  ClockScope clk(PH_LSOLVE, s);
  if (!Z.val) Z.val = dalloc<double>(Z.nnz, s);
  Csr Zt;
  int* perm = nullptr;
  csr_transpose(Z, Zt, &perm, s);  // structure (values are set below)
  double* Bc = dalloc<double>((size_t)nc * k, s);
  for (int a = 0; a < k; ++a) gather(B + (size_t)a * n, cpts, Bc + (size_t)a * nc, nc, s);
  // tentative weights: 1 at the identity entries (C rows), the projection of 0 elsewhere
  if (n) {
    unit_on_c_rows<<<ceil_div(n, 256), 256, 0, s>>>(Zt.rowptr, cf, n, Zt.val); ::clair::count_launch();
  }
  CLAIR_LAUNCHED();
  project_constraint(Zt, cf, Bc, nc, B, k, st, s);
  scatter_vals(Zt.val, perm, Z.val, Z.nnz, s);
  double* zbar = dalloc<double>(std::max(Z.nnz, 1), s);
  unsigned long long* scratch6 = dalloc<unsigned long long>(6, s);
  for (int it = 0; it < iterations; ++it) {
    if (nc) {
      diag_update<<<ceil_div((long long)nc * 32, 256), 256, 0, s>>>(
          Ahat.rowptr, Ahat.col, Ahat.val, Z.rowptr, Z.col, Z.val, cpts, nc, zbar); ::clair::count_launch();
    }
    CLAIR_LAUNCHED();
    gather_vals(zbar, perm, Zt.val, Z.nnz, s);
    LocalStats discard;  // empty F rows are counted once, by the first projection
    discard.dev = scratch6;
    project_constraint(Zt, cf, Bc, nc, nullptr, k, discard, s);
    scatter_vals(Zt.val, perm, zbar, Z.nnz, s);
    if (Z.nnz) {
      add_into<<<ceil_div(Z.nnz, 256), 256, 0, s>>>(zbar, Z.val, Z.nnz); ::clair::count_launch();
    }
    CLAIR_LAUNCHED();
  }
  gather_vals(Z.val, perm, Zt.val, Z.nnz, s);
  dfree(scratch6, s);
  dfree(zbar, s);
  dfree(Bc, s);
  dfree(perm, s);
  if (keep_t)
    *keep_t = Zt;
  else
    Zt.release(s);
}

// ======================================================================================
// The same computation with every temporary carved from one static device array, for
// callers that must not allocate device memory (see clair_local_weights_noalloc).
// ======================================================================================
int scan_ws_blocks(int n);
long long exclusive_scan_ws(const int* in, int* out, int n, cudaStream_t s, bool want_total,
                            long long* sums, int* ovf);
void csr_transpose_ws(const Csr& A, Csr& At, int* perm, int* cnt, long long* sums, int* ovf,
                      cudaStream_t s);
void validate_csr_ws(const int* rowptr, const int* col, int rows, int cols, int nnz,
                     const char* what, int* bad, cudaStream_t s);
void validate_cf_ws(const signed char* cf, int n, int* bad, cudaStream_t s);
const char* last_error();
void clear_error();

// The scratch array.  Host code only ever sees a host-side stand-in for this name; its
// device address comes from cudaGetSymbolAddress, once per device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[CLAIR_NOALLOC_SCRATCH_BYTES];

static std::mutex g_scratch_mutex;
static void* g_scratch_address[256] = {};

// Device address of the scratch array on the current device (looked up on first use).
static unsigned char* scratch_on_current_device() {
  int dev = -1;
  CLAIR_CUDA(cudaGetDevice(&dev));
  CLAIR_REQUIRE(dev >= 0 && dev < 256, CLAIR_ERR_ARG, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_address[dev]) {
    void* p = nullptr;
    CLAIR_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    CLAIR_REQUIRE(p != nullptr, CLAIR_ERR_CUDA, "no device address for the scratch array");
    g_scratch_address[dev] = p;
  }
  return static_cast<unsigned char*>(g_scratch_address[dev]);
}

// Bump allocation of 256-byte aligned pieces; with base == nullptr it only measures.
struct ScratchCursor {
  unsigned char* base = nullptr;
  size_t used = 0;
  template <class T>
  T* take(size_t count) {
    const size_t bytes = ((count ? count : 1) * sizeof(T) + 255) & ~size_t(255);
    T* p = base ? reinterpret_cast<T*>(base + used) : nullptr;
    used += bytes;
    return p;
  }
};

struct NoallocBuffers {
  int *bad, *flag, *pre, *ovf, *cpts, *lists, *counts, *zt_rowptr, *zt_col, *perm, *cnt;
  long long* sums;
  unsigned long long *work, *nempty;
  double *zt_val, *Bc;
};

static void carve(ScratchCursor& c, int n, int nc, int nnzZ, NoallocBuffers& b) {
  b.bad = c.take<int>(1);
  b.ovf = c.take<int>(1);
  b.sums = c.take<long long>(scan_ws_blocks(n) + 1);
  b.flag = c.take<int>(n);
  b.pre = c.take<int>((size_t)n + 1);
  b.cpts = c.take<int>(nc);
  b.lists = c.take<int>((size_t)LS_BUCKETS * (nc > 0 ? nc : 1));
  b.counts = c.take<int>(LS_BUCKETS + 2);
  b.work = c.take<unsigned long long>(5);
  b.zt_rowptr = c.take<int>((size_t)n + 1);
  b.zt_col = c.take<int>(nnzZ);
  b.zt_val = c.take<double>(nnzZ);
  b.perm = c.take<int>(nnzZ);
  b.cnt = c.take<int>((size_t)n + 1);
  b.Bc = c.take<double>(nc);
  b.nempty = c.take<unsigned long long>(1);
}

static size_t noalloc_bytes(int n, int nc, int nnzZ) {
  ScratchCursor c;
  NoallocBuffers b;
  carve(c, n, nc, nnzZ, b);
  return c.used;
}

static void local_weights_noalloc(int n, const Csr& Ahat, const signed char* cf, int nc, Csr& Z,
                                  const double* B, int precision, const NoallocBuffers& b,
                                  LocalStats& st, cudaStream_t s) {
  validate_csr_ws(Ahat.rowptr, Ahat.col, n, n, Ahat.nnz, "Ahat", b.bad, s);
  validate_cf_ws(cf, n, b.bad, s);
  validate_csr_ws(Z.rowptr, Z.col, nc, n, Z.nnz, "Z", b.bad, s);
  // coarse points
  cf_to_int<<<ceil_div(n, 256), 256, 0, s>>>(cf, n, b.flag); ::clair::count_launch();
  CLAIR_LAUNCHED();
  const int nc2 = (int)exclusive_scan_ws(b.flag, b.pre, n, s, true, b.sums, b.ovf);
  CLAIR_REQUIRE(nc2 == nc, CLAIR_ERR_ARG, "nc=%d but cf has %d C-points", nc, nc2);
  coarse_of<<<ceil_div(n, 256), 256, 0, s>>>(cf, b.pre, n, b.cpts); ::clair::count_launch();
  CLAIR_LAUNCHED();
  // bucketed local solves (counters start at zero on every call)
  CLAIR_CUDA(cudaMemsetAsync(b.counts, 0, sizeof(int) * (LS_BUCKETS + 2), s));
  CLAIR_CUDA(cudaMemsetAsync(b.work, 0, 5 * sizeof(unsigned long long), s));
  const int tmed = precision == CLAIR_MIXED ? LS_TMED32 : LS_TMED64;
  if (nc) bucket_rows<<<ceil_div(nc, 256), 256, 0, s>>>(Z.rowptr, nc, tmed, b.lists, b.counts, Z.col,
                                                        b.cpts, Ahat.rowptr, b.counts + LS_BUCKETS,
                                                        b.work + 1); ::clair::count_launch();
  CLAIR_LAUNCHED();
  int counts_h[LS_BUCKETS + 2];
  CLAIR_CUDA(cudaMemcpyAsync(counts_h, b.counts, sizeof(counts_h), cudaMemcpyDeviceToHost, s));
  CLAIR_CUDA(cudaStreamSynchronize(s));
  // every refusal comes before the first write to Z_val: systems above 128 unknowns need
  // a per-call tile buffer, which this entry point does not have
  const int over128 = counts_h[5] + counts_h[6] + counts_h[7];
  CLAIR_REQUIRE(over128 == 0, CLAIR_ERR_CAPACITY,
                "%d local systems larger than 128 unknowns (this entry point solves T <= 128, "
                "use clair_local_weights)", over128);
  if (precision == CLAIR_MIXED)
    launch_solves<float, double>(Ahat, Ahat.val, Z.rowptr, Z.col, b.cpts, b.lists, counts_h, nc,
                                 Z.val, b.work, s, /*big_scratch_forbidden=*/true);
  else
    launch_solves<double, double>(Ahat, Ahat.val, Z.rowptr, Z.col, b.cpts, b.lists, counts_h, nc,
                                  Z.val, b.work, s, /*big_scratch_forbidden=*/true);
  // column view of the weights, projection, values back into the row view
  Csr Zt;
  Zt.rowptr = b.zt_rowptr;
  Zt.col = b.zt_col;
  Zt.val = b.zt_val;
  csr_transpose_ws(Z, Zt, b.perm, b.cnt, b.sums, b.ovf, s);
  gather(B, b.cpts, b.Bc, nc, s);
  CLAIR_CUDA(cudaMemsetAsync(b.nempty, 0, sizeof(unsigned long long), s));
  if (Zt.rows) {
    constexpr int W = 1;  // as project_constraint: the same summation order, the same bits
    project_rows<W><<<ceil_div((long long)Zt.rows * W, 256), 256, 0, s>>>(
        Zt.rowptr, Zt.col, Zt.val, Zt.rows, cf, b.Bc, B, b.nempty); ::clair::count_launch();
  }
  CLAIR_LAUNCHED();
  scatter_vals(Zt.val, b.perm, Z.val, Z.nnz, s);
  unsigned long long h[2] = {0, 0};
  CLAIR_CUDA(cudaMemcpyAsync(&h[0], b.work, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
  CLAIR_CUDA(cudaMemcpyAsync(&h[1], b.nempty, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
  CLAIR_CUDA(cudaStreamSynchronize(s));
  st.singular += (long long)h[0];
  st.empty += (long long)h[1];
}

}  // namespace clair

extern "C" clair_status clair_local_weights_noalloc(
    int n, const int* Ahat_rowptr, const int* Ahat_col, const double* Ahat_val,
    const signed char* cf, int nc, const int* Z_rowptr, const int* Z_col, const double* B,
    int precision, double* Z_val, void* stream, int64_t* singular_out, int64_t* empty_out) {
  using namespace clair;
  clear_error();
  try {
    CLAIR_REQUIRE(Ahat_rowptr && Ahat_col && Ahat_val && cf && Z_rowptr && Z_col && B && Z_val,
                  CLAIR_ERR_ARG, "clair_local_weights_noalloc: null pointer");
    CLAIR_REQUIRE(n > 0 && nc >= 0 && nc <= n, CLAIR_ERR_ARG,
                  "clair_local_weights_noalloc: bad sizes n=%d nc=%d", n, nc);
    CLAIR_REQUIRE(precision == CLAIR_FP64 || precision == CLAIR_MIXED, CLAIR_ERR_ARG,
                  "unknown precision");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int nnzA = 0, nnzZ = 0;
    CLAIR_CUDA(cudaMemcpyAsync(&nnzA, Ahat_rowptr + n, sizeof(int), cudaMemcpyDeviceToHost, s));
    CLAIR_CUDA(cudaMemcpyAsync(&nnzZ, Z_rowptr + nc, sizeof(int), cudaMemcpyDeviceToHost, s));
    CLAIR_CUDA(cudaStreamSynchronize(s));
    CLAIR_REQUIRE(nnzA >= 0 && nnzZ >= 0, CLAIR_ERR_ARG, "negative nnz in a row pointer");
    const size_t need = noalloc_bytes(n, nc, nnzZ);
    CLAIR_REQUIRE(need <= (size_t)CLAIR_NOALLOC_SCRATCH_BYTES, CLAIR_ERR_CAPACITY,
                  "clair_local_weights_noalloc needs %zu bytes of scratch for n=%d, nc=%d, "
                  "nnz(Z)=%d; its fixed limit is %zu bytes (use clair_local_weights)",
                  need, n, nc, nnzZ, (size_t)CLAIR_NOALLOC_SCRATCH_BYTES);
    ScratchCursor cur;
    cur.base = scratch_on_current_device();
    NoallocBuffers buf;
    carve(cur, n, nc, nnzZ, buf);
    Csr Ahat;
    Ahat.rows = Ahat.cols = n;
    Ahat.nnz = nnzA;
    Ahat.rowptr = const_cast<int*>(Ahat_rowptr);
    Ahat.col = const_cast<int*>(Ahat_col);
    Ahat.val = const_cast<double*>(Ahat_val);
    Csr Z;
    Z.rows = nc;
    Z.cols = n;
    Z.nnz = nnzZ;
    Z.rowptr = const_cast<int*>(Z_rowptr);
    Z.col = const_cast<int*>(Z_col);
    Z.val = Z_val;
    LocalStats st;
    try {
      local_weights_noalloc(n, Ahat, cf, nc, Z, B, precision, buf, st, s);
    } catch (...) {
      // a refusal or failure returns only once nothing this call queued still runs
      cudaStreamSynchronize(s);
      throw;
    }
    if (singular_out) *singular_out = st.singular;
    if (empty_out) *empty_out = st.empty;
    if (st.singular) {
      set_error("%lld local blocks had a zero pivot", st.singular);
      return CLAIR_ERR_SINGULAR_BLOCK;
    }
  } catch (const Error& e) {
    return e.st;
  } catch (...) {
    set_error("unexpected host exception");
    return CLAIR_ERR_CUDA;
  }
  return CLAIR_OK;
}
