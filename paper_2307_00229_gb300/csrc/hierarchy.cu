// CLAIR hierarchy: setup (per level: strength, splitting, weight, smoothed modes, R and P
// by Algorithm 1, Galerkin product) and solve (V(1,1) cycles inside right-preconditioned
// flexible GMRES in float64), plus the C ABI declared in include/clair.h.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <memory>
#include <mutex>
#include <vector>

#include "common.cuh"

namespace clair {

// --- functions of the other translation units -----------------------------------------
void strength2(const Csr& M, const double* thr1, double theta1, int mode1, unsigned char* mask1,
               const double* thr2, double theta2, int mode2, unsigned char* mask2,
               cudaStream_t s);
void split_fc(const Csr& A, const Csr& At, const unsigned char* sA, const unsigned char* sAt,
              const int* lbase, signed char* cf, cudaStream_t s);
void aggregate(const Csr& A, const Csr& At, const unsigned char* sA, const unsigned char* sAt,
               const int* lbase, signed char* cf, int* agg, cudaStream_t s);
void aggregate_members(const int* agg, int n, int nc, int** rp_out, int** members_out,
                       cudaStream_t s);
void build_pattern(const Csr& Wm, const unsigned char* sW, const signed char* cf, const int* cpts,
                   int nc, int n, int degree, const int* Mrp, const int* Mcol, Csr& Z,
                   cudaStream_t s);
template <class T>
void jacobi(const Csr& A, const T* vals, const T* dinv, const signed char* cf, int which, T omega,
            const T* b, const T* xin, T* xout, cudaStream_t s, const T* omega_dev = nullptr);
void smooth_modes(const Csr& M, const double* dinv, const signed char* cf, const double* omega_dev,
                  int sweeps, double* Bv, double* tmp, cudaStream_t s);
void smooth_modes_sides(const SmoothSides& sides, int rows, double avg_row, const double* dinv,
                        const signed char* cf, const double* omega_dev, double omega, int sweeps,
                        cudaStream_t s);
void transfer_solve(const Csr& Ahat, const int* cpts, Csr& Z, int precision, LocalStats& st,
                    cudaStream_t s);
void transfer_project(const signed char* cf, const int* cpts, Csr& Z, const double* B, int k,
                      LocalStats& st, Csr* keep_t, cudaStream_t s);
void transfer_solve_pair(const Csr& At, Csr& R, const Csr& A, Csr& Pt, const int* cpts,
                         int precision, LocalStats& st, cudaStream_t s);
void lsolve_config(int precision, int* kind_b1, int* kind_b3, int* blocks_per_sm, int* tuned,
                   bool set);
void transfer_diag(const Csr& Ahat, const signed char* cf, const int* cpts, Csr& Z,
                   const double* B, int k, int iterations, LocalStats& st, Csr* keep_t,
                   cudaStream_t s);
template <class T>
void jacobi_from_zero(int rows, const T* dinv, const signed char* cf, int which, T omega,
                      const T* b, T* x, cudaStream_t s);
struct RitzHost;
RitzHost* ritz_host_alloc(int ninst);
void ritz_host_free(RitzHost* r);
double arnoldi_weight(const Csr& A, const double* dinv, int iters, uint64_t seed,
                      double* omega_dev, RitzHost* rh, cudaStream_t s);
void arnoldi_weight_batched(const Csr& A, const double* dinv, int iters, uint64_t seed,
                            const std::vector<int>& off, double* omega_dev, RitzHost* rh,
                            cudaStream_t s);
void dense_inverse(const Csr& A, const std::vector<int>& off, double* Inv, int** d_off,
                   long long** d_ioff, cudaStream_t s);
template <class T>
void coarse_apply(const T* Inv, const int* d_off, const long long* d_ioff, int nblk, int n,
                  const T* b, T* x, cudaStream_t s);
int coarse_points(const signed char* cf, int n, int** cpts_out, cudaStream_t s);
void transfer_weights(const Csr& Ahat, const signed char* cf, const int* cpts, Csr& Z,
                      const double* B, int precision, LocalStats& st, Csr* keep_t,
                      cudaStream_t s);
const char* last_error();
void clear_error();

// --- hierarchy --------------------------------------------------------------------------
struct Level {
  Csr A, R, P;
  int n = 0, nc = 0;
  double* dinv = nullptr;
  float* dinv32 = nullptr;
  signed char* cf = nullptr;
  int* cpts = nullptr;
  double omega = 1.0;
  double* B_P = nullptr;
  double* B_R = nullptr;
  // batch (block-diagonal instances): host row offsets of the instances on this level,
  // instance and instance base of every row, weights and frozen flags per instance, and
  // the relaxation weights folded into D^-1 per row (pre and post smoothing)
  std::vector<int> off;
  int* inst = nullptr;
  int* lbase = nullptr;
  std::vector<double> omega_inst;
  std::vector<char> frozen;
  double *wpre64 = nullptr, *wpost64 = nullptr;
  float *wpre32 = nullptr, *wpost32 = nullptr;
  // MIXED: this level's part of the cycle runs in FP64 (its transfer weights, or those of
  // a finer level, exceed what FP32 carries; see kCycle64Weight)
  bool cycle64 = false;
  double max_weight = 0.0;
  // cycle work vectors
  double *b64 = nullptr, *x64 = nullptr, *y64 = nullptr, *r64 = nullptr;
  float *b32 = nullptr, *x32 = nullptr, *y32 = nullptr, *r32 = nullptr;
};

// Krylov workspace of one solve call: nrhs right-hand sides of all instances as nseg =
// nrhs * ninst independent processes (segments) in lockstep.  Vectors have N = nrhs * n
// rows (right-hand side r at offset r * n); V (m+1 vectors) and Z (m vectors) are stored
// one vector after another.  Per-segment scalars: the Hessenberg matrices, rotations and
// right-hand sides of the least-squares problems, tolerances and iteration counts.
struct Krylov {
  int nrhs = 0, m = 0, n = 0;
  long long N = 0;
  Segments S;
  double *V = nullptr, *Z = nullptr, *w = nullptr, *r = nullptr;
  double *H = nullptr, *cs = nullptr, *sn = nullptr, *g = nullptr, *y = nullptr;
  double *h1 = nullptr, *h2 = nullptr, *partial = nullptr;
  double *fn2 = nullptr, *fnorm = nullptr, *tol = nullptr, *beta2 = nullptr, *wn2 = nullptr;
  double *inv = nullptr, *summary = nullptr, *cg = nullptr;
  int *active = nullptr, *jend = nullptr, *its = nullptr;
  double* host = nullptr;  // pinned scalars
};

// The captured fine-level cycle: head and tail graphs, replayed one after the other.
struct CycleGraph {
  cudaGraphExec_t head = nullptr, tail = nullptr;
  long long kernels = 0;  // kernels in both
};
inline void destroy_cycle(CycleGraph& c) {
  if (c.head) cudaGraphExecDestroy(c.head);
  if (c.tail) cudaGraphExecDestroy(c.tail);
  c = CycleGraph{};
}

}  // namespace clair

struct clair_hierarchy {
  clair_params p;
  std::vector<clair::Level> lv;
  double* Inv = nullptr;     // coarsest dense inverse (float64, column-major)
  float* Inv32 = nullptr;
  int nL = 0;
  cudaStream_t stream = nullptr;
  clair::Krylov kr;
  clair::LocalStats st;
  double setup_ms = 0.0;
  double phase_ms[clair::PH_COUNT] = {};   // setup, per phase
  double level_phase_ms[32 * clair::PH_COUNT] = {};  // setup, per level and phase
  // event marks of the last setup and solve, read when the statistics are asked for (an
  // instrument, kept off the setup's and the solve's own time)
  std::unique_ptr<clair::PhaseClock> setup_clock, solve_clock;
  double level_span_ms[32] = {};           // setup: main-stream time from level to level
  double solve_ms[clair::PH_COUNT] = {};   // last solve, per phase
  clair::CycleGraph cycle;                  // captured fine-level V(1,1) cycle
  double* vin = nullptr;                    // its fixed input and output vectors
  double* zout = nullptr;
  double* B0 = nullptr;                     // the caller's mode vector, unsmoothed
  int ninst = 1;                            // instances of a block-diagonal batch
  int* coarse_off = nullptr;                // coarsest diagonal blocks (device offsets)
  long long* coarse_ioff = nullptr;         // and their inverses' offsets in Inv
  int coarse_nblk = 1;
  int short_lanes = 0;                      // FP32 short-row lanes chosen for the cycle
  int cycle_lanes_pick = 0;
  bool cycle_fp64 = false;                  // MIXED solve fell back to the FP64 cycle
  int fp64_from = -1;                       // iteration of that fallback (-1: none)
  int kmodes = 1;                           // mode vectors (columns of B)
  std::vector<int> last_its;                // per segment, last solve
  std::vector<double> last_rel;
};

namespace clair {

// Largest transfer weight an FP32 cycle level takes (FP32 keeps about 7 digits: weights of
// this size that cancel to O(1) leave about 4).
constexpr double kCycle64Weight = 1e3;

static void alloc_cycle(Level& L, cudaStream_t s) {
  const int n = L.n;
  L.b64 = dalloc<double>(n, s);
  L.x64 = dalloc<double>(n, s);
  L.y64 = dalloc<double>(n, s);
  L.r64 = dalloc<double>(n, s);
  L.b32 = dalloc<float>(n, s);
  L.x32 = dalloc<float>(n, s);
  L.y32 = dalloc<float>(n, s);
  L.r32 = dalloc<float>(n, s);
}

static void release_level(Level& L, cudaStream_t s) {
  L.A.release(s);
  L.R.release(s);
  L.P.release(s);
  dfree(L.dinv, s);
  dfree(L.dinv32, s);
  dfree(L.cf, s);
  dfree(L.cpts, s);
  dfree(L.B_P, s);
  dfree(L.B_R, s);
  dfree(L.inst, s);
  dfree(L.lbase, s);
  dfree(L.wpre64, s);
  dfree(L.wpost64, s);
  dfree(L.wpre32, s);
  dfree(L.wpost32, s);
  dfree(L.b64, s);
  dfree(L.x64, s);
  dfree(L.y64, s);
  dfree(L.r64, s);
  dfree(L.b32, s);
  dfree(L.x32, s);
  dfree(L.y32, s);
  dfree(L.r32, s);
}

static void release_krylov(Krylov& k, cudaStream_t s) {
  k.S.release(s);
  for (double** p : {&k.V, &k.Z, &k.w, &k.r, &k.H, &k.cs, &k.sn, &k.g, &k.y, &k.h1, &k.h2,
                     &k.partial, &k.fn2, &k.fnorm, &k.tol, &k.beta2, &k.wn2, &k.inv, &k.summary,
                     &k.cg})
    dfree(*p, s);
  dfree(k.active, s);
  dfree(k.jend, s);
  dfree(k.its, s);
  if (k.host) {
    cudaStreamSynchronize(s);
    pinned_put(k.host, sizeof(double) * 4);
  }
  k.host = nullptr;
  k.nrhs = 0;
}

static void release_all(clair_hierarchy* h) {
  cudaStream_t s = h->stream;
  for (auto& L : h->lv) release_level(L, s);
  h->lv.clear();
  dfree(h->Inv, s);
  dfree(h->Inv32, s);
  dfree(h->coarse_off, s);
  dfree(h->coarse_ioff, s);
  release_krylov(h->kr, s);
  destroy_cycle(h->cycle);
  dfree(h->vin, s);
  dfree(h->zout, s);
  dfree(h->B0, s);
}

__global__ void inject(const double* __restrict__ x, const int* __restrict__ cpts, int nc,
                       double* __restrict__ y) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nc) y[i] = x[cpts[i]];
}


// ---- batch of independent instances (block-diagonal operator) ------------------------
// Rows off[i] .. off[i+1]-1 of every level belong to instance i (coarse points are
// numbered in fine order, so the ranges stay contiguous).  An instance that reaches its
// coarsest size is frozen: all its points become C-points (identity transfers, no
// F-points) and its relaxation weights are zero, so it passes unchanged to the batch's
// coarsest level, where its diagonal block is inverted.
__global__ void row_instance(const int* __restrict__ off, int ninst, int n, int* __restrict__ inst,
                             int* __restrict__ lbase) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  int lo = 0, hi = ninst;  // largest i with off[i] <= r
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (off[mid] <= r) lo = mid; else hi = mid;
  }
  inst[r] = lo;
  lbase[r] = off[lo];
}

// cnt[i] = number of C-points of instance i (one block per instance)
__global__ void count_c_instances(const signed char* __restrict__ cf, const int* __restrict__ off,
                                  int* __restrict__ cnt) {
  __shared__ int part[8];
  const int i = blockIdx.x;
  int c = 0;
  for (int r = off[i] + threadIdx.x; r < off[i + 1]; r += blockDim.x) c += cf[r] == 1;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
    cnt[i] = t;
  }
}

__global__ void freeze_rows(const int* __restrict__ inst, const char* __restrict__ frozen, int n,
                            signed char* __restrict__ cf) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n && frozen[inst[r]]) cf[r] = 1;
}

__global__ void point_to_coarse(const int* __restrict__ cpts, int nc, int* __restrict__ cidx) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < nc) cidx[cpts[r]] = r;
}

// aggregate index after freezing renumbered the C-points: the old root's new coarse
// index; frozen instances keep no aggregates
__global__ void remap_aggregates(const int* __restrict__ inst, const char* __restrict__ frozen,
                                 const int* __restrict__ old_cpts, const int* __restrict__ cidx,
                                 int n, int* __restrict__ agg) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const int a = agg[j];
  agg[j] = (a < 0 || frozen[inst[j]]) ? -1 : cidx[old_cpts[a]];
}

// out[r] = weight of r's instance times dinv[r] (the weight folded into D^-1)
template <class T>
__global__ void instance_weights(const int* __restrict__ inst, const double* __restrict__ w,
                                 const T* __restrict__ dinv, int n, T* __restrict__ out) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n) out[r] = (T)w[inst[r]] * dinv[r];
}

__global__ void check_block_diagonal(const int* __restrict__ rowptr, const int* __restrict__ col,
                                     const int* __restrict__ inst, const int* __restrict__ off,
                                     int n, int* __restrict__ bad) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const int lo = off[inst[r]], hi = off[inst[r] + 1];
  for (int e = rowptr[r]; e < rowptr[r + 1]; ++e)
    if (col[e] < lo || col[e] >= hi) {
      atomicAdd(bad, 1);
      return;
    }
}

// out[i] = sum of x^2 over instance i's rows (one block of 256 per instance, fixed order)
__global__ void instance_sumsq(const double* __restrict__ x, const int* __restrict__ off,
                               double* __restrict__ out) {
  __shared__ double part[8];
  const int i = blockIdx.x;
  double a = 0.0;
  for (int r = off[i] + threadIdx.x; r < off[i + 1]; r += blockDim.x) a += x[r] * x[r];
  a = warp_sum(a);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
    out[i] = t;
  }
}

// device copies of a level's instance map
static void level_instances(Level& L, cudaStream_t s) {
  const int ninst = (int)L.off.size() - 1;
  int* d_off = dalloc<int>(ninst + 1, s);
  CLAIR_CUDA(cudaMemcpyAsync(d_off, L.off.data(), sizeof(int) * (ninst + 1), cudaMemcpyHostToDevice, s));
  L.inst = dalloc<int>(L.n, s);
  L.lbase = dalloc<int>(L.n, s);
  if (L.n) {
    row_instance<<<ceil_div(L.n, 256), 256, 0, s>>>(d_off, ninst, L.n, L.inst, L.lbase); ::clair::count_launch();
  }
  CLAIR_LAUNCHED();
  dfree(d_off, s);
}

// per-instance C counts of a level (host)
static std::vector<int> c_counts(const Level& L, const signed char* cf, cudaStream_t s) {
  const int ninst = (int)L.off.size() - 1;
  int* d_off = dalloc<int>(ninst + 1, s);
  int* d_cnt = dalloc<int>(ninst, s);
  CLAIR_CUDA(cudaMemcpyAsync(d_off, L.off.data(), sizeof(int) * (ninst + 1), cudaMemcpyHostToDevice, s));
  count_c_instances<<<ninst, 256, 0, s>>>(cf, d_off, d_cnt); ::clair::count_launch();
  CLAIR_LAUNCHED();
  std::vector<int> cnt(ninst);
  CLAIR_CUDA(cudaMemcpyAsync(cnt.data(), d_cnt, sizeof(int) * ninst, cudaMemcpyDeviceToHost, s));
  CLAIR_CUDA(cudaStreamSynchronize(s));
  dfree(d_off, s);
  dfree(d_cnt, s);
  return cnt;
}

// weights folded into D^-1 for the cycle: pre = omega_i, post = 1 (or omega_i when
// post_weighted), both 0 for a frozen instance
static void batch_cycle_weights(Level& L, bool post_weighted, cudaStream_t s) {
  const int ninst = (int)L.off.size() - 1;
  std::vector<double> w(2 * ninst);
  for (int i = 0; i < ninst; ++i) {
    const bool fz = L.frozen[i] != 0;
    w[i] = fz ? 0.0 : L.omega_inst[i];
    w[ninst + i] = fz ? 0.0 : (post_weighted ? L.omega_inst[i] : 1.0);
  }
  double* dw = dalloc<double>(2 * ninst, s);
  CLAIR_CUDA(cudaMemcpyAsync(dw, w.data(), sizeof(double) * 2 * ninst, cudaMemcpyHostToDevice, s));
  L.wpre64 = dalloc<double>(L.n, s);
  L.wpost64 = dalloc<double>(L.n, s);
  L.wpre32 = dalloc<float>(L.n, s);
  L.wpost32 = dalloc<float>(L.n, s);
  const int g = ceil_div(L.n, 256);
  if (L.n) {
    instance_weights<double><<<g, 256, 0, s>>>(L.inst, dw, L.dinv, L.n, L.wpre64); ::clair::count_launch();
    instance_weights<double><<<g, 256, 0, s>>>(L.inst, dw + ninst, L.dinv, L.n, L.wpost64); ::clair::count_launch();
    instance_weights<float><<<g, 256, 0, s>>>(L.inst, dw, L.dinv32, L.n, L.wpre32); ::clair::count_launch();
    instance_weights<float><<<g, 256, 0, s>>>(L.inst, dw + ninst, L.dinv32, L.n, L.wpost32); ::clair::count_launch();
  }
  CLAIR_LAUNCHED();
  dfree(dw, s);
}

// A second stream and the fork/join events of one setup (released on scope exit).
struct SideStream {
  cudaStream_t s2 = nullptr;
  cudaEvent_t fork = nullptr, split = nullptr, join = nullptr;
  SideStream() {
    // the weight chain's blocks go first, the splitting, patterns and local solves use the
    // SMs it leaves (measured: the reverse order, the main stream first, lengthens every
    // level by its wait for the slower weight chain at the join)
    int lo = 0, hi = 0;
    CLAIR_CUDA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    CLAIR_CUDA(cudaStreamCreateWithPriority(&s2, cudaStreamNonBlocking, hi));
    CLAIR_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    CLAIR_CUDA(cudaEventCreateWithFlags(&split, cudaEventDisableTiming));
    CLAIR_CUDA(cudaEventCreateWithFlags(&join, cudaEventDisableTiming));
  }
  ~SideStream() {
    if (s2) cudaStreamSynchronize(s2);
    if (fork) cudaEventDestroy(fork);
    if (split) cudaEventDestroy(split);
    if (join) cudaEventDestroy(join);
    if (s2) cudaStreamDestroy(s2);
  }
};

// Builds the hierarchy from the fine operator (already copied into h->lv[0].A).
static void setup_levels(clair_hierarchy* h, const double* B0, const signed char* cf_marker) {
  cudaStream_t s = h->stream;
  const clair_params& p = h->p;
  const bool batch = h->ninst > 1;
  const int ninst = h->ninst;
  const int km = h->kmodes;
  const bool sym = p.symmetric != 0;
  {
    Level& L0 = h->lv[0];
    L0.B_P = dalloc<double>((size_t)L0.n * km, s);
    L0.B_R = dalloc<double>((size_t)L0.n * km, s);
    CLAIR_CUDA(cudaMemcpyAsync(L0.B_P, B0, sizeof(double) * L0.n * km, cudaMemcpyDeviceToDevice, s));
    CLAIR_CUDA(cudaMemcpyAsync(L0.B_R, B0, sizeof(double) * L0.n * km, cudaMemcpyDeviceToDevice, s));
  }
  // pinned buffers of the host Ritz steps; declared before the side stream so that the
  // stream (whose destructor waits for it) is gone before they are released
  struct RitzList {
    std::vector<RitzHost*> v;
    void push_back(RitzHost* r) { v.push_back(r); }
    RitzHost* back() { return v.back(); }
    ~RitzList() {
      for (RitzHost* r : v) ritz_host_free(r);
    }
  } ritz;
  SideStream ss;
  // one weight per level (per level and instance for a batch), on the device
  double* omega_dev = dalloc<double>((size_t)p.max_levels * ninst, s);
  int* bad_coarse = dalloc<int>(1, s);  // coarse rows without a usable diagonal
  CLAIR_CUDA(cudaMemsetAsync(bad_coarse, 0, sizeof(int), s));
  // main-stream marks at every level start (level spans for clair_stats)
  struct Marks {
    std::vector<cudaEvent_t> v;
    ~Marks() {
      for (cudaEvent_t e : v) cudaEventDestroy(e);
    }
    void record(cudaStream_t st) {
      cudaEvent_t e;
      CLAIR_CUDA(cudaEventCreate(&e));
      v.push_back(e);
      CLAIR_CUDA(cudaEventRecord(e, st));
    }
  } marks;
  for (int k = 0;; ++k) {
    Level& L = h->lv[k];
    const int n = L.n;
    if (active_clock()) active_clock()->set_level(k);
    marks.record(s);
    L.dinv = dalloc<double>(n, s);
    // the fine operator is checked at once; a coarse operator's count is read with the
    // weights after the last level
    inverse_diagonal(L.A, L.dinv, s, k > 0 ? bad_coarse : nullptr);
    if (!batch) {
      if (n <= p.coarse_max || k + 1 >= p.max_levels) break;
    } else {
      // an instance at its coarsest size (or the level cap) freezes; all frozen: stop
      level_instances(L, s);
      if (L.frozen.empty()) L.frozen.assign(ninst, 0);
      bool all = true;
      for (int i = 0; i < ninst; ++i) {
        const int ni = L.off[i + 1] - L.off[i];
        if (ni <= p.coarse_max || k + 1 >= p.max_levels) L.frozen[i] = 1;
        all = all && L.frozen[i];
      }
      if (all) break;
    }
    // Fork.  Stream s2: relaxation weight (Arnoldi on D^-1 A needs neither the splitting
    // nor A^T, so it starts now), then, once the splitting is known, the mode vectors
    // smoothed with zero right-hand side (A for P, A^T for R), the weight read on the
    // device.  Stream s: splitting, patterns and local lAIR solves.  Join before the
    // projection.
    CLAIR_CUDA(cudaEventRecord(ss.fork, s));
    CLAIR_CUDA(cudaStreamWaitEvent(ss.s2, ss.fork, 0));
    double* om_k = omega_dev + (size_t)k * ninst;
    // enqueued after the first splitting kernels, so that the main stream has work while
    // the host issues the Arnoldi launches
    auto enqueue_weight = [&]() {
      ClockScope clk(PH_WEIGHT, ss.s2);
      ritz.push_back(ritz_host_alloc(ninst));
      if (batch)
        arnoldi_weight_batched(L.A, L.dinv, p.arnoldi_iters, p.seed + (uint64_t)k, L.off, om_k,
                               ritz.back(), ss.s2);
      else
        arnoldi_weight(L.A, L.dinv, p.arnoldi_iters, p.seed + (uint64_t)k, om_k, ritz.back(),
                       ss.s2);
    };

    Csr At;
    int* agg = nullptr;                           // aggregate of each point (Agg coarsening)
    double* rmaxA = dalloc<double>(n, s);
    double* rmaxAt = dalloc<double>(n, s);
    unsigned char* sA = dalloc<unsigned char>(L.A.nnz, s);
    unsigned char* sAt = dalloc<unsigned char>(L.A.nnz, s);
    unsigned char* sR = dalloc<unsigned char>(L.A.nnz, s);
    unsigned char* sP = dalloc<unsigned char>(L.A.nnz, s);
    std::vector<int> cnt;                         // C-points per instance (batch)
    {
      ClockScope clk(PH_SPLIT, s);
      csr_transpose(L.A, At, nullptr, s);
      row_max_offdiag(L.A, rmaxA, s);
      row_max_offdiag(At, rmaxAt, s);
      // coarsening strength S(A, theta_c): on A row-relative, on A^T via A's row maxima;
      // in the same passes the interpolation-strength masks of the two patterns:
      // R: Algorithm 1 on A^T, walked on A, S(A^T) uses the row maxima of A^T
      // P: Algorithm 1 on A,   walked on A^T, S(A) uses the row maxima of A
      strength2(L.A, rmaxA, p.theta_coarsen, 0, sA, rmaxAt, p.theta_interp, 1, sR, s);
      strength2(At, rmaxA, p.theta_coarsen, 1, sAt, rmaxA, p.theta_interp, 1, sP, s);
      enqueue_weight();
      L.cf = dalloc<signed char>(n, s);
      if (k == 0 && cf_marker) {
        // the caller's splitting replaces step a2 on the fine level
        CLAIR_CUDA(cudaMemcpyAsync(L.cf, cf_marker, n, cudaMemcpyDeviceToDevice, s));
      } else if (p.coarsen == CLAIR_COARSEN_AGG) {
        agg = dalloc<int>(n, s);
        aggregate(L.A, At, sA, sAt, L.lbase, L.cf, agg, s);
      } else {
        split_fc(L.A, At, sA, sAt, L.lbase, L.cf, s);
      }
      L.nc = coarse_points(L.cf, n, &L.cpts, s);
      if (batch) {
        // an instance whose splitting leaves no C-point or no F-point ends there
        cnt = c_counts(L, L.cf, s);
        bool all = true, changed = false;
        for (int i = 0; i < ninst; ++i) {
          const int ni = L.off[i + 1] - L.off[i];
          if (!L.frozen[i] && (cnt[i] == 0 || cnt[i] == ni)) L.frozen[i] = 1;
          all = all && L.frozen[i];
          if (L.frozen[i] && cnt[i] != ni) changed = true;
        }
        if (all) {
          L.nc = 0;  // this level is the batch's coarsest
        } else if (changed) {
          char* dfz = dalloc<char>(ninst, s);
          CLAIR_CUDA(cudaMemcpyAsync(dfz, L.frozen.data(), ninst, cudaMemcpyHostToDevice, s));
          freeze_rows<<<ceil_div(n, 256), 256, 0, s>>>(L.inst, dfz, n, L.cf); ::clair::count_launch();
          CLAIR_LAUNCHED();
          int* old_cpts = L.cpts;
          L.cpts = nullptr;
          L.nc = coarse_points(L.cf, n, &L.cpts, s);
          if (agg) {
            int* cidx = dalloc<int>(n, s);
            point_to_coarse<<<ceil_div(L.nc, 256), 256, 0, s>>>(L.cpts, L.nc, cidx); ::clair::count_launch();
            remap_aggregates<<<ceil_div(n, 256), 256, 0, s>>>(L.inst, dfz, old_cpts, cidx, n, agg); ::clair::count_launch();
            CLAIR_LAUNCHED();
            dfree(cidx, s);
          }
          dfree(old_cpts, s);
          dfree(dfz, s);
          for (int i = 0; i < ninst; ++i)
            if (L.frozen[i]) cnt[i] = L.off[i + 1] - L.off[i];
        }
      }
    }
    if (L.nc == 0 || L.nc == n) {
      dfree(agg, s);
      dfree(L.cf, s);
      dfree(L.cpts, s);
      L.nc = 0;
      At.release(s);
      dfree(rmaxA, s);
      dfree(rmaxAt, s);
      dfree(sA, s);
      dfree(sAt, s);
      dfree(sR, s);
      dfree(sP, s);
      break;
    }
    CLAIR_CUDA(cudaEventRecord(ss.split, s));
    Csr Pt;
    int* Mrp = nullptr;
    int* Mcol = nullptr;
    PatternJob jobR, jobP;
    {
      ClockScope clk(PH_PATTERN, s);
      if (agg) aggregate_members(agg, n, L.nc, &Mrp, &Mcol, s);
      if (!sym) jobR = pattern_count(L.A, sR, L.cf, L.cpts, L.nc, n, p.degree, Mrp, Mcol, s);
      jobP = pattern_count(At, sP, L.cf, L.cpts, L.nc, n, p.degree, Mrp, Mcol, s);
    }
    // the mode smoothing on s2 is issued while the counting passes run on s
    CLAIR_CUDA(cudaStreamWaitEvent(ss.s2, ss.split, 0));
    {
      ClockScope clk(PH_SMOOTH, ss.s2);
      // each mode vector separately; the symmetric variant (R = P^T) needs only A's
      double* wd = nullptr;
      if (batch) {
        // each instance's weight folded into D^-1, unit scalar weight
        wd = dalloc<double>(n, ss.s2);
        instance_weights<double><<<ceil_div(n, 256), 256, 0, ss.s2>>>(L.inst, om_k, L.dinv, n, wd); ::clair::count_launch();
        CLAIR_LAUNCHED();
      }
      // every mode of both sides in one launch per relaxation (A for P, A^T for R)
      SmoothSides sides{};
      double* tmps = dalloc<double>((size_t)n * km * (sym ? 1 : 2), ss.s2);
      for (int a = 0; a < km; ++a) {
        for (int side = 0; side < (sym ? 1 : 2); ++side) {
          const Csr& M = side == 0 ? L.A : At;
          const int g = sides.count++;
          sides.rowptr[g] = M.rowptr;
          sides.col[g] = M.col;
          sides.val[g] = M.val;
          sides.x[g] = (side == 0 ? L.B_P : L.B_R) + (size_t)a * n;
          sides.y[g] = tmps + (size_t)g * n;
        }
      }
      smooth_modes_sides(sides, n, (double)L.A.nnz / n, batch ? wd : L.dinv, L.cf,
                         batch ? nullptr : om_k, 1.0, p.b_smooth_iters, ss.s2);
      if (sym)
        for (int a = 0; a < km; ++a)
          CLAIR_CUDA(cudaMemcpyAsync(L.B_R + (size_t)a * n, L.B_P + (size_t)a * n,
                                     sizeof(double) * n, cudaMemcpyDeviceToDevice, ss.s2));
      dfree(tmps, ss.s2);
      dfree(wd, ss.s2);
    }
    CLAIR_CUDA(cudaEventRecord(ss.join, ss.s2));
    {
      ClockScope clk(PH_PATTERN, s);
      // both patterns' entry counts in one host read
      PatternJob* jobs[2];
      Csr* zs[2];
      int nj = 0;
      if (!sym) {
        pattern_scan(jobR, L.R, s);
        jobs[nj] = &jobR;
        zs[nj++] = &L.R;
      }
      pattern_scan(jobP, Pt, s);
      jobs[nj] = &jobP;
      zs[nj++] = &Pt;
      pattern_read(jobs, zs, nj, s);
      if (!sym) pattern_build(jobR, L.R, s);
      pattern_build(jobP, Pt, s);
      dfree(Mrp, s);
      dfree(Mcol, s);
      dfree(agg, s);
    }
    if (p.inverse == CLAIR_INVERSE_EXACT) {
      // exact block inverses: the local solves need no mode vector and overlap the smoothing
      if (sym)
        transfer_solve(L.A, L.cpts, Pt, p.precision, h->st, s);
      else
        transfer_solve_pair(At, L.R, L.A, Pt, L.cpts, p.precision, h->st, s);
      CLAIR_CUDA(cudaStreamWaitEvent(s, ss.join, 0));
      if (!sym) transfer_project(L.cf, L.cpts, L.R, L.B_R, km, h->st, nullptr, s);
      transfer_project(L.cf, L.cpts, Pt, L.B_P, km, h->st, &L.P, s);
    } else {
      // diagonal block inverses: every pass of Algorithm 1's loop projects (needs B)
      CLAIR_CUDA(cudaStreamWaitEvent(s, ss.join, 0));
      if (!sym) transfer_diag(At, L.cf, L.cpts, L.R, L.B_R, km, p.iterations, h->st, nullptr, s);
      transfer_diag(L.A, L.cf, L.cpts, Pt, L.B_P, km, p.iterations, h->st, &L.P, s);
    }
    if (sym)
      L.R = Pt;  // R = P^T: the coarse-row form of P is R
    else
      Pt.release(s);
    dfree(rmaxA, s);
    dfree(rmaxAt, s);
    dfree(sA, s);
    dfree(sAt, s);
    dfree(sR, s);
    dfree(sP, s);
    At.release(s);
    // Galerkin coarse operator A_c = (R A) P
    Csr RA, Ac;
    ClockScope clk(PH_GALERKIN, s);
    spgemm(L.R, L.A, RA, s);
    spgemm(RA, L.P, Ac, s);
    RA.release(s);
    drop_zeros(Ac, s);  // exact cancellations leave no stored zeros
    Level C;
    C.A = Ac;
    C.n = Ac.rows;
    C.B_P = dalloc<double>((size_t)C.n * km, s);
    C.B_R = dalloc<double>((size_t)C.n * km, s);
    if (C.n) {
      for (int a = 0; a < km; ++a) {
        inject<<<ceil_div(C.n, 256), 256, 0, s>>>(L.B_P + (size_t)a * n, L.cpts, C.n,
                                                  C.B_P + (size_t)a * C.n); ::clair::count_launch();
        inject<<<ceil_div(C.n, 256), 256, 0, s>>>(L.B_R + (size_t)a * n, L.cpts, C.n,
                                                  C.B_R + (size_t)a * C.n); ::clair::count_launch();
      }
    }
    CLAIR_LAUNCHED();
    if (batch) {
      C.off.assign(ninst + 1, 0);
      for (int i = 0; i < ninst; ++i) C.off[i + 1] = C.off[i] + cnt[i];
      C.frozen = L.frozen;
    }
    h->lv.push_back(C);
  }
  // the last level's weight chain may still run on s2 (a level that turned out to be the
  // coarsest after its splitting)
  CLAIR_CUDA(cudaEventRecord(ss.join, ss.s2));
  CLAIR_CUDA(cudaStreamWaitEvent(s, ss.join, 0));
  marks.record(s);
  if (active_clock()) active_clock()->set_level((int)h->lv.size() - 1);
  ClockScope clk(PH_COARSE, s);
  // MIXED: the smoothed mode vectors of nearly pure advection shrink by orders of
  // magnitude per level, and the projected weights grow in proportion (1e13 seen); an FP32
  // copy of such R and P loses everything to cancellation.  From the first level whose
  // largest |R| or |P| weight exceeds kCycle64Weight on, the cycle runs in FP64.  The
  // maxima, the weights and the coarse diagonal check come back in one read.
  const int nl = (int)h->lv.size();
  unsigned long long* wmax = dalloc<unsigned long long>(nl, s);
  CLAIR_CUDA(cudaMemsetAsync(wmax, 0, sizeof(unsigned long long) * nl, s));
  {
    SegBatch mx(s, wmax);
    for (int k = 0; k < nl; ++k) {
      Level& L = h->lv[k];
      if (!L.nc) continue;
      mx.add(L.R.val, nullptr, L.R.nnz, k);
      mx.add(L.P.val, nullptr, L.P.nnz, k);
    }
    mx.flush();
  }
  {
    std::vector<double> om((size_t)p.max_levels * ninst, 1.0);
    std::vector<unsigned long long> hw(nl);
    int nbad = 0;
    CLAIR_CUDA(cudaMemcpyAsync(om.data(), omega_dev, sizeof(double) * om.size(),
                               cudaMemcpyDeviceToHost, s));
    CLAIR_CUDA(cudaMemcpyAsync(&nbad, bad_coarse, sizeof(int), cudaMemcpyDeviceToHost, s));
    CLAIR_CUDA(cudaMemcpyAsync(hw.data(), wmax, sizeof(unsigned long long) * nl,
                               cudaMemcpyDeviceToHost, s));
    CLAIR_CUDA(cudaStreamSynchronize(s));
    dfree(bad_coarse, s);
    dfree(wmax, s);
    CLAIR_REQUIRE(nbad == 0, CLAIR_ERR_ARG,
                  "%d coarse rows with a missing, zero or nonfinite diagonal", nbad);
    for (size_t k = 0; k + 1 < marks.v.size() && k < 32; ++k) {
      float ms = 0.f;
      CLAIR_CUDA(cudaEventElapsedTime(&ms, marks.v[k], marks.v[k + 1]));
      h->level_span_ms[k] = ms;
    }
    for (size_t k = 0; k < h->lv.size(); ++k) {
      Level& L = h->lv[k];
      if (!L.nc) continue;
      L.omega = om[k * ninst];
      if (batch) L.omega_inst.assign(om.begin() + k * ninst, om.begin() + (k + 1) * ninst);
    }
    bool on = false;
    for (int k = 0; k < nl; ++k) {
      double w;
      memcpy(&w, &hw[k], sizeof(w));
      h->lv[k].max_weight = w;
      on = on || (p.precision == CLAIR_MIXED && w > kCycle64Weight);
      h->lv[k].cycle64 = on;
    }
  }
  dfree(omega_dev, s);
  // coarsest level: dense inverse; float copies and work vectors everywhere
  Level& last = h->lv.back();
  h->nL = last.n;
  // coarsest level: one dense block, or each instance's diagonal block of a batch
  std::vector<int> blocks = batch ? last.off : std::vector<int>{0, last.n};
  long long inv_size = 0;
  for (size_t i = 0; i + 1 < blocks.size(); ++i) {
    const long long ni = blocks[i + 1] - blocks[i];
    CLAIR_REQUIRE(ni <= 1024, CLAIR_ERR_CAPACITY,
                  "coarsest level has a block of %lld unknowns (> 1024): raise max_levels", ni);
    inv_size += ni * ni;
  }
  h->coarse_nblk = (int)blocks.size() - 1;
  h->Inv = dalloc<double>(std::max<long long>(inv_size, 1), s);
  dense_inverse(last.A, blocks, h->Inv, &h->coarse_off, &h->coarse_ioff, s);
  SegBatch conv(s);
  auto to_float_later = [&](const double* x, float** y, long long n) {
    *y = dalloc<float>(n, s);
    conv.add(x, *y, n);
  };
  to_float_later(h->Inv, &h->Inv32, std::max<long long>(inv_size, 1));
  for (auto& L : h->lv) {
    to_float_later(L.A.val, &L.A.val32, L.A.nnz);
    to_float_later(L.dinv, &L.dinv32, L.n);
    if (L.nc) {
      to_float_later(L.R.val, &L.R.val32, L.R.nnz);
      to_float_later(L.P.val, &L.P.val32, L.P.nnz);
    }
  }
  conv.flush();
  for (auto& L : h->lv) {
    if (L.nc && batch) batch_cycle_weights(L, p.post_weighted != 0, s);
    alloc_cycle(L, s);
  }
}

// --- V(1,1) cycle ---------------------------------------------------------------------
template <class T>
struct Vec {
  static T* b(Level& L);
  static T* x(Level& L);
  static T* y(Level& L);
  static T* r(Level& L);
  static const T* aval(const Csr& M);
  static const T* dinv(const Level& L);
  static const T* wpre(const Level& L);
  static const T* wpost(const Level& L);
};
template <>
struct Vec<double> {
  static double* b(Level& L) { return L.b64; }
  static double* x(Level& L) { return L.x64; }
  static double* y(Level& L) { return L.y64; }
  static double* r(Level& L) { return L.r64; }
  static const double* aval(const Csr& M) { return M.val; }
  static const double* dinv(const Level& L) { return L.dinv; }
  static const double* wpre(const Level& L) { return L.wpre64; }
  static const double* wpost(const Level& L) { return L.wpost64; }
};
template <>
struct Vec<float> {
  static float* b(Level& L) { return L.b32; }
  static float* x(Level& L) { return L.x32; }
  static float* y(Level& L) { return L.y32; }
  static float* r(Level& L) { return L.r32; }
  static const float* aval(const Csr& M) { return M.val32; }
  static const float* dinv(const Level& L) { return L.dinv32; }
  static const float* wpre(const Level& L) { return L.wpre32; }
  static const float* wpost(const Level& L) { return L.wpost32; }
};

template <class T>
static void spmv_t(const Csr& A, const T* x, T* y, T alpha, T beta, cudaStream_t s);
template <>
void spmv_t<double>(const Csr& A, const double* x, double* y, double a, double b, cudaStream_t s) {
  spmv(A, x, y, a, b, s);
}
template <>
void spmv_t<float>(const Csr& A, const float* x, float* y, float a, float b, cudaStream_t s) {
  spmv32(A, x, y, a, b, s);
}
template <class T>
static void residual_t(const Csr& A, const T* b, const T* x, T* r, cudaStream_t s);
template <>
void residual_t<double>(const Csr& A, const double* b, const double* x, double* r, cudaStream_t s) {
  residual(A, b, x, r, s);
}
template <>
void residual_t<float>(const Csr& A, const float* b, const float* x, float* r, cudaStream_t s) {
  residual32(A, b, x, r, s);
}

// Cycle on level k: input in Vec<T>::b(L_k); returns where the output is (Vec<T>::x or
// Vec<T>::y of L_k: the last post-smoothing sweep writes the other buffer, no copy back).
// vcycle_pre is the CFF pre-smoothing from x = 0, vcycle_post the rest (on the coarsest
// level, its solve): the fine level's two halves are captured as graphs of their own.
template <class T>
static T* vcycle_level(clair_hierarchy* h, int k);

template <class T>
static void vcycle_pre(clair_hierarchy* h, int k) {
  if (k == (int)h->lv.size() - 1) return;
  cudaStream_t s = h->stream;
  Level& L = h->lv[k];
  T* b = Vec<T>::b(L);
  T* x = Vec<T>::x(L);
  T* y = Vec<T>::y(L);
  const T* av = Vec<T>::aval(L.A);
  // a batch folds each instance's weight into D^-1 (0 for frozen instances)
  const bool batch = h->ninst > 1;
  const T* dv = batch ? Vec<T>::wpre(L) : Vec<T>::dinv(L);
  const T w = batch ? T(1) : (T)L.omega;
  jacobi_from_zero<T>(L.n, dv, L.cf, 1, w, b, x, s);
  jacobi<T>(L.A, av, dv, L.cf, 0, w, b, x, y, s);
  jacobi<T>(L.A, av, dv, L.cf, 0, w, b, y, x, s);
}

template <class T>
static T* vcycle_post(clair_hierarchy* h, int k) {
  cudaStream_t s = h->stream;
  Level& L = h->lv[k];
  T* b = Vec<T>::b(L);
  T* x = Vec<T>::x(L);
  T* y = Vec<T>::y(L);
  if (k == (int)h->lv.size() - 1) {
    const T* Inv = nullptr;
    if constexpr (sizeof(T) == 8)
      Inv = reinterpret_cast<const T*>(h->Inv);
    else
      Inv = reinterpret_cast<const T*>(h->Inv32);
    coarse_apply<T>(Inv, h->coarse_off, h->coarse_ioff, h->coarse_nblk, L.n, b, x, s);
    return x;
  }
  const T* av = Vec<T>::aval(L.A);
  const bool batch = h->ninst > 1;
  const T* dvpost = batch ? Vec<T>::wpost(L) : Vec<T>::dinv(L);
  const T w = batch ? T(1) : (T)L.omega;
  const T wpost = batch ? T(1) : (h->p.post_weighted ? w : T(1));
  // residual, restriction, coarse cycle, interpolation
  T* r = Vec<T>::r(L);
  residual_t<T>(L.A, b, x, r, s);
  Level& C = h->lv[k + 1];
  spmv_t<T>(L.R, r, Vec<T>::b(C), T(1), T(0), s);
  const T* xc = nullptr;
  if constexpr (sizeof(T) == 4) {
    if (C.cycle64) {  // the coarser levels run in FP64 (MIXED with large weights there)
      to_double(C.b32, C.b64, C.n, s);
      const double* xc64 = vcycle_level<double>(h, k + 1);
      to_float(xc64, C.x32, C.n, s);
      xc = C.x32;
    }
  }
  if (!xc) xc = vcycle_level<T>(h, k + 1);
  spmv_t<T>(L.P, xc, x, T(1), T(1), s);
  // FFC post-smoothing
  jacobi<T>(L.A, av, dvpost, L.cf, 0, wpost, b, x, y, s);
  jacobi<T>(L.A, av, dvpost, L.cf, 0, wpost, b, y, x, s);
  jacobi<T>(L.A, av, dvpost, L.cf, 1, wpost, b, x, y, s);
  return y;
}

template <class T>
static T* vcycle_level(clair_hierarchy* h, int k) {
  vcycle_pre<T>(h, k);
  return vcycle_post<T>(h, k);
}

// z = M^-1 v on level k (float64 in and out), launching every kernel: the input's
// conversion and the pre-smoothing (head), then the rest of the cycle and the output's
// conversion (tail).
static bool precond_fp32(const clair_hierarchy* h, const Level& L) {
  return h->p.precision == CLAIR_MIXED && !h->cycle_fp64 && !L.cycle64;
}
static void precond_head(clair_hierarchy* h, int k, const double* v) {
  Level& L = h->lv[k];
  if (precond_fp32(h, L)) {
    to_float(v, L.b32, L.n, h->stream);
    vcycle_pre<float>(h, k);
  } else {
    copy_f64(v, L.b64, L.n, h->stream);
    vcycle_pre<double>(h, k);
  }
}
static void precond_tail(clair_hierarchy* h, int k, double* z) {
  Level& L = h->lv[k];
  if (precond_fp32(h, L)) {
    const float* out = vcycle_post<float>(h, k);
    to_double(out, z, L.n, h->stream);
  } else {
    const double* out = vcycle_post<double>(h, k);
    copy_f64(out, z, L.n, h->stream);
  }
}
struct LanesScope {  // the hierarchy's row-kernel lane rule for these launches
  int keep;
  explicit LanesScope(int w) : keep(cycle_short_lanes()) { set_cycle_short_lanes(w); }
  ~LanesScope() { set_cycle_short_lanes(keep); }
};
static void apply_precond_direct(clair_hierarchy* h, int k, const double* v, double* z) {
  LanesScope lanes(h->short_lanes);
  precond_head(h, k, v);
  precond_tail(h, k, z);
}

// The fine-level cycle is a fixed sequence of about ten kernels per level; it is captured
// once, with fixed input / output buffers (h->vin, h->zout), into two CUDA graphs that
// are replayed: the head (input conversion and the fine level's pre-smoothing, four
// kernels) and the tail (the rest).  The host's launch of the long tail then overlaps the
// head's execution instead of delaying the cycle's first kernel.  In MIXED precision the
// cycle is captured with each lane rule for short FP32 rows, the replays of each are
// timed, and the fastest is kept.
static cudaGraphExec_t capture_part(clair_hierarchy* h, cudaStream_t cs, bool head) {
  cudaGraph_t g = nullptr;
  cudaGraphExec_t exec = nullptr;
  struct PdlScope {  // the captured kernels chain by programmatic dependence
    PdlScope() { set_pdl_launches(true); }
    ~PdlScope() { set_pdl_launches(false); }
  };
  try {
    CLAIR_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    {
      PdlScope pdl;
      LanesScope lanes(h->short_lanes);
      if (head)
        precond_head(h, 0, h->vin);
      else
        precond_tail(h, 0, h->zout);
    }
    CLAIR_CUDA(cudaStreamEndCapture(cs, &g));
    CLAIR_CUDA(cudaGraphInstantiate(&exec, g, 0));
  } catch (...) {
    cudaGraph_t dummy;
    cudaStreamEndCapture(cs, &dummy);
    if (g) cudaGraphDestroy(g);
    throw;
  }
  cudaGraphDestroy(g);
  return exec;
}

static CycleGraph capture_cycle(clair_hierarchy* h) {
  cudaStream_t cs;
  CLAIR_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaStream_t keep = h->stream;
  h->stream = cs;
  const long long before = launch_count();
  CycleGraph c;
  try {
    c.head = capture_part(h, cs, true);
    c.tail = capture_part(h, cs, false);
  } catch (...) {
    destroy_cycle(c);
    h->stream = keep;
    cudaStreamDestroy(cs);
    throw;
  }
  c.kernels = launch_count() - before;
  count_launches(-c.kernels);  // captured, not launched
  h->stream = keep;
  cudaStreamDestroy(cs);
  return c;
}

static void launch_cycle(const CycleGraph& c, cudaStream_t s) {
  CLAIR_CUDA(cudaGraphLaunch(c.head, s));
  CLAIR_CUDA(cudaGraphLaunch(c.tail, s));
}

static float time_cycle(const CycleGraph& c, cudaStream_t s) {
  cudaEvent_t e0, e1;
  CLAIR_CUDA(cudaEventCreate(&e0));
  CLAIR_CUDA(cudaEventCreate(&e1));
  launch_cycle(c, s);  // warm
  CLAIR_CUDA(cudaEventRecord(e0, s));
  for (int i = 0; i < 3; ++i) launch_cycle(c, s);
  CLAIR_CUDA(cudaEventRecord(e1, s));
  CLAIR_CUDA(cudaEventSynchronize(e1));
  float ms = 0.f;
  CLAIR_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return ms;
}

// The lane rule chosen by the first timed MIXED cycle on each device (-1: not yet timed).
static std::mutex g_lanes_mu;
static int g_lanes_pick[256] = {-1};
static bool g_lanes_init = false;

static int* lanes_slot() {
  int dev = 0;
  CLAIR_CUDA(cudaGetDevice(&dev));
  CLAIR_REQUIRE(dev >= 0 && dev < 256, CLAIR_ERR_ARG, "device ordinal %d out of range", dev);
  if (!g_lanes_init) {
    for (int& v : g_lanes_pick) v = -1;
    g_lanes_init = true;
  }
  return &g_lanes_pick[dev];
}

static void build_cycle_graph(clair_hierarchy* h) {
  if (h->p.precision != CLAIR_MIXED) {
    h->short_lanes = 0;
    h->cycle = capture_cycle(h);
    h->cycle_lanes_pick = 0;
    return;
  }
  {
    std::lock_guard<std::mutex> lock(g_lanes_mu);
    const int known = *lanes_slot();
    if (known >= 0) {  // timed once per device: capture the chosen rule only
      h->short_lanes = h->cycle_lanes_pick = known;
      h->cycle = capture_cycle(h);
      return;
    }
  }
  CLAIR_CUDA(cudaMemsetAsync(h->vin, 0, sizeof(double) * h->lv[0].n, h->stream));
  CycleGraph best;
  float best_ms = 0.f;
  for (int lanes = 0; lanes <= 2; ++lanes) {
    h->short_lanes = lanes;
    CycleGraph e = capture_cycle(h);
    float ms = 0.f;
    try {
      ms = time_cycle(e, h->stream);
      count_launches(4 * e.kernels);
    } catch (...) {
      destroy_cycle(e);
      destroy_cycle(best);
      throw;
    }
    if (!best.head || ms < best_ms) {
      destroy_cycle(best);
      best = e;
      best_ms = ms;
      h->cycle_lanes_pick = lanes;
    } else {
      destroy_cycle(e);
    }
  }
  h->short_lanes = h->cycle_lanes_pick;
  h->cycle = best;
  std::lock_guard<std::mutex> lock(g_lanes_mu);
  *lanes_slot() = h->cycle_lanes_pick;
}

// z = M^-1 v on level k; the fine level replays the captured cycle.
static void apply_precond(clair_hierarchy* h, int k, const double* v, double* z) {
  if (k != 0 || !h->cycle.head || h->cycle_fp64) {
    apply_precond_direct(h, k, v, z);
    return;
  }
  cudaStream_t s = h->stream;
  const size_t bytes = sizeof(double) * h->lv[0].n;
  CLAIR_CUDA(cudaMemcpyAsync(h->vin, v, bytes, cudaMemcpyDeviceToDevice, s));
  launch_cycle(h->cycle, s);
  for (long long i = 0; i < h->cycle.kernels; ++i) count_launch();
  CLAIR_CUDA(cudaMemcpyAsync(z, h->zout, bytes, cudaMemcpyDeviceToDevice, s));
}

// --- Krylov solvers ---------------------------------------------------------------------
static void ensure_krylov(clair_hierarchy* h, int nrhs) {
  cudaStream_t s = h->stream;
  Krylov& k = h->kr;
  const int n = h->lv[0].n, m = h->p.gmres_restart;
  if (k.V && k.nrhs == nrhs && k.m == m && k.n == n) return;
  release_krylov(k, s);
  k.nrhs = nrhs;
  k.m = m;
  k.n = n;
  k.N = (long long)nrhs * n;
  const std::vector<int> off = h->ninst > 1 ? h->lv[0].off : std::vector<int>{0, n};
  k.S.build(nrhs, off, s);
  const long long N = k.N;
  const int nseg = k.S.nseg;
  k.V = dalloc<double>((size_t)std::max(m + 1, 3) * N, s);  // CG keeps z, p, q in V
  k.Z = dalloc<double>((size_t)m * N, s);
  k.w = dalloc<double>(N, s);
  k.r = dalloc<double>(N, s);
  k.H = dalloc<double>((size_t)nseg * m * (m + 1), s);
  k.cs = dalloc<double>((size_t)nseg * m, s);
  k.sn = dalloc<double>((size_t)nseg * m, s);
  k.g = dalloc<double>((size_t)nseg * (m + 1), s);
  k.y = dalloc<double>((size_t)nseg * m, s);
  k.h1 = dalloc<double>((size_t)nseg * (m + 1), s);
  k.h2 = dalloc<double>((size_t)nseg * (m + 1), s);
  k.partial = dalloc<double>((size_t)(m + 1) * std::max(k.S.nchunk, 1), s);
  for (double** p : {&k.fn2, &k.fnorm, &k.tol, &k.beta2, &k.wn2, &k.inv})
    *p = dalloc<double>(nseg, s);
  k.cg = dalloc<double>((size_t)8 * nseg, s);
  k.summary = dalloc<double>(4, s);
  k.active = dalloc<int>(nseg, s);
  k.jend = dalloc<int>(nseg, s);
  k.its = dalloc<int>(nseg, s);
  k.host = static_cast<double*>(pinned_get(sizeof(double) * 4));
}

// (number of active segments, largest residual / tolerance among them)
static void read_summary(clair_hierarchy* h, double* active, double* ratio) {
  CLAIR_CUDA(cudaMemcpyAsync(h->kr.host, h->kr.summary, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                             h->stream));
  CLAIR_CUDA(cudaStreamSynchronize(h->stream));
  *active = h->kr.host[0];
  *ratio = h->kr.host[1];
}

// Z = M^-1 V (every right-hand side), W = A X (every right-hand side), R = F - A U
static void precond_all(clair_hierarchy* h, const double* v, double* z) {
  const Krylov& k = h->kr;
  for (int r = 0; r < k.nrhs; ++r) apply_precond(h, 0, v + (size_t)r * k.n, z + (size_t)r * k.n);
}
static void matvec_all(clair_hierarchy* h, const double* x, double* y) {
  const Krylov& k = h->kr;
  for (int r = 0; r < k.nrhs; ++r)
    spmv(h->lv[0].A, x + (size_t)r * k.n, y + (size_t)r * k.n, 1.0, 0.0, h->stream);
}
static void residual_all(clair_hierarchy* h, const double* f, const double* u, double* r) {
  const Krylov& k = h->kr;
  for (int q = 0; q < k.nrhs; ++q)
    residual(h->lv[0].A, f + (size_t)q * k.n, u + (size_t)q * k.n, r + (size_t)q * k.n, h->stream);
}

// Per-segment results of the finished solve into the hierarchy (host).
static bool finish_segments(clair_hierarchy* h) {
  cudaStream_t s = h->stream;
  Krylov& k = h->kr;
  const int nseg = k.S.nseg;
  std::vector<double> b2(nseg), fn(nseg), tl(nseg);
  h->last_its.assign(nseg, 0);
  CLAIR_CUDA(cudaMemcpyAsync(b2.data(), k.beta2, sizeof(double) * nseg, cudaMemcpyDeviceToHost, s));
  CLAIR_CUDA(cudaMemcpyAsync(fn.data(), k.fnorm, sizeof(double) * nseg, cudaMemcpyDeviceToHost, s));
  CLAIR_CUDA(cudaMemcpyAsync(tl.data(), k.tol, sizeof(double) * nseg, cudaMemcpyDeviceToHost, s));
  CLAIR_CUDA(cudaMemcpyAsync(h->last_its.data(), k.its, sizeof(int) * nseg, cudaMemcpyDeviceToHost, s));
  CLAIR_CUDA(cudaStreamSynchronize(s));
  h->last_rel.assign(nseg, 0.0);
  bool ok = true;
  for (int i = 0; i < nseg; ++i) {
    const double b = sqrt(b2[i]);
    h->last_rel[i] = fn[i] > 0.0 ? b / fn[i] : 0.0;
    if (b > tl[i]) ok = false;
  }
  return ok;
}

// MIXED policy: the FP32 cycle carries ~7 digits; where the hierarchy's weights span more
// than that (near-pure advection after mode smoothing) it stops reducing the residual.  A
// restart cycle that ends unconverged, stalls (less than 2x gain in the worst active
// segment's residual estimate over 10 iterations; its directions are kept: it is still a
// valid flexible preconditioner) or produces a nonfinite estimate (that cycle is
// discarded) hands the rest of the solve to the FP64 cycle of the same hierarchy.
constexpr int kStallWindow = 10;

// Right-preconditioned FGMRES(m) per segment, float64; stops each segment on its true
// residual ||f_s - A u_s|| <= rtol ||f_s|| (restarts act as iterative refinement).
static bool fgmres(clair_hierarchy* h, const double* f, double* u) {
  cudaStream_t s = h->stream;
  Krylov& k = h->kr;
  const Segments& S = k.S;
  const int m = k.m, nseg = S.nseg;
  const long long N = k.N;
  const bool mixed = h->p.precision == CLAIR_MIXED;
  seg_dot(S, f, 0, 1, f, k.fn2, 1, k.partial, s);
  seg_tolerance_launch(S, k.fn2, h->p.rtol, k.tol, k.fnorm, u, s);
  CLAIR_CUDA(cudaMemsetAsync(k.its, 0, sizeof(int) * nseg, s));
  residual_all(h, f, u, k.r);
  seg_dot(S, k.r, 0, 1, k.r, k.beta2, 1, k.partial, s);
  seg_gmres_start_launch(nseg, m, k.beta2, k.tol, k.g, k.inv, k.active, k.jend, k.summary, s);
  double nact = 0, ratio = 0;
  read_summary(h, &nact, &ratio);
  CLAIR_REQUIRE(isfinite(ratio), CLAIR_ERR_NONFINITE, "nonfinite initial residual");
  int its = 0;
  std::vector<double> hist;
  while (nact > 0 && its < h->p.gmres_maxit) {
    seg_scale(S, k.r, k.inv, 1, k.V, s);
    int jmax = 0;
    bool discarded = false, stalled = false;
    hist.clear();
    for (int j = 0; j < m; ++j) {
      double* vj = k.V + (size_t)j * N;
      double* zj = k.Z + (size_t)j * N;
      {
        ClockScope clk(PH_VCYCLE, s);
        precond_all(h, vj, zj);
      }
      ClockScope clk(PH_KRYLOV, s);
      matvec_all(h, zj, k.w);
      seg_dot(S, k.V, N, j + 1, k.w, k.h1, m + 1, k.partial, s);
      seg_axpy(S, k.V, N, j + 1, k.h1, m + 1, k.w, s);
      seg_dot(S, k.V, N, j + 1, k.w, k.h2, m + 1, k.partial, s);
      seg_axpy(S, k.V, N, j + 1, k.h2, m + 1, k.w, s);
      seg_dot(S, k.w, 0, 1, k.w, k.wn2, 1, k.partial, s);
      seg_gmres_givens_launch(nseg, m, j, k.h1, k.h2, m + 1, k.wn2, k.H, k.cs, k.sn, k.g, k.inv,
                              k.active, k.jend, k.its, k.tol, k.summary, s);
      seg_scale(S, k.w, k.inv, 1, k.V + (size_t)(j + 1) * N, s);
      ++its;
      jmax = j + 1;
      read_summary(h, &nact, &ratio);
      if (!isfinite(ratio) && mixed && !h->cycle_fp64) {
        CLAIR_CUDA(cudaMemsetAsync(k.jend, 0, sizeof(int) * nseg, s));  // discard the cycle
        discarded = true;
        break;
      }
      CLAIR_REQUIRE(isfinite(ratio), CLAIR_ERR_NONFINITE, "nonfinite residual estimate");
      if (nact == 0 || its >= h->p.gmres_maxit) break;
      hist.push_back(ratio);
      if (mixed && !h->cycle_fp64 && (int)hist.size() > kStallWindow &&
          ratio > 0.5 * hist[hist.size() - 1 - kStallWindow]) {
        stalled = true;
        break;
      }
    }
    {
      ClockScope clk(PH_KRYLOV, s);
      seg_gmres_backsolve_launch(nseg, m, k.H, k.g, k.jend, k.y, s);
      seg_axpy(S, k.Z, N, jmax, k.y, m, u, s);
      residual_all(h, f, u, k.r);
      seg_dot(S, k.r, 0, 1, k.r, k.beta2, 1, k.partial, s);
      seg_gmres_start_launch(nseg, m, k.beta2, k.tol, k.g, k.inv, k.active, k.jend, k.summary, s);
    }
    read_summary(h, &nact, &ratio);
    CLAIR_REQUIRE(isfinite(ratio), CLAIR_ERR_NONFINITE, "nonfinite residual");
    // (a cycle that stopped on its estimates but not on the true residuals is iterative
    // refinement, and stays in FP32)
    if (nact > 0 && mixed && !h->cycle_fp64 && (discarded || stalled || jmax == m)) {
      h->cycle_fp64 = true;
      h->fp64_from = its;
    }
  }
  return finish_segments(h);
}

// Preconditioned CG per segment (the symmetric case, R = P^T: the V(1,1) cycle with CFF
// pre- and FFC post-smoothing and equal weights is then a symmetric preconditioner).  The
// recursive residual decides convergence; the true residual is checked at the end and a
// segment that misses it restarts from its current iterate.
static bool pcg(clair_hierarchy* h, const double* f, double* u) {
  cudaStream_t s = h->stream;
  Krylov& k = h->kr;
  const Segments& S = k.S;
  const int nseg = S.nseg;
  const long long N = k.N;
  const bool mixed = h->p.precision == CLAIR_MIXED;
  double* zv = k.V;            // M^-1 r
  double* pv = k.V + N;        // search direction
  double* qv = k.V + 2 * N;    // A p
  double* rho = k.cg;
  double* rz = k.cg + nseg;
  double* pq = k.cg + 2 * nseg;
  double* alpha = k.cg + 3 * nseg;
  double* malpha = k.cg + 4 * nseg;
  double* beta = k.cg + 5 * nseg;
  seg_dot(S, f, 0, 1, f, k.fn2, 1, k.partial, s);
  seg_tolerance_launch(S, k.fn2, h->p.rtol, k.tol, k.fnorm, u, s);
  CLAIR_CUDA(cudaMemsetAsync(k.its, 0, sizeof(int) * nseg, s));
  int its = 0;
  double nact = 0, ratio = 0;
  for (;;) {
    residual_all(h, f, u, k.r);
    seg_dot(S, k.r, 0, 1, k.r, k.beta2, 1, k.partial, s);
    {
      ClockScope clk(PH_VCYCLE, s);
      precond_all(h, k.r, zv);
    }
    seg_dot(S, k.r, 0, 1, zv, rz, 1, k.partial, s);
    seg_cg_start_launch(nseg, k.beta2, k.tol, rz, rho, k.active, k.summary, s);
    CLAIR_CUDA(cudaMemcpyAsync(pv, zv, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
    read_summary(h, &nact, &ratio);
    CLAIR_REQUIRE(isfinite(ratio), CLAIR_ERR_NONFINITE, "nonfinite residual");
    if (nact == 0 || its >= h->p.gmres_maxit) break;
    std::vector<double> hist;
    bool stalled = false;
    while (nact > 0 && its < h->p.gmres_maxit) {
      {
        ClockScope clk(PH_KRYLOV, s);
        matvec_all(h, pv, qv);
        seg_dot(S, pv, 0, 1, qv, pq, 1, k.partial, s);
        seg_cg_alpha_launch(nseg, rho, pq, k.active, alpha, malpha, s);
        seg_axpy1(S, pv, alpha, u, s);
        seg_axpy1(S, qv, malpha, k.r, s);
        seg_dot(S, k.r, 0, 1, k.r, k.wn2, 1, k.partial, s);
      }
      {
        ClockScope clk(PH_VCYCLE, s);
        precond_all(h, k.r, zv);
      }
      {
        ClockScope clk(PH_KRYLOV, s);
        seg_dot(S, k.r, 0, 1, zv, rz, 1, k.partial, s);
        seg_cg_beta_launch(nseg, k.wn2, k.tol, rz, rho, k.active, k.its, beta, k.summary, s);
        seg_xpby(S, zv, beta, pv, s);
      }
      ++its;
      read_summary(h, &nact, &ratio);
      CLAIR_REQUIRE(isfinite(ratio), CLAIR_ERR_NONFINITE, "nonfinite CG residual");
      hist.push_back(ratio);
      if (mixed && !h->cycle_fp64 && (int)hist.size() > kStallWindow &&
          ratio > 0.5 * hist[hist.size() - 1 - kStallWindow]) {
        stalled = true;
        break;
      }
    }
    if (stalled) {
      h->cycle_fp64 = true;
      h->fp64_from = its;
    }
  }
  return finish_segments(h);
}

static bool krylov_solve(clair_hierarchy* h, int nrhs, const double* f, double* u) {
  ensure_krylov(h, nrhs);
  h->cycle_fp64 = false;
  h->fp64_from = -1;
  return h->p.krylov == CLAIR_KRYLOV_PCG ? pcg(h, f, u) : fgmres(h, f, u);
}

}  // namespace clair

// =======================================================================================
// C ABI
// =======================================================================================
using namespace clair;

extern "C" {

clair_status clair_params_default(clair_params* p) {
  if (!p) {
    set_error("clair_params_default: null pointer");
    return CLAIR_ERR_ARG;
  }
  p->theta_coarsen = 0.25;
  p->theta_interp = 0.05;
  p->degree = 2;
  p->coarsen = CLAIR_COARSEN_FC;
  p->b_smooth_iters = 5;
  p->arnoldi_iters = 15;
  p->post_weighted = 0;
  p->coarse_max = 128;
  p->max_levels = 25;
  p->precision = CLAIR_FP64;
  p->gmres_restart = 50;
  p->gmres_maxit = 200;
  p->rtol = 1e-8;
  p->seed = 0x5EED;
  p->inverse = CLAIR_INVERSE_EXACT;
  p->iterations = 1;
  p->symmetric = 0;
  p->krylov = CLAIR_KRYLOV_FGMRES;
  return CLAIR_OK;
}

const char* clair_last_error(void) { return last_error(); }

static clair_status setup_common(int ninst, const int* offsets_host, int n, int nnz,
                                 const int* rowptr, const int* col, const double* val, int kmodes,
                                 const double* B, const signed char* cf_marker,
                                 const clair_params* pin, void* stream, clair_h* out) {
  if (out) *out = nullptr;
  CLAIR_API_BEGIN
  CLAIR_REQUIRE(out && rowptr && col && val && B, CLAIR_ERR_ARG, "clair_setup: null pointer");
  CLAIR_REQUIRE(n > 0 && nnz >= n, CLAIR_ERR_ARG, "clair_setup: bad sizes n=%d nnz=%d", n, nnz);
  clair_params p;
  if (pin)
    p = *pin;
  else
    clair_params_default(&p);
  CLAIR_REQUIRE(p.gmres_restart >= 1 && p.gmres_restart <= 64, CLAIR_ERR_ARG,
                "gmres_restart must be in [1, 64]");
  CLAIR_REQUIRE(p.precision == CLAIR_FP64 || p.precision == CLAIR_MIXED, CLAIR_ERR_ARG,
                "unknown precision");
  CLAIR_REQUIRE(p.max_levels >= 1 && p.max_levels <= 32, CLAIR_ERR_ARG, "max_levels in [1,32]");
  CLAIR_REQUIRE(p.coarse_max >= 1 && p.coarse_max <= 1024, CLAIR_ERR_ARG,
                "coarse_max in [1, 1024]");
  CLAIR_REQUIRE(p.arnoldi_iters >= 1 && p.arnoldi_iters <= 60, CLAIR_ERR_ARG,
                "arnoldi_iters in [1, 60]");
  CLAIR_REQUIRE(p.degree == 1 || p.degree == 2, CLAIR_ERR_UNSUPPORTED, "degree must be 1 or 2");
  CLAIR_REQUIRE(p.coarsen == CLAIR_COARSEN_FC || p.coarsen == CLAIR_COARSEN_AGG, CLAIR_ERR_ARG,
                "unknown coarsening type %d", p.coarsen);
  CLAIR_REQUIRE(p.b_smooth_iters >= 0 && p.gmres_maxit >= 1 && p.rtol > 0.0, CLAIR_ERR_ARG,
                "bad iteration counts or rtol");
  CLAIR_REQUIRE(kmodes >= 1 && kmodes <= CLAIR_KMAX, CLAIR_ERR_ARG,
                "k (mode vectors) must be in [1, %d], got %d", CLAIR_KMAX, kmodes);
  CLAIR_REQUIRE(p.inverse == CLAIR_INVERSE_EXACT || p.inverse == CLAIR_INVERSE_DIAG, CLAIR_ERR_ARG,
                "unknown block inverse %d", p.inverse);
  CLAIR_REQUIRE(p.iterations >= 1 && p.iterations <= 100, CLAIR_ERR_ARG,
                "iterations must be in [1, 100]");
  CLAIR_REQUIRE(p.symmetric == 0 || p.symmetric == 1, CLAIR_ERR_ARG, "symmetric must be 0 or 1");
  CLAIR_REQUIRE(p.krylov == CLAIR_KRYLOV_FGMRES || p.krylov == CLAIR_KRYLOV_PCG, CLAIR_ERR_ARG,
                "unknown Krylov method %d", p.krylov);
  CLAIR_REQUIRE(!cf_marker || p.coarsen == CLAIR_COARSEN_FC, CLAIR_ERR_UNSUPPORTED,
                "a caller splitting (cf_marker) needs FC coarsening (aggregates are not given)");
  std::vector<int> off{0, n};
  if (ninst > 1) {
    CLAIR_REQUIRE(offsets_host, CLAIR_ERR_ARG, "clair_setup_batched: null offsets");
    off.assign(offsets_host, offsets_host + ninst + 1);
    CLAIR_REQUIRE(off[0] == 0 && off[ninst] == n, CLAIR_ERR_ARG,
                  "clair_setup_batched: offsets must run from 0 to n");
    for (int i = 0; i < ninst; ++i)
      CLAIR_REQUIRE(off[i + 1] > off[i], CLAIR_ERR_ARG,
                    "clair_setup_batched: instance %d is empty or offsets decrease", i);
    CLAIR_REQUIRE(p.arnoldi_iters <= 15, CLAIR_ERR_UNSUPPORTED,
                  "clair_setup_batched: arnoldi_iters must be <= 15");
  }
  clair_hierarchy* h = new clair_hierarchy();
  h->p = p;
  h->kmodes = kmodes;
  h->ninst = std::max(ninst, 1);
  h->stream = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  try {
    cudaStream_t s = h->stream;
    CLAIR_CUDA(cudaEventCreate(&e0));
    CLAIR_CUDA(cudaEventCreate(&e1));
    CLAIR_CUDA(cudaEventRecord(e0, s));
    Level L0;
    L0.n = n;
    if (h->ninst > 1) L0.off = off;
    L0.A.rows = L0.A.cols = n;
    L0.A.nnz = nnz;
    L0.A.rowptr = dalloc<int>(n + 1, s);
    L0.A.col = dalloc<int>(nnz, s);
    L0.A.val = dalloc<double>(nnz, s);
    h->lv.push_back(L0);
    CLAIR_CUDA(cudaMemcpyAsync(L0.A.rowptr, rowptr, sizeof(int) * (n + 1), cudaMemcpyDeviceToDevice, s));
    CLAIR_CUDA(cudaMemcpyAsync(L0.A.col, col, sizeof(int) * nnz, cudaMemcpyDeviceToDevice, s));
    CLAIR_CUDA(cudaMemcpyAsync(L0.A.val, val, sizeof(double) * nnz, cudaMemcpyDeviceToDevice, s));
    validate_csr(rowptr, col, n, n, nnz, "A", s);
    if (h->ninst > 1) {  // no entry may couple two instances
      int* d_off = dalloc<int>(h->ninst + 1, s);
      int* inst = dalloc<int>(n, s);
      int* base = dalloc<int>(n, s);
      int* bad = dalloc<int>(1, s);
      CLAIR_CUDA(cudaMemcpyAsync(d_off, off.data(), sizeof(int) * (h->ninst + 1),
                                 cudaMemcpyHostToDevice, s));
      CLAIR_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
      row_instance<<<ceil_div(n, 256), 256, 0, s>>>(d_off, h->ninst, n, inst, base); ::clair::count_launch();
      check_block_diagonal<<<ceil_div(n, 256), 256, 0, s>>>(rowptr, col, inst, d_off, n, bad); ::clair::count_launch();
      CLAIR_LAUNCHED();
      int hb = 0;
      CLAIR_CUDA(cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
      CLAIR_CUDA(cudaStreamSynchronize(s));
      dfree(d_off, s);
      dfree(inst, s);
      dfree(base, s);
      dfree(bad, s);
      CLAIR_REQUIRE(hb == 0, CLAIR_ERR_ARG,
                    "clair_setup_batched: %d rows couple two instances (not block-diagonal)", hb);
    }
    CLAIR_REQUIRE(all_finite(val, nnz, s), CLAIR_ERR_NONFINITE, "A has nonfinite values");
    CLAIR_REQUIRE(all_finite(B, (long long)n * kmodes, s), CLAIR_ERR_NONFINITE,
                  "B has nonfinite values");
    if (cf_marker) validate_cf(cf_marker, n, s);
    h->B0 = dalloc<double>((size_t)n * kmodes, s);
    CLAIR_CUDA(cudaMemcpyAsync(h->B0, B, sizeof(double) * n * kmodes, cudaMemcpyDeviceToDevice, s));
    h->setup_clock.reset(new PhaseClock());
    set_active_clock(h->setup_clock.get());
    // per-level counters stay on the device until the end of the setup
    h->st.dev = dalloc<unsigned long long>(6, s);
    CLAIR_CUDA(cudaMemsetAsync(h->st.dev, 0, 6 * sizeof(unsigned long long), s));
    setup_levels(h, B, cf_marker);
    set_active_clock(nullptr);
    h->vin = dalloc<double>(n, s);
    h->zout = dalloc<double>(n, s);
    // captured and instantiated on the host while the stream finishes the setup
    build_cycle_graph(h);
    h->st.absorb_device(s);  // the one synchronisation at the end
    dfree(h->st.dev, s);
    CLAIR_CUDA(cudaEventRecord(e1, s));
    CLAIR_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    CLAIR_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    h->setup_ms = ms;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  } catch (...) {
    set_active_clock(nullptr);
    release_all(h);
    delete h;
    throw;
  }
  *out = h;
  CLAIR_API_END
}

clair_status clair_setup(int n, int nnz, const int* rowptr, const int* col, const double* val,
                         int k, const double* B, const signed char* cf_marker,
                         const clair_params* p, void* stream, clair_h* out) {
  return setup_common(1, nullptr, n, nnz, rowptr, col, val, k, B, cf_marker, p, stream, out);
}

clair_status clair_setup_batched(int ninst, const int* offsets_host, int n, int nnz,
                                 const int* rowptr, const int* col, const double* val, int k,
                                 const double* B, const signed char* cf_marker,
                                 const clair_params* p, void* stream, clair_h* out) {
  if (out) *out = nullptr;
  if (ninst < 1) {
    set_error("clair_setup_batched: ninst must be >= 1");
    return CLAIR_ERR_ARG;
  }
  return setup_common(ninst, offsets_host, n, nnz, rowptr, col, val, k, B, cf_marker, p, stream,
                      out);
}

clair_status clair_batch_view(clair_h h, int level, int* ninst, int* offsets_host,
                              double* omega_host, signed char* frozen_host) {
  CLAIR_API_BEGIN
  CLAIR_REQUIRE(h && ninst, CLAIR_ERR_ARG, "clair_batch_view: null pointer");
  CLAIR_REQUIRE(level >= 0 && level < (int)h->lv.size(), CLAIR_ERR_ARG, "bad level %d", level);
  const Level& L = h->lv[level];
  *ninst = h->ninst;
  for (int i = 0; i < h->ninst; ++i) {
    if (offsets_host) {
      offsets_host[i] = h->ninst > 1 ? L.off[i] : 0;
      offsets_host[i + 1] = h->ninst > 1 ? L.off[i + 1] : L.n;
    }
    if (omega_host)
      omega_host[i] = (h->ninst > 1 && !L.omega_inst.empty()) ? L.omega_inst[i] : L.omega;
    if (frozen_host)
      frozen_host[i] = (h->ninst > 1 && !L.frozen.empty()) ? L.frozen[i] : (L.nc ? 0 : 1);
  }
  CLAIR_API_END
}

clair_status clair_setup_adjoint(clair_h fwd, void* stream, clair_h* adj) {
  if (adj) *adj = nullptr;
  CLAIR_API_BEGIN
  CLAIR_REQUIRE(fwd && adj, CLAIR_ERR_ARG, "clair_setup_adjoint: null pointer");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const Csr& A = fwd->lv[0].A;
  Csr At;
  csr_transpose(A, At, nullptr, s);
  clair_status st;
  try {
    st = setup_common(fwd->ninst, fwd->ninst > 1 ? fwd->lv[0].off.data() : nullptr, A.rows, A.nnz,
                      At.rowptr, At.col, At.val, fwd->kmodes, fwd->B0, nullptr, &fwd->p, stream,
                      adj);
  } catch (...) {
    At.release(s);
    throw;
  }
  At.release(s);
  CLAIR_CUDA(cudaStreamSynchronize(s));
  return st;
  CLAIR_API_END
}

clair_status clair_solve(clair_h h, const double* f, double* u, int nrhs, void* stream,
                         int* iters, double* relres) {
  CLAIR_API_BEGIN
  CLAIR_REQUIRE(h && f && u, CLAIR_ERR_ARG, "clair_solve: null pointer");
  CLAIR_REQUIRE(nrhs >= 1 && (long long)nrhs * h->lv[0].n < (1LL << 40), CLAIR_ERR_ARG,
                "clair_solve: nrhs must be >= 1 (got %d)", nrhs);
  cudaStream_t keep = h->stream;
  h->stream = static_cast<cudaStream_t>(stream);
  bool ok = false;
  h->solve_clock.reset(new PhaseClock());
  set_active_clock(h->solve_clock.get());
  for (double& v : h->solve_ms) v = 0.0;
  try {
    ok = krylov_solve(h, nrhs, f, u);
  } catch (...) {
    set_active_clock(nullptr);
    h->stream = keep;
    throw;
  }
  set_active_clock(nullptr);
  h->stream = keep;
  const int ninst = h->ninst;
  for (int r = 0; r < nrhs; ++r) {
    int it = 0;
    double rel = 0.0;
    for (int i = 0; i < ninst; ++i) {
      it = std::max(it, h->last_its[(size_t)r * ninst + i]);
      rel = std::max(rel, h->last_rel[(size_t)r * ninst + i]);
    }
    if (iters) iters[r] = it;
    if (relres) relres[r] = rel;
  }
  if (!ok) {
    set_error("the Krylov solver did not reach rtol within gmres_maxit for every right-hand side");
    return CLAIR_ERR_NOT_CONVERGED;
  }
  CLAIR_API_END
}

clair_status clair_solve_detail(clair_h h, int* nseg, int* iters_host, double* relres_host) {
  CLAIR_API_BEGIN
  CLAIR_REQUIRE(h && nseg, CLAIR_ERR_ARG, "clair_solve_detail: null pointer");
  *nseg = (int)h->last_its.size();
  for (size_t i = 0; i < h->last_its.size(); ++i) {
    if (iters_host) iters_host[i] = h->last_its[i];
    if (relres_host) relres_host[i] = h->last_rel[i];
  }
  CLAIR_API_END
}

clair_status clair_vcycle(clair_h h, int level, const double* b, double* x, void* stream) {
  CLAIR_API_BEGIN
  CLAIR_REQUIRE(h && b && x, CLAIR_ERR_ARG, "clair_vcycle: null pointer");
  CLAIR_REQUIRE(level >= 0 && level < (int)h->lv.size(), CLAIR_ERR_ARG, "bad level %d", level);
  cudaStream_t keep = h->stream;
  h->stream = static_cast<cudaStream_t>(stream);
  try {
    apply_precond(h, level, b, x);
  } catch (...) {
    h->stream = keep;
    throw;
  }
  h->stream = keep;
  CLAIR_API_END
}

clair_status clair_stats(clair_h h, clair_stats_t* o) {
  CLAIR_API_BEGIN
  CLAIR_REQUIRE(h && o, CLAIR_ERR_ARG, "clair_stats: null pointer");
  if (h->setup_clock) {
    h->setup_clock->collect(h->phase_ms, h->level_phase_ms, 32);
    h->setup_clock.reset();
  }
  if (h->solve_clock) {
    h->solve_clock->collect(h->solve_ms);
    h->solve_clock.reset();
  }
  memset(o, 0, sizeof(*o));
  o->levels = (int)h->lv.size();
  double nnz0 = h->lv[0].A.nnz, sum = 0.0;
  for (size_t k = 0; k < h->lv.size() && k < 32; ++k) {
    const Level& L = h->lv[k];
    o->n[k] = L.n;
    o->nnz[k] = L.A.nnz;
    o->nnz_R[k] = L.nc ? L.R.nnz : 0;
    o->nnz_P[k] = L.nc ? L.P.nnz : 0;
    o->omega[k] = L.omega;
    sum += L.A.nnz;
    o->r_rows += L.nc;
    o->p_cols += L.nc;
  }
  o->operator_complexity = sum / nnz0;
  for (int b = 0; b < 7; ++b) o->t_hist[b] = h->st.hist[b];
  o->singular_blocks = h->st.singular;
  o->empty_constraints = h->st.empty;
  o->setup_ms = h->setup_ms;
  for (int i = 0; i < PH_COUNT && i < 10; ++i) {
    o->phase_ms[i] = h->phase_ms[i];
    o->solve_phase_ms[i] = h->solve_ms[i];
  }
  o->lsolve_flops = (2.0 / 3.0) * h->st.sum_t3 + 2.0 * h->st.sum_t2;
  double minb = 0.0;
  for (const Level& L : h->lv)
    if (L.nc) minb += 2.0 * 12.0 * L.A.nnz + 12.0 * (double)L.R.nnz + 12.0 * (double)L.P.nnz;
  o->lsolve_min_bytes = minb;
  o->lsolve_gathered = h->st.gathered;
  o->fp64_cycle_from = h->fp64_from;
  o->k = h->kmodes;
  o->lsolve_kind_b1 = h->st.config_kind_b1;
  o->lsolve_kind_b3 = h->st.config_kind_b3;
  o->lsolve_blocks_per_sm = h->st.config_blocks_per_sm;
  o->lsolve_tuned = h->st.config_tuned;
  o->cycle_short_lanes = h->short_lanes;
  for (int k = 0; k < 32; ++k) {
    o->level_span_ms[k] = h->level_span_ms[k];
    for (int q = 0; q < 8; ++q) o->level_phase_ms[k][q] = h->level_phase_ms[k * PH_COUNT + q];
  }
  o->cycle64_from = -1;
  for (size_t k = 0; k < h->lv.size(); ++k)
    if (h->lv[k].cycle64) {
      o->cycle64_from = (int)k;
      break;
    }
  CLAIR_API_END
}

int64_t clair_kernel_launches(void) { return launch_count(); }

clair_status clair_lsolve_config(int precision, int set, int* kind_b1, int* kind_b3,
                                 int* blocks_per_sm, int* tuned) {
  CLAIR_API_BEGIN
  CLAIR_REQUIRE(kind_b1 && kind_b3 && blocks_per_sm && tuned, CLAIR_ERR_ARG,
                "clair_lsolve_config: null pointer");
  CLAIR_REQUIRE(precision == CLAIR_FP64 || precision == CLAIR_MIXED, CLAIR_ERR_ARG,
                "unknown precision");
  if (set) {
    CLAIR_REQUIRE((*kind_b1 == 1 || *kind_b1 == 2) && (*kind_b3 == 3 || *kind_b3 == 4) &&
                      *blocks_per_sm >= 0,
                  CLAIR_ERR_ARG,
                  "clair_lsolve_config: kind_b1 in {1, 2}, kind_b3 in {3, 4}, blocks_per_sm >= 0");
  }
  lsolve_config(precision, kind_b1, kind_b3, blocks_per_sm, tuned, set != 0);
  CLAIR_API_END
}

clair_status clair_spgemm(int m, int kdim, int ncols, const int* A_rowptr, const int* A_col,
                          const double* A_val, const int* B_rowptr, const int* B_col,
                          const double* B_val, void* stream, int* rowptr_out, int64_t* nnz_out,
                          int64_t cap, int* col_out, double* val_out) {
  CLAIR_API_BEGIN
  CLAIR_REQUIRE(A_rowptr && A_col && A_val && B_rowptr && B_col && B_val && rowptr_out && nnz_out,
                CLAIR_ERR_ARG, "clair_spgemm: null pointer");
  CLAIR_REQUIRE(m > 0 && kdim > 0 && ncols > 0, CLAIR_ERR_ARG, "clair_spgemm: bad sizes");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int nnzA = 0, nnzB = 0;
  CLAIR_CUDA(cudaMemcpyAsync(&nnzA, A_rowptr + m, sizeof(int), cudaMemcpyDeviceToHost, s));
  CLAIR_CUDA(cudaMemcpyAsync(&nnzB, B_rowptr + kdim, sizeof(int), cudaMemcpyDeviceToHost, s));
  CLAIR_CUDA(cudaStreamSynchronize(s));
  validate_csr(A_rowptr, A_col, m, kdim, nnzA, "A", s);
  validate_csr(B_rowptr, B_col, kdim, ncols, nnzB, "B", s);
  Csr A, B, C;
  A.rows = m;
  A.cols = kdim;
  A.nnz = nnzA;
  A.rowptr = const_cast<int*>(A_rowptr);
  A.col = const_cast<int*>(A_col);
  A.val = const_cast<double*>(A_val);
  B.rows = kdim;
  B.cols = ncols;
  B.nnz = nnzB;
  B.rowptr = const_cast<int*>(B_rowptr);
  B.col = const_cast<int*>(B_col);
  B.val = const_cast<double*>(B_val);
  spgemm(A, B, C, s);
  *nnz_out = C.nnz;
  try {
    CLAIR_CUDA(cudaMemcpyAsync(rowptr_out, C.rowptr, sizeof(int) * (m + 1), cudaMemcpyDeviceToDevice, s));
    if (col_out && val_out) {
      CLAIR_REQUIRE(C.nnz <= cap, CLAIR_ERR_CAPACITY, "clair_spgemm: nnz(C) = %d exceeds cap %lld",
                    C.nnz, (long long)cap);
      CLAIR_CUDA(cudaMemcpyAsync(col_out, C.col, sizeof(int) * C.nnz, cudaMemcpyDeviceToDevice, s));
      CLAIR_CUDA(cudaMemcpyAsync(val_out, C.val, sizeof(double) * C.nnz, cudaMemcpyDeviceToDevice, s));
    }
  } catch (...) {
    C.release(s);
    cudaStreamSynchronize(s);
    throw;
  }
  C.release(s);
  CLAIR_CUDA(cudaStreamSynchronize(s));
  CLAIR_API_END
}

int clair_compiled_arch(void) {
#ifdef __CUDA_ARCH_LIST__
  return __CUDA_ARCH_LIST__;
#else
  return 0;
#endif
}

clair_status clair_level_view(clair_h h, int level, int* n, int* nc, int* nnz_A,
                              const int** A_rowptr, const int** A_col, const double** A_val,
                              int* nnz_R, const int** R_rowptr, const int** R_col,
                              const double** R_val, int* nnz_P, const int** P_rowptr,
                              const int** P_col, const double** P_val, const signed char** cf,
                              const double** B_P, const double** B_R, double* omega) {
  CLAIR_API_BEGIN
  CLAIR_REQUIRE(h, CLAIR_ERR_ARG, "clair_level_view: null handle");
  CLAIR_REQUIRE(level >= 0 && level < (int)h->lv.size(), CLAIR_ERR_ARG, "bad level %d", level);
  const Level& L = h->lv[level];
  if (n) *n = L.n;
  if (nc) *nc = L.nc;
  if (nnz_A) *nnz_A = L.A.nnz;
  if (A_rowptr) *A_rowptr = L.A.rowptr;
  if (A_col) *A_col = L.A.col;
  if (A_val) *A_val = L.A.val;
  const bool has = L.nc > 0;
  if (nnz_R) *nnz_R = has ? L.R.nnz : 0;
  if (R_rowptr) *R_rowptr = has ? L.R.rowptr : nullptr;
  if (R_col) *R_col = has ? L.R.col : nullptr;
  if (R_val) *R_val = has ? L.R.val : nullptr;
  if (nnz_P) *nnz_P = has ? L.P.nnz : 0;
  if (P_rowptr) *P_rowptr = has ? L.P.rowptr : nullptr;
  if (P_col) *P_col = has ? L.P.col : nullptr;
  if (P_val) *P_val = has ? L.P.val : nullptr;
  if (cf) *cf = has ? L.cf : nullptr;
  if (B_P) *B_P = has ? L.B_P : nullptr;
  if (B_R) *B_R = has ? L.B_R : nullptr;
  if (omega) *omega = L.omega;
  CLAIR_API_END
}

clair_status clair_free(clair_h h) {
  CLAIR_API_BEGIN
  if (!h) return CLAIR_OK;
  release_all(h);
  cudaStreamSynchronize(h->stream);
  delete h;
  CLAIR_API_END
}

clair_status clair_local_weights(int n, const int* Ahat_rowptr, const int* Ahat_col,
                                 const double* Ahat_val, const signed char* cf, int nc,
                                 const int* Z_rowptr, const int* Z_col, const double* B,
                                 int precision, double* Z_val, void* stream,
                                 int64_t* singular_out, int64_t* empty_out) {
  CLAIR_API_BEGIN
  CLAIR_REQUIRE(Ahat_rowptr && Ahat_col && Ahat_val && cf && Z_rowptr && Z_col && B && Z_val,
                CLAIR_ERR_ARG, "clair_local_weights: null pointer");
  CLAIR_REQUIRE(n > 0 && nc >= 0 && nc <= n, CLAIR_ERR_ARG, "clair_local_weights: bad sizes");
  CLAIR_REQUIRE(precision == CLAIR_FP64 || precision == CLAIR_MIXED, CLAIR_ERR_ARG,
                "unknown precision");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int nnzA = 0;
  CLAIR_CUDA(cudaMemcpyAsync(&nnzA, Ahat_rowptr + n, sizeof(int), cudaMemcpyDeviceToHost, s));
  CLAIR_CUDA(cudaStreamSynchronize(s));
  validate_csr(Ahat_rowptr, Ahat_col, n, n, nnzA, "Ahat", s);
  validate_cf(cf, n, s);
  int* cpts = nullptr;
  const int nc2 = coarse_points(cf, n, &cpts, s);
  if (nc2 != nc) {
    dfree(cpts, s);
    CLAIR_REQUIRE(false, CLAIR_ERR_ARG, "nc=%d but cf has %d C-points", nc, nc2);
  }
  Csr Ahat;
  Ahat.rows = Ahat.cols = n;
  Ahat.nnz = nnzA;
  Ahat.rowptr = const_cast<int*>(Ahat_rowptr);
  Ahat.col = const_cast<int*>(Ahat_col);
  Ahat.val = const_cast<double*>(Ahat_val);
  int nnzZ = 0;
  CLAIR_CUDA(cudaMemcpyAsync(&nnzZ, Z_rowptr + nc, sizeof(int), cudaMemcpyDeviceToHost, s));
  CLAIR_CUDA(cudaStreamSynchronize(s));
  try {
    validate_csr(Z_rowptr, Z_col, nc, n, nnzZ, "Z", s);
  } catch (...) {
    dfree(cpts, s);
    throw;
  }
  Csr Z;
  Z.rows = nc;
  Z.cols = n;
  Z.nnz = nnzZ;
  Z.rowptr = const_cast<int*>(Z_rowptr);
  Z.col = const_cast<int*>(Z_col);
  Z.val = Z_val;
  LocalStats st;
  try {
    transfer_weights(Ahat, cf, cpts, Z, B, precision, st, nullptr, s);
  } catch (...) {
    dfree(cpts, s);
    throw;
  }
  dfree(cpts, s);
  CLAIR_CUDA(cudaStreamSynchronize(s));
  if (singular_out) *singular_out = st.singular;
  if (empty_out) *empty_out = st.empty;
  if (st.singular) {
    set_error("%lld local blocks had a zero pivot", st.singular);
    return CLAIR_ERR_SINGULAR_BLOCK;
  }
  CLAIR_API_END
}

}  // extern "C"
