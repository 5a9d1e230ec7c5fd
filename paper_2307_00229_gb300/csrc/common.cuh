// Internal helpers shared by the CUDA translation units of the CLAIR library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <string>
#include <vector>

#include "../../include/clair.h"

namespace clair {

// ------------------------------------------------------------------------------------
// Errors: every entry point returns a status; the message of the last failure is kept
// per host thread.
// ------------------------------------------------------------------------------------
void set_error(const char* fmt, ...);
void clear_error();

struct Error {
  clair_status st;
};

#define CLAIR_CUDA(call)                                                                  \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess) {                                                              \
      ::clair::set_error("%s:%d %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e_)); \
      throw ::clair::Error{CLAIR_ERR_CUDA};                                               \
    }                                                                                     \
  } while (0)

#define CLAIR_LAUNCHED() CLAIR_CUDA(cudaGetLastError())

#define CLAIR_REQUIRE(cond, status, ...)  \
  do {                                    \
    if (!(cond)) {                        \
      ::clair::set_error(__VA_ARGS__);    \
      throw ::clair::Error{status};       \
    }                                     \
  } while (0)

// ------------------------------------------------------------------------------------
// Stream-ordered device buffers.
// ------------------------------------------------------------------------------------
// The library's own stream-ordered pool on the current device.  It keeps freed memory
// for reuse (release threshold = unlimited) instead of returning it to the driver at every
// synchronisation, so repeated setups do not re-map their temporaries.
cudaMemPool_t library_pool();

template <class T>
T* dalloc(size_t count, cudaStream_t s) {
  void* p = nullptr;
  if (count == 0) count = 1;
  CLAIR_CUDA(cudaMallocFromPoolAsync(&p, count * sizeof(T), library_pool(), s));
  return static_cast<T*>(p);
}

template <class T>
void dfree(T*& p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
  p = nullptr;
}

// Device CSR matrix (values in float64 and, optionally, a float32 copy).
struct Csr {
  int rows = 0, cols = 0, nnz = 0;
  int* rowptr = nullptr;
  int* col = nullptr;
  double* val = nullptr;
  float* val32 = nullptr;
  void release(cudaStream_t s) {
    dfree(rowptr, s);
    dfree(col, s);
    dfree(val, s);
    dfree(val32, s);
  }
};

inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

// Body of every C-ABI entry point: host exceptions become status codes and the message
// stays readable through clair_last_error().
#define CLAIR_API_BEGIN \
  ::clair::clear_error(); \
  try {
#define CLAIR_API_END                                    \
  }                                                      \
  catch (const ::clair::Error& e) {                      \
    return e.st;                                         \
  }                                                      \
  catch (...) {                                          \
    ::clair::set_error("unexpected host exception");     \
    return CLAIR_ERR_CUDA;                               \
  }                                                      \
  return CLAIR_OK;

// Pinned host memory for small per-setup and per-solve buffers, recycled by size class
// for the life of the process (returned with the size it was taken with).
void* pinned_get(size_t bytes);
void pinned_put(void* p, size_t bytes);

// Number of SMs of the current device (cached per process).
int sm_count();

// Runs `set` once per device and `tag` (function attributes such as the dynamic
// shared-memory limit belong to the current device's context), under a lock so that
// host threads driving several devices do not race.  The tag is the address of the
// kernel whose attributes `set` installs, so every template instantiation has its own.
void once_per_device(const void* tag, void (*set)());

// ------------------------------------------------------------------------------------
// Device utilities.
// ------------------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v, unsigned mask = 0xffffffffu) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o);
  return v;
}

template <int W, class T>
__device__ __forceinline__ T group_sum(T v) {
#pragma unroll
  for (int o = W / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, W);
  return v;
}

// Sum over CSR entries e0 <= e < e1 of val[e] * x[col[e]], in increasing e (lane `lane`
// of W takes every W-th entry).  The row's indices and values are loaded eight (one lane
// per row) or four (W lanes) at a time before their gathers, so a row costs two dependent
// memory round trips per batch instead of two per entry; the order and the contraction
// (acc + v * x into one fma) are the same as one entry at a time.
template <int W, class T, class X>
__device__ __forceinline__ T csr_row_dot(const int* __restrict__ col, const T* __restrict__ val,
                                         const X* __restrict__ x, int e0, int e1, int lane) {
  T acc = 0;
  if constexpr (W == 1) {
    for (int eb = e0; eb < e1; eb += 8) {
      int c[8];
      T v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const bool in = eb + q < e1;
        c[q] = in ? col[eb + q] : 0;
        v[q] = in ? val[eb + q] : T(0);
      }
#pragma unroll
      for (int q = 0; q < 8; ++q)
        if (eb + q < e1) acc += v[q] * __ldg(&x[c[q]]);
    }
  } else {
    // four entries per lane in flight: indices and values first, then the four gathers,
    // then the same running sum in the same order as one entry at a time
    int e = e0 + lane;
    for (; e + 3 * W < e1; e += 4 * W) {
      const int c0 = col[e], c1 = col[e + W], c2 = col[e + 2 * W], c3 = col[e + 3 * W];
      const T v0 = val[e], v1 = val[e + W], v2 = val[e + 2 * W], v3 = val[e + 3 * W];
      const X x0 = __ldg(&x[c0]), x1 = __ldg(&x[c1]), x2 = __ldg(&x[c2]), x3 = __ldg(&x[c3]);
      acc += v0 * x0;
      acc += v1 * x1;
      acc += v2 * x2;
      acc += v3 * x3;
    }
    for (; e < e1; e += W) acc += val[e] * __ldg(&x[col[e]]);
  }
  return acc;
}

// splitmix64 (Steele, Lea & Flood 2014): draw i of the stream seeded with `seed`.
__device__ __forceinline__ double splitmix_pm1(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return 2.0 * ((double)(z >> 11) * (1.0 / 9007199254740992.0)) - 1.0;
}

// 'lowbias32' integer hash (C. Wellons, hash-prospector); a bijection of uint32.
__host__ __device__ __forceinline__ uint32_t lowbias32(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7feb352du;
  x ^= x >> 15;
  x *= 0x846ca68bu;
  x ^= x >> 16;
  return x;
}

// ------------------------------------------------------------------------------------
// Host-callable building blocks (sparse.cu).
// ------------------------------------------------------------------------------------
// out[0] = 0, out[i+1] = sum_{k<=i} in[k]; returns out[n] (synchronises s).
// want_total: returns out[n] after synchronising s; a device int `extra_dev` (optional) is
// read back into *extra_host by the same synchronisation.
long long exclusive_scan(const int* in, int* out, int n, cudaStream_t s, bool want_total = true,
                         const int* extra_dev = nullptr, int* extra_host = nullptr);
// Transpose (structure + values; perm[k] = source entry of output entry k); output
// arrays are allocated here.  Rows of the result are sorted by column.
void csr_transpose(const Csr& A, Csr& At, int** perm, cudaStream_t s);
// max_{j != i} |a_ij| per row (0 for rows without off-diagonal entries).
void row_max_offdiag(const Csr& A, double* out, cudaStream_t s);
// y = alpha * A x + beta * y   (y may alias nothing; beta = 0 ignores y's input)
void spmv(const Csr& A, const double* x, double* y, double alpha, double beta, cudaStream_t s);
void spmv32(const Csr& A, const float* x, float* y, float alpha, float beta, cudaStream_t s);
// r = b - A x
void residual(const Csr& A, const double* b, const double* x, double* r, cudaStream_t s);
void residual32(const Csr& A, const float* b, const float* x, float* r, cudaStream_t s);
// C = A * B (sparse-sparse, deterministic summation in A's row order, no FMA contraction)
void spgemm(const Csr& A, const Csr& B, Csr& C, cudaStream_t s);
// Removes entries whose value is exactly zero (structure follows the values).
void drop_zeros(Csr& C, cudaStream_t s);
// Inverse diagonal (error if a diagonal entry is missing or zero).
// dinv = 1 / diag(A); rows with a missing, zero or nonfinite diagonal are an error, raised
// here (bad_acc null, one host synchronisation) or counted into *bad_acc for the caller.
void inverse_diagonal(const Csr& A, double* dinv, cudaStream_t s, int* bad_acc = nullptr);

// The sparsity pattern of Algorithm 1 in two stages, so that other work can be issued
// between them: pattern_count launches the counting pass, pattern_fill reads the count
// back and builds the rows (and releases the job's buffers).
struct PatternJob {
  Csr Wm;
  const unsigned char* sW = nullptr;
  const signed char* cf = nullptr;
  const int* cpts = nullptr;
  int nc = 0, n = 0, degree = 0;
  const int* Mrp = nullptr;
  const int* Mcol = nullptr;
  int* count = nullptr;
  int* err = nullptr;
  int* start = nullptr;
  int* buf = nullptr;
  long long cap = 0;
  unsigned long long* bump = nullptr;
  unsigned char* done = nullptr;  // points counted by the short-row group pass
  int* ovf = nullptr;             // scan overflow flag (device)
};
PatternJob pattern_count(const Csr& Wm, const unsigned char* sW, const signed char* cf,
                         const int* cpts, int nc, int n, int degree, const int* Mrp,
                         const int* Mcol, cudaStream_t s);
void pattern_fill(PatternJob& j, Csr& Z, cudaStream_t s);
// pattern_fill in three steps, so that several patterns share one host read: the row
// pointers (device only), the entry counts and overflow flags of all jobs (one
// synchronisation), then the rows
void pattern_scan(PatternJob& j, Csr& Z, cudaStream_t s);
void pattern_read(PatternJob* const* jobs, Csr* const* Z, int k, cudaStream_t s);
void pattern_build(PatternJob& j, Csr& Z, cudaStream_t s);
void exclusive_scan_into(const int* in, int* out, int n, int* ovf, cudaStream_t s);

// Vectors relaxed together by the mode smoothing: side g = blockIdx.y relaxes x[g] with its
// own operator (A for the P side, A^T for the R side, one entry per mode) and ping-pongs
// with y[g]; D^-1, the splitting and the weight are shared.
struct SmoothSides {
  static constexpr int kMax = 2 * CLAIR_KMAX;
  const int* rowptr[kMax];
  const int* col[kMax];
  const double* val[kMax];
  double* x[kMax];
  double* y[kMax];
  int count;
};
// Float copies.
void to_float(const double* x, float* y, long long n, cudaStream_t s);
// y = x as a kernel (a node the cycle graph can chain by programmatic dependence)
void copy_f64(const double* x, double* y, long long n, cudaStream_t s);
void to_double(const float* x, double* y, long long n, cudaStream_t s);
// Deterministic dot products: out[j] = <V_j, w> for j < m (V column-major n x m, ld = n).
void multi_dot(const double* V, int m, const double* w, int n, double* out, double* partial,
               cudaStream_t s);
// w -= V[:, :m] * h  (h device)
void multi_axpy(const double* V, int m, const double* h, double* w, int n, cudaStream_t s);
// Gather: y[i] = x[idx[i]]
void gather(const double* x, const int* idx, double* y, int n, cudaStream_t s);
void gather_vals(const double* x, const int* perm, double* y, int n, cudaStream_t s);
void scatter_vals(const double* x, const int* perm, double* y, int n, cudaStream_t s);
// Caller-input validation (synchronises); throws CLAIR_ERR_ARG with a message.
void validate_csr(const int* rowptr, const int* col, int rows, int cols, int nnz, const char* what,
                  cudaStream_t s);
void validate_cf(const signed char* cf, int n, cudaStream_t s);
// *out = max(*out, max |x|) as the bits of a non-negative double (asynchronous).
void absmax_into(const double* x, long long n, unsigned long long* out, cudaStream_t s);

// Up to kMax (source, length) segments for one launch: FP64 -> FP32 copies (dst), or the
// largest |x| of each segment folded into out[slot] (as the bits of a nonnegative double).
struct SegList {
  static constexpr int kMax = 48;
  const double* src[kMax];
  float* dst[kMax];
  long long n[kMax];
  int slot[kMax];
  int count = 0;
};
// Collects segments and launches them kMax at a time (out null: conversions, else maxima).
struct SegBatch {
  SegBatch(cudaStream_t st, unsigned long long* o = nullptr) : s(st), out(o) {}
  void add(const double* src, float* dst, long long n, int slot = 0);
  void flush();
  cudaStream_t s;
  unsigned long long* out;
  SegList cur;
};
// Nonfinite check over a buffer; returns true if all finite (synchronises).
bool all_finite(const double* x, long long n, cudaStream_t s);

int partial_blocks();  // number of blocks used by the deterministic reductions

// Lanes per row of the FP32 row kernels (SpMV, residual, Jacobi sweeps): 0 = the power of
// two at or above the mean row length; 1 = about four entries per lane (one thread per
// row up to 8 entries), the FP64 rule.  A per-thread setting, chosen per hierarchy by
// timing its cycle graph.
int cycle_short_lanes();
void set_cycle_short_lanes(int lanes);

// Programmatic dependent launch for the captured V-cycle.  While pdl_launches() is set
// (the capture of the cycle graph), the cycle's row kernels are launched with
// programmatic stream serialization: a kernel's blocks may be scheduled while its
// predecessor runs, and wait at pdl_prologue() until the predecessor has completed and
// its writes are visible, so the graph's kernel-to-kernel gaps shrink to that wait.
// Launched without the attribute, the prologue returns at once.
bool pdl_launches();
void set_pdl_launches(bool on);

__device__ __forceinline__ void pdl_prologue() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <class... KArgs, class... Args>
inline void launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                     Args... args) {
  if (!pdl_launches()) {
    kernel<<<grid, block, smem, s>>>(args...);
    return;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  CLAIR_CUDA(cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...));
}

// ------------------------------------------------------------------------------------
// Segmented Krylov building blocks (krylov.cu): independent Krylov processes in lockstep,
// one per segment = (right-hand side, instance) of a long vector.
// ------------------------------------------------------------------------------------
struct Segments {
  int nseg = 0, nchunk = 0;
  long long len = 0;              // nrhs * n rows
  int* chunk_seg = nullptr;       // [nchunk] segment of each chunk
  long long* chunk_lo = nullptr;  // [nchunk] first row of each chunk
  long long* chunk_hi = nullptr;  // [nchunk] one past its last row
  int* seg_chunk0 = nullptr;      // [nseg + 1] first chunk of each segment
  // segment r * ninst + i = rows r * n + off[i] .. r * n + off[i + 1] - 1
  void build(int nrhs, const std::vector<int>& off, cudaStream_t s);
  void release(cudaStream_t s);
};
// out[seg * ldo + q] = <V_q, w> over the segment's rows (V_q at V + q * ldv), q < m
void seg_dot(const Segments& S, const double* V, long long ldv, int m, const double* w,
             double* out, int ldo, double* partial, cudaStream_t s);
// w -= sum_q coef[seg * ldc + q] V_q on each segment
void seg_axpy(const Segments& S, const double* V, long long ldv, int m, const double* coef,
              int ldc, double* w, cudaStream_t s);
// y = x * f[seg * ldf]
void seg_scale(const Segments& S, const double* x, const double* f, int ldf, double* y,
               cudaStream_t s);
// y += a[seg] x ;  z = x + b[seg] z
void seg_axpy1(const Segments& S, const double* x, const double* a, double* y, cudaStream_t s);
void seg_xpby(const Segments& S, const double* x, const double* b, double* z, cudaStream_t s);
void seg_tolerance_launch(const Segments& S, const double* fn2, double rtol, double* tol,
                          double* fnorm, double* u, cudaStream_t s);
void seg_gmres_start_launch(int nseg, int m, const double* beta2, const double* tol, double* g,
                            double* inv, int* active, int* jend, double* summary, cudaStream_t s);
void seg_gmres_givens_launch(int nseg, int m, int j, const double* h1, const double* h2, int ldh12,
                             const double* wn2, double* H, double* cs, double* sn, double* g,
                             double* inv, int* active, int* jend, int* its, const double* tol,
                             double* summary, cudaStream_t s);
void seg_gmres_backsolve_launch(int nseg, int m, const double* H, const double* g, const int* jend,
                                double* ny, cudaStream_t s);
void seg_cg_start_launch(int nseg, const double* rr, const double* tol, const double* rz,
                         double* rho, int* active, double* summary, cudaStream_t s);
void seg_cg_alpha_launch(int nseg, const double* rho, const double* pq, const int* active,
                         double* alpha, double* malpha, cudaStream_t s);
void seg_cg_beta_launch(int nseg, const double* rr, const double* tol, const double* rho_new,
                        double* rho, int* active, int* its, double* beta, double* summary,
                        cudaStream_t s);

// Counters of the batched local solves: zero-pivot blocks, F-points skipped by the
// projection, systems per size bucket (T <= 8, 16, 32, 64, 128, larger), and the
// algorithmic work: sum over systems of T^3, T^2 and T, and the gathered A entries.
struct LocalStats {
  long long singular = 0, empty = 0;
  long long hist[7] = {0, 0, 0, 0, 0, 0, 0};
  double sum_t3 = 0, sum_t2 = 0, sum_t = 0;
  long long gathered = 0;
  // execution configuration of the last persistent local-solve launch
  int config_kind_b1 = -1, config_kind_b3 = -1, config_blocks_per_sm = 0, config_tuned = 0;
  // Optional device counters [singular, empty, sum T^3, sum T^2, sum T, gathered]: when set,
  // kernels add into them and no host read happens per call (read once by the owner).
  unsigned long long* dev = nullptr;
  void absorb_device(cudaStream_t s);  // adds the device counters in, zeroes them (syncs)
};

// Kernel launches issued by this library (monotonic, process-wide).
void count_launch();
void count_launches(long long delta);  // graph replays (+), captures that issued nothing (-)
long long launch_count();

// Device time per phase, measured with CUDA events on the launching stream.  Phases are
// nested by nobody: begin() closes nothing, end() closes the last begin().
enum Phase {
  PH_SPLIT = 0,   // transpose, row maxima, strength, C/F splitting
  PH_WEIGHT,      // Arnoldi relaxation weight
  PH_SMOOTH,      // mode-vector smoothing
  PH_PATTERN,     // transfer sparsity patterns
  PH_LSOLVE,      // batched local gathers + solves (the hot kernels)
  PH_PROJECT,     // transposes + constraint projection
  PH_GALERKIN,    // R A P
  PH_COARSE,      // coarsest inverse, float copies
  PH_VCYCLE,      // V(1,1) cycles
  PH_KRYLOV,      // FGMRES orthogonalisation, residuals, updates
  PH_COUNT
};

class PhaseClock {
 public:
  int begin(int ph, cudaStream_t s);    // returns the mark to close
  void end(int mark, cudaStream_t s);
  // synchronises; adds elapsed ms per phase (and, with level_ms, per level and phase:
  // level_ms[level * PH_COUNT + phase] for levels below max_levels); clears
  void collect(double* ms_out, double* level_ms = nullptr, int max_levels = 0);
  void set_level(int level) { level_ = level; }
  ~PhaseClock();

 private:
  struct Mark {
    int ph, level;
    cudaEvent_t a, b;
  };
  Mark* marks_ = nullptr;
  int n_ = 0, cap_ = 0, level_ = 0;
};
PhaseClock* active_clock();
void set_active_clock(PhaseClock* c);

struct ClockScope {  // times the launches a block of host code makes on `s` as one phase
  ClockScope(int ph, cudaStream_t s) : s_(s) {
    if (active_clock()) mark_ = active_clock()->begin(ph, s);
  }
  ~ClockScope() {
    if (active_clock() && mark_ >= 0) active_clock()->end(mark_, s_);
  }
  cudaStream_t s_;
  int mark_ = -1;
};

}  // namespace clair
