// Sparse building blocks of the CLAIR library: scan, deterministic CSR transpose,
// row maxima, sub-warp SpMV, deterministic Gustavson SpGEMM for the Galerkin product
// A_c = R A P (Section 1), and fixed-order reductions for the FP64 Krylov solver.
#include <stdarg.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <set>
#include <utility>
#include <vector>

#include "common.cuh"

namespace clair {

static thread_local std::string g_last_error;

void set_error(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
}

const char* last_error() { return g_last_error.c_str(); }
void clear_error() { g_last_error.clear(); }

int sm_count() {
  static int cached = 0;
  if (!cached) {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    cached = v > 0 ? v : 148;
  }
  return cached;
}

int partial_blocks() { return 2 * sm_count(); }

void once_per_device(const void* tag, void (*set)()) {
  static std::mutex mu;
  static std::set<std::pair<int, const void*>> done;
  int dev = 0;
  CLAIR_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  if (done.count({dev, tag})) return;
  set();
  done.insert({dev, tag});
}

// Pinned host blocks, kept for the life of the process: a setup takes a few small ones
// per level (the Ritz steps) and a solve one (the Krylov summary), and pinning pages in
// the driver costs far more than the copies they serve.  Blocks are recycled by size
// class (powers of two from 256 bytes); portable, so any device's context may use them.
static std::mutex g_pinned_mu;
static std::vector<void*> g_pinned_free[48];

static int pinned_class(size_t bytes, size_t* rounded) {
  int c = 8;
  while (((size_t)1 << c) < bytes) ++c;
  *rounded = (size_t)1 << c;
  return c;
}

void* pinned_get(size_t bytes) {
  size_t rb = 0;
  const int c = pinned_class(bytes, &rb);
  {
    std::lock_guard<std::mutex> lock(g_pinned_mu);
    if (!g_pinned_free[c].empty()) {
      void* p = g_pinned_free[c].back();
      g_pinned_free[c].pop_back();
      return p;
    }
  }
  void* p = nullptr;
  CLAIR_CUDA(cudaHostAlloc(&p, rb, cudaHostAllocPortable));
  return p;
}

void pinned_put(void* p, size_t bytes) {
  if (!p) return;
  size_t rb = 0;
  const int c = pinned_class(bytes, &rb);
  std::lock_guard<std::mutex> lock(g_pinned_mu);
  g_pinned_free[c].push_back(p);
}

cudaMemPool_t library_pool() {
  static std::mutex mu;
  static cudaMemPool_t pools[256] = {};
  int dev = 0;
  CLAIR_CUDA(cudaGetDevice(&dev));
  CLAIR_REQUIRE(dev >= 0 && dev < 256, CLAIR_ERR_ARG, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lock(mu);
  if (!pools[dev]) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool;
    CLAIR_CUDA(cudaMemPoolCreate(&pool, &props));
    uint64_t keep = ~0ull;
    CLAIR_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
    pools[dev] = pool;
  }
  return pools[dev];
}

static std::atomic<long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void count_launches(long long delta) { g_launches.fetch_add(delta, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(); }

static thread_local PhaseClock* g_clock = nullptr;
PhaseClock* active_clock() { return g_clock; }
void set_active_clock(PhaseClock* c) { g_clock = c; }

int PhaseClock::begin(int ph, cudaStream_t s) {
  if (n_ == cap_) {
    int cap = cap_ ? 2 * cap_ : 64;
    Mark* m = new Mark[cap];
    for (int i = 0; i < n_; ++i) m[i] = marks_[i];
    delete[] marks_;
    marks_ = m;
    cap_ = cap;
  }
  Mark& m = marks_[n_++];
  m.ph = ph;
  m.level = level_;
  cudaEventCreate(&m.a);
  cudaEventCreate(&m.b);
  cudaEventRecord(m.a, s);
  return n_ - 1;
}

void PhaseClock::end(int mark, cudaStream_t s) {
  if (mark >= 0 && mark < n_) cudaEventRecord(marks_[mark].b, s);
}

void PhaseClock::collect(double* ms_out, double* level_ms, int max_levels) {
  for (int i = 0; i < n_; ++i) cudaEventSynchronize(marks_[i].b);
  for (int i = 0; i < n_; ++i) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, marks_[i].a, marks_[i].b) == cudaSuccess) {
      ms_out[marks_[i].ph] += ms;
      if (level_ms && marks_[i].level < max_levels)
        level_ms[marks_[i].level * PH_COUNT + marks_[i].ph] += ms;
    }
    cudaEventDestroy(marks_[i].a);
    cudaEventDestroy(marks_[i].b);
  }
  n_ = 0;
}

PhaseClock::~PhaseClock() {
  for (int i = 0; i < n_; ++i) {
    cudaEventDestroy(marks_[i].a);
    cudaEventDestroy(marks_[i].b);
  }
  delete[] marks_;
}

// ------------------------------------------------------------------------------------
// Exclusive scan (three phases: block sums, scan of sums in one block, block scans).
// ------------------------------------------------------------------------------------
constexpr int SCAN_THREADS = 512;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

template <class T>
__device__ T block_inclusive_scan(T v, T* sh) {
  // Hillis-Steele over warps then across warp totals; blockDim.x == SCAN_THREADS.
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  if (lane == 31) sh[wid] = v;
  __syncthreads();
  if (wid == 0) {
    T w = lane < (SCAN_THREADS / 32) ? sh[lane] : T(0);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T t = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += t;
    }
    sh[lane] = w;
  }
  __syncthreads();
  if (wid > 0) v += sh[wid - 1];
  __syncthreads();
  return v;
}

__global__ void scan_block_sums(const int* __restrict__ in, int n, long long* __restrict__ sums) {
  __shared__ long long sh[32];
  long long acc = 0;
  const long long base = (long long)blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    long long i = base + k;
    if (i < n) acc += in[i];
  }
  acc = block_inclusive_scan(acc, sh);
  if (threadIdx.x == SCAN_THREADS - 1) sums[blockIdx.x] = acc;
}

__global__ void scan_sums(long long* sums, int nb) {
  // single block; nb <= SCAN_TILE
  __shared__ long long sh[32];
  long long loc[SCAN_ITEMS];
  long long acc = 0;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    int i = threadIdx.x * SCAN_ITEMS + k;
    loc[k] = i < nb ? sums[i] : 0;
    acc += loc[k];
  }
  long long incl = block_inclusive_scan(acc, sh);
  long long run = incl - acc;  // exclusive prefix of this thread
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    int i = threadIdx.x * SCAN_ITEMS + k;
    if (i < nb) sums[i] = run;  // exclusive block offsets
    run += loc[k];
  }
}

__global__ void scan_apply(const int* __restrict__ in, int n, const long long* __restrict__ offs,
                           int* __restrict__ out, int* __restrict__ overflow) {
  __shared__ long long sh[32];
  long long loc[SCAN_ITEMS];
  long long acc = 0;
  const long long base = (long long)blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    long long i = base + k;
    loc[k] = i < n ? in[i] : 0;
    acc += loc[k];
  }
  long long incl = block_inclusive_scan(acc, sh);
  long long run = offs[blockIdx.x] + incl - acc;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    long long i = base + k;
    run += loc[k];
    if (i < n) {
      if (run > 0x7fffffffLL) *overflow = 1;
      out[i + 1] = (int)run;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) out[0] = 0;
}

// The whole scan in one block (n <= SCAN_TILE, every coarse level): one launch instead of
// three; writes the overflow flag whether or not it is set.
__global__ void scan_single(const int* __restrict__ in, int n, int* __restrict__ out,
                            int* __restrict__ overflow) {
  __shared__ long long sh[32];
  __shared__ int s_ovf;
  if (threadIdx.x == 0) s_ovf = 0;
  long long loc[SCAN_ITEMS];
  long long acc = 0;
  const int base = threadIdx.x * SCAN_ITEMS;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    const int i = base + k;
    loc[k] = i < n ? in[i] : 0;
    acc += loc[k];
  }
  long long run = block_inclusive_scan(acc, sh) - acc;  // (its barriers order s_ovf = 0)
  bool ov = false;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    const int i = base + k;
    run += loc[k];
    if (i < n) {
      ov = ov || run > 0x7fffffffLL;
      out[i + 1] = (int)run;
    }
  }
  if (ov) s_ovf = 1;
  if (threadIdx.x == 0) out[0] = 0;
  __syncthreads();
  if (threadIdx.x == 0) *overflow = s_ovf;
}

// out = exclusive scan of in (out[n] = total), *ovf = 1 if the total exceeds int32; no
// host synchronisation (the caller reads out[n] and *ovf when it synchronises anyway).
void exclusive_scan_into(const int* in, int* out, int n, int* ovf, cudaStream_t s) {
  const int nb = std::max(1, ceil_div(n, SCAN_TILE));
  CLAIR_REQUIRE(nb <= SCAN_TILE, CLAIR_ERR_CAPACITY, "scan of %d items exceeds capacity", n);
  CLAIR_CUDA(cudaMemsetAsync(ovf, 0, sizeof(int), s));
  if (nb == 1) {
    scan_single<<<1, SCAN_THREADS, 0, s>>>(in, n, out, ovf); ::clair::count_launch();
  } else {
    long long* sums = dalloc<long long>(nb + 1, s);
    scan_block_sums<<<nb, SCAN_THREADS, 0, s>>>(in, n, sums); ::clair::count_launch();
    scan_sums<<<1, SCAN_THREADS, 0, s>>>(sums, nb); ::clair::count_launch();
    scan_apply<<<nb, SCAN_THREADS, 0, s>>>(in, n, sums, out, ovf); ::clair::count_launch();
    dfree(sums, s);
  }
  CLAIR_LAUNCHED();
}

long long exclusive_scan(const int* in, int* out, int n, cudaStream_t s, bool want_total,
                         const int* extra_dev, int* extra_host) {
  const int nb = std::max(1, ceil_div(n, SCAN_TILE));
  CLAIR_REQUIRE(nb <= SCAN_TILE, CLAIR_ERR_CAPACITY, "scan of %d items exceeds capacity", n);
  long long* sums = nullptr;
  int* ovf = dalloc<int>(1, s);
  if (nb == 1) {
    scan_single<<<1, SCAN_THREADS, 0, s>>>(in, n, out, ovf); ::clair::count_launch();
  } else {
    sums = dalloc<long long>(nb + 1, s);
    CLAIR_CUDA(cudaMemsetAsync(ovf, 0, sizeof(int), s));
    scan_block_sums<<<nb, SCAN_THREADS, 0, s>>>(in, n, sums); ::clair::count_launch();
    scan_sums<<<1, SCAN_THREADS, 0, s>>>(sums, nb); ::clair::count_launch();
    scan_apply<<<nb, SCAN_THREADS, 0, s>>>(in, n, sums, out, ovf); ::clair::count_launch();
  }
  CLAIR_LAUNCHED();
  long long total = 0;
  if (want_total) {
    int total32 = 0, h_ovf = 0;
    CLAIR_CUDA(cudaMemcpyAsync(&total32, out + n, sizeof(int), cudaMemcpyDeviceToHost, s));
    CLAIR_CUDA(cudaMemcpyAsync(&h_ovf, ovf, sizeof(int), cudaMemcpyDeviceToHost, s));
    if (extra_dev)
      CLAIR_CUDA(cudaMemcpyAsync(extra_host, extra_dev, sizeof(int), cudaMemcpyDeviceToHost, s));
    CLAIR_CUDA(cudaStreamSynchronize(s));
    CLAIR_REQUIRE(!h_ovf, CLAIR_ERR_CAPACITY, "scan total exceeds int32");
    total = total32;
  }
  dfree(sums, s);
  dfree(ovf, s);
  return total;
}

// ------------------------------------------------------------------------------------
// CSR transpose: column counts, scan, atomic fill, then a per-row insertion sort makes
// the result independent of the atomic order.
// ------------------------------------------------------------------------------------
__global__ void count_cols(const int* __restrict__ col, int nnz, int* __restrict__ cnt) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nnz;
       e += (long long)gridDim.x * blockDim.x)
    atomicAdd(&cnt[col[e]], 1);
}

// W lanes per row, so a long row is not one thread's chain of atomics; the slot order
// within a column is arbitrary here and fixed by the segment sort that follows.
template <int W>
__global__ void transpose_fill(const int* __restrict__ rowptr, const int* __restrict__ col,
                               int rows, int* __restrict__ cursor, int* __restrict__ col_t,
                               int* __restrict__ perm) {
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long r = g / W;
  if (r >= rows) return;
  for (int e = rowptr[r] + (int)(g % W); e < rowptr[r + 1]; e += W) {
    const int pos = atomicAdd(&cursor[col[e]], 1);
    col_t[pos] = (int)r;
    perm[pos] = e;
  }
}

__global__ void sort_segments(const int* __restrict__ rowptr, int rows, int* __restrict__ key,
                              int* __restrict__ perm) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  const int b = rowptr[r], e = rowptr[r + 1];
  for (int i = b + 1; i < e; ++i) {
    int k = key[i], p = perm[i], j = i - 1;
    while (j >= b && key[j] > k) {
      key[j + 1] = key[j];
      perm[j + 1] = perm[j];
      --j;
    }
    key[j + 1] = k;
    perm[j + 1] = p;
  }
}

// W lanes per segment: every entry goes to its rank among the segment's (distinct) keys.
template <int W>
__global__ void sort_segments_warp(const int* __restrict__ rowptr, int rows,
                                   const int* __restrict__ key, const int* __restrict__ perm,
                                   int* __restrict__ key_out, int* __restrict__ perm_out) {
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long w = g / W;
  if (w >= rows) return;
  const int b = rowptr[w], L = rowptr[w + 1] - b;
  for (int t = (int)(g % W); t < L; t += W) {
    const int k = key[b + t];
    int rank = 0;
    for (int u = 0; u < L; ++u) rank += key[b + u] < k;
    key_out[b + rank] = k;
    perm_out[b + rank] = perm[b + t];
  }
}

__global__ void gather_kernel(const double* __restrict__ x, const int* __restrict__ idx,
                              double* __restrict__ y, int n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = x[idx[i]];
}

__global__ void scatter_kernel(const double* __restrict__ x, const int* __restrict__ idx,
                               double* __restrict__ y, int n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[idx[i]] = x[i];
}

static int grid_for(long long n, int threads = 256) {
  long long g = (n + threads - 1) / threads;
  long long cap = 32LL * sm_count();
  return (int)std::max(1LL, std::min(g, cap));
}

void gather(const double* x, const int* idx, double* y, int n, cudaStream_t s) {
  if (n <= 0) return;
  gather_kernel<<<grid_for(n), 256, 0, s>>>(x, idx, y, n); ::clair::count_launch();
  CLAIR_LAUNCHED();
}
void gather_vals(const double* x, const int* perm, double* y, int n, cudaStream_t s) {
  gather(x, perm, y, n, s);
}
void scatter_vals(const double* x, const int* perm, double* y, int n, cudaStream_t s) {
  if (n <= 0) return;
  scatter_kernel<<<grid_for(n), 256, 0, s>>>(x, perm, y, n); ::clair::count_launch();
  CLAIR_LAUNCHED();
}

void csr_transpose(const Csr& A, Csr& At, int** perm_out, cudaStream_t s) {
  At.rows = A.cols;
  At.cols = A.rows;
  At.nnz = A.nnz;
  int* cnt = dalloc<int>(A.cols + 1, s);
  CLAIR_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * (A.cols + 1), s));
  if (A.nnz) count_cols<<<grid_for(A.nnz), 256, 0, s>>>(A.col, A.nnz, cnt); ::clair::count_launch();
  At.rowptr = dalloc<int>(A.cols + 1, s);
  exclusive_scan(cnt, At.rowptr, A.cols, s, false);
  CLAIR_CUDA(cudaMemcpyAsync(cnt, At.rowptr, sizeof(int) * A.cols, cudaMemcpyDeviceToDevice, s));
  int* col_fill = dalloc<int>(A.nnz, s);
  int* perm_fill = dalloc<int>(A.nnz, s);
  At.col = dalloc<int>(A.nnz, s);
  int* perm = dalloc<int>(A.nnz, s);
  if (A.rows) {
    const double mean = (double)A.nnz / A.rows;
    const int W = mean <= 2.0 ? 1 : mean <= 8.0 ? 4 : mean <= 32.0 ? 8 : 32;
    const int grid = (int)ceil_div((long long)A.rows * W, 256);
    switch (W) {
      case 1: transpose_fill<1><<<grid, 256, 0, s>>>(A.rowptr, A.col, A.rows, cnt, col_fill, perm_fill); break;
      case 4: transpose_fill<4><<<grid, 256, 0, s>>>(A.rowptr, A.col, A.rows, cnt, col_fill, perm_fill); break;
      case 8: transpose_fill<8><<<grid, 256, 0, s>>>(A.rowptr, A.col, A.rows, cnt, col_fill, perm_fill); break;
      default: transpose_fill<32><<<grid, 256, 0, s>>>(A.rowptr, A.col, A.rows, cnt, col_fill, perm_fill); break;
    }
    ::clair::count_launch();
  }
  if (At.rows) {
    const double mean = (double)A.nnz / At.rows;
    const int W = mean <= 4.0 ? 4 : mean <= 8.0 ? 8 : mean <= 16.0 ? 16 : 32;
    const int grid = ceil_div((long long)At.rows * W, 256);
    switch (W) {
      case 4: sort_segments_warp<4><<<grid, 256, 0, s>>>(At.rowptr, At.rows, col_fill, perm_fill, At.col, perm); break;
      case 8: sort_segments_warp<8><<<grid, 256, 0, s>>>(At.rowptr, At.rows, col_fill, perm_fill, At.col, perm); break;
      case 16: sort_segments_warp<16><<<grid, 256, 0, s>>>(At.rowptr, At.rows, col_fill, perm_fill, At.col, perm); break;
      default: sort_segments_warp<32><<<grid, 256, 0, s>>>(At.rowptr, At.rows, col_fill, perm_fill, At.col, perm); break;
    }
    ::clair::count_launch();
  }
  CLAIR_LAUNCHED();
  dfree(col_fill, s);
  dfree(perm_fill, s);
  if (A.val) {
    At.val = dalloc<double>(A.nnz, s);
    gather(A.val, perm, At.val, A.nnz, s);
  }
  dfree(cnt, s);
  if (perm_out)
    *perm_out = perm;
  else
    dfree(perm, s);
}

// ------------------------------------------------------------------------------------
// Row kernels with W lanes per row.  FP64 kernels use one thread per row: on this GPU an
// FP64 warp instruction costs the SM's FP64 unit about 16 cycles however few lanes are
// active, so sub-warp groups (idle lanes, shuffle-add trees) waste most of it.  FP32
// kernels use W lanes per row, W the power of two at or above the mean row length.
// ------------------------------------------------------------------------------------
// FP32: W >= the mean row length.  FP64: an FP64 warp instruction costs about the same
// with 1 or 32 active lanes, so short rows run one per thread; long rows (coarse levels)
// would then be one thread's chain of dependent index and value loads, so they get lanes
// at about four entries per lane.
static thread_local int g_short_lanes = 0;
int cycle_short_lanes() { return g_short_lanes; }
void set_cycle_short_lanes(int lanes) { g_short_lanes = lanes; }
static thread_local bool g_pdl = false;
bool pdl_launches() { return g_pdl; }
void set_pdl_launches(bool on) { g_pdl = on; }

static int lanes_for(const Csr& A, bool fp64) {
  double avg = A.rows ? (double)A.nnz / A.rows : 1.0;
  if (fp64 || g_short_lanes == 1) {
    if (avg <= 8.0) return 1;
    int w = 2;
    while (w < 32 && 4 * w < avg) w <<= 1;
    return w;
  }
  if (g_short_lanes == 2) {  // FP32, about eight entries per lane (one thread up to 16 entries)
    if (avg <= 16.0) return 1;
    int w = 2;
    while (w < 32 && 8 * w < avg) w <<= 1;
    return w;
  }
  int w = 2;
  while (w < 32 && w < avg) w <<= 1;
  return w;
}

template <int W>
__global__ void rowmax_kernel(const int* __restrict__ rowptr, const int* __restrict__ col,
                              const double* __restrict__ val, int rows, double* __restrict__ out) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int r = (int)(t / W), lane = (int)(t % W);
  const bool ok = r < rows;  // no early exit: every lane takes part in the shuffles
  double m = 0.0;
  if (ok)
    for (int e = rowptr[r] + lane; e < rowptr[r + 1]; e += W)
      if (col[e] != r) m = fmax(m, fabs(val[e]));
#pragma unroll
  for (int o = W / 2; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o, W));
  if (ok && lane == 0) out[r] = m;
}

#define CLAIR_DISPATCH_W(W, ...)             \
  switch (W) {                               \
    case 1: { constexpr int WW = 1; __VA_ARGS__; ::clair::count_launch(); } break;   \
    case 2: { constexpr int WW = 2; __VA_ARGS__; ::clair::count_launch(); } break;   \
    case 4: { constexpr int WW = 4; __VA_ARGS__; ::clair::count_launch(); } break;   \
    case 8: { constexpr int WW = 8; __VA_ARGS__; ::clair::count_launch(); } break;   \
    case 16: { constexpr int WW = 16; __VA_ARGS__; ::clair::count_launch(); } break; \
    default: { constexpr int WW = 32; __VA_ARGS__; ::clair::count_launch(); } break; \
  }

void row_max_offdiag(const Csr& A, double* out, cudaStream_t s) {
  if (!A.rows) return;
  int W = lanes_for(A, true);
  long long threads = (long long)A.rows * W;
  int blocks = ceil_div(threads, 256);
  CLAIR_DISPATCH_W(W, rowmax_kernel<WW><<<blocks, 256, 0, s>>>(A.rowptr, A.col, A.val, A.rows, out));
  CLAIR_LAUNCHED();
}

template <int W, class T, bool RESID>
__global__ void spmv_kernel(const int* __restrict__ rowptr, const int* __restrict__ col,
                            const T* __restrict__ val, int rows, const T* __restrict__ x,
                            const T* __restrict__ b, T* __restrict__ y, T alpha, T beta) {
  pdl_prologue();
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int r = (int)(t / W), lane = (int)(t % W);
  const bool ok = r < rows;  // no early exit: every lane takes part in the shuffles
  T acc = 0;
  if (ok)
    acc = csr_row_dot<W>(col, val, x, rowptr[r], rowptr[r + 1], lane);
  acc = group_sum<W>(acc);
  if (ok && lane == 0) {
    if (RESID)
      y[r] = b[r] - acc;
    else
      y[r] = beta == T(0) ? alpha * acc : alpha * acc + beta * y[r];
  }
}

template <class T, bool RESID>
static void spmv_launch(const Csr& A, const T* vals, const T* x, const T* b, T* y, T alpha, T beta,
                        cudaStream_t s) {
  if (!A.rows) return;
  int W = lanes_for(A, sizeof(T) == 8);
  long long threads = (long long)A.rows * W;
  int blocks = ceil_div(threads, 256);
  CLAIR_DISPATCH_W(W, launch_k(spmv_kernel<WW, T, RESID>, blocks, 256, 0, s, A.rowptr, A.col, vals,
                                A.rows, x, b, y, alpha, beta));
  CLAIR_LAUNCHED();
}

void spmv(const Csr& A, const double* x, double* y, double alpha, double beta, cudaStream_t s) {
  spmv_launch<double, false>(A, A.val, x, nullptr, y, alpha, beta, s);
}
void spmv32(const Csr& A, const float* x, float* y, float alpha, float beta, cudaStream_t s) {
  spmv_launch<float, false>(A, A.val32, x, nullptr, y, alpha, beta, s);
}
void residual(const Csr& A, const double* b, const double* x, double* r, cudaStream_t s) {
  spmv_launch<double, true>(A, A.val, x, b, r, 1.0, 0.0, s);
}
void residual32(const Csr& A, const float* b, const float* x, float* r, cudaStream_t s) {
  spmv_launch<float, true>(A, A.val32, x, b, r, 1.f, 0.f, s);
}

// W lanes per row; the row's last entry in column r is its diagonal.
template <int W>
__global__ void inv_diag_kernel(const int* __restrict__ rowptr, const int* __restrict__ col,
                                const double* __restrict__ val, int rows, double* __restrict__ dinv,
                                int* __restrict__ bad) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int r = (int)(t / W), sub = (int)(t % W);
  int last = -1;
  if (r < rows)
    for (int e = rowptr[r] + sub; e < rowptr[r + 1]; e += W)
      if (col[e] == r) last = e;
#pragma unroll
  for (int o = W / 2; o > 0; o >>= 1) last = max(last, __shfl_xor_sync(0xffffffffu, last, o, W));
  if (r >= rows || sub != 0) return;
  const double d = last >= 0 ? val[last] : 0.0;
  if (d == 0.0 || !isfinite(d)) atomicAdd(bad, 1);
  dinv[r] = d != 0.0 ? 1.0 / d : 0.0;
}

void inverse_diagonal(const Csr& A, double* dinv, cudaStream_t s, int* bad_acc) {
  const double avg = A.rows ? (double)A.nnz / A.rows : 1.0;
  int W = 1;
  while (W < 32 && 4 * W < avg) W <<= 1;
  const int blocks = (int)ceil_div((long long)A.rows * W, 256);
  if (bad_acc) {  // the caller reads the count later, at a synchronisation it makes anyway
    if (A.rows)
      CLAIR_DISPATCH_W(W, (inv_diag_kernel<WW><<<blocks, 256, 0, s>>>(A.rowptr, A.col, A.val,
                                                                       A.rows, dinv, bad_acc)));
    CLAIR_LAUNCHED();
    return;
  }
  int* bad = dalloc<int>(1, s);
  CLAIR_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
  if (A.rows)
    CLAIR_DISPATCH_W(W, (inv_diag_kernel<WW><<<blocks, 256, 0, s>>>(A.rowptr, A.col, A.val, A.rows,
                                                                     dinv, bad)));
  CLAIR_LAUNCHED();
  int h = 0;
  CLAIR_CUDA(cudaMemcpyAsync(&h, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
  CLAIR_CUDA(cudaStreamSynchronize(s));
  dfree(bad, s);
  CLAIR_REQUIRE(h == 0, CLAIR_ERR_ARG, "%d rows with a missing, zero or nonfinite diagonal", h);
}

__global__ void to_float_kernel(const double* __restrict__ x, float* __restrict__ y, long long n) {
  pdl_prologue();
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = (float)x[i];
}
__global__ void to_double_kernel(const float* __restrict__ x, double* __restrict__ y, long long n) {
  pdl_prologue();
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = (double)x[i];
}
__global__ void copy_f64_kernel(const double* __restrict__ x, double* __restrict__ y, long long n) {
  pdl_prologue();
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = x[i];
}
void copy_f64(const double* x, double* y, long long n, cudaStream_t s) {
  if (n <= 0) return;
  launch_k(copy_f64_kernel, grid_for(n), 256, 0, s, x, y, n); ::clair::count_launch();
  CLAIR_LAUNCHED();
}
void to_float(const double* x, float* y, long long n, cudaStream_t s) {
  if (n <= 0) return;
  launch_k(to_float_kernel, grid_for(n), 256, 0, s, x, y, n); ::clair::count_launch();
  CLAIR_LAUNCHED();
}
void to_double(const float* x, double* y, long long n, cudaStream_t s) {
  if (n <= 0) return;
  launch_k(to_double_kernel, grid_for(n), 256, 0, s, x, y, n); ::clair::count_launch();
  CLAIR_LAUNCHED();
}

// ------------------------------------------------------------------------------------
// Deterministic multi-dot: partial sums per block in a fixed order, then a fixed-order
// reduction of the partials.
// ------------------------------------------------------------------------------------
constexpr int DOT_THREADS = 256;
constexpr int DOT_GROUP = 8;

__global__ void multi_dot_partial(const double* __restrict__ V, int m, const double* __restrict__ w,
                                  long long n, double* __restrict__ partial) {
  __shared__ double sh[DOT_GROUP][DOT_THREADS / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int j0 = 0; j0 < m; j0 += DOT_GROUP) {
    double acc[DOT_GROUP];
#pragma unroll
    for (int g = 0; g < DOT_GROUP; ++g) acc[g] = 0.0;
    for (long long i = blockIdx.x * (long long)DOT_THREADS + threadIdx.x; i < n;
         i += (long long)gridDim.x * DOT_THREADS) {
      const double wi = w[i];
#pragma unroll
      for (int g = 0; g < DOT_GROUP; ++g)
        if (j0 + g < m) acc[g] = fma(V[(long long)(j0 + g) * n + i], wi, acc[g]);
    }
#pragma unroll
    for (int g = 0; g < DOT_GROUP; ++g) {
      double v = warp_sum(acc[g]);
      if (lane == 0) sh[g][wid] = v;
    }
    __syncthreads();
    if (threadIdx.x < DOT_GROUP && j0 + threadIdx.x < m) {
      double v = 0.0;
      for (int k = 0; k < DOT_THREADS / 32; ++k) v += sh[threadIdx.x][k];
      partial[(long long)(j0 + threadIdx.x) * gridDim.x + blockIdx.x] = v;
    }
    __syncthreads();
  }
}

__global__ void multi_dot_final(const double* __restrict__ partial, int nblocks, int m,
                                double* __restrict__ out) {
  // one warp per vector, fixed order
  const int j = blockIdx.x;
  if (j >= m) return;
  double v = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += 32) v += partial[(long long)j * nblocks + b];
  v = warp_sum(v);
  if (threadIdx.x == 0) out[j] = v;
}

void multi_dot(const double* V, int m, const double* w, int n, double* out, double* partial,
               cudaStream_t s) {
  if (m <= 0) return;
  int nb = partial_blocks();
  multi_dot_partial<<<nb, DOT_THREADS, 0, s>>>(V, m, w, n, partial); ::clair::count_launch();
  multi_dot_final<<<m, 32, 0, s>>>(partial, nb, m, out); ::clair::count_launch();
  CLAIR_LAUNCHED();
}

__global__ void multi_axpy_kernel(const double* __restrict__ V, int m, const double* __restrict__ h,
                                  double* __restrict__ w, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    double acc = w[i];
    for (int j = 0; j < m; ++j) acc = fma(-h[j], V[(long long)j * n + i], acc);
    w[i] = acc;
  }
}

void multi_axpy(const double* V, int m, const double* h, double* w, int n, cudaStream_t s) {
  if (m <= 0 || n <= 0) return;
  multi_axpy_kernel<<<grid_for(n), 256, 0, s>>>(V, m, h, w, n); ::clair::count_launch();
  CLAIR_LAUNCHED();
}

__global__ void finite_kernel(const double* __restrict__ x, long long n, int* bad) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    if (!isfinite(x[i])) *bad = 1;
}

// max |x| (non-negative doubles order as their bit patterns)
__global__ void absmax_kernel(const double* __restrict__ x, long long n,
                              unsigned long long* __restrict__ out) {
  double m = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    m = fmax(m, fabs(x[i]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m > 0.0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

void absmax_into(const double* x, long long n, unsigned long long* out, cudaStream_t s) {
  if (n <= 0) return;
  absmax_kernel<<<grid_for(n), 256, 0, s>>>(x, n, out); ::clair::count_launch();
  CLAIR_LAUNCHED();
}

// Many short conversions or maxima in one launch: blockIdx.y picks the segment, the x
// blocks stride over it (the end of a setup holds a few per level).
__global__ void to_float_segments(SegList L) {
  const int g = blockIdx.y;
  const double* __restrict__ x = L.src[g];
  float* __restrict__ y = L.dst[g];
  const long long n = L.n[g];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = (float)x[i];
}

__global__ void absmax_segments(SegList L, unsigned long long* __restrict__ out) {
  const int g = blockIdx.y;
  const double* __restrict__ x = L.src[g];
  const long long n = L.n[g];
  double m = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    m = fmax(m, fabs(x[i]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m > 0.0)
    atomicMax(out + L.slot[g], (unsigned long long)__double_as_longlong(m));
}

static dim3 seg_grid(const SegList& L) {
  long long mx = 1;
  for (int g = 0; g < L.count; ++g) mx = std::max(mx, L.n[g]);
  return dim3((unsigned)std::min<long long>(ceil_div(mx, 256), 4LL * sm_count()), (unsigned)L.count);
}

void SegBatch::add(const double* src, float* dst, long long n, int slot) {
  if (n <= 0) return;
  if (cur.count == SegList::kMax) flush();
  cur.src[cur.count] = src;
  cur.dst[cur.count] = dst;
  cur.n[cur.count] = n;
  cur.slot[cur.count] = slot;
  ++cur.count;
}

void SegBatch::flush() {
  if (!cur.count) return;
  if (out)
    absmax_segments<<<seg_grid(cur), 256, 0, s>>>(cur, out);
  else
    to_float_segments<<<seg_grid(cur), 256, 0, s>>>(cur);
  ::clair::count_launch();
  CLAIR_LAUNCHED();
  cur.count = 0;
}

bool all_finite(const double* x, long long n, cudaStream_t s) {
  if (n <= 0) return true;
  int* bad = dalloc<int>(1, s);
  CLAIR_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
  finite_kernel<<<grid_for(n), 256, 0, s>>>(x, n, bad); ::clair::count_launch();
  CLAIR_LAUNCHED();
  int h = 0;
  CLAIR_CUDA(cudaMemcpyAsync(&h, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
  CLAIR_CUDA(cudaStreamSynchronize(s));
  dfree(bad, s);
  return h == 0;
}

// ------------------------------------------------------------------------------------
// Input validation of a caller's CSR: rowptr[0] = 0, nondecreasing, rowptr[rows] = nnz,
// columns in [0, cols) and strictly increasing within each row.
// ------------------------------------------------------------------------------------
__global__ void validate_rows(const int* __restrict__ rowptr, const int* __restrict__ col, int rows,
                              int cols, int nnz, int* __restrict__ bad) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  const int b = rowptr[r], e = rowptr[r + 1];
  if ((r == 0 && b != 0) || e < b || b < 0 || e > nnz || (r == rows - 1 && e != nnz)) {
    atomicAdd(bad, 1);
    return;
  }
  int prev = -1;
  for (int k = b; k < e; ++k) {
    const int c = col[k];
    if (c < 0 || c >= cols || c <= prev) {
      atomicAdd(bad, 1);
      return;
    }
    prev = c;
  }
}

__global__ void validate_flags(const signed char* __restrict__ f, int n, int* __restrict__ bad) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && f[i] != 0 && f[i] != 1) atomicAdd(bad, 1);
}

void validate_csr(const int* rowptr, const int* col, int rows, int cols, int nnz, const char* what,
                  cudaStream_t s) {
  CLAIR_REQUIRE(rows >= 0 && nnz >= 0, CLAIR_ERR_ARG, "%s: negative size", what);
  if (!rows) return;
  int* bad = dalloc<int>(1, s);
  CLAIR_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
  int h_rp[2] = {0, 0};
  CLAIR_CUDA(cudaMemcpyAsync(&h_rp[0], rowptr, sizeof(int), cudaMemcpyDeviceToHost, s));
  CLAIR_CUDA(cudaMemcpyAsync(&h_rp[1], rowptr + rows, sizeof(int), cudaMemcpyDeviceToHost, s));
  CLAIR_CUDA(cudaStreamSynchronize(s));
  if (h_rp[0] == 0 && h_rp[1] == nnz) {
    validate_rows<<<ceil_div(rows, 256), 256, 0, s>>>(rowptr, col, rows, cols, nnz, bad); ::clair::count_launch();
    CLAIR_LAUNCHED();
  }
  int h = 0;
  CLAIR_CUDA(cudaMemcpyAsync(&h, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
  CLAIR_CUDA(cudaStreamSynchronize(s));
  dfree(bad, s);
  CLAIR_REQUIRE(h_rp[0] == 0 && h_rp[1] == nnz, CLAIR_ERR_ARG,
                "%s: rowptr[0]=%d rowptr[rows]=%d, expected 0 and %d", what, h_rp[0], h_rp[1], nnz);
  CLAIR_REQUIRE(h == 0, CLAIR_ERR_ARG,
                "%s: %d rows with bad row pointers or unsorted/out-of-range columns", what, h);
}

void validate_cf(const signed char* cf, int n, cudaStream_t s) {
  if (!n) return;
  int* bad = dalloc<int>(1, s);
  CLAIR_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
  validate_flags<<<ceil_div(n, 256), 256, 0, s>>>(cf, n, bad); ::clair::count_launch();
  CLAIR_LAUNCHED();
  int h = 0;
  CLAIR_CUDA(cudaMemcpyAsync(&h, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
  CLAIR_CUDA(cudaStreamSynchronize(s));
  dfree(bad, s);
  CLAIR_REQUIRE(h == 0, CLAIR_ERR_ARG, "cf has %d entries other than 0/1", h);
}

// ------------------------------------------------------------------------------------
// SpGEMM C = A B (Gustavson).  One warp per row of A; the row's entries k are taken in
// stored (ascending column) order and, for each k, the lanes add a_ik * b_kj for the
// distinct j of row k into a shared-memory hash table.  Every output entry therefore
// sums its products in increasing k, with separate multiply and add (no contraction),
// independent of scheduling.  Rows whose product count exceeds the small table go to a
// one-warp-per-block path with a large dynamic table.
// ------------------------------------------------------------------------------------
constexpr int SG_LARGE = 16384;       // slots (large path)

__device__ __forceinline__ int sg_hash(int key, int cap) {
  return (int)(((unsigned)key * 2654435761u) & (unsigned)(cap - 1));
}

// Inserts key; returns slot (or -1 if the table is full).
__device__ __forceinline__ int sg_insert(int* keys, int cap, int key, bool* is_new) {
  int h = sg_hash(key, cap);
  for (int probe = 0; probe < cap; ++probe) {
    int prev = atomicCAS(&keys[h], -1, key);
    if (prev == -1) {
      *is_new = true;
      return h;
    }
    if (prev == key) {
      *is_new = false;
      return h;
    }
    h = (h + 1) & (cap - 1);
  }
  return -1;
}

// One warp processes row r.  NUMERIC = false: count[r] = number of distinct columns, or
// -1 if they do not fit the table (the row is then redone with a larger one).
// NUMERIC = true (the table holds at least twice the row's count): writes the row sorted
// by column.  keys/vals: the warp's table of `cap` slots.
template <bool NUMERIC>
__device__ void spgemm_row(int r, const int* __restrict__ Arp, const int* __restrict__ Acol,
                           const double* __restrict__ Aval, const int* __restrict__ Brp,
                           const int* __restrict__ Bcol, const double* __restrict__ Bval, int* keys,
                           double* vals, int cap, int* __restrict__ count,
                           const int* __restrict__ Crp, int* __restrict__ Ccol,
                           double* __restrict__ Cval) {
  const int lane = threadIdx.x & 31;
  for (int s = lane; s < cap; s += 32) {
    keys[s] = -1;
    if (NUMERIC) vals[s] = 0.0;
  }
  __syncwarp();
  int mine = 0;
  bool full = false;
  for (int ea = Arp[r]; ea < Arp[r + 1]; ++ea) {
    const int k = Acol[ea];
    const double a = NUMERIC ? Aval[ea] : 0.0;
    for (int eb = Brp[k] + lane; eb < Brp[k + 1]; eb += 32) {
      bool is_new;
      const int slot = sg_insert(keys, cap, Bcol[eb], &is_new);
      if (slot < 0) {
        full = true;
        break;
      }
      if (is_new) ++mine;
      if (NUMERIC) vals[slot] = __dadd_rn(vals[slot], __dmul_rn(a, Bval[eb]));
    }
    if (__any_sync(0xffffffffu, full)) break;  // uniform across the warp
  }
  if (!NUMERIC) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
    const bool overflow = __any_sync(0xffffffffu, full);  // all lanes vote
    if (lane == 0) count[r] = overflow ? -1 : mine;
    return;
  }
  // compact the occupied slots to the front (each 32-slot chunk is read before any of
  // its positions is written), then place every entry at its rank among the row's keys
  __syncwarp();
  int total = 0;
  for (int c = 0; c < cap; c += 32) {
    const int key = keys[c + lane];
    const double v = vals[c + lane];
    const unsigned occ = __ballot_sync(0xffffffffu, key >= 0);
    __syncwarp();
    if (key >= 0) {
      const int dst = total + __popc(occ & ((1u << lane) - 1u));
      keys[dst] = key;
      vals[dst] = v;
    }
    total += __popc(occ);
    __syncwarp();
  }
  const int base = Crp[r];
  for (int t = lane; t < total; t += 32) {
    const int key = keys[t];
    int rank = 0;
    for (int u = 0; u < total; ++u) rank += keys[u] < key;
    Ccol[base + rank] = key;
    Cval[base + rank] = vals[t];
  }
}

// The same row product with all 32 lanes on the row's flattened product list: product p
// (k-major order: entry ea of A's row, then the entries of B's row Acol[ea]) is found from
// a warp-scanned prefix of the B-row lengths.  Products are taken 32 at a time; within a
// chunk, lanes whose products share a column are combined by the lowest such lane in lane
// order before one add into the table, so every sum has a fixed order.  The row uses a
// table of rcap <= CAP slots sized from its product count (symbolic) or its exact
// output count (numeric), so clearing and compacting cost what the row needs.
// Tiers: CAP 128 / prefix 128 with eight warps per block for the bulk of the rows (a small
// table keeps eight warps' tables in 19 KB of shared memory, so occupancy is not limited
// by it), CAP 512 / prefix 512 with four warps, CAP 4096 / prefix 2048 with one warp, then
// the sequential large table above.
constexpr int SG_CAP0 = 128, SG_PRE0 = 128, SG_WARPS0 = 8;
constexpr int SG_CAP1 = 512, SG_PRE1 = 512, SG_WARPS1 = 4;
constexpr int SG_CAP2 = 4096, SG_PRE2 = 2048;

__device__ __forceinline__ int sg_pow2_at_least(int v, int lo, int hi) {
  int c = lo;
  while (c < v && c < hi) c <<= 1;
  return c;
}

template <bool NUMERIC, int CAP, int PCAP>
__device__ void spgemm_row_flat(int r, const int* __restrict__ Arp, const int* __restrict__ Acol,
                                const double* __restrict__ Aval, const int* __restrict__ Brp,
                                const int* __restrict__ Bcol, const double* __restrict__ Bval,
                                int* keys, double* vals, int* prefix, int* bst, double* stage,
                                int* __restrict__ count, const int* __restrict__ Crp,
                                int* __restrict__ Ccol, double* __restrict__ Cval) {
  const int lane = threadIdx.x & 31;
  const int a0 = Arp[r], nA = Arp[r + 1] - a0;  // nA <= PCAP (checked by the caller)
  // prefix[t] = number of products of A entries 0..t-1; bst[t] = start of B's row Acol[t]
  int base = 0;
  for (int c = 0; c < nA; c += 32) {
    int len = 0;
    if (c + lane < nA) {
      const int k = Acol[a0 + c + lane];
      const int b0 = Brp[k];
      len = Brp[k + 1] - b0;
      bst[c + lane] = b0;
    }
    int incl = len;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (c + lane < nA) prefix[c + lane + 1] = base + incl;
    base += __shfl_sync(0xffffffffu, incl, 31);
  }
  if (lane == 0) prefix[0] = 0;
  const int total = base;
  const int rcap = sg_pow2_at_least(2 * (NUMERIC ? (Crp[r + 1] - Crp[r]) : total), 32, CAP);
  for (int s = lane; s < rcap; s += 32) {
    keys[s] = -1;
    if (NUMERIC) vals[s] = 0.0;
  }
  __syncwarp();
  // product p: A entry lo (largest t with prefix[t] <= p), B entry bst[lo] + p - prefix[lo];
  // the next chunk's loads are issued before this chunk's table inserts
  auto locate = [&](int p, int& col, double& prod) {
    int lo = 0, hi = nA;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (prefix[mid] <= p) lo = mid; else hi = mid;
    }
    const int eb = bst[lo] + (p - prefix[lo]);
    col = Bcol[eb];
    if (NUMERIC) prod = __dmul_rn(Aval[a0 + lo], Bval[eb]);
  };
  int ncol = -1;
  double nprod = 0.0;
  if (lane < total) locate(lane, ncol, nprod);
  int mine = 0;
  bool full = false;
  for (int p0 = 0; p0 < total; p0 += 32) {
    const int col = ncol;
    const double prod = nprod;
    const bool here = p0 + lane < total;
    if (p0 + 32 + lane < total) locate(p0 + 32 + lane, ncol, nprod);
    int slot = -1;
    if (here) {
      bool is_new = false;
      slot = sg_insert(keys, rcap, col, &is_new);
      if (slot < 0) full = true;
      if (is_new) ++mine;
    }
    if (__any_sync(0xffffffffu, full)) break;
    if (NUMERIC) {
      stage[lane] = prod;
      const unsigned grp = __match_any_sync(0xffffffffu, slot);
      __syncwarp();
      if (slot >= 0 && lane == __ffs(grp) - 1) {
        double sum = prod;
        for (unsigned g = grp & (grp - 1); g; g &= g - 1) sum = __dadd_rn(sum, stage[__ffs(g) - 1]);
        vals[slot] = __dadd_rn(vals[slot], sum);
      }
      __syncwarp();
    }
  }
  if (!NUMERIC) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
    const bool overflow = __any_sync(0xffffffffu, full);  // all lanes vote
    if (lane == 0) count[r] = overflow ? -1 : mine;
    return;
  }
  __syncwarp();
  int ntot = 0;
  for (int c = 0; c < rcap; c += 32) {
    const int key = keys[c + lane];
    const double v = vals[c + lane];
    const unsigned occ = __ballot_sync(0xffffffffu, key >= 0);
    __syncwarp();
    if (key >= 0) {
      const int dst = ntot + __popc(occ & ((1u << lane) - 1u));
      keys[dst] = key;
      vals[dst] = v;
    }
    ntot += __popc(occ);
    __syncwarp();
  }
  const int obase = Crp[r];
  for (int t = lane; t < ntot; t += 32) {
    const int key = keys[t];
    int rank = 0;
    for (int u = 0; u < ntot; ++u) rank += keys[u] < key;
    Ccol[obase + rank] = key;
    Cval[obase + rank] = vals[t];
  }
}

// shared memory of one warp of a flat tier: stage, (vals), keys, prefix, B-row starts
__host__ __device__ constexpr size_t sg_warp_bytes(bool numeric, int cap, int pcap) {
  return sizeof(double) * 32 + (numeric ? sizeof(double) * cap : 0) + sizeof(int) * cap +
         sizeof(int) * (pcap + 8) + sizeof(int) * pcap;
}

// One warp per row, rows 0..nrows-1 or list[0..nrows-1].  Symbolic: rows whose A row is
// longer than PCAP get count -1 (next tier).  Numeric: rows whose output count exceeds
// CAP/2 or whose A row exceeds PCAP are left to the next tier.
template <bool NUMERIC, int CAP, int PCAP, int WARPS>
__global__ void __launch_bounds__(32 * WARPS)
spgemm_flat(const int* __restrict__ Arp, const int* __restrict__ Acol,
            const double* __restrict__ Aval, const int* __restrict__ list, int nrows,
            const int* __restrict__ dnrows, const int* __restrict__ Brp,
            const int* __restrict__ Bcol, const double* __restrict__ Bval,
            int* __restrict__ count, const int* __restrict__ Crp, int* __restrict__ Ccol,
            double* __restrict__ Cval) {
  extern __shared__ __align__(16) unsigned char sg_smem[];
  const int w = threadIdx.x >> 5;
  unsigned char* mine = sg_smem + (size_t)w * sg_warp_bytes(NUMERIC, CAP, PCAP);
  double* stage = reinterpret_cast<double*>(mine);
  double* vals = NUMERIC ? stage + 32 : nullptr;
  int* keys = reinterpret_cast<int*>(mine + sizeof(double) * 32 +
                                     (NUMERIC ? sizeof(double) * CAP : 0));
  int* prefix = keys + CAP;
  int* bst = prefix + PCAP + 8;
  if (dnrows) nrows = *dnrows;  // rows listed by the previous tier, counted on the device
  for (int idx = blockIdx.x * WARPS + w; idx < nrows; idx += gridDim.x * WARPS) {  // warp-uniform
    const int r = list ? list[idx] : idx;
    const bool long_row = (Arp[r + 1] - Arp[r]) > PCAP;
    if (!NUMERIC && long_row) {
      if ((threadIdx.x & 31) == 0) count[r] = -1;
      continue;
    }
    if (NUMERIC && ((Crp[r + 1] - Crp[r]) > CAP / 2 || long_row)) continue;
    spgemm_row_flat<NUMERIC, CAP, PCAP>(r, Arp, Acol, Aval, Brp, Bcol, Bval, keys, vals, prefix,
                                        bst, stage, count, Crp, Ccol, Cval);
    __syncwarp();
  }
}

// Large dynamic table, one warp per listed row (sequential over the A row's entries); the
// list's length is read on the device.
template <bool NUMERIC>
__global__ void __launch_bounds__(32)
spgemm_large(const int* __restrict__ Arp, const int* __restrict__ Acol,
             const double* __restrict__ Aval, const int* __restrict__ list,
             const int* __restrict__ dnrows, const int* __restrict__ Brp,
             const int* __restrict__ Bcol, const double* __restrict__ Bval,
             int* __restrict__ count, const int* __restrict__ Crp, int* __restrict__ Ccol,
             double* __restrict__ Cval) {
  extern __shared__ unsigned char smem[];
  double* vals = reinterpret_cast<double*>(smem);
  int* keys = reinterpret_cast<int*>(smem + (NUMERIC ? sizeof(double) * SG_LARGE : 0));
  const int nrows = *dnrows;
  for (int idx = blockIdx.x; idx < nrows; idx += gridDim.x) {
    if (NUMERIC && count[list[idx]] > SG_LARGE) continue;  // the dense tier writes it
    spgemm_row<NUMERIC>(list[idx], Arp, Acol, Aval, Brp, Bcol, Bval, keys,
                        NUMERIC ? vals : nullptr, SG_LARGE, count, Crp, Ccol, Cval);
    __syncwarp();
  }
}

// Rows beyond the large table (more than SG_LARGE distinct columns: coarse levels of 3D
// problems with slow coarsening): one warp per listed row with a dense accumulator over
// all of B's columns and a column bitmap, both in global memory (one slot per block,
// left zeroed after each row).  Products are added in the row's A order, all lanes of one
// A entry before the next (distinct columns within a B row), as in the other tiers; the
// outputs come out in column order from the bitmap.
template <bool NUMERIC>
__global__ void __launch_bounds__(32)
spgemm_dense(const int* __restrict__ Arp, const int* __restrict__ Acol,
             const double* __restrict__ Aval, const int* __restrict__ list,
             const int* __restrict__ dnrows, const int* __restrict__ Brp,
             const int* __restrict__ Bcol, const double* __restrict__ Bval, int ncols,
             double* __restrict__ dense, unsigned* __restrict__ bits, int* __restrict__ count,
             const int* __restrict__ Crp, int* __restrict__ Ccol, double* __restrict__ Cval) {
  const int lane = threadIdx.x;
  const int nwords = (ncols + 31) >> 5;
  double* acc = dense + (size_t)blockIdx.x * ncols;
  unsigned* bw = bits + (size_t)blockIdx.x * nwords;
  const int nrows = *dnrows;
  for (int idx = blockIdx.x; idx < nrows; idx += gridDim.x) {
    const int r = list[idx];
    if (NUMERIC && count[r] <= SG_LARGE) continue;  // held by the large table
    for (int ea = Arp[r]; ea < Arp[r + 1]; ++ea) {
      const int k = Acol[ea];
      const double a = NUMERIC ? Aval[ea] : 0.0;
      for (int eb = Brp[k] + lane; eb < Brp[k + 1]; eb += 32) {
        const int c = Bcol[eb];
        if (NUMERIC) acc[c] = __dadd_rn(acc[c], __dmul_rn(a, Bval[eb]));
        atomicOr(&bw[c >> 5], 1u << (c & 31));
      }
      __syncwarp();  // the next A entry's products may hit the same columns
    }
    __threadfence_block();
    __syncwarp();
    int total = 0;
    const int base = NUMERIC ? Crp[r] : 0;
    for (int w0 = 0; w0 < nwords; w0 += 32) {
      const int w = w0 + lane;
      unsigned word = w < nwords ? bw[w] : 0u;
      const int cnt = __popc(word);
      int incl = cnt;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
      }
      if (NUMERIC) {
        int pos = base + total + incl - cnt;
        while (word) {
          const int b = __ffs(word) - 1;
          word &= word - 1;
          const int c = w * 32 + b;
          Ccol[pos] = c;
          Cval[pos] = acc[c];
          acc[c] = 0.0;
          ++pos;
        }
      }
      if (w < nwords) bw[w] = 0u;
      total += __shfl_sync(0xffffffffu, incl, 31);
    }
    if (!NUMERIC && lane == 0) count[r] = total;
    __syncwarp();
  }
}

// One CTA per row for long products (coarse levels: thousands of products per row, few
// rows).  Warp w takes a contiguous range of the row's A entries (ranges in increasing k)
// and forms its products into a private shared table as the flat tiers do; the tables are
// then merged into one in warp order, so every output is (((t_0 + t_1) + t_2) + ...) of
// the warps' partial sums: deterministic, independent of scheduling.  A row whose A row
// exceeds SGC_WARPS * SGC_PCAP entries, or whose warp tables or merged table overflow,
// gets count -1 (symbolic) and goes to the large table.
constexpr int SGC_WARPS = 8;
constexpr int SGC_WCAP = 512;   // slots of each warp's table (two numeric blocks fit an SM)
constexpr int SGC_MCAP = 4096;  // slots of the merged table
constexpr int SGC_PCAP = 256;   // A entries per warp
// Output order by a column bitmap over B's columns: rank(key) = set bits below key.  The
// bitmap reuses the warp value tables (SGC_WARPS * SGC_WCAP doubles = 2 * that many
// 32-bit words), and one prefix per group of 8 words reuses the warp key tables.
constexpr int SGC_BITWORDS = 2 * SGC_WARPS * SGC_WCAP;   // 8192 words: 262144 columns
constexpr int SGC_BITGROUPS = SGC_BITWORDS / 8;

__host__ __device__ constexpr size_t sgc_bytes(bool numeric) {
  return SGC_WARPS * (sizeof(int) * SGC_WCAP + (numeric ? sizeof(double) * SGC_WCAP : 0) +
                      sizeof(int) * (SGC_PCAP + 8) + sizeof(double) * 32) +
         sizeof(int) * SGC_MCAP + (numeric ? sizeof(double) * SGC_MCAP : 0) +
         sizeof(int) * (32 * SGC_WARPS + 8);
}

template <bool NUMERIC>
__global__ void __launch_bounds__(32 * SGC_WARPS, 2)  // shared memory: 2 numeric or 4 symbolic blocks per SM
spgemm_cta(const int* __restrict__ Arp, const int* __restrict__ Acol,
           const double* __restrict__ Aval, const int* __restrict__ Brp,
           const int* __restrict__ Bcol, const double* __restrict__ Bval, int rows,
           int ncols, const int* __restrict__ route, int* __restrict__ count,
           const int* __restrict__ Crp, int* __restrict__ Ccol, double* __restrict__ Cval) {
  extern __shared__ __align__(16) unsigned char sgc_smem[];
  constexpr int NT = 32 * SGC_WARPS;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, t = threadIdx.x;
  // layout: doubles first (8-byte aligned), then ints
  double* wvals_all = reinterpret_cast<double*>(sgc_smem);                       // WARPS x WCAP
  double* mvals = wvals_all + (NUMERIC ? SGC_WARPS * SGC_WCAP : 0);              // MCAP
  double* stage_all = mvals + (NUMERIC ? SGC_MCAP : 0);                          // WARPS x 32
  int* wkeys_all = reinterpret_cast<int*>(stage_all + SGC_WARPS * 32);           // WARPS x WCAP
  int* mkeys = wkeys_all + SGC_WARPS * SGC_WCAP;                                 // MCAP
  int* pre_all = mkeys + SGC_MCAP;                                               // WARPS x (PCAP+8)
  int* part = pre_all + SGC_WARPS * (SGC_PCAP + 8);                              // NT + 8
  __shared__ int s_full, s_total;
  double* wvals = wvals_all + w * SGC_WCAP;
  double* stage = stage_all + w * 32;
  int* wkeys = wkeys_all + w * SGC_WCAP;
  for (int r = blockIdx.x; r < rows; r += gridDim.x) {  // block-uniform
    const int a0 = Arp[r], nA = Arp[r + 1] - a0;
    if (nA > SGC_WARPS * SGC_PCAP) {
      if (!NUMERIC && t == 0) count[r] = -1;
      continue;
    }
    if (NUMERIC && route[r]) continue;  // the large table computes this row
    if (t == 0) {
      s_full = 0;
      s_total = 0;
    }
    for (int q = t; q < SGC_MCAP; q += NT) {
      mkeys[q] = -1;
      if (NUMERIC) mvals[q] = 0.0;
    }
    for (int q = lane; q < SGC_WCAP; q += 32) {
      wkeys[q] = -1;
      if (NUMERIC) wvals[q] = 0.0;
    }
    __syncthreads();  // the row's flags are reset before any warp can raise one
    // this warp's A entries [lo, hi), 32 at a time: lane q holds entry q's B-row start,
    // length and value in registers; the chunk's products (k-major) are taken 32 at a
    // time, each lane finding its product's entry by a binary search over the lanes'
    // exclusive prefix (shuffles), so a product costs one dependent load of B
    const int chunk = (nA + SGC_WARPS - 1) / SGC_WARPS;
    const int lo = min(nA, w * chunk), hi = min(nA, lo + chunk), nw = hi - lo;
    bool full = false;
    for (int c0 = 0; c0 < nw; c0 += 32) {
      int bst = 0, len = 0;
      double av = 0.0;
      if (c0 + lane < nw) {
        const int ea = a0 + lo + c0 + lane;
        const int k = Acol[ea];
        bst = Brp[k];
        len = Brp[k + 1] - bst;
        if (NUMERIC) av = Aval[ea];
      }
      int incl = len;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
      }
      const int excl = incl - len;
      const int tot = __shfl_sync(0xffffffffu, incl, 31);
      for (int p0 = 0; p0 < tot; p0 += 32) {
        const int p = p0 + lane;
        int l = 0, h = 32;  // largest lane l with excl_l <= p (lanes past the chunk: excl = tot)
#pragma unroll
        for (int it = 0; it < 5; ++it) {
          const int mid = (l + h) >> 1;
          if (__shfl_sync(0xffffffffu, excl, mid) <= p) l = mid; else h = mid;
        }
        const int ob = __shfl_sync(0xffffffffu, bst, l);
        const int oe = __shfl_sync(0xffffffffu, excl, l);
        const double oa = NUMERIC ? __shfl_sync(0xffffffffu, av, l) : 0.0;
        int slot = -1;
        double prod = 0.0;
        if (p < tot) {
          const int eb = ob + (p - oe);
          bool is_new = false;
          slot = sg_insert(wkeys, SGC_WCAP, Bcol[eb], &is_new);
          if (slot < 0) full = true;
          if (NUMERIC) prod = __dmul_rn(oa, Bval[eb]);
        }
        if (__any_sync(0xffffffffu, full)) break;
        if (NUMERIC) {
          stage[lane] = prod;
          const unsigned grp = __match_any_sync(0xffffffffu, slot);
          __syncwarp();
          if (slot >= 0 && lane == __ffs(grp) - 1) {
            double sum = prod;
            for (unsigned g = grp & (grp - 1); g; g &= g - 1) sum = __dadd_rn(sum, stage[__ffs(g) - 1]);
            wvals[slot] = __dadd_rn(wvals[slot], sum);
          }
          __syncwarp();
        }
      }
      if (__any_sync(0xffffffffu, full)) break;
    }
    const bool wfull = __any_sync(0xffffffffu, full);  // the whole warp votes
    if (wfull && lane == 0) s_full = 1;
    __syncthreads();
    // merge the warp tables into the merged table, one warp's table after another
    for (int v = 0; v < SGC_WARPS && !s_full; ++v) {
      const int* vk = wkeys_all + v * SGC_WCAP;
      const double* vv = wvals_all + v * SGC_WCAP;
      for (int q = t; q < SGC_WCAP; q += NT) {
        const int key = vk[q];
        if (key < 0) continue;
        bool is_new = false;
        const int slot = sg_insert(mkeys, SGC_MCAP, key, &is_new);
        if (slot < 0) {
          s_full = 1;
        } else {
          if (is_new) atomicAdd(&s_total, 1);
          if (NUMERIC) mvals[slot] = __dadd_rn(mvals[slot], vv[q]);  // keys distinct per table
        }
      }
      __syncthreads();
    }
    if (s_full) {  // block-uniform after the barrier
      if (!NUMERIC && t == 0) count[r] = -1;
      __syncthreads();
      continue;
    }
    const int ntot = s_total;
    if (!NUMERIC) {
      if (t == 0) count[r] = ntot;
      __syncthreads();
      continue;
    }
    const int cbase = Crp[r];
    const int nwords = (ncols + 31) >> 5;
    if (nwords <= SGC_BITWORDS) {
      // every output's position is the number of the row's columns below it: set one bit
      // per column, prefix the bit counts of 8-word groups, then count within the group
      unsigned* bits = reinterpret_cast<unsigned*>(wvals_all);
      int* gpre = wkeys_all;
      const int ngroups = (nwords + 7) >> 3;
      for (int q = t; q < ngroups * 8; q += NT) bits[q] = 0u;
      __syncthreads();
      for (int q = t; q < SGC_MCAP; q += NT) {
        const int key = mkeys[q];
        if (key >= 0) atomicOr(&bits[key >> 5], 1u << (key & 31));
      }
      __syncthreads();
      constexpr int GPT = SGC_BITGROUPS / NT;  // groups per thread, consecutive
      const int g0 = t * GPT, g1 = min(ngroups, g0 + GPT);
      int sum = 0;
      for (int u = g0 * 8; u < g1 * 8; ++u) sum += __popc(bits[u]);
      int incl = sum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
      }
      if (lane == 31) part[w] = incl;
      __syncthreads();
      if (w == 0) {
        int x = lane < SGC_WARPS ? part[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int v = __shfl_up_sync(0xffffffffu, x, o);
          if (lane >= o) x += v;
        }
        if (lane < SGC_WARPS) part[lane] = x;  // inclusive warp totals
      }
      __syncthreads();
      int run = incl - sum + (w > 0 ? part[w - 1] : 0);
      for (int g = g0; g < g1; ++g) {
        gpre[g] = run;
        for (int u = 0; u < 8; ++u) run += __popc(bits[g * 8 + u]);
      }
      __syncthreads();
      for (int q = t; q < SGC_MCAP; q += NT) {
        const int key = mkeys[q];
        if (key < 0) continue;
        const int wd = key >> 5, g = key >> 8;
        int rank = gpre[g] + __popc(bits[wd] & ((1u << (key & 31)) - 1u));
        for (int u = g * 8; u < wd; ++u) rank += __popc(bits[u]);
        Ccol[cbase + rank] = key;
        Cval[cbase + rank] = mvals[q];
      }
      __syncthreads();
      continue;
    }
    // wider B: compact the merged table (thread t owns slots [t*16, t*16+16)) into warp
    // 0's arrays and rank each key by counting the smaller ones
    constexpr int PER = SGC_MCAP / NT;
    int c = 0;
    for (int q = t * PER; q < (t + 1) * PER; ++q) c += mkeys[q] >= 0;
    part[t + 1] = c;
    if (t == 0) part[0] = 0;
    __syncthreads();
    if (t == 0)
      for (int q = 1; q <= NT; ++q) part[q] += part[q - 1];
    __syncthreads();
    int o = part[t];
    for (int q = t * PER; q < (t + 1) * PER; ++q)
      if (mkeys[q] >= 0) {
        wkeys_all[o] = mkeys[q];
        wvals_all[o] = mvals[q];
        ++o;
      }
    __syncthreads();
    for (int q = t; q < ntot; q += NT) {
      const int key = wkeys_all[q];
      int rank = 0;
      for (int u = 0; u < ntot; ++u) rank += wkeys_all[u] < key;
      Ccol[cbase + rank] = key;
      Cval[cbase + rank] = wvals_all[q];
    }
    __syncthreads();
  }
}

__global__ void sg_mark_rows(const int* __restrict__ list, const int* __restrict__ dn,
                             int* __restrict__ route) {
  const int n = *dn;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x)
    route[list[q]] = 1;
}

// Lists (from `src` rows, or all rows when src == nullptr) the rows with count == -1
// (mode 0) or, mode 1, the rows a numeric tier left out: more than `lim_cnt` output
// entries or more than `lim_nA` A entries.
__global__ void spgemm_collect(const int* __restrict__ count, const int* __restrict__ Crp,
                               const int* __restrict__ Arp, const int* __restrict__ src,
                               int nsrc, const int* __restrict__ dnsrc, int mode, int lim_cnt,
                               int lim_nA, int* __restrict__ list, int* __restrict__ n) {
  if (dnsrc) nsrc = *dnsrc;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nsrc; t += gridDim.x * blockDim.x) {
    const int r = src ? src[t] : t;
    const bool take = mode == 0 ? count[r] < 0
                                : ((Crp[r + 1] - Crp[r]) > lim_cnt || (Arp[r + 1] - Arp[r]) > lim_nA);
    if (take) list[atomicAdd(n, 1)] = r;
  }
}

__global__ void count_nonzero(const int* __restrict__ rowptr, const double* __restrict__ val, int rows,
                              int* __restrict__ cnt) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  int c = 0;
  for (int e = rowptr[r]; e < rowptr[r + 1]; ++e) c += val[e] != 0.0;
  cnt[r] = c;
}

__global__ void copy_nonzero(const int* __restrict__ rowptr, const int* __restrict__ col,
                             const double* __restrict__ val, int rows, const int* __restrict__ out_rp,
                             int* __restrict__ out_col, double* __restrict__ out_val) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  int o = out_rp[r];
  for (int e = rowptr[r]; e < rowptr[r + 1]; ++e)
    if (val[e] != 0.0) {
      out_col[o] = col[e];
      out_val[o] = val[e];
      ++o;
    }
}

void drop_zeros(Csr& C, cudaStream_t s) {
  const int rows = C.rows;
  int* cnt = dalloc<int>(rows + 1, s);
  if (rows) count_nonzero<<<ceil_div(rows, 256), 256, 0, s>>>(C.rowptr, C.val, rows, cnt); ::clair::count_launch();
  CLAIR_LAUNCHED();
  int* rp = dalloc<int>(rows + 1, s);
  const int nnz = (int)exclusive_scan(cnt, rp, rows, s, true);
  if (nnz == C.nnz) {
    dfree(cnt, s);
    dfree(rp, s);
    return;
  }
  int* col = dalloc<int>(nnz, s);
  double* val = dalloc<double>(nnz, s);
  if (rows) copy_nonzero<<<ceil_div(rows, 256), 256, 0, s>>>(C.rowptr, C.col, C.val, rows, rp, col, val); ::clair::count_launch();
  CLAIR_LAUNCHED();
  dfree(cnt, s);
  dfree(C.rowptr, s);
  dfree(C.col, s);
  dfree(C.val, s);
  C.rowptr = rp;
  C.col = col;
  C.val = val;
  C.nnz = nnz;
}

// The dense tier for the `dn` rows listed in `list` (symbolic: count; numeric: values).
// Its accumulators are allocated only when rows reach it; the host reads the list length
// with the scan that follows the symbolic pass, so `still` rows need no further check.
struct DenseTier {
  double* dense = nullptr;
  unsigned* bits = nullptr;
  int slots = 0;
  void ensure(int ncols, int rows, cudaStream_t s) {
    if (dense) return;
    slots = std::max(1, std::min(rows, 2 * sm_count()));
    const size_t nwords = (size_t)(ncols + 31) / 32;
    dense = dalloc<double>((size_t)slots * ncols, s);
    bits = dalloc<unsigned>((size_t)slots * nwords, s);
    CLAIR_CUDA(cudaMemsetAsync(dense, 0, sizeof(double) * slots * ncols, s));
    CLAIR_CUDA(cudaMemsetAsync(bits, 0, sizeof(unsigned) * slots * nwords, s));
  }
  void release(cudaStream_t s) {
    dfree(dense, s);
    dfree(bits, s);
  }
};

// Long products: the CTA-per-row kernel for every row, the large table for the rows it
// could not hold.
static void spgemm_cta_path(const Csr& A, const Csr& B, Csr& C, cudaStream_t s) {
  const int rows = A.rows;
  once_per_device((const void*)spgemm_cta<true>, [] {
    CLAIR_CUDA(cudaFuncSetAttribute(spgemm_cta<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)sgc_bytes(false)));
    CLAIR_CUDA(cudaFuncSetAttribute(spgemm_cta<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)sgc_bytes(true)));
    CLAIR_CUDA(cudaFuncSetAttribute(spgemm_large<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)(sizeof(int) * SG_LARGE)));
    CLAIR_CUDA(cudaFuncSetAttribute(spgemm_large<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)((sizeof(int) + sizeof(double)) * SG_LARGE)));
  });
  const int sms = sm_count();
  int* count = dalloc<int>(rows + 1, s);
  int* route = dalloc<int>(rows, s);
  int* list = dalloc<int>(rows, s);
  int* list2 = dalloc<int>(rows, s);
  int* nlist = dalloc<int>(2, s);
  CLAIR_CUDA(cudaMemsetAsync(route, 0, sizeof(int) * rows, s));
  CLAIR_CUDA(cudaMemsetAsync(nlist, 0, 2 * sizeof(int), s));
  const int gsym = std::min(rows, 4 * sms), gnum = std::min(rows, 2 * sms);
  spgemm_cta<false><<<gsym, 32 * SGC_WARPS, sgc_bytes(false), s>>>(
      A.rowptr, A.col, A.val, B.rowptr, B.col, B.val, rows, B.cols, route, count, nullptr, nullptr,
      nullptr); ::clair::count_launch();
  spgemm_collect<<<std::max(1, std::min(ceil_div(rows, 256), sms * 8)), 256, 0, s>>>(
      count, nullptr, A.rowptr, nullptr, rows, nullptr, 0, 0, 0, list, nlist); ::clair::count_launch();
  sg_mark_rows<<<std::max(1, std::min(ceil_div(rows, 256), sms * 8)), 256, 0, s>>>(list, nlist, route); ::clair::count_launch();
  spgemm_large<false><<<std::max(1, std::min(rows, sms)), 32, sizeof(int) * SG_LARGE, s>>>(
      A.rowptr, A.col, A.val, list, nlist, B.rowptr, B.col, B.val, count, nullptr, nullptr, nullptr); ::clair::count_launch();
  spgemm_collect<<<std::max(1, std::min(ceil_div(rows, 256), sms * 8)), 256, 0, s>>>(
      count, nullptr, A.rowptr, list, rows, nlist, 0, 0, 0, list2, nlist + 1); ::clair::count_launch();
  CLAIR_LAUNCHED();
  // rows no table could hold (list2, nlist[1], read back with the scan total) go to the
  // dense tier, and the scan is redone
  C.rowptr = dalloc<int>(rows + 1, s);
  int still = 0;
  C.nnz = (int)exclusive_scan(count, C.rowptr, rows, s, true, nlist + 1, &still);
  DenseTier dt;
  const bool may_overflow = still > 0;
  if (may_overflow) {
    dt.ensure(B.cols, still, s);
    spgemm_dense<false><<<dt.slots, 32, 0, s>>>(A.rowptr, A.col, A.val, list2, nlist + 1, B.rowptr,
                                                B.col, B.val, B.cols, dt.dense, dt.bits, count,
                                                nullptr, nullptr, nullptr); ::clair::count_launch();
    CLAIR_LAUNCHED();
    C.nnz = (int)exclusive_scan(count, C.rowptr, rows, s, true);
  }
  C.col = dalloc<int>(C.nnz, s);
  C.val = dalloc<double>(C.nnz, s);
  spgemm_cta<true><<<gnum, 32 * SGC_WARPS, sgc_bytes(true), s>>>(
      A.rowptr, A.col, A.val, B.rowptr, B.col, B.val, rows, B.cols, route, count, C.rowptr, C.col,
      C.val); ::clair::count_launch();
  spgemm_large<true><<<std::max(1, std::min(rows, sms)), 32, (sizeof(int) + sizeof(double)) * SG_LARGE, s>>>(
      A.rowptr, A.col, A.val, list, nlist, B.rowptr, B.col, B.val, count, C.rowptr, C.col, C.val); ::clair::count_launch();
  if (may_overflow) {
    spgemm_dense<true><<<dt.slots, 32, 0, s>>>(A.rowptr, A.col, A.val, list2, nlist + 1, B.rowptr,
                                               B.col, B.val, B.cols, dt.dense, dt.bits, count,
                                               C.rowptr, C.col, C.val); ::clair::count_launch();
  }
  CLAIR_LAUNCHED();
  dt.release(s);
  dfree(count, s);
  dfree(route, s);
  dfree(list, s);
  dfree(list2, s);
  dfree(nlist, s);
}

// Tier 0 runs over every row; each later tier (and the large table) runs over the rows the
// previous one listed, with a grid-stride loop over a count it reads on the device, so the
// tiers follow one another without a host round trip.  The host reads back once, with the
// output size (symbolic) and the rows no table could hold.
void spgemm(const Csr& A, const Csr& B, Csr& C, cudaStream_t s) {
  C.rows = A.rows;
  C.cols = B.cols;
  const int rows = A.rows;
  // long products (mean products per row ~ mean A row x mean B row): one CTA per row
  const double mean_products =
      (rows ? (double)A.nnz / rows : 0.0) * (B.rows ? (double)B.nnz / B.rows : 0.0);
  // (thresholds measured on the 1024^2 hierarchy: the flat tiers win from 1024 to 2048
  // products per row on levels of many rows, the CTA path on short matrices)
  if (rows && (mean_products >= 2048.0 || (mean_products >= 1024.0 && rows < 8192))) {
    spgemm_cta_path(A, B, C, s);
    return;
  }
  int* count = dalloc<int>(rows + 1, s);
  int* lists[2] = {dalloc<int>(std::max(rows, 1), s), dalloc<int>(std::max(rows, 1), s)};
  int* nlist = dalloc<int>(8, s);
  struct Tier {
    int cap, pcap, warps;
    void (*sym)(const int*, const int*, const double*, const int*, int, const int*, const int*,
                const int*, const double*, int*, const int*, int*, double*);
    void (*num)(const int*, const int*, const double*, const int*, int, const int*, const int*,
                const int*, const double*, int*, const int*, int*, double*);
  };
  const Tier tiers[3] = {
      {SG_CAP0, SG_PRE0, SG_WARPS0, spgemm_flat<false, SG_CAP0, SG_PRE0, SG_WARPS0>,
       spgemm_flat<true, SG_CAP0, SG_PRE0, SG_WARPS0>},
      {SG_CAP1, SG_PRE1, SG_WARPS1, spgemm_flat<false, SG_CAP1, SG_PRE1, SG_WARPS1>,
       spgemm_flat<true, SG_CAP1, SG_PRE1, SG_WARPS1>},
      {SG_CAP2, SG_PRE2, 1, spgemm_flat<false, SG_CAP2, SG_PRE2, 1>,
       spgemm_flat<true, SG_CAP2, SG_PRE2, 1>}};
  const size_t large_sym = sizeof(int) * SG_LARGE;
  const size_t large_num = (sizeof(int) + sizeof(double)) * SG_LARGE;
  once_per_device((const void*)spgemm_flat<true, SG_CAP0, SG_PRE0, SG_WARPS0>, [] {
    auto both = [](auto sym, auto num, size_t sym_bytes, size_t num_bytes) {
      CLAIR_CUDA(cudaFuncSetAttribute(sym, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)sym_bytes));
      CLAIR_CUDA(cudaFuncSetAttribute(num, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)num_bytes));
    };
    both(spgemm_flat<false, SG_CAP0, SG_PRE0, SG_WARPS0>, spgemm_flat<true, SG_CAP0, SG_PRE0, SG_WARPS0>,
         SG_WARPS0 * sg_warp_bytes(false, SG_CAP0, SG_PRE0),
         SG_WARPS0 * sg_warp_bytes(true, SG_CAP0, SG_PRE0));
    both(spgemm_flat<false, SG_CAP1, SG_PRE1, SG_WARPS1>, spgemm_flat<true, SG_CAP1, SG_PRE1, SG_WARPS1>,
         SG_WARPS1 * sg_warp_bytes(false, SG_CAP1, SG_PRE1),
         SG_WARPS1 * sg_warp_bytes(true, SG_CAP1, SG_PRE1));
    both(spgemm_flat<false, SG_CAP2, SG_PRE2, 1>, spgemm_flat<true, SG_CAP2, SG_PRE2, 1>,
         sg_warp_bytes(false, SG_CAP2, SG_PRE2), sg_warp_bytes(true, SG_CAP2, SG_PRE2));
    both(spgemm_large<false>, spgemm_large<true>, sizeof(int) * SG_LARGE,
         (sizeof(int) + sizeof(double)) * SG_LARGE);
  });
  const int sms = sm_count();
  // grid of a tier over listed rows: enough warps to fill the GPU, never more than the rows
  auto grid_for_list = [&](int warps_per_block, int blocks_per_sm) {
    return std::max(1, std::min(ceil_div(rows, warps_per_block), sms * blocks_per_sm));
  };
  // ---- symbolic ----
  CLAIR_CUDA(cudaMemsetAsync(nlist, 0, 8 * sizeof(int), s));
  {
    const int* src = nullptr;
    const int* dn = nullptr;
    int cur = 0;
    for (int t = 0; t < 4; ++t) {
      if (t < 3) {
        const Tier& T = tiers[t];
        const size_t sm = T.warps * sg_warp_bytes(false, T.cap, T.pcap);
        const int grid = t == 0 ? std::max(1, ceil_div(rows, T.warps)) : grid_for_list(T.warps, 8);
        T.sym<<<grid, 32 * T.warps, sm, s>>>(A.rowptr, A.col, A.val, src, rows, dn, B.rowptr, B.col,
                                            B.val, count, nullptr, nullptr, nullptr); ::clair::count_launch();
      } else {
        spgemm_large<false><<<std::max(1, std::min(rows, sms)), 32, large_sym, s>>>(
            A.rowptr, A.col, A.val, src, dn, B.rowptr, B.col, B.val, count, nullptr, nullptr,
            nullptr); ::clair::count_launch();
      }
      spgemm_collect<<<std::max(1, std::min(ceil_div(rows, 256), sms * 8)), 256, 0, s>>>(
          count, nullptr, A.rowptr, src, rows, dn, 0, 0, 0, lists[cur], nlist + t); ::clair::count_launch();
      CLAIR_LAUNCHED();
      src = lists[cur];
      dn = nlist + t;
      cur ^= 1;
    }
  }
  // rows still unplaced after the large table (lists[1], nlist[3], read back with the scan
  // total) go to the dense tier, and the scan is redone; they keep a list of their own for
  // the numeric pass
  C.rowptr = dalloc<int>(rows + 1, s);
  int still = 0;
  C.nnz = (int)exclusive_scan(count, C.rowptr, rows, s, true, nlist + 3, &still);
  DenseTier dt;
  int* dense_list = nullptr;
  const bool may_overflow = still > 0;
  if (may_overflow) {
    dt.ensure(B.cols, still, s);
    dense_list = dalloc<int>(std::max(rows, 1), s);
    CLAIR_CUDA(cudaMemcpyAsync(dense_list, lists[1], sizeof(int) * rows, cudaMemcpyDeviceToDevice, s));
    CLAIR_CUDA(cudaMemcpyAsync(nlist + 4, nlist + 3, sizeof(int), cudaMemcpyDeviceToDevice, s));
    spgemm_dense<false><<<dt.slots, 32, 0, s>>>(A.rowptr, A.col, A.val, dense_list, nlist + 4,
                                                B.rowptr, B.col, B.val, B.cols, dt.dense, dt.bits,
                                                count, nullptr, nullptr, nullptr); ::clair::count_launch();
    CLAIR_LAUNCHED();
    C.nnz = (int)exclusive_scan(count, C.rowptr, rows, s, true);
  }
  C.col = dalloc<int>(C.nnz, s);
  C.val = dalloc<double>(C.nnz, s);
  // ---- numeric: each row in the first tier that holds it (output count <= cap / 2, A row
  // <= prefix capacity) ----
  CLAIR_CUDA(cudaMemsetAsync(nlist, 0, 4 * sizeof(int), s));
  {
    const int* src = nullptr;
    const int* dn = nullptr;
    int cur = 0;
    for (int t = 0; t < 4; ++t) {
      if (t < 3) {
        const Tier& T = tiers[t];
        const size_t sm = T.warps * sg_warp_bytes(true, T.cap, T.pcap);
        const int grid = t == 0 ? std::max(1, ceil_div(rows, T.warps)) : grid_for_list(T.warps, 8);
        T.num<<<grid, 32 * T.warps, sm, s>>>(A.rowptr, A.col, A.val, src, rows, dn, B.rowptr, B.col,
                                            B.val, count, C.rowptr, C.col, C.val); ::clair::count_launch();
        spgemm_collect<<<std::max(1, std::min(ceil_div(rows, 256), sms * 8)), 256, 0, s>>>(
            count, C.rowptr, A.rowptr, src, rows, dn, 1, T.cap / 2, T.pcap, lists[cur],
            nlist + t); ::clair::count_launch();
        CLAIR_LAUNCHED();
        src = lists[cur];
        dn = nlist + t;
        cur ^= 1;
      } else {
        spgemm_large<true><<<std::max(1, std::min(rows, sms)), 32, large_num, s>>>(
            A.rowptr, A.col, A.val, src, dn, B.rowptr, B.col, B.val, count, C.rowptr, C.col,
            C.val); ::clair::count_launch();
        CLAIR_LAUNCHED();
      }
    }
  }
  if (may_overflow) {
    spgemm_dense<true><<<dt.slots, 32, 0, s>>>(A.rowptr, A.col, A.val, dense_list, nlist + 4,
                                               B.rowptr, B.col, B.val, B.cols, dt.dense, dt.bits,
                                               count, C.rowptr, C.col, C.val); ::clair::count_launch();
    CLAIR_LAUNCHED();
  }
  dt.release(s);
  dfree(dense_list, s);
  dfree(count, s);
  dfree(lists[0], s);
  dfree(lists[1], s);
  dfree(nlist, s);
}

// ------------------------------------------------------------------------------------
// Variants that take every temporary from a caller-provided workspace instead of
// allocating it (for the entry point that must not allocate device memory).
// ------------------------------------------------------------------------------------
int scan_ws_blocks(int n) { return std::max(1, ceil_div(n, SCAN_TILE)); }

long long exclusive_scan_ws(const int* in, int* out, int n, cudaStream_t s, bool want_total,
                            long long* sums, int* ovf) {
  const int nb = scan_ws_blocks(n);
  CLAIR_REQUIRE(nb <= SCAN_TILE, CLAIR_ERR_CAPACITY, "scan of %d items exceeds capacity", n);
  CLAIR_CUDA(cudaMemsetAsync(ovf, 0, sizeof(int), s));
  scan_block_sums<<<nb, SCAN_THREADS, 0, s>>>(in, n, sums); ::clair::count_launch();
  scan_sums<<<1, SCAN_THREADS, 0, s>>>(sums, nb); ::clair::count_launch();
  scan_apply<<<nb, SCAN_THREADS, 0, s>>>(in, n, sums, out, ovf); ::clair::count_launch();
  CLAIR_LAUNCHED();
  long long total = 0;
  if (want_total) {
    int total32 = 0, h_ovf = 0;
    CLAIR_CUDA(cudaMemcpyAsync(&total32, out + n, sizeof(int), cudaMemcpyDeviceToHost, s));
    CLAIR_CUDA(cudaMemcpyAsync(&h_ovf, ovf, sizeof(int), cudaMemcpyDeviceToHost, s));
    CLAIR_CUDA(cudaStreamSynchronize(s));
    CLAIR_REQUIRE(!h_ovf, CLAIR_ERR_CAPACITY, "scan total exceeds int32");
    total = total32;
  }
  return total;
}

// At.rowptr (A.cols + 1), At.col and At.val (A.nnz each, val optional) are caller buffers;
// perm (A.nnz), cnt (A.cols + 1), sums (scan_ws_blocks(A.cols) + 1) and ovf are workspace.
void csr_transpose_ws(const Csr& A, Csr& At, int* perm, int* cnt, long long* sums, int* ovf,
                      cudaStream_t s) {
  At.rows = A.cols;
  At.cols = A.rows;
  At.nnz = A.nnz;
  CLAIR_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * (A.cols + 1), s));
  if (A.nnz) count_cols<<<grid_for(A.nnz), 256, 0, s>>>(A.col, A.nnz, cnt); ::clair::count_launch();
  exclusive_scan_ws(cnt, At.rowptr, A.cols, s, false, sums, ovf);
  CLAIR_CUDA(cudaMemcpyAsync(cnt, At.rowptr, sizeof(int) * A.cols, cudaMemcpyDeviceToDevice, s));
  if (A.rows) transpose_fill<1><<<ceil_div(A.rows, 256), 256, 0, s>>>(A.rowptr, A.col, A.rows, cnt,
                                                                        At.col, perm); ::clair::count_launch();
  if (At.rows) sort_segments<<<ceil_div(At.rows, 128), 128, 0, s>>>(At.rowptr, At.rows, At.col, perm); ::clair::count_launch();
  CLAIR_LAUNCHED();
  if (A.val && At.val) gather(A.val, perm, At.val, A.nnz, s);
}

void validate_csr_ws(const int* rowptr, const int* col, int rows, int cols, int nnz,
                     const char* what, int* bad, cudaStream_t s) {
  CLAIR_REQUIRE(rows >= 0 && nnz >= 0, CLAIR_ERR_ARG, "%s: negative size", what);
  if (!rows) return;
  CLAIR_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
  int h_rp[2] = {0, 0};
  CLAIR_CUDA(cudaMemcpyAsync(&h_rp[0], rowptr, sizeof(int), cudaMemcpyDeviceToHost, s));
  CLAIR_CUDA(cudaMemcpyAsync(&h_rp[1], rowptr + rows, sizeof(int), cudaMemcpyDeviceToHost, s));
  CLAIR_CUDA(cudaStreamSynchronize(s));
  CLAIR_REQUIRE(h_rp[0] == 0 && h_rp[1] == nnz, CLAIR_ERR_ARG,
                "%s: rowptr[0]=%d rowptr[rows]=%d, expected 0 and %d", what, h_rp[0], h_rp[1], nnz);
  validate_rows<<<ceil_div(rows, 256), 256, 0, s>>>(rowptr, col, rows, cols, nnz, bad); ::clair::count_launch();
  CLAIR_LAUNCHED();
  int h = 0;
  CLAIR_CUDA(cudaMemcpyAsync(&h, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
  CLAIR_CUDA(cudaStreamSynchronize(s));
  CLAIR_REQUIRE(h == 0, CLAIR_ERR_ARG,
                "%s: %d rows with bad row pointers or unsorted/out-of-range columns", what, h);
}

void validate_cf_ws(const signed char* cf, int n, int* bad, cudaStream_t s) {
  if (!n) return;
  CLAIR_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
  validate_flags<<<ceil_div(n, 256), 256, 0, s>>>(cf, n, bad); ::clair::count_launch();
  CLAIR_LAUNCHED();
  int h = 0;
  CLAIR_CUDA(cudaMemcpyAsync(&h, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
  CLAIR_CUDA(cudaStreamSynchronize(s));
  CLAIR_REQUIRE(h == 0, CLAIR_ERR_ARG, "cf has %d entries other than 0/1", h);
}

}  // namespace clair
