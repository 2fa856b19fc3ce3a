// Shared helpers of the APLICUR CUDA library: error handling, device buffers,
// deterministic reductions and the "last block finishes" pattern.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <stdexcept>
#include <string>
#include <utility>
#include <vector>

namespace apl {

// Internal failures are C++ exceptions; the C ABI layer converts them to status codes.
struct Error : std::runtime_error {
  int code;
  Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

enum { ST_OK = 0, ST_EINVAL = 1, ST_ENOMEM = 2, ST_ECUDA = 3, ST_ENOTCONV = 4,
       ST_EBREAKDOWN = 5, ST_ETIMEOUT = 6 };

#define APL_CUDA(call)                                                                    \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      throw ::apl::Error(e_ == cudaErrorMemoryAllocation ? ::apl::ST_ENOMEM : ::apl::ST_ECUDA, \
                         std::string(#call) + ": " + cudaGetErrorString(e_));             \
  } while (0)

// Kernel launch accounting: every launch site calls APL_LAUNCH_CHECK; launches made
// while a graph is being captured are counted when the graph is replayed instead.
void note_launch();
void add_launches(long long n);
long long launch_count();
struct CaptureScope {
  CaptureScope();
  ~CaptureScope();
};

// Device-time accounting by kernel family, active while a solve with profiling runs on
// this thread.  Categories: 0 A z pass, 1 A^T u pass, 2 preconditioner passes (bytes);
// 3 FP64 GEMM, 4 FP64 Jacobi sweeps (FP64 flops); 5 LUPP selection (bytes);
// 6 FP32 Jacobi sweeps (FP32 flops).
enum { PROF_NCAT = 7, PROF_GEMM = 3, PROF_JACOBI = 4, PROF_LUPP = 5, PROF_JACOBI32 = 6 };
struct ProfSink {
  cudaStream_t st = nullptr;
  std::vector<cudaEvent_t> pool;
  struct Rec { int cat; double work; int e0, e1; };
  std::vector<Rec> recs;
  double ms[PROF_NCAT] = {0};
  double work[PROF_NCAT] = {0};
  long long n[PROF_NCAT] = {0};
  ~ProfSink();
  int event();                  // record a fresh event on st, return its index
  void harvest();               // synchronise and accumulate all pending records
  void add(int cat, double ms_, double work_, long long cnt);
};
// The sink of the calling thread (NULL when profiling is off or a graph is captured).
ProfSink* prof_sink();
void prof_set_sink(ProfSink* s);
// Open a timed region on stream st; returns a token for prof_end (or -1 when off).
int prof_begin(cudaStream_t st);
void prof_end(cudaStream_t st, int token, int cat, double work);
void prof_set_work(int token_rec, double work);  // adjust the last record's work

#define APL_LAUNCH_CHECK()            \
  do {                                \
    APL_CUDA(cudaGetLastError());     \
    ::apl::note_launch();             \
  } while (0)

#define APL_REQUIRE(cond, msg)                                         \
  do {                                                                 \
    if (!(cond)) throw ::apl::Error(::apl::ST_EINVAL, (msg));          \
  } while (0)

inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Caller-supplied device allocator (aplicur_options alloc / free_ / alloc_ctx).  Empty:
// the library's own stream-ordered cudaMallocAsync / cudaFreeAsync.
struct Allocator {
  void* (*alloc)(size_t bytes, void* stream, void* ctx) = nullptr;
  void (*free_)(void* p, size_t bytes, void* stream, void* ctx) = nullptr;
  void* ctx = nullptr;
};
// The allocator installed on the calling thread for the duration of a C ABI call (NULL:
// the library's own).  Worker threads of batched solves inherit the caller's.
const Allocator* current_allocator();
struct AllocScope {
  const Allocator* prev;
  explicit AllocScope(const Allocator* a);
  ~AllocScope();
};
void note_internal_alloc();
long long internal_alloc_count();

// Device buffer owned by the library (stream-ordered allocation, through the caller's
// allocator when one is installed; freed by the allocator that made it).
template <typename T>
struct DBuf {
  T* p = nullptr;
  size_t n = 0;
  cudaStream_t st = nullptr;
  Allocator al;
  DBuf() = default;
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  ~DBuf() { release(); }
  void release() {
    if (p) {
      if (al.free_) al.free_(p, n * sizeof(T), st, al.ctx);
      else cudaFreeAsync(p, st);
    }
    p = nullptr;
    n = 0;
  }
  // (Re)allocate to hold `count` elements; contents are not kept.
  void alloc(size_t count, cudaStream_t s) {
    if (count <= n && p) { st = s; return; }
    release();
    st = s;
    if (count == 0) return;
    const Allocator* a = current_allocator();
    if (a && a->alloc) {
      p = static_cast<T*>(a->alloc(count * sizeof(T), s, a->ctx));
      if (!p) throw Error(ST_ENOMEM, "the caller's allocator returned NULL");
      al = *a;
    } else {
      APL_CUDA(cudaMallocAsync((void**)&p, count * sizeof(T), s));
      al = Allocator();
      note_internal_alloc();
    }
    n = count;
  }
  void zero(cudaStream_t s) {
    if (p && n) APL_CUDA(cudaMemsetAsync(p, 0, n * sizeof(T), s));
  }
  T* get() const { return p; }
  void swap(DBuf& o) {
    std::swap(p, o.p);
    std::swap(n, o.n);
    std::swap(st, o.st);
    std::swap(al, o.al);
  }
};

// Scratch buffers of the dense routines (split-K partial sums, Cholesky QR temporary,
// Jacobi copies).  They belong to the calling context, whose stream carries every use,
// so growing one is stream-ordered (cudaFreeAsync/cudaMallocAsync on that stream) and
// contexts driven from different threads never share or free each other's buffers.
// The context installs its workspace for the duration of a call with DenseWorkScope.
struct DenseWork {
  DBuf<double> splitk, qrtmp, jw64, jtmp, jw2;
  DBuf<float> jb32, jw32;
  DBuf<float> gah, gal, gbh, gbl;  // hi / lo operands of the compensated GEMM
  DBuf<float> tth, ttl;            // hi / lo of the triangle of a compensated solve
  bool fp64_gemm = false;  // GEMMs on the FP64 units instead of compensated FP32
};
DenseWork& dense_work();  // the workspace installed on the calling thread (throws if none)
// Run the dense products of a scope on the FP64 units (retry of a breakdown).
struct Fp64Scope {
  bool prev;
  Fp64Scope() : prev(dense_work().fp64_gemm) { dense_work().fp64_gemm = true; }
  ~Fp64Scope() { dense_work().fp64_gemm = prev; }
};
struct DenseWorkScope {
  DenseWork* prev;
  explicit DenseWorkScope(DenseWork* w);
  ~DenseWorkScope();
};

// ---- device reductions (fixed order -> bitwise reproducible) -------------------------

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Block sum; result valid in thread 0.  `sh` needs blockDim.x/32 doubles.
__device__ __forceinline__ double block_sum(double v, double* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double r = 0.0;
  if (wid == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    r = (lane < nw) ? sh[lane] : 0.0;
    r = warp_sum(r);
  }
  return r;
}

// Returns true in every thread of the block that finished last among all blocks of
// the grid.  Writers must have stored their partial results before calling.
// The counter is reset by the last block so graphs can replay the kernel.
__device__ __forceinline__ bool last_block_done(unsigned int* counter) {
  __shared__ bool is_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int total = gridDim.x * gridDim.y * gridDim.z;
    const unsigned int t = atomicAdd(counter, 1u);
    is_last = (t == total - 1);
    if (is_last) *counter = 0u;
  }
  __syncthreads();
  if (is_last) __threadfence();
  return is_last;
}

// Sum of n partials in fixed order by one block; result in thread 0.
__device__ __forceinline__ double block_sum_partials(const double* part, int n, double* sh) {
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) v += __ldcg(part + i);
  return block_sum(v, sh);
}

template <typename T> __device__ __forceinline__ double to_d(T v) { return (double)v; }

}  // namespace apl
