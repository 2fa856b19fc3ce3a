// Dense FP64 kernels for the ell x ell and n x b work of the CUR and preconditioner
// steps: tiled GEMM, blocked triangular solves, single-CTA Cholesky, Cholesky QR2 and a
// parallel one-sided (Hestenes) Jacobi SVD.
#include <algorithm>
#include <cstring>
#include <atomic>
#include <numeric>

#include "dense.cuh"
#include "df32.cuh"

namespace apl {

namespace {
std::atomic<long long> g_launches{0};
thread_local int g_capture_depth = 0;
}  // namespace
void note_launch() {
  if (g_capture_depth == 0) g_launches.fetch_add(1, std::memory_order_relaxed);
}
void add_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(); }
CaptureScope::CaptureScope() { ++g_capture_depth; }
CaptureScope::~CaptureScope() { --g_capture_depth; }

namespace {
thread_local const Allocator* g_alloc = nullptr;
std::atomic<long long> g_internal_allocs{0};
}  // namespace
const Allocator* current_allocator() { return g_alloc; }
AllocScope::AllocScope(const Allocator* a) : prev(g_alloc) { g_alloc = a; }
AllocScope::~AllocScope() { g_alloc = prev; }
void note_internal_alloc() { g_internal_allocs.fetch_add(1, std::memory_order_relaxed); }
long long internal_alloc_count() { return g_internal_allocs.load(); }

namespace {
thread_local ProfSink* g_sink = nullptr;
thread_local DenseWork* g_work = nullptr;
}
ProfSink* prof_sink() { return g_capture_depth == 0 ? g_sink : nullptr; }
DenseWork& dense_work() {
  APL_REQUIRE(g_work != nullptr, "internal: dense routine called without a workspace");
  return *g_work;
}
DenseWorkScope::DenseWorkScope(DenseWork* w) : prev(g_work) { g_work = w; }
DenseWorkScope::~DenseWorkScope() { g_work = prev; }
void prof_set_sink(ProfSink* s) { g_sink = s; }
ProfSink::~ProfSink() {
  for (cudaEvent_t e : pool) cudaEventDestroy(e);
}
int ProfSink::event() {
  const int used = (int)(recs.size() * 2);
  while ((int)pool.size() < used + 2) {
    cudaEvent_t e;
    APL_CUDA(cudaEventCreate(&e));
    pool.push_back(e);
  }
  return used;
}
void ProfSink::add(int cat, double ms_, double work_, long long cnt) {
  ms[cat] += ms_;
  work[cat] += work_;
  n[cat] += cnt;
}
void ProfSink::harvest() {
  if (recs.empty()) return;
  APL_CUDA(cudaStreamSynchronize(st));
  for (const Rec& r : recs) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, pool[r.e0], pool[r.e1]) == cudaSuccess) add(r.cat, t, r.work, 1);
    else (void)cudaGetLastError();
  }
  recs.clear();
}
int prof_begin(cudaStream_t st) {
  ProfSink* s = prof_sink();
  if (!s) return -1;
  if (s->recs.size() >= 4096) s->harvest();
  const int e0 = s->event();
  s->st = st;
  APL_CUDA(cudaEventRecord(s->pool[e0], st));
  s->recs.push_back(ProfSink::Rec{-1, 0.0, e0, e0 + 1});
  return (int)s->recs.size() - 1;
}
void prof_end(cudaStream_t st, int token, int cat, double work) {
  ProfSink* s = prof_sink();
  if (!s || token < 0 || token >= (int)s->recs.size()) return;
  ProfSink::Rec& r = s->recs[token];
  r.cat = cat;
  r.work = work;
  APL_CUDA(cudaEventRecord(s->pool[r.e1], st));
}
void prof_set_work(int token, double work) {
  ProfSink* s = prof_sink();
  if (!s || token < 0 || token >= (int)s->recs.size()) return;
  s->recs[token].work = work;
}

// ------------------------------------------------------------------------------------
// Triangular solve.  Diagonal blocks (<= 64) are solved by one thread per right-hand
// vector; the rest is GEMM updates.
// ------------------------------------------------------------------------------------
namespace {
constexpr int TNB = 64;

// Solve T x = b for `nvec` vectors of length `len` (<= 64), one warp per vector; lane q
// holds x_q and x_{q+32}.  T(r, c) = Tm[r * trs + c * tcs]; lower: forward substitution,
// else backward.  Vector v element i at X[v * vstride + i * estride].  Column (axpy)
// form: at step i the lane holding x_i finishes it, broadcasts it, and every lane removes
// T(q, i) x_i from its later entries, so no step needs a warp reduction.
__global__ void __launch_bounds__(256) trsv_block_kernel(int64_t nvec, int len,
                                                         double* __restrict__ X,
                                                         int64_t vstride, int64_t estride,
                                                         const double* __restrict__ Tm,
                                                         int64_t trs, int64_t tcs, int lower,
                                                         int unit) {
  __shared__ double Ts[TNB][TNB + 1];
  for (int e = threadIdx.x; e < len * len; e += blockDim.x) {
    const int r = e % len, c = e / len;
    Ts[r][c] = Tm[r * trs + c * tcs];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (v >= nvec) return;
  double* x = X + v * vstride;
  double x0 = lane < len ? x[lane * estride] : 0.0;
  double x1 = lane + 32 < len ? x[(lane + 32) * estride] : 0.0;
  const int c0 = lane, c1 = lane + 32;
  for (int t = 0; t < len; ++t) {
    const int i = lower ? t : len - 1 - t;
    if (!unit && lane == (i & 31)) {
      if (i < 32) x0 /= Ts[i][i]; else x1 /= Ts[i][i];
    }
    const double xi = __shfl_sync(0xffffffffu, i < 32 ? x0 : x1, i & 31);
    if (lower) {
      if (c0 > i && c0 < len) x0 = fma(-Ts[c0][i], xi, x0);
      if (c1 > i && c1 < len) x1 = fma(-Ts[c1][i], xi, x1);
    } else {
      if (c0 < i) x0 = fma(-Ts[c0][i], xi, x0);
      if (c1 < i) x1 = fma(-Ts[c1][i], xi, x1);
    }
  }
  if (lane < len) x[lane * estride] = x0;
  if (lane + 32 < len) x[(lane + 32) * estride] = x1;
}

// The same solve in compensated FP32: T as FP32 hi/lo in shared memory, the diagonal's
// reciprocals formed once in FP64 and split, x carried as hi/lo pairs; each update
// x_q -= T(q, i) x_i is an exact hi product plus cross terms, combined by TwoSum (about
// 2^-46 relative per operation), with no FP64 instruction in the substitution loop.
__device__ __forceinline__ void df_mul_sub(float& xh, float& xl, float th, float tl, float yh,
                                           float yl) {
  // (xh, xl) -= (th + tl) (yh + yl)
  const float p = __fmul_rn(th, yh);
  const float e = __fmaf_rn(th, yh, -p);
  const float cross = __fmaf_rn(th, yl, __fmul_rn(tl, yh));
  float s1, e1;
  df_two_sum(xh, -p, s1, e1);
  const float lo = __fsub_rn(__fadd_rn(e1, xl), __fadd_rn(e, cross));
  df_two_sum(s1, lo, xh, xl);
}
__device__ __forceinline__ void df_mul(float& xh, float& xl, float rh, float rl) {
  const float p = __fmul_rn(xh, rh);
  const float e = __fmaf_rn(xh, rh, -p);
  const float lo = __fmaf_rn(xh, rl, __fmaf_rn(xl, rh, e));
  df_two_sum(p, lo, xh, xl);
}

// The FP32 hi / lo parts of T come split once per triangular solve (Thg, Tlg, element
// (r, c) at r * trs2 + c * tcs2): every block of the grid would otherwise repeat the FP64
// split of the whole diagonal block, at GB300's FP64 rate.
__global__ void __launch_bounds__(256) trsv_block_df_kernel(int64_t nvec, int len,
                                                            double* __restrict__ X,
                                                            int64_t vstride, int64_t estride,
                                                            const double* __restrict__ Tm,
                                                            int64_t trs, int64_t tcs, int lower,
                                                            int unit,
                                                            const float* __restrict__ Thg,
                                                            const float* __restrict__ Tlg,
                                                            int64_t trs2, int64_t tcs2) {
  __shared__ float Th[TNB][TNB + 1], Tl[TNB][TNB + 1];
  __shared__ float Rh[TNB], Rl[TNB];
  for (int e = threadIdx.x; e < len * len; e += blockDim.x) {
    const int r = e % len, c = e / len;
    Th[r][c] = Thg[r * trs2 + c * tcs2];
    Tl[r][c] = Tlg[r * trs2 + c * tcs2];
  }
  if (threadIdx.x < len) {
    const double rv = unit ? 1.0 : 1.0 / Tm[threadIdx.x * trs + threadIdx.x * tcs];
    const float h = __double2float_rn(rv);
    Rh[threadIdx.x] = h;
    Rl[threadIdx.x] = __double2float_rn(rv - (double)h);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (v >= nvec) return;
  double* x = X + v * vstride;
  const double d0 = lane < len ? x[lane * estride] : 0.0;
  const double d1 = lane + 32 < len ? x[(lane + 32) * estride] : 0.0;
  float x0h = __double2float_rn(d0), x0l = __double2float_rn(d0 - (double)x0h);
  float x1h = __double2float_rn(d1), x1l = __double2float_rn(d1 - (double)x1h);
  const int c0 = lane, c1 = lane + 32;
  for (int t = 0; t < len; ++t) {
    const int i = lower ? t : len - 1 - t;
    if (!unit && lane == (i & 31)) {
      if (i < 32) df_mul(x0h, x0l, Rh[i], Rl[i]);
      else df_mul(x1h, x1l, Rh[i], Rl[i]);
    }
    const float yh = __shfl_sync(0xffffffffu, i < 32 ? x0h : x1h, i & 31);
    const float yl = __shfl_sync(0xffffffffu, i < 32 ? x0l : x1l, i & 31);
    if (lower) {
      if (c0 > i && c0 < len) df_mul_sub(x0h, x0l, Th[c0][i], Tl[c0][i], yh, yl);
      if (c1 > i && c1 < len) df_mul_sub(x1h, x1l, Th[c1][i], Tl[c1][i], yh, yl);
    } else {
      if (c0 < i) df_mul_sub(x0h, x0l, Th[c0][i], Tl[c0][i], yh, yl);
      if (c1 < i) df_mul_sub(x1h, x1l, Th[c1][i], Tl[c1][i], yh, yl);
    }
  }
  if (lane < len) x[lane * estride] = (double)x0h + (double)x0l;
  if (lane + 32 < len) x[(lane + 32) * estride] = (double)x1h + (double)x1l;
}

// Pointer/trans to the sub-block op(A)[r0:, c0:] for use as a GEMM operand.
inline const double* opblk(const double* A, int64_t lda, bool trans, int64_t r0, int64_t c0) {
  return trans ? A + c0 + r0 * lda : A + r0 + c0 * lda;
}
}  // namespace

void dtrsm(cudaStream_t st, bool left, char uplo, bool trans, bool unit, int64_t M, int64_t N,
           const double* A, int64_t lda, double* B, int64_t ldb) {
  if (M <= 0 || N <= 0) return;
  const bool effLower = (uplo == 'L') != trans;  // shape of op(A)
  const int64_t dim = left ? M : N;
  const int64_t nblk = cdiv(dim, TNB);
  const bool fp64 = dense_work().fp64_gemm;
  // compensated form: the dim x dim triangle split once into compact FP32 hi / lo arrays
  const float *Th = nullptr, *Tl = nullptr;
  if (!fp64) {
    DenseWork& wk = dense_work();
    wk.tth.alloc((size_t)dim * dim, st);
    wk.ttl.alloc((size_t)dim * dim, st);
    split_hilo(st, dim, dim, A, lda, wk.tth.p, wk.ttl.p);
    Th = wk.tth.p;
    Tl = wk.ttl.p;
  }
  auto diag = [&](int64_t k0, int64_t kb) {
    // element (r, c) of op(A)_kk; the same element of the compact split at r rs2 + c cs2
    const double* base = A + k0 + k0 * lda;
    const int64_t rs = trans ? lda : 1, cs = trans ? 1 : lda;
    const int64_t rs2 = trans ? dim : 1, cs2 = trans ? 1 : dim;
    const float* bh = fp64 ? nullptr : Th + k0 + k0 * dim;
    const float* bl = fp64 ? nullptr : Tl + k0 + k0 * dim;
    if (left) {
      const int64_t nvec = N;
      if (fp64)
        trsv_block_kernel<<<(unsigned)cdiv(nvec * 32, 256), 256, 0, st>>>(
            nvec, (int)kb, B + k0, ldb, 1, base, rs, cs, effLower ? 1 : 0, unit ? 1 : 0);
      else
        trsv_block_df_kernel<<<(unsigned)cdiv(nvec * 32, 256), 256, 0, st>>>(
            nvec, (int)kb, B + k0, ldb, 1, base, rs, cs, effLower ? 1 : 0, unit ? 1 : 0, bh,
            bl, rs2, cs2);
    } else {
      // X T = B  <=>  T^T x^T = b^T : matrix element (r, c) of T^T = T(c, r)
      const int64_t nvec = M;
      if (fp64)
        trsv_block_kernel<<<(unsigned)cdiv(nvec * 32, 256), 256, 0, st>>>(
            nvec, (int)kb, B + k0 * ldb, 1, ldb, base, cs, rs, effLower ? 0 : 1, unit ? 1 : 0);
      else
        trsv_block_df_kernel<<<(unsigned)cdiv(nvec * 32, 256), 256, 0, st>>>(
            nvec, (int)kb, B + k0 * ldb, 1, ldb, base, cs, rs, effLower ? 0 : 1, unit ? 1 : 0,
            bh, bl, cs2, rs2);
    }
    APL_LAUNCH_CHECK();
  };
  if (left) {
    if (effLower) {
      for (int64_t b = 0; b < nblk; ++b) {
        const int64_t k0 = b * TNB, kb = std::min<int64_t>(TNB, M - k0);
        diag(k0, kb);
        if (k0 + kb < M)
          dgemm(st, trans, 0, M - k0 - kb, N, kb, -1.0, opblk(A, lda, trans, k0 + kb, k0), lda,
                B + k0, ldb, 1.0, B + k0 + kb, ldb);
      }
    } else {
      for (int64_t b = nblk - 1; b >= 0; --b) {
        const int64_t k0 = b * TNB, kb = std::min<int64_t>(TNB, M - k0);
        diag(k0, kb);
        if (k0 > 0)
          dgemm(st, trans, 0, k0, N, kb, -1.0, opblk(A, lda, trans, 0, k0), lda, B + k0, ldb,
                1.0, B, ldb);
      }
    }
  } else {
    if (!effLower) {  // op(A) upper: forward over column blocks
      for (int64_t b = 0; b < nblk; ++b) {
        const int64_t k0 = b * TNB, kb = std::min<int64_t>(TNB, N - k0);
        diag(k0, kb);
        if (k0 + kb < N)
          dgemm(st, 0, trans, M, N - k0 - kb, kb, -1.0, B + k0 * ldb, ldb,
                opblk(A, lda, trans, k0, k0 + kb), lda, 1.0, B + (k0 + kb) * ldb, ldb);
      }
    } else {
      for (int64_t b = nblk - 1; b >= 0; --b) {
        const int64_t k0 = b * TNB, kb = std::min<int64_t>(TNB, N - k0);
        diag(k0, kb);
        if (k0 > 0)
          dgemm(st, 0, trans, M, k0, kb, -1.0, B + k0 * ldb, ldb, opblk(A, lda, trans, k0, 0),
                lda, 1.0, B, ldb);
      }
    }
  }
}

// ------------------------------------------------------------------------------------
// Cholesky (upper), blocked: a shared-memory kernel factors each diagonal block of at
// most 64, a triangular solve forms the block row and a GEMM updates the trailing part.
// ------------------------------------------------------------------------------------
namespace {
constexpr int PNB = 64;

__global__ void __launch_bounds__(256) potrf_small_kernel(int nb, double* A, int64_t lda,
                                                          int* info, int64_t koff) {
  __shared__ double S[PNB][PNB + 1];
  __shared__ int bad;
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    const int r = e % nb, c = e / nb;
    S[r][c] = A[r + c * lda];
  }
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int k = 0; k < nb; ++k) {
    if (threadIdx.x == 0) {
      const double d = S[k][k];
      if (!(d > 0.0) || !isfinite(d)) bad = k + 1;
      else S[k][k] = sqrt(d);
    }
    __syncthreads();
    if (bad) break;
    const double dk = S[k][k];
    for (int j = k + 1 + threadIdx.x; j < nb; j += blockDim.x) S[k][j] /= dk;
    __syncthreads();
    const int t = nb - k - 1;
    for (int e = threadIdx.x; e < t * t; e += blockDim.x) {
      const int i = k + 1 + e / t, j = k + 1 + e % t;
      if (j >= i) S[i][j] -= S[k][i] * S[k][j];
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    const int r = e % nb, c = e / nb;
    A[r + c * lda] = r <= c ? S[r][c] : 0.0;
  }
  if (threadIdx.x == 0 && bad && *info == 0) *info = (int)koff + bad;
}
}  // namespace

void dpotrf_upper(cudaStream_t st, int64_t n, double* A, int64_t lda, int* info_dev) {
  if (n <= 0) return;
  APL_CUDA(cudaMemsetAsync(info_dev, 0, sizeof(int), st));
  for (int64_t k0 = 0; k0 < n; k0 += PNB) {
    const int64_t kb = std::min<int64_t>(PNB, n - k0);
    double* Akk = A + k0 + k0 * lda;
    potrf_small_kernel<<<1, 256, 0, st>>>((int)kb, Akk, lda, info_dev, k0);
    APL_LAUNCH_CHECK();
    const int64_t rest = n - k0 - kb;
    if (rest > 0) {
      double* Akr = A + k0 + (k0 + kb) * lda;
      dtrsm(st, true, 'U', true, false, kb, rest, Akk, lda, Akr, lda);
      dgemm(st, 1, 0, rest, rest, kb, -1.0, Akr, lda, Akr, lda, 1.0,
            A + (k0 + kb) + (k0 + kb) * lda, lda);
    }
  }
  dzero_lower(st, n, A, lda);
}

namespace {

// E <- E T^{-1} for upper triangular T (k x k): T^{-1} by a left triangular solve on the
// identity (contiguous columns), then one GEMM; E's rows are never walked with a stride.
void right_upper_inverse_apply(cudaStream_t st, int64_t n, int64_t k, double* E, int64_t lde,
                               const double* T, int64_t ldt, double* Tinv) {
  dset2d(st, k, k, 0.0, Tinv, k);
  dset_diag(st, k, 1.0, Tinv, k);
  dtrsm(st, true, 'U', false, false, k, k, T, ldt, Tinv, k);
  DBuf<double>& tmp = dense_work().qrtmp;
  tmp.alloc((size_t)n * k, st);
  dgemm(st, 0, 0, n, k, k, 1.0, E, lde, Tinv, k, 0.0, tmp.p, n);
  dcopy2d(st, n, k, tmp.p, n, E, lde, false);
}
}  // namespace

bool cholqr2(cudaStream_t st, int64_t n, int64_t k, double* E, int64_t lde, double* R,
             int64_t ldr, double* work, int* info_dev) {
  // work: 3 k x k blocks
  double* G = work;
  double* R1 = work + k * k;
  double* Ti = work + 2 * k * k;
  int info = 0;
  auto first_gram = [&]() {
    dgemm(st, 1, 0, k, k, n, 1.0, E, lde, E, lde, 0.0, G, k);
    dpotrf_upper(st, k, G, k, info_dev);
    APL_CUDA(cudaMemcpyAsync(&info, info_dev, sizeof(int), cudaMemcpyDeviceToHost, st));
    APL_CUDA(cudaStreamSynchronize(st));
  };
  first_gram();
  if (info && !dense_work().fp64_gemm) {
    // E is untouched so far: redo the first Gram with FP64 products
    Fp64Scope f64;
    first_gram();
  }
  if (info) return false;
  dcopy2d(st, k, k, G, k, R1, k, false);
  right_upper_inverse_apply(st, n, k, E, lde, R1, k, Ti);
  dgemm(st, 1, 0, k, k, n, 1.0, E, lde, E, lde, 0.0, G, k);
  dpotrf_upper(st, k, G, k, info_dev);
  APL_CUDA(cudaMemcpyAsync(&info, info_dev, sizeof(int), cudaMemcpyDeviceToHost, st));
  APL_CUDA(cudaStreamSynchronize(st));
  if (info) return false;
  right_upper_inverse_apply(st, n, k, E, lde, G, k, Ti);
  // R = R2 R1 (both upper; lower parts are zero)
  dgemm(st, 0, 0, k, k, k, 1.0, G, k, R1, k, 0.0, R, ldr);
  dzero_lower(st, k, R, ldr);
  return true;
}

// ------------------------------------------------------------------------------------
// One-sided (Hestenes) Jacobi on the columns of B.  Round-robin ordering: in round r the
// N (even) columns form N/2 disjoint pairs; one block rotates one pair.  At convergence
// the columns of B are mutually orthogonal, their norms are the singular values of B and
// the normalised columns its left singular vectors.  Applied to B = M^T this yields the
// singular values and the right singular vectors of M.
//
// Two stages, because FP64 arithmetic is scarce on this part and FP32 is not: stage 1
// sweeps an FP32 copy of B and accumulates the rotations in W (FP32); W is then made
// orthogonal to FP64 accuracy (Newton-Schulz) and applied to B in FP64, which leaves the
// singular values untouched to FP64 rounding.  Stage 2 sweeps B in FP64 from this nearly
// orthogonal start down to the l * eps threshold; its result alone fixes the accuracy.
// ------------------------------------------------------------------------------------
namespace {
__device__ __forceinline__ int64_t rr_elem(int64_t pos, int64_t r, int64_t N) {
  return pos == 0 ? 0 : 1 + ((pos - 1 + r) % (N - 1));
}

__global__ void __launch_bounds__(256) jacobi_round_kernel(int64_t l, int64_t N, int64_t r,
                                                           double* __restrict__ B, int64_t ldb,
                                                           double tol, int* rotated) {
  __shared__ double sh[3][8];
  __shared__ double cs[2];
  __shared__ int doit;
  const int64_t k = blockIdx.x;
  int64_t p = rr_elem(k, r, N), q = rr_elem(N - 1 - k, r, N);
  if (p >= l || q >= l) return;
  if (p > q) { const int64_t t = p; p = q; q = t; }
  double* bp = B + p * ldb;
  double* bq = B + q * ldb;
  double a = 0.0, b = 0.0, g = 0.0;
  for (int64_t i = threadIdx.x; i < l; i += blockDim.x) {
    const double x = bp[i], y = bq[i];
    a = fma(x, x, a);
    b = fma(y, y, b);
    g = fma(x, y, g);
  }
  a = warp_sum(a);
  b = warp_sum(b);
  g = warp_sum(g);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) { sh[0][wid] = a; sh[1][wid] = b; sh[2][wid] = g; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double A_ = 0, B_ = 0, G_ = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { A_ += sh[0][w]; B_ += sh[1][w]; G_ += sh[2][w]; }
    doit = 0;
    if (A_ > 0.0 && B_ > 0.0 && fabs(G_) > tol * sqrt(A_) * sqrt(B_)) {
      const double zeta = (B_ - A_) / (2.0 * G_);
      const double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
      const double c = 1.0 / sqrt(1.0 + t * t);
      cs[0] = c;
      cs[1] = c * t;
      doit = 1;
      atomicAdd(rotated, 1);
    }
  }
  __syncthreads();
  if (!doit) return;
  const double c = cs[0], s = cs[1];
  for (int64_t i = threadIdx.x; i < l; i += blockDim.x) {
    const double x = bp[i], y = bq[i];
    bp[i] = c * x - s * y;
    bq[i] = s * x + c * y;
  }
}

__global__ void col_norms_kernel(int64_t rows, int64_t cols, const double* M, int64_t ldm,
                                 double* out) {
  __shared__ double sh[32];
  const int64_t c = blockIdx.x;
  if (c >= cols) return;
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < rows; i += blockDim.x) {
    const double x = M[i + c * ldm];
    s = fma(x, x, s);
  }
  s = block_sum(s, sh);
  if (threadIdx.x == 0) out[c] = sqrt(s);
}

// dst(:, q) = src(:, idx[q]) / sig[q]  (zero column when sig[q] == 0)
__global__ void gather_normalise_kernel(int64_t rows, const double* src, int64_t lds,
                                        const int* idx, const double* sig, int64_t k, double* dst,
                                        int64_t ldd) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= rows * k) return;
  const int64_t r = e % rows, q = e / rows;
  const double sq = sig[q];
  dst[r + q * ldd] = sq > 0.0 ? src[r + (int64_t)idx[q] * lds] / sq : 0.0;
}
}  // namespace

namespace {
// FP32 stage, block-cyclic: the l columns form NB (even) blocks of JW columns; in block
// round r the blocks form NB/2 disjoint pairs (round robin) and one CTA takes one pair.
// The CTA holds its 2 JW columns in shared memory and rotates every (P-column, Q-column)
// pair in JW inner rounds of JW disjoint pairs (two warps per pair); in block round 0 it
// first rotates the pairs inside P and inside Q.  Over the NB - 1 block rounds of a sweep
// every pair of columns meets once, as in a scalar cyclic sweep.  The rotations are
// accumulated in a 2JW x 2JW matrix R and applied to the matching columns of W at the
// end (W <- W R).  Angles are computed in FP32: this stage only has to bring the columns
// close to orthogonal; the second (compensated or FP64) stage decides the accuracy.
constexpr int JW = 8;
constexpr int JW2 = 2 * JW;
constexpr int kJac32SmemCap = 220 * 1024;  // dynamic shared memory cap of the FP32 stage
constexpr int kJac32Wpp = 2;                // warps per column pair in the FP32 stage (4 measured slower)

// Column stride of the FP32 stage's shared copy: l rounded up to a multiple of 4, so every
// column starts on a 16-byte boundary and is read as float4; the pad holds zeros.
inline int64_t jac32_ld(int64_t l) { return (l + 3) & ~int64_t(3); }

__device__ __forceinline__ float warp_allsumf(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Barrier of the warps of pair slot pw (64 threads, or 32 * wpp); id 0 is
// __syncthreads'.
__device__ __forceinline__ void pair_bar(int pw, int nthreads = 64) {
  asm volatile("bar.sync %0, %1;" ::"r"(pw + 1), "r"(nthreads) : "memory");
}

// One pair (p, q) handled by WPP warps (interleaved float4 stretches; `half` is the
// warp's part).  Only g = x^T y is a dot product: the squared norms a, b of the CTA's
// columns live in nrm and follow the rotation exactly in exact arithmetic (a - t g,
// b + t g); a norm that the update would lose to cancellation (below 1/16 of its old
// value) is summed again from the rotated column.  The warps meet at their own named
// barrier and add their parts in the same order, so all take the same rotation.  All
// threads of the block call this; it ends with a block-wide barrier, since the next
// inner round reads columns that other pairs rotated.  Part 0 also rotates the columns
// p, q of the accumulated rotation R.
template <int WPP>
__device__ __forceinline__ void jac32_pair2(float* __restrict__ cp, float* __restrict__ cq,
                                            float* __restrict__ R, float* __restrict__ nrm,
                                            int p, int q, bool valid, int64_t n4, float tol,
                                            int lane, int half, int pw, float* xch, int& rot,
                                            float& mx) {
  float4* p4 = reinterpret_cast<float4*>(cp);
  float4* q4 = reinterpret_cast<float4*>(cq);
  float g0 = 0.f, g1 = 0.f;
  if (valid) {
#pragma unroll 2
    for (int k = lane + 32 * half; k < (int)n4; k += 32 * WPP) {
      const float4 x = p4[k], y = q4[k];
      g0 = fmaf(x.x, y.x, g0);
      g1 = fmaf(x.y, y.y, g1);
      g0 = fmaf(x.z, y.z, g0);
      g1 = fmaf(x.w, y.w, g1);
    }
  }
  float g = warp_allsumf(g0 + g1);
  // read before the pair barrier: part 0 rewrites them after it, so every warp of the
  // pair sees the same values
  const float a = nrm[p], b = nrm[q];
  if (lane == 0) xch[half] = g;
  pair_bar(pw, 32 * WPP);
  g = xch[0];
#pragma unroll
  for (int w = 1; w < WPP; ++w) g += xch[w];
  // no barrier before xch is written again: that happens after the closing barrier below
  // the angle needs only FP32 accuracy here (the next stage decides the final one), so
  // it is formed with the approximate reciprocal square root and division
  const float relg =
      (valid && a > 0.f && b > 0.f) ? fabsf(g) * (rsqrtf(a) * rsqrtf(b)) : 0.f;
  if (!(relg > tol)) {
    __syncthreads();
    return;
  }
  mx = fmaxf(mx, relg);
  const float zeta = __fdividef(b - a, 2.f * g);
  const float az = fabsf(zeta);
  // tan of the rotation angle, the smaller root; 1 / (2 zeta) once zeta^2 would overflow
  float t;
  if (az < 1e15f) {
    const float q = 1.f + zeta * zeta;
    t = __fdividef(1.f, az + q * rsqrtf(q));
  } else {
    t = __fdividef(0.5f, az);
  }
  t = zeta >= 0.f ? t : -t;
  const float c = rsqrtf(1.f + t * t), sn = c * t;
  float na = a - t * g, nb = b + t * g;
  const bool refresh = !(na >= 0.0625f * a) || !(nb >= 0.0625f * b);
  float sa = 0.f, sb = 0.f;
#pragma unroll 2
  for (int k = lane + 32 * half; k < (int)n4; k += 32 * WPP) {
    const float4 x = p4[k], y = q4[k];
    float4 u, v;
    u.x = c * x.x - sn * y.x;
    u.y = c * x.y - sn * y.y;
    u.z = c * x.z - sn * y.z;
    u.w = c * x.w - sn * y.w;
    v.x = sn * x.x + c * y.x;
    v.y = sn * x.y + c * y.y;
    v.z = sn * x.z + c * y.z;
    v.w = sn * x.w + c * y.w;
    p4[k] = u;
    q4[k] = v;
    if (refresh) {
      sa = fmaf(u.x, u.x, fmaf(u.y, u.y, fmaf(u.z, u.z, fmaf(u.w, u.w, sa))));
      sb = fmaf(v.x, v.x, fmaf(v.y, v.y, fmaf(v.z, v.z, fmaf(v.w, v.w, sb))));
    }
  }
  if (refresh) {  // the same decision on every warp of the pair
    sa = warp_allsumf(sa);
    sb = warp_allsumf(sb);
    if (lane == 0) { xch[WPP + 2 * half] = sa; xch[WPP + 1 + 2 * half] = sb; }
    pair_bar(pw, 32 * WPP);
    na = xch[WPP];
    nb = xch[WPP + 1];
#pragma unroll
    for (int w = 1; w < WPP; ++w) {
      na += xch[WPP + 2 * w];
      nb += xch[WPP + 1 + 2 * w];
    }
  }
  if (half == 0) {
    if (lane < JW2) {
      const float u = R[lane * JW2 + p], v = R[lane * JW2 + q];
      R[lane * JW2 + p] = c * u - sn * v;
      R[lane * JW2 + q] = sn * u + c * v;
    }
    if (lane == 0) { nrm[p] = na; nrm[q] = nb; }
    ++rot;
  }
  __syncthreads();
}

// Bulk-copy (TMA) helpers: one thread moves whole columns between global and shared
// memory; loads complete on an mbarrier (transaction bytes), stores in a bulk group.
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
// Waits for the phase with the given parity; false once the wait ran past its bound.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity) {
  for (long long it = 0; it < (1LL << 24); ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes,
                                          uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ void bulk_store(void* dst, const void* src, unsigned bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst),
               "r"(smem_addr(src)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit_and_drain() {
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
// generic-proxy writes to shared memory become visible to the bulk-copy (async) proxy
__device__ __forceinline__ void fence_async_shared() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// grid NB/2, block 32 * WPP * JW threads (WPP warps per pair).  B and W are l x l with column
// stride ls = jac32_ld(l) (zero pad rows), so every column is one 16-byte aligned bulk
// copy.  Dynamic shared memory: JW2 columns of B, with WPRE also JW2 columns of W
// (fetched with B, so the fetch overlaps the rotations), then R.  Without WPRE the W
// columns are fetched into the B area after B has been stored.  rotated[0] counts
// rotations, rotated[1] holds the largest rotated |cos| of the sweep (as float bits;
// non-negative floats order like their bits), rotated[2] is set when a wait gave up.
template <bool WPRE, int WPP>
__global__ void __launch_bounds__(32 * WPP * JW) jacobi32_block_kernel(int64_t l, int64_t ls,
                                                                 int64_t NB, int64_t r,
                                                                 float* __restrict__ B,
                                                                 float* __restrict__ W,
                                                                 float tol, int* rotated) {
  extern __shared__ __align__(128) float jsm[];
  float* cols = jsm;                                  // JW2 columns of B, stride ls
  float* wsm = WPRE ? jsm + (size_t)JW2 * ls : jsm;   // JW2 columns of W
  float* R = jsm + (size_t)(WPRE ? 2 : 1) * JW2 * ls;  // JW2 x JW2, R[row * JW2 + col]
  __shared__ __align__(8) uint64_t mbar;
  __shared__ int gcol[JW2];
  __shared__ float nrm[JW2];
  __shared__ int cta_rot, nvalid;
  __shared__ unsigned int cta_max;
  __shared__ float xch[JW][3 * WPP];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int pw = warp / WPP, half = warp % WPP;  // pair slot and part of this warp
  const int64_t k = blockIdx.x;
  const int64_t bp = rr_elem(k, r, NB), bq = rr_elem(NB - 1 - k, r, NB);
  if (threadIdx.x < JW2) {
    const int64_t blk = threadIdx.x < JW ? bp : bq;
    const int64_t c = blk * JW + (threadIdx.x % JW);
    gcol[threadIdx.x] = c < l ? (int)c : -1;
  }
  if (threadIdx.x == 0) {
    cta_rot = 0;
    cta_max = 0u;
    mbar_init(&mbar, 1);
  }
  for (int e = threadIdx.x; e < JW2 * JW2; e += blockDim.x)
    R[e] = (e / JW2 == e % JW2) ? 1.f : 0.f;
  __syncthreads();
  // columns past l (the last block of an odd count) stay zero
  for (int c = 0; c < JW2; ++c)
    if (gcol[c] < 0)
      for (int64_t i = threadIdx.x; i < ls; i += blockDim.x) {
        cols[(size_t)c * ls + i] = 0.f;
        if (WPRE) wsm[(size_t)c * ls + i] = 0.f;
      }
  const unsigned colbytes = (unsigned)(ls * sizeof(float));
  if (threadIdx.x == 0) {
    int nv = 0;
    for (int c = 0; c < JW2; ++c) nv += gcol[c] >= 0;
    nvalid = nv;
    mbar_expect_tx(&mbar, (unsigned)nv * colbytes * (WPRE ? 2u : 1u));
    for (int c = 0; c < JW2; ++c)
      if (gcol[c] >= 0) {
        bulk_load(cols + (size_t)c * ls, B + (int64_t)gcol[c] * ls, colbytes, &mbar);
        if (WPRE) bulk_load(wsm + (size_t)c * ls, W + (int64_t)gcol[c] * ls, colbytes, &mbar);
      }
  }
  if (!mbar_wait_bounded(&mbar, 0)) {
    if (threadIdx.x == 0) atomicExch(rotated + 2, 1);
    mbar_wait_bounded(&mbar, 0);  // the copies in flight target this block's memory
    return;
  }
  __syncthreads();  // the zero columns written by other threads
  const int64_t n4 = ls / 4;
  if (warp < JW2) {
    // squared column norms, one warp per column
    const float4* c4 = reinterpret_cast<const float4*>(cols + (size_t)warp * ls);
    float s0 = 0.f, s1 = 0.f;
    for (int64_t q = lane; q < n4; q += 32) {
      const float4 x = c4[q];
      s0 = fmaf(x.x, x.x, fmaf(x.z, x.z, s0));
      s1 = fmaf(x.y, x.y, fmaf(x.w, x.w, s1));
    }
    const float s = warp_allsumf(s0 + s1);
    if (lane == 0) nrm[warp] = s;
  }
  __syncthreads();
  int rot = 0;
  float mx = 0.f;
  if (r == 0) {
    // pairs inside each block: JW - 1 round-robin rounds of JW/2 pairs per block
    for (int ir = 0; ir < JW - 1; ++ir) {
      const int t = pw % (JW / 2), side = pw / (JW / 2);
      int p = (int)rr_elem(t, ir, JW), q = (int)rr_elem(JW - 1 - t, ir, JW);
      if (p > q) { const int z = p; p = q; q = z; }
      p += side * JW;
      q += side * JW;
      jac32_pair2<WPP>(cols + (size_t)p * ls, cols + (size_t)q * ls, R, nrm, p, q,
                  gcol[p] >= 0 && gcol[q] >= 0, n4, tol, lane, half, pw, xch[pw], rot, mx);
    }
  }
  for (int ir = 0; ir < JW; ++ir) {
    const int p = pw, q = JW + (pw + ir) % JW;
    jac32_pair2<WPP>(cols + (size_t)p * ls, cols + (size_t)q * ls, R, nrm, p, q,
                gcol[p] >= 0 && gcol[q] >= 0, n4, tol, lane, half, pw, xch[pw], rot, mx);
  }
  if (lane == 0 && half == 0 && rot) {
    atomicAdd(&cta_rot, rot);
    atomicMax(&cta_max, __float_as_uint(mx));
  }
  __syncthreads();
  if (cta_rot == 0) return;  // nothing rotated: B and W stay as they are
  if (threadIdx.x == 0) {
    atomicAdd(rotated, cta_rot);
    atomicMax(reinterpret_cast<unsigned int*>(rotated + 1), cta_max);
  }
  if (!WPRE) {
    // store B, then fetch W into the same columns
    fence_async_shared();
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int c = 0; c < JW2; ++c)
        if (gcol[c] >= 0) bulk_store(B + (int64_t)gcol[c] * ls, cols + (size_t)c * ls, colbytes);
      bulk_commit_and_drain();
      mbar_expect_tx(&mbar, (unsigned)nvalid * colbytes);
      for (int c = 0; c < JW2; ++c)
        if (gcol[c] >= 0) bulk_load(cols + (size_t)c * ls, W + (int64_t)gcol[c] * ls, colbytes, &mbar);
    }
    if (!mbar_wait_bounded(&mbar, 1)) {
      if (threadIdx.x == 0) atomicExch(rotated + 2, 1);
      mbar_wait_bounded(&mbar, 1);
      return;
    }
  }
  // W(:, cols) <- W(:, cols) R in shared memory, one row per thread and pass, the 16
  // outputs in two halves of 8; R rows are read as float4
  const float4* R4 = reinterpret_cast<const float4*>(R);
  for (int64_t i = threadIdx.x; i < l; i += blockDim.x) {
    float w[JW2];
#pragma unroll
    for (int c = 0; c < JW2; ++c) w[c] = wsm[(size_t)c * ls + i];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float o[JW];
#pragma unroll
      for (int j = 0; j < JW; ++j) o[j] = 0.f;
#pragma unroll
      for (int c = 0; c < JW2; ++c) {
        const float4 r0 = R4[(c * JW2 + h * JW) / 4], r1 = R4[(c * JW2 + h * JW) / 4 + 1];
        o[0] = fmaf(w[c], r0.x, o[0]);
        o[1] = fmaf(w[c], r0.y, o[1]);
        o[2] = fmaf(w[c], r0.z, o[2]);
        o[3] = fmaf(w[c], r0.w, o[3]);
        o[4] = fmaf(w[c], r1.x, o[4]);
        o[5] = fmaf(w[c], r1.y, o[5]);
        o[6] = fmaf(w[c], r1.z, o[6]);
        o[7] = fmaf(w[c], r1.w, o[7]);
      }
#pragma unroll
      for (int j = 0; j < JW; ++j) wsm[(size_t)(h * JW + j) * ls + i] = o[j];
    }
  }
  fence_async_shared();
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int c = 0; c < JW2; ++c)
      if (gcol[c] >= 0) {
        if (WPRE) bulk_store(B + (int64_t)gcol[c] * ls, cols + (size_t)c * ls, colbytes);
        bulk_store(W + (int64_t)gcol[c] * ls, wsm + (size_t)c * ls, colbytes);
      }
    bulk_commit_and_drain();
  }
}

// Stage 2 in compensated FP32, block-cyclic like stage 1: the CTA's 16 columns live in
// shared memory as FP32 hi/lo pairs (48 of the 53 bits of B); dot products are summed as
// unevaluated FP32 pairs (TwoSum) and the rotation is applied in compensated FP32.
// Singular values depend on the off-diagonal only to second order, so the threshold
// (set above the dot-product noise, about 1e-12) leaves them accurate to rounding; the
// vectors carry first-order errors at the threshold.
// (h, l) <- c * x with c = ch + cl and x = xh + xl
__device__ __forceinline__ void df_scale(float ch, float cl, float xh, float xl, float& h,
                                         float& l) {
  h = __fmul_rn(ch, xh);
  const float e = __fmaf_rn(ch, xh, -h);
  l = __fmaf_rn(ch, xl, __fmaf_rn(cl, xh, e));
}
// acc += x * y (pairs)
__device__ __forceinline__ void df_dot_add(float& s, float& c, float xh, float xl, float yh,
                                           float yl) {
  const float p = __fmul_rn(xh, yh);
  const float e = __fmaf_rn(xh, yh, -p);
  const float cross = __fmaf_rn(xh, yl, __fmul_rn(xl, yh));
  float t, err;
  df_two_sum(s, p, t, err);
  s = t;
  c = __fadd_rn(c, __fadd_rn(err, __fadd_rn(e, cross)));
}

// (s, c) + (t, d) as unevaluated FP32 pairs; TwoSum's error term is exact, so the sum is
// the same bitwise in either operand order (butterfly reductions agree on every lane).
__device__ __forceinline__ void df_add(float& s, float& c, float t, float d) {
  float h, e;
  df_two_sum(s, t, h, e);
  const float lo = __fadd_rn(e, __fadd_rn(c, d));
  s = __fadd_rn(h, lo);
  c = __fsub_rn(lo, __fsub_rn(s, h));
}
__device__ __forceinline__ void df_warp_allsum(float& s, float& c) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float t = __shfl_xor_sync(0xffffffffu, s, o);
    const float d = __shfl_xor_sync(0xffffffffu, c, o);
    df_add(s, c, t, d);
  }
}
// 1/sqrt(v) for v = vh + vl as a pair, by two Newton steps from the FP32 estimate; the
// result (ch, cl) satisfies ch^2 (vh + vl) = 1 to about 2^-46.
__device__ __forceinline__ void df_rsqrt(float vh, float vl, float& ch, float& cl) {
  float y = rsqrtf(vh), yl = 0.f;
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    // r = 1 - v y^2 (small), y <- y + y r / 2
    const float q = __fmul_rn(y, y);
    const float qe = __fmaf_rn(y, y, -q);
    const float q2 = __fmaf_rn(2.f * y, yl, qe);  // low part of (y + yl)^2
    const float p = __fmul_rn(vh, q);
    const float pe = __fmaf_rn(vh, q, -p);
    const float plo = __fmaf_rn(vh, q2, __fmaf_rn(vl, q, pe));
    const float r = __fsub_rn(__fsub_rn(1.f, p), plo);
    const float corr = __fmul_rn(0.5f * y, r);
    float h, e;
    df_two_sum(y, __fadd_rn(yl, corr), h, e);
    y = h;
    yl = e;
  }
  ch = y;
  cl = yl;
}

// (h, l) <- (xh + xl) + d for a small FP32 d, renormalised
__device__ __forceinline__ void df_nudge(float xh, float xl, float d, float& h, float& l) {
  float r, e;
  df_two_sum(xh, d, r, e);
  const float lo = __fadd_rn(e, xl);
  h = __fadd_rn(r, lo);
  l = __fsub_rn(lo, __fsub_rn(h, r));
}

// x' = c x - s y and y' = s x + c y for one hi/lo element, c = (ch, cl), s = (sh, sl)
__device__ __forceinline__ void df_rotate(float ch, float cl, float sh, float sl, float xh,
                                          float xl, float yh, float yl, float& uh, float& ul,
                                          float& vh, float& vl) {
  float cxh, cxl, syh, syl, sxh, sxl, cyh, cyl;
  df_scale(ch, cl, xh, xl, cxh, cxl);
  df_scale(sh, sl, yh, yl, syh, syl);
  df_scale(sh, sl, xh, xl, sxh, sxl);
  df_scale(ch, cl, yh, yl, cyh, cyl);
  float r, er;
  df_two_sum(cxh, -syh, r, er);
  df_two_sum(r, __fadd_rn(er, __fsub_rn(cxl, syl)), uh, ul);
  df_two_sum(sxh, cyh, r, er);
  df_two_sum(r, __fadd_rn(er, __fadd_rn(sxl, cyl)), vh, vl);
}

// One pair (p, q) of columns handled by two warps (interleaved stretches of float4 = two
// hi/lo elements).  Only g = x^T y is a compensated dot product: the squared norms, kept
// as pairs (nh, nl) for the CTA's columns, follow the rotation as a - t g and b + t g.
// That is exact for the exact root t; the FP32 t is off only to second order in its
// rounding, as the angle is a stationary point of |x'|^2.  A norm that the update would
// lose to cancellation (below 1/16 of its old value) is summed again from the rotated
// column.  The halves meet at the pair's own named barrier and add in half order, so both
// warps form the same rotation.  The angle comes from FP32 arithmetic on the compensated
// sums (an approximate angle only slows convergence); its cosine and sine are formed as
// pairs with c^2 + s^2 = 1 to about 2^-46, so every rotation is orthogonal to that
// accuracy.  All threads of the block call this; it ends with a block-wide barrier.
__device__ __forceinline__ void jacdf_pair2(float4* __restrict__ cp, float4* __restrict__ cq,
                                            float* __restrict__ nh, float* __restrict__ nl,
                                            int p, int q, bool valid, int64_t n2, float tol,
                                            int lane, int half, int pw, float* xch, int& rot,
                                            float& mx) {
  float gs = 0.f, gc = 0.f, hs = 0.f, hc = 0.f;
  if (valid) {
#pragma unroll 2
    for (int k = lane + 32 * half; k < (int)n2; k += 64) {
      const float4 x = cp[k], y = cq[k];
      df_dot_add(gs, gc, x.x, x.y, y.x, y.y);
      df_dot_add(hs, hc, x.z, x.w, y.z, y.w);
    }
  }
  df_add(gs, gc, hs, hc);
  df_warp_allsum(gs, gc);
  // read before the pair barrier: half 0 rewrites them after it, so both warps see the
  // same values
  const float A = nh[p], Al = nl[p], Bv = nh[q], Bl = nl[q];
  if (lane == 0) { xch[2 * half] = gs; xch[2 * half + 1] = gc; }
  pair_bar(pw);
  float G = xch[0], Gl = xch[1];
  df_add(G, Gl, xch[2], xch[3]);
  // no barrier before xch is written again: that happens after the closing barrier below
  const float relg = (valid && A > 0.f && Bv > 0.f) ? fabsf(G) / (sqrtf(A) * sqrtf(Bv)) : 0.f;
  if (!(relg > tol)) {
    __syncthreads();  // the next inner round reads columns other warps may still rotate
    return;
  }
  mx = fmaxf(mx, relg);
  // zeta = (b - a) / (2 g) with b - a formed from the pairs (no cancellation loss)
  float dh = Bv, dl = Bl;
  df_add(dh, dl, -A, -Al);
  const float zeta = __fdiv_rn(__fadd_rn(dh, dl), 2.f * G);
  const float az = fabsf(zeta);
  float t = az < 1e15f ? 1.f / (az + sqrtf(1.f + zeta * zeta)) : 0.5f / az;
  t = zeta >= 0.f ? t : -t;
  // c = 1 / sqrt(1 + t^2), s = c t, as pairs
  const float t2 = __fmul_rn(t, t);
  const float t2e = __fmaf_rn(t, t, -t2);
  float vh, vl;
  df_two_sum(1.f, t2, vh, vl);
  vl = __fadd_rn(vl, t2e);
  float ch, cl;
  df_rsqrt(vh, vl, ch, cl);
  const float sh = __fmul_rn(ch, t);
  const float sl = __fmaf_rn(cl, t, __fmaf_rn(ch, t, -sh));
  // t g as a pair, then the updated norms
  const float tg = __fmul_rn(t, G);
  const float tgl = __fmaf_rn(t, Gl, __fmaf_rn(t, G, -tg));
  float NA = A, NAl = Al, NB = Bv, NBl = Bl;
  df_add(NA, NAl, -tg, -tgl);
  df_add(NB, NBl, tg, tgl);
  const bool refresh = !(NA >= 0.0625f * A) || !(NB >= 0.0625f * Bv);
  float as = 0.f, ac = 0.f, bs = 0.f, bc = 0.f;
  // |t| <= 2^-23: x' = x + (c - 1) x - s y with the small update formed in FP32 from the
  // high parts; what it drops (s y_lo, s_lo y, the update's rounding) is below
  // 2^-23 |s| |y|, the compensated rotation's own error level
  const bool small = fabsf(t) <= 1.1920928955078125e-7f;
  const float em = __fadd_rn(__fsub_rn(ch, 1.f), cl);  // c - 1
#pragma unroll 2
  for (int k = lane + 32 * half; k < (int)n2; k += 64) {
    const float4 x = cp[k];
    const float4 y = cq[k];
    float4 u, v;
    if (small) {
      df_nudge(x.x, x.y, __fmaf_rn(-sh, y.x, __fmul_rn(em, x.x)), u.x, u.y);
      df_nudge(x.z, x.w, __fmaf_rn(-sh, y.z, __fmul_rn(em, x.z)), u.z, u.w);
      df_nudge(y.x, y.y, __fmaf_rn(sh, x.x, __fmul_rn(em, y.x)), v.x, v.y);
      df_nudge(y.z, y.w, __fmaf_rn(sh, x.z, __fmul_rn(em, y.z)), v.z, v.w);
    } else {
      df_rotate(ch, cl, sh, sl, x.x, x.y, y.x, y.y, u.x, u.y, v.x, v.y);
      df_rotate(ch, cl, sh, sl, x.z, x.w, y.z, y.w, u.z, u.w, v.z, v.w);
    }
    cp[k] = u;
    cq[k] = v;
    if (refresh) {
      df_dot_add(as, ac, u.x, u.y, u.x, u.y);
      df_dot_add(as, ac, u.z, u.w, u.z, u.w);
      df_dot_add(bs, bc, v.x, v.y, v.x, v.y);
      df_dot_add(bs, bc, v.z, v.w, v.z, v.w);
    }
  }
  if (refresh) {  // the same decision on both warps of the pair
    df_warp_allsum(as, ac);
    df_warp_allsum(bs, bc);
    if (lane == 0) {
      float* o = xch + 4 + 4 * half;
      o[0] = as; o[1] = ac; o[2] = bs; o[3] = bc;
    }
    pair_bar(pw);
    NA = xch[4]; NAl = xch[5];
    df_add(NA, NAl, xch[8], xch[9]);
    NB = xch[6]; NBl = xch[7];
    df_add(NB, NBl, xch[10], xch[11]);
  }
  if (half == 0) {
    if (lane == 0) { nh[p] = NA; nl[p] = NAl; nh[q] = NB; nl[q] = NBl; }
    ++rot;
  }
  __syncthreads();
}

// Column stride (in hi/lo elements) of the compensated stage's working copy: l rounded up
// to even, so every column is one 16-byte aligned bulk copy; the pad holds zeros.
inline int64_t jacdf_ld(int64_t l) { return (l + 1) & ~int64_t(1); }

// D (hi/lo pairs, column stride ldd) <- B (l x l FP64, ld ldb); pad rows zero
__global__ void split_df_kernel(int64_t l, const double* __restrict__ B, int64_t ldb,
                                float2* __restrict__ D, int64_t ldd) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ldd * l) return;
  const int64_t r = e % ldd, c = e / ldd;
  float2 v = make_float2(0.f, 0.f);
  if (r < l) {
    const double x = B[r + c * ldb];
    v.x = __double2float_rn(x);
    v.y = __double2float_rn(x - (double)v.x);
  }
  D[e] = v;
}
// B <- D as FP64 (hi + lo)
__global__ void join_df_kernel(int64_t l, const float2* __restrict__ D, int64_t ldd,
                               double* __restrict__ B, int64_t ldb) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= l * l) return;
  const int64_t r = e % l, c = e / l;
  const float2 v = D[r + c * ldd];
  B[r + c * ldb] = (double)v.x + (double)v.y;
}

// grid NB/2, block 64 * JW threads (two warps per pair).  D holds the l columns as FP32
// hi/lo pairs with column stride ls = jacdf_ld(l) (zero pad rows); the block's JW2
// columns arrive in shared memory as bulk copies and leave the same way.  Dynamic shared
// memory JW2 * ls float2.  rotated[0] counts rotations, rotated[1] holds the largest
// rotated |cos| of the sweep (as float bits; non-negative floats order like their bits),
// rotated[2] is set when a wait gave up.
__global__ void __launch_bounds__(64 * JW) jacobi_df_block_kernel(int64_t l, int64_t ls,
                                                                  int64_t NB, int64_t r,
                                                                  float2* __restrict__ D,
                                                                  float tol, int* rotated) {
  extern __shared__ __align__(128) float2 dsm[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ int gcol[JW2];
  __shared__ float nh[JW2], nl[JW2];
  __shared__ int cta_rot;
  __shared__ unsigned int cta_max;
  __shared__ float xch[JW][12];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int pw = warp >> 1, half = warp & 1;  // pair slot and half of this warp
  const int64_t k = blockIdx.x;
  const int64_t bp = rr_elem(k, r, NB), bq = rr_elem(NB - 1 - k, r, NB);
  if (threadIdx.x < JW2) {
    const int64_t blk = threadIdx.x < JW ? bp : bq;
    const int64_t c = blk * JW + (threadIdx.x % JW);
    gcol[threadIdx.x] = c < l ? (int)c : -1;
  }
  if (threadIdx.x == 0) {
    cta_rot = 0;
    cta_max = 0u;
    mbar_init(&mbar, 1);
  }
  __syncthreads();
  for (int c = 0; c < JW2; ++c)
    if (gcol[c] < 0)
      for (int64_t i = threadIdx.x; i < ls; i += blockDim.x)
        dsm[(size_t)c * ls + i] = make_float2(0.f, 0.f);
  const unsigned colbytes = (unsigned)(ls * sizeof(float2));
  if (threadIdx.x == 0) {
    int nv = 0;
    for (int c = 0; c < JW2; ++c) nv += gcol[c] >= 0;
    mbar_expect_tx(&mbar, (unsigned)nv * colbytes);
    for (int c = 0; c < JW2; ++c)
      if (gcol[c] >= 0)
        bulk_load(dsm + (size_t)c * ls, D + (int64_t)gcol[c] * ls, colbytes, &mbar);
  }
  if (!mbar_wait_bounded(&mbar, 0)) {
    if (threadIdx.x == 0) atomicExch(rotated + 2, 1);
    mbar_wait_bounded(&mbar, 0);  // the copies in flight target this block's memory
    return;
  }
  __syncthreads();  // the zero columns written by other threads
  const int64_t n2 = ls / 2;
  {
    // squared column norms as pairs, one warp per column (the block has JW2 warps)
    const float4* c4 = reinterpret_cast<const float4*>(dsm + (size_t)warp * ls);
    float s0 = 0.f, e0 = 0.f, s1 = 0.f, e1 = 0.f;
    for (int64_t q = lane; q < n2; q += 32) {
      const float4 x = c4[q];
      df_dot_add(s0, e0, x.x, x.y, x.x, x.y);
      df_dot_add(s1, e1, x.z, x.w, x.z, x.w);
    }
    df_add(s0, e0, s1, e1);
    df_warp_allsum(s0, e0);
    if (lane == 0) { nh[warp] = s0; nl[warp] = e0; }
  }
  __syncthreads();
  float4* d4 = reinterpret_cast<float4*>(dsm);
  int rot = 0;
  float mx = 0.f;
  if (r == 0) {
    for (int ir = 0; ir < JW - 1; ++ir) {
      const int t = pw % (JW / 2), side = pw / (JW / 2);
      int p = (int)rr_elem(t, ir, JW), q = (int)rr_elem(JW - 1 - t, ir, JW);
      if (p > q) { const int z = p; p = q; q = z; }
      p += side * JW;
      q += side * JW;
      jacdf_pair2(d4 + (size_t)p * n2, d4 + (size_t)q * n2, nh, nl, p, q,
                  gcol[p] >= 0 && gcol[q] >= 0, n2, tol, lane, half, pw, xch[pw], rot, mx);
    }
  }
  for (int ir = 0; ir < JW; ++ir) {
    const int p = pw, q = JW + (pw + ir) % JW;
    jacdf_pair2(d4 + (size_t)p * n2, d4 + (size_t)q * n2, nh, nl, p, q,
                gcol[p] >= 0 && gcol[q] >= 0, n2, tol, lane, half, pw, xch[pw], rot, mx);
  }
  if (lane == 0 && half == 0 && rot) {
    atomicAdd(&cta_rot, rot);
    atomicMax(&cta_max, __float_as_uint(mx));
  }
  __syncthreads();
  if (cta_rot == 0) return;
  fence_async_shared();
  __syncthreads();
  if (threadIdx.x == 0) {
    atomicAdd(rotated, cta_rot);
    atomicMax(reinterpret_cast<unsigned int*>(rotated + 1), cta_max);
    for (int c = 0; c < JW2; ++c)
      if (gcol[c] >= 0) bulk_store(D + (int64_t)gcol[c] * ls, dsm + (size_t)c * ls, colbytes);
    bulk_commit_and_drain();
  }
}

// d (ldd x l, FP32) <- s (l x l, FP64, ld lds); rows l .. ldd-1 of d are zero
__global__ void d2f_kernel(int64_t l, const double* s, int64_t lds, float* d, int64_t ldd) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ldd * l) return;
  const int64_t r = e % ldd, c = e / ldd;
  d[e] = r < l ? (float)s[r + c * lds] : 0.f;
}
// d (l x l, FP64, ld l) <- s (l x l, FP32, ld lds)
__global__ void f2d_kernel(int64_t l, const float* s, int64_t lds, double* d) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= l * l) return;
  const int64_t r = e % l, c = e / l;
  d[e] = (double)s[r + c * lds];
}
// W (ldw x n) <- the identity, zero pad rows
__global__ void eye32_kernel(int64_t n, float* W, int64_t ldw) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < ldw * n) W[e] = (e % ldw == e / ldw) ? 1.f : 0.f;
}


// Run sweeps of `round` (a lambda launching round r) as one captured graph per sweep
// until a sweep rotates nothing; returns the sweep count.
template <typename F>
int run_sweeps(cudaStream_t st, int64_t N, int max_sweeps, int* flag_dev, F&& round,
               int prof_cat, double flops_per_sweep, double flops_per_rot,
               double stop_max = 0.0) {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  APL_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  {
    CaptureScope cs;
    try {
      for (int64_t r = 0; r < N - 1; ++r) round(r);
    } catch (...) {
      cudaStreamEndCapture(st, &graph);
      if (graph) cudaGraphDestroy(graph);
      throw;
    }
  }
  APL_CUDA(cudaStreamEndCapture(st, &graph));
  cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  APL_CUDA(e);
  struct Guard {
    cudaGraphExec_t e;
    ~Guard() { cudaGraphExecDestroy(e); }
  } guard{exec};
  int sweeps = 0;
  for (; sweeps < max_sweeps;) {
    APL_CUDA(cudaMemsetAsync(flag_dev, 0, 3 * sizeof(int), st));
    const int tok = prof_cat >= 0 ? prof_begin(st) : -1;
    APL_CUDA(cudaGraphLaunch(exec, st));
    add_launches(N - 1);
    if (tok >= 0) prof_end(st, tok, prof_cat, 0.0);
    ++sweeps;
    int fl[3] = {0, 0, 0};
    APL_CUDA(cudaMemcpyAsync(fl, flag_dev, 3 * sizeof(int), cudaMemcpyDeviceToHost, st));
    APL_CUDA(cudaStreamSynchronize(st));
    if (fl[2]) throw Error(ST_ETIMEOUT, "Jacobi sweep: a bulk-copy wait ran past its bound");
    const int rot = fl[0];
    if (tok >= 0) prof_set_work(tok, flops_per_sweep + flops_per_rot * rot);
    if (rot == 0) break;
    // every rotation of this sweep was below stop_max: the cyclic sweep converges
    // quadratically, so what remains is of order stop_max^2, far under the threshold
    float mx;
    std::memcpy(&mx, &fl[1], sizeof(float));
    if (stop_max > 0.0 && (double)mx <= stop_max) break;
  }
  return sweeps;
}
}  // namespace

namespace {
// v <- y / ||y||_2 and lam <- ||y||_2, one block
__global__ void __launch_bounds__(1024) normalize_kernel(int64_t n, const double* __restrict__ y,
                                                         double* __restrict__ v, double* lam) {
  __shared__ double part[32];
  __shared__ double nrm;
  double ss = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) ss = fma(y[i], y[i], ss);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = ss;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
    nrm = sqrt(t);
    *lam = nrm;
  }
  __syncthreads();
  const double inv = nrm > 0.0 ? 1.0 / nrm : 1.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) v[i] = y[i] * inv;
}
// a fixed start vector with no special structure: 1 + ((7919 i) mod 101) / 101
__global__ void start_vector_kernel(int64_t n, double* v) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = 1.0 + (double)((7919 * i) % 101) / 101.0;
}
}  // namespace

double power_sigma_min(cudaStream_t st, int64_t L, const double* Minv, int64_t ldm, double* work,
                       int iters) {
  if (L <= 0) return 0.0;
  double* v = work;
  double* t = work + L;
  double* y = work + 2 * L;
  double* lam = work + 3 * L;
  start_vector_kernel<<<(unsigned)cdiv(L, 256), 256, 0, st>>>(L, y);
  APL_LAUNCH_CHECK();
  normalize_kernel<<<1, 1024, 0, st>>>(L, y, v, lam);
  APL_LAUNCH_CHECK();
  for (int it = 0; it < iters; ++it) {
    dgemm(st, 0, 0, L, 1, L, 1.0, Minv, ldm, v, L, 0.0, t, L);  // t = M^{-1} v
    dgemm(st, 1, 0, L, 1, L, 1.0, Minv, ldm, t, L, 0.0, y, L);  // y = M^{-T} t
    normalize_kernel<<<1, 1024, 0, st>>>(L, y, v, lam);
    APL_LAUNCH_CHECK();
  }
  double h = 0.0;
  APL_CUDA(cudaMemcpyAsync(&h, lam, sizeof(double), cudaMemcpyDeviceToHost, st));
  APL_CUDA(cudaStreamSynchronize(st));
  return h > 0.0 ? 1.0 / std::sqrt(h) : 0.0;
}

int jacobi_left(cudaStream_t st, int64_t l, double* B, int64_t ldb, double* U, int64_t ldu,
                double* sigma, int* flag_dev, const double* W0, int64_t l0, double* Wout,
                int64_t* wout_l) {
  if (wout_l) *wout_l = 0;
  if (l <= 0) return 0;
  const int64_t N = (l % 2) ? l + 1 : l;
  int sweeps = 0;
  const size_t smem = ((size_t)JW2 * jac32_ld(l) + JW2 * JW2) * sizeof(float);
  if (l > 1 && smem <= (size_t)kJac32SmemCap) {
    // warm start: B(:, 0:l0) <- B(:, 0:l0) W0 with the orthogonal W0 of an earlier
    // factorisation whose matrix was close to this one's leading block (singular values
    // unchanged, the sweeps start nearly converged on those columns)
    const bool warm = W0 && l0 > 0 && l0 <= l;
    if (warm) {
      DenseWork& wk0 = dense_work();
      wk0.jtmp.alloc(l * l, st);
      dgemm(st, 0, 0, l, l0, l0, 1.0, B, ldb, W0, l0, 0.0, wk0.jtmp.p, l);
      dcopy2d(st, l, l0, wk0.jtmp.p, l, B, ldb, false);
    }
    // Stage 1 (FP32): sweeps on an FP32 copy that accumulate the rotation W until the
    // columns are orthogonal to FP32 accuracy; then B <- B W in FP64.  Skipped when the
    // CTA's two column blocks do not fit in shared memory (l above about 3600).
    const int64_t l2 = l * l;
    const int64_t ls = jac32_ld(l);
    DenseWork& wk = dense_work();
    wk.jb32.alloc(ls * l, st);
    wk.jw32.alloc(ls * l, st);
    wk.jw64.alloc(l2, st);
    wk.jtmp.alloc(l2, st);
    wk.jw2.alloc(l2, st);
    float* B32 = wk.jb32.p;
    float* W32 = wk.jw32.p;
    // the sweep kernels move whole columns with bulk copies: 16-byte aligned bases
    APL_REQUIRE(((uintptr_t)B32 & 15) == 0 && ((uintptr_t)W32 & 15) == 0,
                "jacobi_left: work buffers not 16-byte aligned");
    d2f_kernel<<<(unsigned)cdiv(ls * l, 256), 256, 0, st>>>(l, B, ldb, B32, ls);
    APL_LAUNCH_CHECK();
    eye32_kernel<<<(unsigned)cdiv(ls * l, 256), 256, 0, st>>>(l, W32, ls);
    APL_LAUNCH_CHECK();
    // FP32 dot products summed lane-wise then by a 5-level tree: the relative error of
    // g / sqrt(a b) stays below (l/32 + 5) u32; the threshold sits above twice that
    const double tol32 = std::max(6e-6, 2.0 * ((double)l / 32.0 + 5.0) * 5.960464477539063e-8);
    const int64_t nb = cdiv(l, (int64_t)JW);
    const int64_t NB = nb + (nb % 2);
    // W's columns ride along with B's when both fit in shared memory
    const size_t smem_pre = ((size_t)2 * JW2 * ls + JW2 * JW2) * sizeof(float);
    const bool wpre = smem_pre <= (size_t)kJac32SmemCap;
    // one value for every call: threads that build preconditioners concurrently must not
    // lower the cap under each other's launches
    APL_CUDA(cudaFuncSetAttribute(jacobi32_block_kernel<true, kJac32Wpp>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, kJac32SmemCap));
    APL_CUDA(cudaFuncSetAttribute(jacobi32_block_kernel<false, kJac32Wpp>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, kJac32SmemCap));
    // per pair and sweep: the dot product g (2 l) and the rotation (6 l); the norms follow
    // the rotations
    const double flops32 = 8.0 * (double)l * (double)l * (double)(l - 1) / 2.0;
    // A sweep whose rotations all had |cos| <= 5e-3 ends the stage: the next would find
    // about the square of that, and the compensated stage converges from there in as
    // many sweeps as from the fully converged FP32 start.
    sweeps += run_sweeps(st, NB, 40, flag_dev, [&](int64_t r) {
      if (wpre)
        jacobi32_block_kernel<true, kJac32Wpp><<<(unsigned)(NB / 2), 32 * kJac32Wpp * JW,
                                                 smem_pre, st>>>(l, ls, NB, r, B32, W32,
                                                                 (float)tol32, flag_dev);
      else
        jacobi32_block_kernel<false, kJac32Wpp><<<(unsigned)(NB / 2), 32 * kJac32Wpp * JW,
                                                  smem, st>>>(l, ls, NB, r, B32, W32,
                                                              (float)tol32, flag_dev);
      APL_LAUNCH_CHECK();
    }, PROF_JACOBI32, flops32, 0.0, 5e-3);
    f2d_kernel<<<(unsigned)cdiv(l2, 256), 256, 0, st>>>(l, W32, ls, wk.jw64.p);
    APL_LAUNCH_CHECK();
    // W is orthogonal only to FP32 accuracy; two Newton-Schulz steps
    // W <- W (3 I - W^T W) / 2 make it orthogonal to FP64 accuracy, so B W keeps the
    // singular values of B exactly (to rounding)
    double* Wd = wk.jw64.p;
    double* Wn = wk.jw2.p;
    double* G = wk.jtmp.p;
    for (int it = 0; it < 2; ++it) {
      dgemm(st, 1, 0, l, l, l, -0.5, Wd, l, Wd, l, 0.0, G, l);
      dadd_diag(st, l, 1.5, G, l);
      dgemm(st, 0, 0, l, l, l, 1.0, Wd, l, G, l, 0.0, Wn, l);
      std::swap(Wd, Wn);
    }
    dgemm(st, 0, 0, l, l, l, 1.0, B, ldb, Wd, l, 0.0, G, l);
    dcopy2d(st, l, l, G, l, B, ldb, false);
    if (Wout) {
      // the whole rotation of this stage, diag(W0, I) Wd, for the next warm start
      if (warm) {
        dgemm(st, 0, 0, l0, l, l0, 1.0, W0, l0, Wd, l, 0.0, Wout, l);
        if (l > l0) dcopy2d(st, l - l0, l, Wd + l0, l, Wout + l0, l, false);
      } else {
        dcopy2d(st, l, l, Wd, l, Wout, l, false);
      }
      if (wout_l) *wout_l = l;
    }
  }
  const size_t smem_df = (size_t)JW2 * jacdf_ld(l) * sizeof(float2);
  if (l > 1 && !dense_work().fp64_gemm && smem_df <= (size_t)kJac32SmemCap) {
    // Stage 2 in compensated FP32 (default): block-cyclic sweeps on hi/lo columns.
    // Threshold above the noise of the compensated dot products, about (l/64 + 6) 2^-46
    // relative; a sweep whose rotations were all below 1e-2 sqrt(tol) ends the iteration
    // (the next sweep would find at most about the square of that).
    const double tol = std::max(1e-13, 4.0 * ((double)l / 64.0 + 6.0) * 1.4210854715202004e-14);
    const int64_t nb = cdiv(l, (int64_t)JW);
    const int64_t NB = nb + (nb % 2);
    APL_CUDA(cudaFuncSetAttribute(jacobi_df_block_kernel,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, kJac32SmemCap));
    const double pairs = (double)(l * (l - 1)) / 2.0;
    // the sweeps work on a hi/lo copy of B: split once here, joined once after
    const int64_t ls = jacdf_ld(l);
    DenseWork& wk = dense_work();
    wk.jb32.alloc(2 * ls * l, st);
    float2* D = reinterpret_cast<float2*>(wk.jb32.p);
    APL_REQUIRE(((uintptr_t)D & 15) == 0, "jacobi_left: work buffer not 16-byte aligned");
    split_df_kernel<<<(unsigned)cdiv(ls * l, 256), 256, 0, st>>>(l, B, ldb, D, ls);
    APL_LAUNCH_CHECK();
    sweeps += run_sweeps(st, NB, 60, flag_dev, [&](int64_t r) {
      jacobi_df_block_kernel<<<(unsigned)(NB / 2), 64 * JW, smem_df, st>>>(l, ls, NB, r, D,
                                                                          (float)tol, flag_dev);
      APL_LAUNCH_CHECK();
    }, PROF_JACOBI, 2.0 * (double)l * pairs, 6.0 * (double)l, 1e-2 * std::sqrt(tol));
    join_df_kernel<<<(unsigned)cdiv(l * l, 256), 256, 0, st>>>(l, D, ls, B, ldb);
    APL_LAUNCH_CHECK();
  } else if (l > 1) {
    // Stage 2 (FP64): sweeps from the nearly orthogonal start down to l * eps
    const double tol = std::max(1e-15, (double)l * 1.1102230246251565e-16);
    const double pairs = (double)(l * (l - 1)) / 2.0;
    sweeps += run_sweeps(st, N, 60, flag_dev, [&](int64_t r) {
      jacobi_round_kernel<<<(unsigned)(N / 2), 256, 0, st>>>(l, N, r, B, ldb, tol, flag_dev);
      APL_LAUNCH_CHECK();
    }, PROF_JACOBI, 6.0 * (double)l * pairs, 6.0 * (double)l);
  }
  col_norms_kernel<<<(unsigned)l, 256, 0, st>>>(l, l, B, ldb, sigma);
  APL_LAUNCH_CHECK();
  std::vector<double> sg(l);
  APL_CUDA(cudaMemcpyAsync(sg.data(), sigma, l * sizeof(double), cudaMemcpyDeviceToHost, st));
  APL_CUDA(cudaStreamSynchronize(st));
  std::vector<int> perm(l);
  std::iota(perm.begin(), perm.end(), 0);
  std::stable_sort(perm.begin(), perm.end(), [&](int a, int b) { return sg[a] > sg[b]; });
  std::vector<double> ss(l);
  for (int64_t i = 0; i < l; ++i) ss[i] = sg[perm[i]];
  DBuf<int> perm_dev;
  perm_dev.alloc(l, st);
  APL_CUDA(cudaMemcpyAsync(perm_dev.p, perm.data(), l * sizeof(int), cudaMemcpyHostToDevice, st));
  APL_CUDA(cudaMemcpyAsync(sigma, ss.data(), l * sizeof(double), cudaMemcpyHostToDevice, st));
  gather_normalise_kernel<<<(unsigned)cdiv(l * l, 256), 256, 0, st>>>(l, B, ldb, perm_dev.p, sigma,
                                                                     l, U, ldu);
  APL_LAUNCH_CHECK();
  APL_CUDA(cudaStreamSynchronize(st));
  return sweeps;
}

// ------------------------------------------------------------------------------------
// Elementwise helpers
// ------------------------------------------------------------------------------------
namespace {
__global__ void copy2d_kernel(int64_t rows, int64_t cols, const double* src, int64_t lds,
                              double* dst, int64_t ldd, int transpose) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= rows * cols) return;
  const int64_t r = e % rows, c = e / rows;
  if (transpose) dst[c + r * ldd] = src[r + c * lds];
  else dst[r + c * ldd] = src[r + c * lds];
}
__global__ void set2d_kernel(int64_t rows, int64_t cols, double v, double* dst, int64_t ldd) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= rows * cols) return;
  dst[e % rows + (e / rows) * ldd] = v;
}
__global__ void set_diag_kernel(int64_t n, double v, double* A, int64_t lda) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) A[i + i * lda] = v;
}
__global__ void zero_lower_kernel(int64_t n, double* A, int64_t lda) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * n) return;
  const int64_t r = e % n, c = e / n;
  if (r > c) A[r + c * lda] = 0.0;
}
__global__ void gather_cols_kernel(int64_t rows, const double* src, int64_t lds, const int* idx,
                                   int64_t k, double* dst, int64_t ldd) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= rows * k) return;
  const int64_t r = e % rows, q = e / rows;
  dst[r + q * ldd] = src[r + (int64_t)idx[q] * lds];
}
}  // namespace

void dcopy2d(cudaStream_t st, int64_t rows, int64_t cols, const double* src, int64_t lds,
             double* dst, int64_t ldd, bool transpose) {
  if (rows <= 0 || cols <= 0) return;
  copy2d_kernel<<<(unsigned)cdiv(rows * cols, 256), 256, 0, st>>>(rows, cols, src, lds, dst, ldd,
                                                                  transpose ? 1 : 0);
  APL_LAUNCH_CHECK();
}
void dset2d(cudaStream_t st, int64_t rows, int64_t cols, double v, double* dst, int64_t ldd) {
  if (rows <= 0 || cols <= 0) return;
  set2d_kernel<<<(unsigned)cdiv(rows * cols, 256), 256, 0, st>>>(rows, cols, v, dst, ldd);
  APL_LAUNCH_CHECK();
}
__global__ void add_diag_kernel(int64_t n, double v, double* A, int64_t lda) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) A[i + i * lda] += v;
}
void dadd_diag(cudaStream_t st, int64_t n, double v, double* A, int64_t lda) {
  if (n <= 0) return;
  add_diag_kernel<<<(unsigned)cdiv(n, 256), 256, 0, st>>>(n, v, A, lda);
  APL_LAUNCH_CHECK();
}
void dset_diag(cudaStream_t st, int64_t n, double v, double* A, int64_t lda) {
  if (n <= 0) return;
  set_diag_kernel<<<(unsigned)cdiv(n, 256), 256, 0, st>>>(n, v, A, lda);
  APL_LAUNCH_CHECK();
}
void dzero_lower(cudaStream_t st, int64_t n, double* A, int64_t lda) {
  if (n <= 1) return;
  zero_lower_kernel<<<(unsigned)cdiv(n * n, 256), 256, 0, st>>>(n, A, lda);
  APL_LAUNCH_CHECK();
}
void dgather_cols(cudaStream_t st, int64_t rows, const double* src, int64_t lds, const int* idx,
                  int64_t k, double* dst, int64_t ldd) {
  if (rows <= 0 || k <= 0) return;
  gather_cols_kernel<<<(unsigned)cdiv(rows * k, 256), 256, 0, st>>>(rows, src, lds, idx, k, dst,
                                                                    ldd);
  APL_LAUNCH_CHECK();
}

}  // namespace apl
