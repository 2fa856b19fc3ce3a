// Dense FP64 kernels for the ell x ell and n x b work of the CUR and preconditioner
// steps: tiled GEMM, blocked triangular solves, single-CTA Cholesky, Cholesky QR2 and a
// parallel one-sided (Hestenes) Jacobi SVD.
#include <algorithm>
#include <atomic>
#include <numeric>

#include "dense.cuh"

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

// ------------------------------------------------------------------------------------
// GEMM: 64 x 64 output tile per 256-thread block, 4 x 4 outputs per thread, K step 16.
// ------------------------------------------------------------------------------------
namespace {
constexpr int GBM = 64, GBN = 64, GBK = 16;

__global__ void __launch_bounds__(256) dgemm_kernel(int transA, int transB, int64_t M,
                                                    int64_t N, int64_t K, double alpha,
                                                    const double* __restrict__ A, int64_t lda,
                                                    const double* __restrict__ B, int64_t ldb,
                                                    double beta, double* __restrict__ C,
                                                    int64_t ldc) {
  __shared__ double As[GBK][GBM + 1];
  __shared__ double Bs[GBK][GBN + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t m0 = (int64_t)blockIdx.x * GBM, n0 = (int64_t)blockIdx.y * GBN;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

  for (int64_t k0 = 0; k0 < K; k0 += GBK) {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int lin = threadIdx.x + e * 256;  // 0..1023
      int mm, kk;
      if (!transA) { mm = lin & 63; kk = lin >> 6; } else { kk = lin & 15; mm = lin >> 4; }
      const int64_t gm = m0 + mm, gk = k0 + kk;
      double v = 0.0;
      if (gm < M && gk < K) v = transA ? A[gk + gm * lda] : A[gm + gk * lda];
      As[kk][mm] = v;
      int nn;
      if (!transB) { kk = lin & 15; nn = lin >> 4; } else { nn = lin & 63; kk = lin >> 6; }
      const int64_t gn = n0 + nn, gk2 = k0 + kk;
      double w = 0.0;
      if (gn < N && gk2 < K) w = transB ? B[gn + gk2 * ldb] : B[gk2 + gn * ldb];
      Bs[kk][nn] = w;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GBK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t gm = m0 + ty + 16 * i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t gn = n0 + tx + 16 * j;
      if (gn >= N) continue;
      double* c = C + gm + gn * ldc;
      *c = (beta == 0.0) ? alpha * acc[i][j] : alpha * acc[i][j] + beta * *c;
    }
  }
}
}  // namespace

void dgemm(cudaStream_t st, int transA, int transB, int64_t M, int64_t N, int64_t K,
           double alpha, const double* A, int64_t lda, const double* B, int64_t ldb,
           double beta, double* C, int64_t ldc) {
  if (M <= 0 || N <= 0) return;
  if (K <= 0) {
    if (beta == 0.0) dset2d(st, M, N, 0.0, C, ldc);
    else if (beta != 1.0) {
      // scale C by beta through a zero-K gemm is not needed by callers
      throw Error(ST_EINVAL, "dgemm: K == 0 with beta not in {0, 1}");
    }
    return;
  }
  dim3 grid((unsigned)cdiv(M, GBM), (unsigned)cdiv(N, GBN));
  APL_REQUIRE(grid.y <= 65535, "dgemm: N too large");
  dgemm_kernel<<<grid, 256, 0, st>>>(transA, transB, M, N, K, alpha, A, lda, B, ldb, beta, C,
                                     ldc);
  APL_LAUNCH_CHECK();
}

// ------------------------------------------------------------------------------------
// Triangular solve.  Diagonal blocks (<= 64) are solved by one thread per right-hand
// vector; the rest is GEMM updates.
// ------------------------------------------------------------------------------------
namespace {
constexpr int TNB = 64;

// Solve T x = b for `nvec` vectors of length `len`.  T(r, c) = Tm[r * trs + c * tcs];
// lower: forward substitution, else backward.  Vector v element i at
// X[v * vstride + i * estride].
__global__ void trsv_block_kernel(int64_t nvec, int len, double* __restrict__ X,
                                  int64_t vstride, int64_t estride,
                                  const double* __restrict__ Tm, int64_t trs, int64_t tcs,
                                  int lower, int unit) {
  __shared__ double Ts[TNB][TNB + 1];
  for (int e = threadIdx.x; e < len * len; e += blockDim.x) {
    const int r = e % len, c = e / len;
    Ts[r][c] = Tm[r * trs + c * tcs];
  }
  __syncthreads();
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nvec) return;
  double* x = X + v * vstride;
  double loc[TNB];
  for (int i = 0; i < len; ++i) loc[i] = x[i * estride];
  if (lower) {
    for (int i = 0; i < len; ++i) {
      double s = loc[i];
      for (int c = 0; c < i; ++c) s -= Ts[i][c] * loc[c];
      loc[i] = unit ? s : s / Ts[i][i];
    }
  } else {
    for (int i = len - 1; i >= 0; --i) {
      double s = loc[i];
      for (int c = i + 1; c < len; ++c) s -= Ts[i][c] * loc[c];
      loc[i] = unit ? s : s / Ts[i][i];
    }
  }
  for (int i = 0; i < len; ++i) x[i * estride] = loc[i];
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
  auto diag = [&](int64_t k0, int64_t kb) {
    // element (r, c) of op(A)_kk
    const double* base = A + k0 + k0 * lda;
    int64_t rs = trans ? lda : 1, cs = trans ? 1 : lda;
    if (left) {
      const int64_t nvec = N;
      trsv_block_kernel<<<(unsigned)cdiv(nvec, 64), 64, 0, st>>>(
          nvec, (int)kb, B + k0, ldb, 1, base, rs, cs, effLower ? 1 : 0, unit ? 1 : 0);
    } else {
      // X T = B  <=>  T^T x^T = b^T : matrix element (r, c) of T^T = T(c, r)
      const int64_t nvec = M;
      trsv_block_kernel<<<(unsigned)cdiv(nvec, 64), 64, 0, st>>>(
          nvec, (int)kb, B + k0 * ldb, 1, ldb, base, cs, rs, effLower ? 0 : 1, unit ? 1 : 0);
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
// Cholesky (upper), one CTA, right-looking, in global memory.
// ------------------------------------------------------------------------------------
namespace {
__global__ void __launch_bounds__(1024) potrf_upper_kernel(int64_t n, double* A, int64_t lda,
                                                           int* info) {
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int64_t k = 0; k < n; ++k) {
    if (threadIdx.x == 0) {
      const double d = A[k + k * lda];
      if (!(d > 0.0) || !isfinite(d)) {
        bad = (int)k + 1;
      } else {
        A[k + k * lda] = sqrt(d);
      }
    }
    __syncthreads();
    if (bad) break;
    const double dk = A[k + k * lda];
    for (int64_t j = k + 1 + threadIdx.x; j < n; j += blockDim.x) A[k + j * lda] /= dk;
    __syncthreads();
    // trailing update of the upper triangle: A[i, j] -= A[k, i] A[k, j], k < i <= j
    const int64_t t = n - k - 1;
    const int64_t total = t * (t + 1) / 2;
    for (int64_t e = threadIdx.x; e < total; e += blockDim.x) {
      // map e -> (i, j) with i <= j over the t x t trailing block, column-major packed
      int64_t j = (int64_t)((sqrt(8.0 * (double)e + 1.0) - 1.0) * 0.5);
      while ((j + 1) * (j + 2) / 2 <= e) ++j;
      while (j * (j + 1) / 2 > e) --j;
      const int64_t i = e - j * (j + 1) / 2;
      const int64_t gi = k + 1 + i, gj = k + 1 + j;
      A[gi + gj * lda] -= A[k + gi * lda] * A[k + gj * lda];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *info = bad;
  // zero the strictly lower part
  for (int64_t e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int64_t r = e % n, c = e / n;
    if (r > c) A[r + c * lda] = 0.0;
  }
}
}  // namespace

void dpotrf_upper(cudaStream_t st, int64_t n, double* A, int64_t lda, int* info_dev) {
  if (n <= 0) return;
  potrf_upper_kernel<<<1, 1024, 0, st>>>(n, A, lda, info_dev);
  APL_LAUNCH_CHECK();
}

bool cholqr2(cudaStream_t st, int64_t n, int64_t k, double* E, int64_t lde, double* R,
             int64_t ldr, double* work, int* info_dev) {
  // work: 2 k x k blocks
  double* G = work;
  double* R1 = work + k * k;
  int info = 0;
  dgemm(st, 1, 0, k, k, n, 1.0, E, lde, E, lde, 0.0, G, k);
  dpotrf_upper(st, k, G, k, info_dev);
  APL_CUDA(cudaMemcpyAsync(&info, info_dev, sizeof(int), cudaMemcpyDeviceToHost, st));
  APL_CUDA(cudaStreamSynchronize(st));
  if (info) return false;
  dcopy2d(st, k, k, G, k, R1, k, false);
  dtrsm(st, false, 'U', false, false, n, k, R1, k, E, lde);
  dgemm(st, 1, 0, k, k, n, 1.0, E, lde, E, lde, 0.0, G, k);
  dpotrf_upper(st, k, G, k, info_dev);
  APL_CUDA(cudaMemcpyAsync(&info, info_dev, sizeof(int), cudaMemcpyDeviceToHost, st));
  APL_CUDA(cudaStreamSynchronize(st));
  if (info) return false;
  dtrsm(st, false, 'U', false, false, n, k, G, k, E, lde);
  // R = R2 R1 (both upper; lower parts are zero)
  dgemm(st, 0, 0, k, k, k, 1.0, G, k, R1, k, 0.0, R, ldr);
  dzero_lower(st, k, R, ldr);
  return true;
}

// ------------------------------------------------------------------------------------
// One-sided Jacobi SVD.  Round-robin ordering: in round r the N (even) columns form
// N/2 disjoint pairs; one block rotates one pair of M and of V.
// ------------------------------------------------------------------------------------
namespace {
__device__ __forceinline__ int64_t rr_elem(int64_t pos, int64_t r, int64_t N) {
  return pos == 0 ? 0 : 1 + ((pos - 1 + r) % (N - 1));
}

__global__ void __launch_bounds__(256) jacobi_round_kernel(int64_t l, int64_t N, int64_t r,
                                                           double* __restrict__ M, int64_t ldm,
                                                           double* __restrict__ V, int64_t ldv,
                                                           double tol, int* rotated) {
  __shared__ double sh[3][8];
  __shared__ double cs[2];
  __shared__ int doit;
  const int64_t k = blockIdx.x;
  int64_t p = rr_elem(k, r, N), q = rr_elem(N - 1 - k, r, N);
  if (p >= l || q >= l) return;
  if (p > q) { const int64_t t = p; p = q; q = t; }
  double* mp = M + p * ldm;
  double* mq = M + q * ldm;
  double a = 0.0, b = 0.0, g = 0.0;
  for (int64_t i = threadIdx.x; i < l; i += blockDim.x) {
    const double x = mp[i], y = mq[i];
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
    const double x = mp[i], y = mq[i];
    mp[i] = c * x - s * y;
    mq[i] = s * x + c * y;
  }
  double* vp = V + p * ldv;
  double* vq = V + q * ldv;
  for (int64_t i = threadIdx.x; i < l; i += blockDim.x) {
    const double x = vp[i], y = vq[i];
    vp[i] = c * x - s * y;
    vq[i] = s * x + c * y;
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

__global__ void eye_kernel(int64_t n, double* V, int64_t ldv) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * n) return;
  const int64_t r = e % n, c = e / n;
  V[r + c * ldv] = (r == c) ? 1.0 : 0.0;
}
}  // namespace

int jacobi_svd(cudaStream_t st, int64_t l, double* M, int64_t ldm, double* V, int64_t ldv,
               double* sigma, double* work, int* flag_dev) {
  if (l <= 0) return 0;
  eye_kernel<<<(unsigned)cdiv(l * l, 256), 256, 0, st>>>(l, V, ldv);
  APL_LAUNCH_CHECK();
  const int64_t N = (l % 2) ? l + 1 : l;
  const double tol = 1e-15;
  int sweeps = 0;
  if (l > 1) {
    for (; sweeps < 60;) {
      APL_CUDA(cudaMemsetAsync(flag_dev, 0, sizeof(int), st));
      for (int64_t r = 0; r < N - 1; ++r) {
        jacobi_round_kernel<<<(unsigned)(N / 2), 256, 0, st>>>(l, N, r, M, ldm, V, ldv, tol,
                                                                 flag_dev);
      }
      APL_LAUNCH_CHECK();
      ++sweeps;
      int rot = 0;
      APL_CUDA(cudaMemcpyAsync(&rot, flag_dev, sizeof(int), cudaMemcpyDeviceToHost, st));
      APL_CUDA(cudaStreamSynchronize(st));
      if (rot == 0) break;
    }
  }
  col_norms_kernel<<<(unsigned)l, 256, 0, st>>>(l, l, M, ldm, sigma);
  APL_LAUNCH_CHECK();
  // sort descending (stable) and permute the columns of V
  std::vector<double> sg(l);
  APL_CUDA(cudaMemcpyAsync(sg.data(), sigma, l * sizeof(double), cudaMemcpyDeviceToHost, st));
  APL_CUDA(cudaStreamSynchronize(st));
  std::vector<int> perm(l);
  std::iota(perm.begin(), perm.end(), 0);
  std::stable_sort(perm.begin(), perm.end(), [&](int a, int b) { return sg[a] > sg[b]; });
  bool ident = true;
  for (int64_t i = 0; i < l; ++i) ident = ident && perm[i] == i;
  if (!ident) {
    std::vector<double> ss(l);
    for (int64_t i = 0; i < l; ++i) ss[i] = sg[perm[i]];
    int* perm_dev = reinterpret_cast<int*>(work + l * l);
    APL_CUDA(cudaMemcpyAsync(perm_dev, perm.data(), l * sizeof(int), cudaMemcpyHostToDevice, st));
    dgather_cols(st, l, V, ldv, perm_dev, l, work, l);
    dcopy2d(st, l, l, work, l, V, ldv, false);
    APL_CUDA(cudaMemcpyAsync(sigma, ss.data(), l * sizeof(double), cudaMemcpyHostToDevice, st));
    APL_CUDA(cudaStreamSynchronize(st));
  }
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
