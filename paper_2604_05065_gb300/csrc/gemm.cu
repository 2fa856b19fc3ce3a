// Dense matrix products for the rank steps and preconditioner builds (dgemm): an FP64
// form and the default compensated-FP32 form, with split-K for tall inner dimensions.
#include <algorithm>

#include "dense.cuh"
#include "df32.cuh"

namespace apl {

// ------------------------------------------------------------------------------------
// GEMM: 64 x 64 output tile per 256-thread block, 4 x 4 outputs per thread, K step 16.
// Two arithmetic forms: FP64 (dgemm_kernel) and compensated FP32 (df32gemm_kernel, the
// default; the context's DenseWork selects).
// ------------------------------------------------------------------------------------
namespace {
constexpr int GBM = 64, GBN = 64, GBK = 16;

// blockIdx.z selects a K range of length kchunk; with part != NULL the block writes its
// unscaled partial product to part + z * M * N (leading dimension M) instead of C.
__global__ void __launch_bounds__(256) dgemm_kernel(int transA, int transB, int64_t M,
                                                    int64_t N, int64_t K, double alpha,
                                                    const double* __restrict__ A, int64_t lda,
                                                    const double* __restrict__ B, int64_t ldb,
                                                    double beta, double* __restrict__ C,
                                                    int64_t ldc, int64_t kchunk,
                                                    double* __restrict__ part) {
  __shared__ double As[GBK][GBM + 1];
  __shared__ double Bs[GBK][GBN + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t m0 = (int64_t)blockIdx.x * GBM, n0 = (int64_t)blockIdx.y * GBN;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

  const int64_t kbeg = (int64_t)blockIdx.z * kchunk;
  const int64_t kend = kbeg + kchunk < K ? kbeg + kchunk : K;
  for (int64_t k0 = kbeg; k0 < kend; k0 += GBK) {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int lin = threadIdx.x + e * 256;  // 0..1023
      int mm, kk;
      if (!transA) { mm = lin & 63; kk = lin >> 6; } else { kk = lin & 15; mm = lin >> 4; }
      const int64_t gm = m0 + mm, gk = k0 + kk;
      double v = 0.0;
      if (gm < M && gk < kend) v = transA ? A[gk + gm * lda] : A[gm + gk * lda];
      As[kk][mm] = v;
      int nn;
      if (!transB) { kk = lin & 15; nn = lin >> 4; } else { nn = lin & 63; kk = lin >> 6; }
      const int64_t gn = n0 + nn, gk2 = k0 + kk;
      double w = 0.0;
      if (gn < N && gk2 < kend) w = transB ? B[gn + gk2 * ldb] : B[gk2 + gn * ldb];
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
      if (part) {
        part[(int64_t)blockIdx.z * M * N + gm + gn * M] = acc[i][j];
      } else {
        double* c = C + gm + gn * ldc;
        *c = (beta == 0.0) ? alpha * acc[i][j] : alpha * acc[i][j] + beta * *c;
      }
    }
  }
}

// The same tiling with compensated FP32 arithmetic.  Every FP64 operand is split once per
// call into FP32 hi + lo arrays (split2_kernel, both operands in one launch; hi + lo keeps
// 48 of its 53 bits), a product is formed exactly in its hi * hi part (an FMA gives the
// rounding error) plus the two cross terms, and the running sum is an unevaluated FP32 pair
// updated by Knuth's TwoSum.  The result is accurate to about 2^-46 relative to
// sum |a_i b_i| and the inner loop has only FP32 instructions, which GB300 issues at over
// 64 times its FP64 rate.  The operands arrive compact: op(A) source rows x cols with
// leading dimension = rows (same for B).
__global__ void split_kernel(int64_t rows, int64_t cols, const double* __restrict__ src,
                             int64_t ld, float* __restrict__ hi, float* __restrict__ lo) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= rows * cols) return;
  const int64_t r = e % rows, c = e / rows;
  const double v = src[r + c * ld];
  const float h = __double2float_rn(v);
  hi[e] = h;
  lo[e] = __double2float_rn(v - (double)h);
}

// Both operands of one product in one launch: elements below ar * ac are op(A)'s source
// block, the rest B's (the same split as split_kernel).
__global__ void split2_kernel(int64_t ar, int64_t ac, const double* __restrict__ A,
                              int64_t lda, float* __restrict__ ah, float* __restrict__ al,
                              int64_t br, int64_t bc, const double* __restrict__ B,
                              int64_t ldb, float* __restrict__ bh, float* __restrict__ bl) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t na = ar * ac;
  double v;
  float *hi, *lo;
  if (e < na) {
    v = A[e % ar + (e / ar) * lda];
    hi = ah;
    lo = al;
  } else {
    e -= na;
    if (e >= br * bc) return;
    v = B[e % br + (e / br) * ldb];
    hi = bh;
    lo = bl;
  }
  const float h = __double2float_rn(v);
  hi[e] = h;
  lo[e] = __double2float_rn(v - (double)h);
}

// R consecutive floats of a hi row and of a lo row of a shared tile (one 16-byte load each
// for R = 4, one 8-byte load for R = 2).
template <int R>
__device__ __forceinline__ void load_row(const float* h, const float* l, float* oh, float* ol) {
  if constexpr (R == 4) {
    const float4 a = *reinterpret_cast<const float4*>(h);
    const float4 b = *reinterpret_cast<const float4*>(l);
    oh[0] = a.x; oh[1] = a.y; oh[2] = a.z; oh[3] = a.w;
    ol[0] = b.x; ol[1] = b.y; ol[2] = b.z; ol[3] = b.w;
  } else {
    static_assert(R == 2, "R is 2 or 4");
    const float2 a = *reinterpret_cast<const float2*>(h);
    const float2 b = *reinterpret_cast<const float2*>(l);
    oh[0] = a.x; oh[1] = a.y;
    ol[0] = b.x; ol[1] = b.y;
  }
}

// R x R outputs per thread on a 16 x 16 thread grid: a (16 R) x (16 R) output tile, thread
// (tx, ty) owning rows ty R ... ty R + R - 1 and columns tx R ... tx R + R - 1.  R = 4
// (64 x 64 tiles) is the default; R = 2 (32 x 32) serves launches whose 64 x 64 tiles would
// not fill one wave of the GPU (the small updates of the blocked triangular solve and
// Cholesky), with four times as many blocks.  Each output's sum runs over k in the same
// order in both, so the two give bitwise the same result.
template <int R>
__global__ void __launch_bounds__(256) df32gemm_kernel(int transA, int transB, int64_t M,
                                                       int64_t N, int64_t K, double alpha,
                                                       const float* __restrict__ Ahi,
                                                       const float* __restrict__ Alo,
                                                       int64_t lda,
                                                       const float* __restrict__ Bhi,
                                                       const float* __restrict__ Blo,
                                                       int64_t ldb, double beta,
                                                       double* __restrict__ C, int64_t ldc,
                                                       int64_t kchunk,
                                                       double* __restrict__ part) {
  constexpr int TM = 16 * R;                     // tile rows = tile columns
  constexpr int LG = R == 4 ? 6 : (R == 2 ? 5 : 4);  // log2(TM)
  static_assert(TM == (1 << LG), "tile size");
  // rows padded by 4 floats: each thread reads its R consecutive entries of a row with one
  // 16-byte (R = 4) or 8-byte (R = 2) load
  constexpr int TP = TM + 4;
  __shared__ __align__(16) float Ah[GBK][TP];
  __shared__ __align__(16) float Al[GBK][TP];
  __shared__ __align__(16) float Bh[GBK][TP];
  __shared__ __align__(16) float Bl[GBK][TP];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t m0 = (int64_t)blockIdx.x * TM, n0 = (int64_t)blockIdx.y * TM;
  float s[R][R], c[R][R];
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int j = 0; j < R; ++j) { s[i][j] = 0.f; c[i][j] = 0.f; }

  const int64_t kbeg = (int64_t)blockIdx.z * kchunk;
  const int64_t kend = kbeg + kchunk < K ? kbeg + kchunk : K;
  // the next K chunk is fetched into registers while the current one is multiplied
  float pah[R], pal[R], pbh[R], pbl[R];
  auto fetch = [&](int64_t k0) {
#pragma unroll
    for (int e = 0; e < R; ++e) {
      const int lin = threadIdx.x + e * 256;
      int mm, kk;
      if (!transA) { mm = lin & (TM - 1); kk = lin >> LG; } else { kk = lin & 15; mm = lin >> 4; }
      const int64_t gm = m0 + mm, gk = k0 + kk;
      pah[e] = 0.f;
      pal[e] = 0.f;
      if (gm < M && gk < kend) {
        const int64_t o = transA ? gk + gm * lda : gm + gk * lda;
        pah[e] = Ahi[o];
        pal[e] = Alo[o];
      }
      int nn;
      if (!transB) { kk = lin & 15; nn = lin >> 4; } else { nn = lin & (TM - 1); kk = lin >> LG; }
      const int64_t gn = n0 + nn, gk2 = k0 + kk;
      pbh[e] = 0.f;
      pbl[e] = 0.f;
      if (gn < N && gk2 < kend) {
        const int64_t o = transB ? gn + gk2 * ldb : gk2 + gn * ldb;
        pbh[e] = Bhi[o];
        pbl[e] = Blo[o];
      }
    }
  };
  if (kbeg < kend) fetch(kbeg);
  for (int64_t k0 = kbeg; k0 < kend; k0 += GBK) {
#pragma unroll
    for (int e = 0; e < R; ++e) {
      const int lin = threadIdx.x + e * 256;
      int mm, kk;
      if (!transA) { mm = lin & (TM - 1); kk = lin >> LG; } else { kk = lin & 15; mm = lin >> 4; }
      Ah[kk][mm] = pah[e];
      Al[kk][mm] = pal[e];
      int nn;
      if (!transB) { kk = lin & 15; nn = lin >> 4; } else { nn = lin & (TM - 1); kk = lin >> LG; }
      Bh[kk][nn] = pbh[e];
      Bl[kk][nn] = pbl[e];
    }
    __syncthreads();
    if (k0 + GBK < kend) fetch(k0 + GBK);
#pragma unroll 4
    for (int kk = 0; kk < GBK; ++kk) {
      float ah[R], al[R], bh[R], bl[R];
      load_row<R>(&Ah[kk][ty * R], &Al[kk][ty * R], ah, al);
      load_row<R>(&Bh[kk][tx * R], &Bl[kk][tx * R], bh, bl);
#pragma unroll
      for (int i = 0; i < R; ++i)
#pragma unroll
        for (int j = 0; j < R; ++j) {
          const float p = __fmul_rn(ah[i], bh[j]);
          float x = __fmaf_rn(ah[i], bh[j], -p);
          x = __fmaf_rn(ah[i], bl[j], x);
          x = __fmaf_rn(al[i], bh[j], x);
          const float t = __fadd_rn(s[i][j], p);
          const float bv = __fsub_rn(t, s[i][j]);
          const float err = __fadd_rn(__fsub_rn(s[i][j], __fsub_rn(t, bv)), __fsub_rn(p, bv));
          s[i][j] = t;
          c[i][j] = __fadd_rn(c[i][j], __fadd_rn(err, x));
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int64_t gm = m0 + ty * R + i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int64_t gn = n0 + tx * R + j;
      if (gn >= N) continue;
      const double acc = (double)s[i][j] + (double)c[i][j];
      if (part) {
        part[(int64_t)blockIdx.z * M * N + gm + gn * M] = acc;
      } else {
        double* cp = C + gm + gn * ldc;
        *cp = (beta == 0.0) ? alpha * acc : alpha * acc + beta * *cp;
      }
    }
  }
}

// SMs of the device current at the first call (a launch-shape heuristic only).
int sm_count() {
  static const int n = [] {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 152;
  }();
  return n;
}

// C = alpha * sum_z part[z] + beta * C, summing the splits in a fixed order.
__global__ void splitk_reduce_kernel(int64_t M, int64_t N, int splits, const double* part,
                                     double alpha, double beta, double* C, int64_t ldc) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= M * N) return;
  double acc = 0.0;
  for (int z = 0; z < splits; ++z) acc += part[(int64_t)z * M * N + e];
  const int64_t r = e % M, c = e / M;
  double* out = C + r + c * ldc;
  *out = (beta == 0.0) ? alpha * acc : alpha * acc + beta * *out;
}

}  // namespace

void split_hilo(cudaStream_t st, int64_t rows, int64_t cols, const double* A, int64_t ld,
                float* hi, float* lo) {
  if (rows <= 0 || cols <= 0) return;
  split_kernel<<<(unsigned)cdiv(rows * cols, 256), 256, 0, st>>>(rows, cols, A, ld, hi, lo);
  APL_LAUNCH_CHECK();
}

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
  // split K when the output tiles alone cannot fill the GPU (tall inner dimension)
  const int64_t tiles = (int64_t)grid.x * grid.y;
  int64_t splits = 1;
  const bool fp64 = dense_work().fp64_gemm;
  if (tiles < 2 * 152 && K >= 256) {
    splits = std::min<int64_t>(cdiv(4 * 152, tiles), K / 128);
    splits = std::min<int64_t>(splits, 64);
    splits = std::max<int64_t>(1, std::min<int64_t>(splits, (int64_t)(1 << 24) / (M * N)));
  } else if (!fp64 && K >= 512) {
    // a few waves of tiles: split K when that fills the last wave much better (the grid
    // runs in waves of `resident` blocks; split-K costs a partial write and a reduction)
    static const int64_t resident = [] {
      int per = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, df32gemm_kernel<4>, 256, 0);
      return (int64_t)std::max(1, sm_count() * std::max(per, 1));
    }();
    auto fill = [&](int64_t sp) {
      const int64_t b = tiles * sp;
      return (double)b / (double)(cdiv(b, resident) * resident);
    };
    const double f1 = fill(1);
    if (f1 < 0.8) {
      int64_t best = 1;
      double bf = f1;
      for (int64_t sp = 2; sp <= 4 && K / sp >= 256; ++sp) {
        const double f = fill(sp);
        if (f > bf + 0.05) { best = sp; bf = f; }
      }
      if ((int64_t)(1 << 24) / (M * N) >= best) splits = best;
    }
  }
  const int tok = prof_begin(st);
  // compensated FP32: operands split once into compact hi / lo arrays
  const float *Ah = nullptr, *Al = nullptr, *Bh = nullptr, *Bl = nullptr;
  int64_t lda2 = lda, ldb2 = ldb;
  if (!fp64) {
    DenseWork& wk = dense_work();
    const int64_t ar = transA ? K : M, ac = transA ? M : K;
    const int64_t br = transB ? N : K, bc = transB ? K : N;
    wk.gah.alloc((size_t)ar * ac, st);
    wk.gal.alloc((size_t)ar * ac, st);
    wk.gbh.alloc((size_t)br * bc, st);
    wk.gbl.alloc((size_t)br * bc, st);
    split2_kernel<<<(unsigned)cdiv(ar * ac + br * bc, 256), 256, 0, st>>>(
        ar, ac, A, lda, wk.gah.p, wk.gal.p, br, bc, B, ldb, wk.gbh.p, wk.gbl.p);
    APL_LAUNCH_CHECK();
    Ah = wk.gah.p; Al = wk.gal.p; Bh = wk.gbh.p; Bl = wk.gbl.p;
    lda2 = ar;
    ldb2 = br;
  }
  if (splits > 1) {
    const int64_t kchunk = cdiv(cdiv(K, splits), GBK) * GBK;
    splits = cdiv(K, kchunk);
    dense_work().splitk.alloc((size_t)splits * M * N, st);
    grid.z = (unsigned)splits;
    if (fp64)
      dgemm_kernel<<<grid, 256, 0, st>>>(transA, transB, M, N, K, 1.0, A, lda, B, ldb, 0.0, C,
                                         ldc, kchunk, dense_work().splitk.p);
    else
      df32gemm_kernel<4><<<grid, 256, 0, st>>>(transA, transB, M, N, K, 1.0, Ah, Al, lda2, Bh,
                                               Bl, ldb2, 0.0, C, ldc, kchunk,
                                               dense_work().splitk.p);
    APL_LAUNCH_CHECK();
    splitk_reduce_kernel<<<(unsigned)cdiv(M * N, 256), 256, 0, st>>>(M, N, (int)splits,
                                                                     dense_work().splitk.p, alpha, beta, C,
                                                                     ldc);
  } else if (fp64) {
    dgemm_kernel<<<grid, 256, 0, st>>>(transA, transB, M, N, K, alpha, A, lda, B, ldb, beta, C,
                                       ldc, K, nullptr);
  } else if (tiles < sm_count()) {
    // less than one wave of 64 x 64 tiles: 32 x 32 tiles, four times the blocks
    const dim3 g2((unsigned)cdiv(M, 32), (unsigned)cdiv(N, 32));
    df32gemm_kernel<2><<<g2, 256, 0, st>>>(transA, transB, M, N, K, alpha, Ah, Al, lda2, Bh, Bl,
                                           ldb2, beta, C, ldc, K, nullptr);
  } else {
    df32gemm_kernel<4><<<grid, 256, 0, st>>>(transA, transB, M, N, K, alpha, Ah, Al, lda2, Bh,
                                             Bl, ldb2, beta, C, ldc, K, nullptr);
  }
  APL_LAUNCH_CHECK();
  prof_end(st, tok, PROF_GEMM, 2.0 * (double)M * (double)N * (double)K);
}

}  // namespace apl
