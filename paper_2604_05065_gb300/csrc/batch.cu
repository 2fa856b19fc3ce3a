// Grouped multi-right-hand-side LSQR phases for a batch of problems (see batch.cuh).
//
// One iteration for all (problem, right-hand side) pairs of a phase is
//   gn   A pass        U <- ca A Z - cb U (rows of A), U_bot <- ca delta Z - cb U_bot
//   beta               beta = ||U||, su = 1/beta                      (per pair)
//   gt   A^T pass      G = su (A^T U_top + delta U_bot)
//   gt   Q^T G         q                                              (preconditioned)
//   gt   VM^T q        t = c (VM^T q)
//   gn   VM t          s
//   gn   expansion     V <- G + Q s - cprev V          (V = alpha v = P^-1 g - beta v)
//   gt, gt, gn         the same three steps on V
//   gn   expansion     Z <- V + Q s                    (Z = P^-1 V)
//   alpha              alpha = ||V||, Givens rotation, stopping tests (per pair)
//   vec                x += xc D,  D <- sv Z - dc D
// which is Golub-Kahan bidiagonalisation of [A; delta I] P^-1 with
// P^-1 w = w + Q_R V_M (c (V_M^T Q_R^T w)) applied through the implicit Vhat = Q_R V_M
// (Eq. preconditioner2).  z = P^-1 v is formed from v every iteration: the FP32 vectors
// would drift apart under a separate recursion for z.  Every kernel walks a work list of
// (problem, tile) items, so one
// launch serves the whole batch; an item whose problem has no live pair returns at
// once.  The loop is captured in a CUDA graph.
#include <algorithm>
#include <cmath>
#include <numeric>

#include "batch.cuh"
#include "df32.cuh"

namespace apl {

namespace {

constexpr int BT = 256;      // threads per block of every grouped kernel
constexpr int GT_CHUNK = 128;  // rows of X staged per chunk in the transposed products
constexpr int ROWS_ITEM = 256; // rows of A per A-pass item
constexpr int VEC_ITEM = 1024; // rows per elementwise item
constexpr int kGnSmemCap = 200 * 1024;  // dynamic shared memory cap of the row products

enum : int {
  K_AZ = 0,      // dense rows of A: U_top <- ca A Z - cb U_top
  K_AZ_CSR = 1,  // CSR rows of A
  K_BOT = 2,     // bottom rows: U_bot <- ca delta Z - cb U_bot
  K_GTA = 3,     // dense columns of A: G = su (A^T U_top + delta U_bot)
  K_GTA_CSC = 4, // CSC columns of A
  K_GTQ = 5,     // q = Q^T G
  K_GTV = 6,     // t = c (VM^T q)
  K_GNV = 7,     // s = VM t
  K_GTQV = 8,    // q = Q^T V
  K_EXPV = 9,    // V <- G + Q s - cprev V
  K_EXPZ = 10,   // Z <- V + Q s
  K_RES = 11,    // residual rows, dense: R = B - A X (compensated FP32)
  K_RES_CSR = 12,
  K_RES_BOT = 13,  // bottom residual rows: -delta X
  K_GTR = 14,      // h = A^T R - mu X, dense columns (compensated FP32)
  K_GTR_CSC = 15,
  K_VEC = 16       // elementwise rows of n
};

enum : int { BR_NONE = 0, BR_EXACT = 1, BR_PS2 = 2, BR_PS1 = 3, BR_INNER = 4, BR_DYNAMIC = 5,
             BR_CHECK = 6, BR_MAXIT = 7 };

__device__ __forceinline__ float warp_allsum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Partial sums of squares per right-hand side of one item: each thread holds the sum for
// r = tid % NR; fixed summation order.
template <int NR>
__device__ __forceinline__ void store_partials(double sq, double* red, double* out) {
  red[threadIdx.x] = sq;
  __syncthreads();
  if (threadIdx.x < NR) {
    double s = 0.0;
    for (int t = threadIdx.x; t < BT; t += NR) s += red[t];
    out[threadIdx.x] = s;
  }
}

// ---- row-oriented products: Y(i, r) = sum_j M(i, j) X(j, r), X staged in shared memory --

template <int NR, int RW>
__global__ void __launch_bounds__(BT) gn_kernel(const BItem* __restrict__ items,
                                                const BProb* __restrict__ probs,
                                                const BPair* __restrict__ pairs,
                                                const int* __restrict__ plive,
                                                double* __restrict__ part) {
  extern __shared__ float xs[];
  __shared__ double red[BT];
  __shared__ float cA[NR], cB[NR];
  const BItem it = items[blockIdx.x];
  if (plive[it.p] == 0) return;
  const BProb& P = probs[it.p];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int kind = it.kind;
  if (tid < NR) {
    const BPair& c = pairs[(int64_t)it.p * NR + tid];
    cA[tid] = (float)c.ca;
    cB[tid] = (float)(kind == K_EXPV ? c.cprev : kind == K_EXPZ ? 0.0 : c.cb);
  }
  double sq = 0.0;
  if (kind == K_BOT) {
    __syncthreads();
    const float dl = (float)P.delta;
    const int r = tid % NR;
    for (int64_t e = it.r0 * NR + tid; e < it.r1 * NR; e += BT) {
      float* u = P.U + P.m * NR + e;
      const float v = cA[r] * dl * P.Z[e] - cB[r] * *u;
      *u = v;
      sq += (double)v * v;
    }
    store_partials<NR>(sq, red, part + (int64_t)blockIdx.x * NR);
    return;
  }
  if (kind == K_AZ_CSR) {
    __syncthreads();
    constexpr int RPW = 32 / NR;  // rows per warp pass
    const int r = lane % NR;
    for (int64_t i = it.r0 + warp * RPW + lane / NR; i < it.r1; i += (BT / 32) * RPW) {
      float acc = 0.f;
      for (int k = P.rowptr[i]; k < P.rowptr[i + 1]; ++k)
        acc = fmaf(P.vals[k], P.Z[(int64_t)P.colidx[k] * NR + r], acc);
      float* u = P.U + i * NR + r;
      const float v = cA[r] * acc - cB[r] * *u;
      *u = v;
      sq += (double)v * v;
    }
    store_partials<NR>(sq, red, part + (int64_t)blockIdx.x * NR);
    return;
  }
  // dense row products
  const float* M;
  const float* X;
  int64_t ld, K;
  int xstride = NR, xoff = 0;
  switch (kind) {
    case K_AZ: M = P.A; ld = P.lda; K = P.n; X = P.Z; break;
    case K_GNV: M = P.VM; ld = P.ell; K = P.ell; X = P.t; break;
    default: M = P.Q; ld = P.ell; K = P.ell; X = P.s; break;  // K_EXPV, K_EXPZ
  }
  for (int64_t e = tid; e < K * NR; e += BT) {
    const int64_t j = e / NR;
    xs[e] = X[j * xstride + xoff + (e - j * NR)];
  }
  __syncthreads();
  const bool v4 = kind == K_AZ && P.vec4;
  for (int64_t row = it.r0 + warp * RW; row < it.r1; row += (BT / 32) * RW) {
    float acc[RW][NR];
#pragma unroll
    for (int w = 0; w < RW; ++w)
#pragma unroll
      for (int r = 0; r < NR; ++r) acc[w][r] = 0.f;
    const float* mrow[RW];
#pragma unroll
    for (int w = 0; w < RW; ++w) mrow[w] = M + (row + w < it.r1 ? row + w : row) * ld;
    int64_t j0 = 0;
    if (v4) {
      const int64_t K4 = K & ~(int64_t)3;
      for (int64_t j = 4 * lane; j < K4; j += 128) {
        float4 a[RW];
#pragma unroll
        for (int w = 0; w < RW; ++w) a[w] = __ldg(reinterpret_cast<const float4*>(mrow[w] + j));
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float4* xv4 = reinterpret_cast<const float4*>(xs + (j + q) * NR);
#pragma unroll
          for (int r4 = 0; r4 < NR / 4; ++r4) {
            const float4 xv = xv4[r4];
#pragma unroll
            for (int w = 0; w < RW; ++w) {
              const float av = q == 0 ? a[w].x : q == 1 ? a[w].y : q == 2 ? a[w].z : a[w].w;
              acc[w][4 * r4 + 0] = fmaf(av, xv.x, acc[w][4 * r4 + 0]);
              acc[w][4 * r4 + 1] = fmaf(av, xv.y, acc[w][4 * r4 + 1]);
              acc[w][4 * r4 + 2] = fmaf(av, xv.z, acc[w][4 * r4 + 2]);
              acc[w][4 * r4 + 3] = fmaf(av, xv.w, acc[w][4 * r4 + 3]);
            }
          }
        }
      }
      j0 = K4;
    }
    for (int64_t j = j0 + lane; j < K; j += 32) {
      float a[RW];
#pragma unroll
      for (int w = 0; w < RW; ++w) a[w] = __ldg(mrow[w] + j);
      const float4* xv4 = reinterpret_cast<const float4*>(xs + j * NR);
#pragma unroll
      for (int r4 = 0; r4 < NR / 4; ++r4) {
        const float4 xv = xv4[r4];
#pragma unroll
        for (int w = 0; w < RW; ++w) {
          acc[w][4 * r4 + 0] = fmaf(a[w], xv.x, acc[w][4 * r4 + 0]);
          acc[w][4 * r4 + 1] = fmaf(a[w], xv.y, acc[w][4 * r4 + 1]);
          acc[w][4 * r4 + 2] = fmaf(a[w], xv.z, acc[w][4 * r4 + 2]);
          acc[w][4 * r4 + 3] = fmaf(a[w], xv.w, acc[w][4 * r4 + 3]);
        }
      }
    }
#pragma unroll
    for (int w = 0; w < RW; ++w)
#pragma unroll
      for (int r = 0; r < NR; ++r) acc[w][r] = warp_allsum(acc[w][r]);
    // lane (w * NR + r) % 32 finishes output (row + w, r)
#pragma unroll
    for (int w = 0; w < RW; ++w) {
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        if (((w * NR + r) & 31) != lane) continue;
        const int64_t i = row + w;
        if (i >= it.r1) continue;
        const float v = acc[w][r];
        if (kind == K_AZ) {
          float* u = P.U + i * NR + r;
          const float o = cA[r] * v - cB[r] * *u;
          *u = o;
          sq += (double)o * o;
        } else if (kind == K_GNV) {
          P.s[i * NR + r] = v;
        } else if (kind == K_EXPV) {
          float* y = P.V + i * NR + r;
          const float o = P.G[i * NR + r] + v - cB[r] * *y;
          *y = o;
          sq += (double)o * o;
        } else {
          P.Z[i * NR + r] = P.V[i * NR + r] + v;
        }
      }
    }
  }
  if (kind == K_AZ || kind == K_EXPV) {
    // lanes own r = lane % NR (RW * NR is a multiple of 32 or NR divides 32)
    __syncthreads();
    store_partials<NR>(sq, red, part + (int64_t)blockIdx.x * NR);
  }
}

// ---- column-oriented products: Y(j, r) = sum_i M(i, j) X(i, r) ---------------------------

template <int NR, int CW>
__global__ void __launch_bounds__(BT) gt_kernel(const BItem* __restrict__ items,
                                                const BProb* __restrict__ probs,
                                                const BPair* __restrict__ pairs,
                                                const int* __restrict__ plive) {
  extern __shared__ float gsm[];
  float* xch = gsm;                    // GT_CHUNK x NR
  float* red = gsm + GT_CHUNK * NR;    // 8 warps x (CW * NR * 32)
  __shared__ float sc[NR];
  const BItem it = items[blockIdx.x];
  if (plive[it.p] == 0) return;
  const BProb& P = probs[it.p];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int kind = it.kind;
  if (tid < NR) sc[tid] = (float)pairs[(int64_t)it.p * NR + tid].su;
  if (kind == K_GTA_CSC) {
    __syncthreads();
    constexpr int CPW = 32 / NR;
    const int r = lane % NR;
    const float dl = (float)P.delta;
    for (int64_t j = it.r0 + warp * CPW + lane / NR; j < it.r1; j += (BT / 32) * CPW) {
      float acc = 0.f;
      for (int k = P.colptr[j]; k < P.colptr[j + 1]; ++k)
        acc = fmaf(P.cvals[k], P.U[(int64_t)P.rowidx[k] * NR + r], acc);
      P.G[j * NR + r] = sc[r] * (acc + dl * P.U[(P.m + j) * NR + r]);
    }
    return;
  }
  const float* M;
  const float* X;
  int64_t ld, rows;
  switch (kind) {
    case K_GTA: M = P.A; ld = P.lda; rows = P.m; X = P.U; break;
    case K_GTQ: M = P.Q; ld = P.ell; rows = P.n; X = P.G; break;
    case K_GTQV: M = P.Q; ld = P.ell; rows = P.n; X = P.V; break;
    default: M = P.VM; ld = P.ell; rows = P.ell; X = P.q; break;  // K_GTV
  }
  float acc[CW][NR];
#pragma unroll
  for (int c = 0; c < CW; ++c)
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[c][r] = 0.f;
  int64_t col[CW];
  bool ok[CW];
#pragma unroll
  for (int c = 0; c < CW; ++c) {
    col[c] = it.r0 + lane + 32 * c;
    ok[c] = col[c] < it.r1;
  }
  for (int64_t i0 = 0; i0 < rows; i0 += GT_CHUNK) {
    const int nr = (int)(rows - i0 < GT_CHUNK ? rows - i0 : GT_CHUNK);
    __syncthreads();
    for (int e = tid; e < nr * NR; e += BT) xch[e] = X[i0 * NR + e];
    __syncthreads();
#pragma unroll 4
    for (int ii = warp; ii < nr; ii += BT / 32) {
      const float* mr = M + (i0 + ii) * ld;
      float a[CW];
#pragma unroll
      for (int c = 0; c < CW; ++c) a[c] = ok[c] ? __ldg(mr + col[c]) : 0.f;
      const float4* xv4 = reinterpret_cast<const float4*>(xch + ii * NR);
#pragma unroll
      for (int r4 = 0; r4 < NR / 4; ++r4) {
        const float4 xv = xv4[r4];
#pragma unroll
        for (int c = 0; c < CW; ++c) {
          acc[c][4 * r4 + 0] = fmaf(a[c], xv.x, acc[c][4 * r4 + 0]);
          acc[c][4 * r4 + 1] = fmaf(a[c], xv.y, acc[c][4 * r4 + 1]);
          acc[c][4 * r4 + 2] = fmaf(a[c], xv.z, acc[c][4 * r4 + 2]);
          acc[c][4 * r4 + 3] = fmaf(a[c], xv.w, acc[c][4 * r4 + 3]);
        }
      }
    }
  }
#pragma unroll
  for (int c = 0; c < CW; ++c)
#pragma unroll
    for (int r = 0; r < NR; ++r) red[warp * (CW * NR * 32) + (c * NR + r) * 32 + lane] = acc[c][r];
  __syncthreads();
  for (int e = tid; e < CW * NR * 32; e += BT) {
    float v = 0.f;
#pragma unroll
    for (int w = 0; w < BT / 32; ++w) v += red[w * (CW * NR * 32) + e];
    const int ln = e & 31, cr = e >> 5, c = cr / NR, r = cr - c * NR;
    const int64_t j = it.r0 + ln + 32 * c;
    if (j >= it.r1) continue;
    if (kind == K_GTA) {
      P.G[j * NR + r] = sc[r] * (v + (float)P.delta * P.U[(P.m + j) * NR + r]);
    } else if (kind == K_GTQ || kind == K_GTQV) {
      P.q[j * NR + r] = v;
    } else {
      P.t[j * NR + r] = P.c1[j] * v;
    }
  }
}

// ---- per-pair scalar steps -------------------------------------------------------------

__global__ void beta_kernel(int npairs, int NR, const BProb* __restrict__ probs,
                            BPair* __restrict__ pairs, const double* __restrict__ part,
                            const double* __restrict__ gpart, int init) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= npairs) return;
  BPair& c = pairs[e];
  if (!c.live) return;
  const int p = e / NR, r = e - p * NR;
  const BProb& P = probs[p];
  double s = 0.0;
  if (init) {
    // beta_1 = ||[0; g / delta]||: the stopping tests of a phase (Paige-Saunders and the
    // dynamic rule) read the residual estimate of this correction system
    double g2 = 0.0;
    for (int k = P.g0; k < P.g1; ++k) g2 += gpart[(int64_t)k * NR + r];
    s = g2 / (P.delta * P.delta);
  } else {
    for (int k = P.b0; k < P.b1; ++k) s += part[(int64_t)k * NR + r];
  }
  const double beta = sqrt(s);
  c.su = beta > 0.0 ? 1.0 / beta : 0.0;
  if (init) {
    c.beta = beta;
    c.beta1 = beta;
    c.phibar = beta;
    c.cprev = 0.0;
    c.anorm2 = 0.0;
    if (beta == 0.0) {
      c.live = 0;
      c.reason = BR_EXACT;
      c.ca = c.cb = c.cprev = c.su = 0.0;
    }
  } else {
    c.anorm2 += c.alpha * c.alpha + beta * beta;
    c.cprev = beta * c.sv;
    c.beta = beta;
  }
}

// Dynamic stopping test of Section 5.3.2: stop when cvgdiff = phibar_prev - phibar is
// below sigma_ell or cvgrate_1 / cvgrate_j > nu (a non-positive rate counts as an infinite
// ratio).
__device__ __forceinline__ bool bdyn_stop(double phibar_prev, double phibar, double rate1,
                                          double nu, double sig_ell) {
  if (!isfinite(nu)) return false;
  if (phibar_prev - phibar < sig_ell) return true;
  if (phibar <= 0.0) return false;
  const double rate = log(phibar_prev / phibar);
  if (rate <= 0.0) return true;
  return rate1 / rate > nu;
}

__global__ void alpha_kernel(int npairs, int NR, const BProb* __restrict__ probs,
                             BPair* __restrict__ pairs, const double* __restrict__ part, int init,
                             int* __restrict__ plive, int* __restrict__ live_count) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= npairs) return;
  BPair& c = pairs[e];
  if (!c.live) { c.upd = 0; return; }
  const int p = e / NR, r = e - p * NR;
  const BProb& P = probs[p];
  double s = 0.0;
  for (int k = P.a0; k < P.a1; ++k) s += part[(int64_t)k * NR + r];
  const double alpha = sqrt(s);
  if (init) {
    c.alpha = alpha;
    c.rhobar = alpha;
    c.sv = alpha > 0.0 ? 1.0 / alpha : 0.0;
    c.upd = 1;
    c.it = 0;
    c.arnorm0 = alpha * c.beta1;
    c.xc = 0.0;
    c.dc = 0.0;
    if (alpha == 0.0) { c.live = 0; c.reason = BR_EXACT; }
  } else {
    const double beta = c.beta;
    const double rho = sqrt(c.rhobar * c.rhobar + beta * beta);
    const double cc = c.rhobar / rho, sn = beta / rho;
    const double theta = sn * alpha;
    c.rhobar = -cc * alpha;
    const double phi = cc * c.phibar;
    const double phibar_prev = c.phibar;
    const double phibar = sn * c.phibar;
    c.phibar = phibar;
    c.phibar_prev = phibar_prev;
    c.xc = phi / rho;
    c.dc = theta / rho;
    c.upd = 2;
    c.alpha = alpha;
    c.sv = alpha > 0.0 ? 1.0 / alpha : 0.0;
    const long long it = ++c.it;
    if (it == 1) c.rate1 = phibar > 0.0 ? log(phibar_prev / phibar) : INFINITY;
    int reason = BR_NONE;
    const double ca = fabs(cc);
    const double arn = phibar * alpha * ca;  // ||Abar^T rbar||
    if (beta == 0.0 || alpha == 0.0) reason = BR_EXACT;
    else if (alpha * ca <= c.eps * sqrt(c.anorm2)) reason = BR_PS2;
    else if (phibar <= c.eps * c.beta1) reason = BR_PS1;
    else if (c.inner > 0.0 && arn <= c.inner * c.arnorm0) reason = BR_INNER;
    else if (bdyn_stop(phibar_prev, phibar, c.rate1, c.nu, c.sig_ell)) reason = BR_DYNAMIC;
    else if (c.tol > 0.0 && c.normP * phibar * alpha * ca / c.norm_ref <= c.tol) reason = BR_CHECK;
    else if (it >= c.maxit) reason = BR_MAXIT;
    if (reason != BR_NONE) { c.live = 0; c.reason = reason; }
  }
  // coefficients of the next A pass: U <- sv A Z - alpha su U.  A pair that stopped
  // gets zero coefficients, so its columns decay to zero instead of running on with
  // stale scales (the x update of this iteration still applies).
  if (c.live) {
    c.ca = c.sv;
    c.cb = c.alpha * c.su;
  } else {
    c.ca = c.cb = c.cprev = c.su = 0.0;
  }
  if (c.live) {
    atomicAdd(&plive[p], 1);
    atomicAdd(live_count, 1);
  }
  (void)r;
}

// x += xc D ; D <- sv Z - dc D   (upd 2);   D <- sv Z   (upd 1)
template <int NR>
__global__ void vec_kernel(const BItem* __restrict__ items, const BProb* __restrict__ probs,
                           const BPair* __restrict__ pairs) {
  const BItem it = items[blockIdx.x];
  const BProb& P = probs[it.p];
  const BPair* pp = pairs + (int64_t)it.p * NR;
  for (int64_t e = it.r0 * NR + threadIdx.x; e < it.r1 * NR; e += BT) {
    const BPair& c = pp[e % NR];
    if (c.upd == 0) continue;
    const double z = c.sv * (double)P.Z[e];
    if (c.upd == 1) {
      P.D[e] = z;
    } else {
      const double d = P.D[e];
      P.X[e] += c.xc * d;
      P.D[e] = z - c.dc * d;
    }
  }
}

// Xh + Xl = X (FP32 hi/lo split)
template <int NR>
__global__ void split_x_kernel(const BItem* __restrict__ items, const BProb* __restrict__ probs) {
  const BItem it = items[blockIdx.x];
  const BProb& P = probs[it.p];
  for (int64_t e = it.r0 * NR + threadIdx.x; e < it.r1 * NR; e += BT) {
    const double v = P.X[e];
    const float h = __double2float_rn(v);
    P.Xh[e] = h;
    P.Xl[e] = __double2float_rn(v - (double)h);
  }
}

// Residual rows r = B - A X with compensated FP32 products (r also split into Rh + Rl)
// and the bottom rows -delta X; partial sums of their squares, whose total is
// ||[b - A x; -delta x]||^2, the norm of the warm-start right-hand side of the phase.
// With init, U_top = 0 (the phase solves for the correction with right-hand side
// [0; g / delta], see gtr_kernel).
template <int NR>
__global__ void __launch_bounds__(BT) res_kernel(const BItem* __restrict__ items,
                                                 const BProb* __restrict__ probs,
                                                 const int* __restrict__ plive,
                                                 double* __restrict__ part, int init) {
  __shared__ double red[BT];
  const BItem it = items[blockIdx.x];
  if (plive[it.p] == 0) return;
  const BProb& P = probs[it.p];
  const int r = threadIdx.x % NR;
  double sq = 0.0;
  if (it.kind == K_RES_BOT) {
    for (int64_t j = it.r0 + threadIdx.x / NR; j < it.r1; j += BT / NR) {
      const double v = -P.delta * P.X[j * NR + r];
      sq += v * v;
    }
  } else {
    for (int64_t i = it.r0 + threadIdx.x / NR; i < it.r1; i += BT / NR) {
      DF acc{0.f, 0.f};
      if (it.kind == K_RES) {
        const float* ar = P.A + i * P.lda;
        for (int64_t j = 0; j < P.n; ++j) df_fma(acc, __ldg(ar + j), P.Xh[j * NR + r], P.Xl[j * NR + r]);
      } else {
        for (int k = P.rowptr[i]; k < P.rowptr[i + 1]; ++k) {
          const int64_t j = P.colidx[k];
          df_fma(acc, P.vals[k], P.Xh[j * NR + r], P.Xl[j * NR + r]);
        }
      }
      const double v = (P.B ? P.B[i * NR + r] : 0.0) - df_val(acc);
      const float h = __double2float_rn(v);
      P.Rh[i * NR + r] = h;
      P.Rl[i * NR + r] = __double2float_rn(v - (double)h);
      if (init) P.U[i * NR + r] = 0.f;
      sq += v * v;
    }
  }
  store_partials<NR>(sq, red, part + (int64_t)blockIdx.x * NR);
}

// g = A^T r - mu X with compensated FP32 products (the normal-equation residual of x);
// partial sums of g^2.  With init, U_bot = g / delta: LSQR on [A; delta I] P^-1 with
// right-hand side [0; g / delta] has the normal equations (A^T A + mu I) dx = g, the same
// as the warm start of the paper (right-hand side [b - A x; -delta x]), so in exact
// arithmetic both produce the same iterates; but every vector of this form shrinks with
// g, so FP32 products keep their relative accuracy as the refinement converges.
template <int NR>
__global__ void __launch_bounds__(BT) gtr_kernel(const BItem* __restrict__ items,
                                                 const BProb* __restrict__ probs,
                                                 const int* __restrict__ plive,
                                                 double* __restrict__ part, int init) {
  __shared__ double red[BT];
  const BItem it = items[blockIdx.x];
  if (plive[it.p] == 0) return;
  const BProb& P = probs[it.p];
  const int r = threadIdx.x % NR;
  double sq = 0.0;
  for (int64_t j = it.r0 + threadIdx.x / NR; j < it.r1; j += BT / NR) {
    DF acc{0.f, 0.f};
    if (it.kind == K_GTR) {
      for (int64_t i = 0; i < P.m; ++i)
        df_fma(acc, __ldg(P.A + i * P.lda + j), P.Rh[i * NR + r], P.Rl[i * NR + r]);
    } else {
      for (int k = P.colptr[j]; k < P.colptr[j + 1]; ++k) {
        const int64_t i = P.rowidx[k];
        df_fma(acc, P.cvals[k], P.Rh[i * NR + r], P.Rl[i * NR + r]);
      }
    }
    double h = df_val(acc) - P.mu * P.X[j * NR + r];
    if (P.Gx) h += P.Gx[j * NR + r];
    if (init) P.U[(P.m + j) * NR + r] = (float)(h / P.delta);
    sq += h * h;
  }
  store_partials<NR>(sq, red, part + (int64_t)blockIdx.x * NR);
}

__global__ void ne_kernel(int npairs, int NR, const BProb* __restrict__ probs,
                          const double* __restrict__ part, double* __restrict__ out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= npairs) return;
  const int p = e / NR, r = e - p * NR;
  const BProb& P = probs[p];
  double s = 0.0;
  for (int k = P.g0; k < P.g1; ++k) s += part[(int64_t)k * NR + r];
  out[e] = sqrt(s);
}

// FP64 column-major (ld) -> FP32 row-major transpose: dst[i * cols + j] = src[i + j * ld]
__global__ void to_f32_rowmajor(int64_t rows, int64_t cols, const double* __restrict__ src,
                                int64_t ld, float* __restrict__ dst) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= rows * cols) return;
  const int64_t i = e / cols, j = e - i * cols;
  dst[e] = (float)src[i + j * ld];
}

__global__ void to_f32(int64_t n, const double* __restrict__ src, float* __restrict__ dst) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) dst[e] = (float)src[e];
}

// B (m x RS, row-major, padded columns zero) from b (m x R column-major)
__global__ void pack_rhs(int64_t m, int R, int RS, const double* __restrict__ b,
                         double* __restrict__ B) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m * RS) return;
  const int64_t i = e / RS;
  const int r = (int)(e - i * RS);
  B[e] = r < R ? b[i + (int64_t)r * m] : 0.0;
}

// x (n x R column-major) from X (n x RS row-major)
__global__ void unpack_x(int64_t n, int R, int RS, const double* __restrict__ X,
                         double* __restrict__ x) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * R) return;
  const int64_t r = e / n, i = e - r * n;
  x[e] = X[i * RS + r];
}

template <int NR>
void gn_launch(cudaStream_t st, const BItem* items, int n, int rw, size_t smem, const BProb* probs,
               const BPair* pairs, const int* plive, double* part) {
  if (n == 0) return;
  if (rw == 2) {
    gn_kernel<NR, 2><<<n, BT, smem, st>>>(items, probs, pairs, plive, part);
  } else {
    gn_kernel<NR, 4><<<n, BT, smem, st>>>(items, probs, pairs, plive, part);
  }
  APL_LAUNCH_CHECK();
}

template <int NR>
size_t gt_smem(int cw) { return ((size_t)GT_CHUNK * NR + (size_t)(BT / 32) * cw * NR * 32) * sizeof(float); }

template <int NR>
void gt_launch(cudaStream_t st, const BItem* items, int n, int cw, const BProb* probs,
               const BPair* pairs, const int* plive) {
  if (n == 0) return;
  const size_t sm = gt_smem<NR>(cw);
  if (cw == 1) gt_kernel<NR, 1><<<n, BT, sm, st>>>(items, probs, pairs, plive);
  else if (cw == 2) gt_kernel<NR, 2><<<n, BT, sm, st>>>(items, probs, pairs, plive);
  else gt_kernel<NR, 4><<<n, BT, sm, st>>>(items, probs, pairs, plive);
  APL_LAUNCH_CHECK();
}

template <int NR>
void set_attrs(size_t gn_smem) {
  // the cap, not this batch's need: engines in other threads use the same kernels
  (void)gn_smem;
  APL_CUDA(cudaFuncSetAttribute(gn_kernel<NR, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kGnSmemCap));
  APL_CUDA(cudaFuncSetAttribute(gn_kernel<NR, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, kGnSmemCap));
  APL_CUDA(cudaFuncSetAttribute(gt_kernel<NR, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gt_smem<NR>(1)));
  APL_CUDA(cudaFuncSetAttribute(gt_kernel<NR, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gt_smem<NR>(2)));
  APL_CUDA(cudaFuncSetAttribute(gt_kernel<NR, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gt_smem<NR>(4)));
}

}  // namespace

// ======================================================================================

BatchEngine::~BatchEngine() {}

void BatchEngine::setup(cudaStream_t st, const std::vector<BatchSrc>& src, int R, double mu) {
  APL_REQUIRE(R >= 1 && R <= BATCH_MAX_RHS, "batched solves take 1 to 16 right-hand sides");
  st_ = st;
  R_ = R;
  RS_ = R <= 4 ? 4 : 16;
  mu_ = mu;
  delta_ = std::sqrt(mu);
  const int np = (int)src.size();
  hp_.assign(np, BProb{});
  qf_.reset(new DBuf<float>[np]);
  vmf_.reset(new DBuf<float>[np]);
  c1f_.reset(new DBuf<float>[np]);
  fvec_.reset(new DBuf<float>[np]);
  dvec_.reset(new DBuf<double>[np]);
  int64_t nmax = 0;
  for (int p = 0; p < np; ++p) {
    const MatView& A = src[p].A;
    APL_REQUIRE(A.dtype == 1, "batched solves take FP32 matrices");
    BProb& P = hp_[p];
    P.m = A.m; P.n = A.n; P.fmt = A.fmt; P.lda = A.ld;
    P.delta = delta_; P.mu = mu;
    P.A = (const float*)A.vals;
    P.rowptr = A.rowptr; P.colidx = A.colidx; P.vals = (const float*)A.vals;
    P.colptr = A.colptr; P.rowidx = A.rowidx; P.cvals = (const float*)A.cvals;
    P.vec4 = (A.fmt == 0 && A.ld % 4 == 0 && ((uintptr_t)A.vals % 16) == 0) ? 1 : 0;
    nmax = std::max(nmax, A.n);
    const int64_t m = A.m, n = A.n, rs = RS_;
    // FP32 vectors: U (m+n), V, Z, G, q (n), t, s (2n), Xh, Xl (n), Rh, Rl (m)
    const int64_t nf = rs * ((m + n) + 4 * n + 4 * n + 2 * n + 2 * m);
    fvec_[p].alloc(nf, st);
    fvec_[p].zero(st);
    float* f = fvec_[p].p;
    P.U = f; f += rs * (m + n);
    P.V = f; f += rs * n;
    P.Z = f; f += rs * n;
    P.G = f; f += rs * n;
    P.q = f; f += rs * n;
    P.t = f; f += rs * n;
    P.s = f; f += rs * n;
    P.Xh = f; f += rs * n;
    P.Xl = f; f += rs * n;
    P.Rh = f; f += rs * m;
    P.Rl = f; f += rs * m;
    // FP64 vectors: X, D (n), B (m)
    const int64_t nd = rs * (2 * n + m);
    dvec_[p].alloc(nd, st);
    dvec_[p].zero(st);
    double* d = dvec_[p].p;
    P.X = d; d += rs * n;
    P.D = d; d += rs * n;
    double* Bp = d;
    P.B = Bp;
    pack_rhs<<<(unsigned)cdiv(m * rs, 256), 256, 0, st>>>(m, R, RS_, src[p].b, Bp);
    APL_LAUNCH_CHECK();
  }
  gn_smem_ = (size_t)nmax * RS_ * sizeof(float);
  APL_REQUIRE(gn_smem_ <= (size_t)kGnSmemCap,
              "batched solves need n * (nrhs rounded up to 4 or 16) * 4 bytes <= 200 KiB");
  if (RS_ == 4) set_attrs<4>(gn_smem_); else set_attrs<16>(gn_smem_);
  dp_.alloc(np, st);
  pairs_.alloc((size_t)np * RS_, st);
  live_count_.alloc(1 + np, st);
  normP_.assign(np, 1.0);
  sig_ell_.assign(np, 0.0);
  // ||A^T b|| for every pair: the normal-equation residual at x = 0 with unit reference
  std::vector<char> all((size_t)np * R_, 1);
  norm_ref_.assign((size_t)np * RS_, 1.0);
  std::vector<double> nb;
  ne_residual(all, nb);
  for (int p = 0; p < np; ++p)
    for (int r = 0; r < R_; ++r) norm_ref_[(size_t)p * RS_ + r] = nb[(size_t)p * R_ + r];
}

void BatchEngine::begin_adjoint(const std::vector<const double*>& gx) {
  const int np = nprob();
  APL_REQUIRE((int)gx.size() == np, "adjoint: one gradient per problem");
  if (!adj_) adj_.reset(new DBuf<double>[np]);
  saved_ref_ = norm_ref_;
  saved_b_.assign(np, nullptr);
  for (int p = 0; p < np; ++p) {
    BProb& P = hp_[p];
    const int64_t n = P.n, rs = RS_;
    adj_[p].alloc((size_t)2 * n * rs, st_);
    double* sx = adj_[p].p;
    double* g = adj_[p].p + n * rs;
    APL_CUDA(cudaMemcpyAsync(sx, P.X, n * rs * sizeof(double), cudaMemcpyDeviceToDevice, st_));
    pack_rhs<<<(unsigned)cdiv(n * rs, 256), 256, 0, st_>>>(n, R_, RS_, gx[p], g);
    APL_LAUNCH_CHECK();
    saved_b_[p] = P.B;
    P.B = nullptr;
    P.Gx = g;
    // ||g|| per pair as the residual reference (host copy: n x R values per problem)
    std::vector<double> hg((size_t)n * R_);
    APL_CUDA(cudaMemcpyAsync(hg.data(), gx[p], hg.size() * sizeof(double), cudaMemcpyDeviceToHost, st_));
    APL_CUDA(cudaStreamSynchronize(st_));
    for (int r = 0; r < R_; ++r) {
      double ss = 0.0;
      for (int64_t j = 0; j < n; ++j) ss += hg[j + (size_t)r * n] * hg[j + (size_t)r * n];
      norm_ref_[(size_t)p * RS_ + r] = std::sqrt(ss);
    }
  }
  zero_x();
  APL_CUDA(cudaStreamSynchronize(st_));
}

void BatchEngine::end_adjoint() {
  const int np = nprob();
  if (saved_b_.empty()) return;
  for (int p = 0; p < np; ++p) {
    BProb& P = hp_[p];
    APL_CUDA(cudaMemcpyAsync(P.X, adj_[p].p, (size_t)P.n * RS_ * sizeof(double),
                             cudaMemcpyDeviceToDevice, st_));
    P.B = saved_b_[p];
    P.Gx = nullptr;
  }
  norm_ref_ = saved_ref_;
  saved_b_.clear();
  APL_CUDA(cudaStreamSynchronize(st_));
}

void BatchEngine::set_precond(int p, const PrecondDev& Pd) {
  BProb& P = hp_[p];
  const int64_t L = Pd.ell, n = P.n;
  P.ell = (int)L;
  if (L == 0) { clear_precond(p); return; }
  qf_[p].alloc((size_t)n * L, st_);
  vmf_[p].alloc((size_t)L * L, st_);
  c1f_[p].alloc(L, st_);
  to_f32_rowmajor<<<(unsigned)cdiv(n * L, 256), 256, 0, st_>>>(n, L, Pd.Q, Pd.ldq, qf_[p].p);
  APL_LAUNCH_CHECK();
  to_f32_rowmajor<<<(unsigned)cdiv(L * L, 256), 256, 0, st_>>>(L, L, Pd.VM, L, vmf_[p].p);
  APL_LAUNCH_CHECK();
  to_f32<<<(unsigned)cdiv(L, 256), 256, 0, st_>>>(L, Pd.coef, c1f_[p].p);
  APL_LAUNCH_CHECK();
  APL_CUDA(cudaStreamSynchronize(st_));
  P.Q = qf_[p].p; P.VM = vmf_[p].p; P.c1 = c1f_[p].p;
  normP_[p] = Pd.normP;
  sig_ell_[p] = Pd.sig_ell;
  items_dirty_ = true;
}

void BatchEngine::clear_precond(int p) {
  BProb& P = hp_[p];
  P.ell = 0;
  P.Q = nullptr; P.VM = nullptr; P.c1 = nullptr;
  normP_[p] = 1.0;
  sig_ell_[p] = 0.0;
  items_dirty_ = true;
}

void BatchEngine::zero_x() {
  for (int p = 0; p < nprob(); ++p)
    APL_CUDA(cudaMemsetAsync(hp_[p].X, 0, (size_t)hp_[p].n * RS_ * sizeof(double), st_));
}

void BatchEngine::get_x(int p, double* x_out) const {
  const BProb& P = hp_[p];
  unpack_x<<<(unsigned)cdiv(P.n * R_, 256), 256, 0, st_>>>(P.n, R_, RS_, P.X, x_out);
  APL_LAUNCH_CHECK();
}

// Work lists for the problems with active != 0 (host flags), largest problems first.
void BatchEngine::build_items() {
  const int np = nprob();
  std::vector<int> order(np);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    const double wa = hp_[a].fmt == 0 ? (double)hp_[a].m * hp_[a].n : 8.0 * hp_[a].m;
    const double wb = hp_[b].fmt == 0 ? (double)hp_[b].m * hp_[b].n : 8.0 * hp_[b].m;
    return wa > wb;
  });
  std::vector<BItem> ap, gta, gtq, gtqv, gtv, gnv, ex, exz, vec, res, gtr;
  for (int p : order) {
    BProb& P = hp_[p];
    P.b0 = P.b1 = P.a0 = P.a1 = P.g0 = P.g1 = P.q0 = P.q1 = 0;
    if (!P.active) continue;
    const int64_t m = P.m, n = P.n, L = P.ell;
    P.b0 = (int)ap.size();
    for (int64_t i = 0; i < m; i += ROWS_ITEM)
      ap.push_back({p, P.fmt == 0 ? K_AZ : K_AZ_CSR, i, std::min(m, i + ROWS_ITEM)});
    for (int64_t j = 0; j < n; j += VEC_ITEM) ap.push_back({p, K_BOT, j, std::min(n, j + VEC_ITEM)});
    P.b1 = (int)ap.size();
    const int64_t cwid = P.fmt == 0 ? 32 * cw_ : 64;
    for (int64_t j = 0; j < n; j += cwid)
      gta.push_back({p, P.fmt == 0 ? K_GTA : K_GTA_CSC, j, std::min(n, j + cwid)});
    for (int64_t k = 0; k < L; k += 32 * cw_) {
      gtq.push_back({p, K_GTQ, k, std::min(L, k + 32 * cw_)});
      gtqv.push_back({p, K_GTQV, k, std::min(L, k + 32 * cw_)});
      gtv.push_back({p, K_GTV, k, std::min(L, k + 32 * cw_)});
    }
    for (int64_t k = 0; k < L; k += 64) {
      gnv.push_back({p, K_GNV, k, std::min(L, k + 64)});
    }
    P.a0 = (int)ex.size();
    for (int64_t j = 0; j < n; j += 64) ex.push_back({p, K_EXPV, j, std::min(n, j + 64)});
    P.a1 = (int)ex.size();
    for (int64_t j = 0; j < n; j += 64) exz.push_back({p, K_EXPZ, j, std::min(n, j + 64)});
    for (int64_t j = 0; j < n; j += VEC_ITEM) vec.push_back({p, K_VEC, j, std::min(n, j + VEC_ITEM)});
    P.q0 = (int)res.size();
    for (int64_t i = 0; i < m; i += 64)
      res.push_back({p, P.fmt == 0 ? K_RES : K_RES_CSR, i, std::min(m, i + 64)});
    for (int64_t j = 0; j < n; j += VEC_ITEM) res.push_back({p, K_RES_BOT, j, std::min(n, j + VEC_ITEM)});
    P.q1 = (int)res.size();
    P.g0 = (int)gtr.size();
    const int64_t gw = 16;
    for (int64_t j = 0; j < n; j += gw)
      gtr.push_back({p, P.fmt == 0 ? K_GTR : K_GTR_CSC, j, std::min(n, j + gw)});
    P.g1 = (int)gtr.size();
  }
  auto up = [&](DBuf<BItem>& d, const std::vector<BItem>& h, int& cnt) {
    cnt = (int)h.size();
    if (h.empty()) return;
    d.alloc(h.size(), st_);
    APL_CUDA(cudaMemcpyAsync(d.p, h.data(), h.size() * sizeof(BItem), cudaMemcpyHostToDevice, st_));
  };
  up(it_apass_, ap, n_apass_);
  up(it_gta_, gta, n_gta_);
  up(it_gtq_, gtq, n_gtq_);
  up(it_gtqv_, gtqv, n_gtqv_);
  up(it_expz_, exz, n_expz_);
  up(it_gtv_, gtv, n_gtv_);
  up(it_gnv_, gnv, n_gnv_);
  up(it_exp_, ex, n_exp_);
  up(it_vec_, vec, n_vec_);
  up(it_res_, res, n_res_);
  up(it_gtr_, gtr, n_gtr_);
  const size_t npart = (size_t)std::max({n_apass_, n_exp_, n_res_, 1}) * RS_;
  part_.alloc(npart, st_);
  ne_part_.alloc((size_t)std::max(n_gtr_, 1) * RS_, st_);
  APL_CUDA(cudaStreamSynchronize(st_));
  items_dirty_ = false;
}

void BatchEngine::upload_probs() {
  APL_CUDA(cudaMemcpyAsync(dp_.p, hp_.data(), hp_.size() * sizeof(BProb), cudaMemcpyHostToDevice, st_));
}

void BatchEngine::launch_gn(const DBuf<BItem>& items, int nitems, int rw) {
  if (RS_ == 4) gn_launch<4>(st_, items.p, nitems, rw, gn_smem_, dp_.p, pairs_.p, live_count_.p + 1, part_.p);
  else gn_launch<16>(st_, items.p, nitems, rw, gn_smem_, dp_.p, pairs_.p, live_count_.p + 1, part_.p);
}

void BatchEngine::launch_gt(const DBuf<BItem>& items, int nitems, int cw) {
  if (RS_ == 4) gt_launch<4>(st_, items.p, nitems, cw, dp_.p, pairs_.p, live_count_.p + 1);
  else gt_launch<16>(st_, items.p, nitems, cw, dp_.p, pairs_.p, live_count_.p + 1);
}

void BatchEngine::launch_residual(bool init) {
  if (n_vec_) {
    if (RS_ == 4) split_x_kernel<4><<<n_vec_, BT, 0, st_>>>(it_vec_.p, dp_.p);
    else split_x_kernel<16><<<n_vec_, BT, 0, st_>>>(it_vec_.p, dp_.p);
    APL_LAUNCH_CHECK();
  }
  if (n_res_) {
    if (RS_ == 4) res_kernel<4><<<n_res_, BT, 0, st_>>>(it_res_.p, dp_.p, live_count_.p + 1, part_.p, init);
    else res_kernel<16><<<n_res_, BT, 0, st_>>>(it_res_.p, dp_.p, live_count_.p + 1, part_.p, init);
    APL_LAUNCH_CHECK();
  }
}

void BatchEngine::launch_gtr(bool init) {
  if (!n_gtr_) return;
  if (RS_ == 4) gtr_kernel<4><<<n_gtr_, BT, 0, st_>>>(it_gtr_.p, dp_.p, live_count_.p + 1, ne_part_.p, init);
  else gtr_kernel<16><<<n_gtr_, BT, 0, st_>>>(it_gtr_.p, dp_.p, live_count_.p + 1, ne_part_.p, init);
  APL_LAUNCH_CHECK();
}

void BatchEngine::launch_iteration(bool init) {
  const int npairs = nprob() * RS_;
  const unsigned pb = (unsigned)cdiv(npairs, 128);
  int64_t launches = 0;
  if (init) {
    launch_residual(true);
    launch_gtr(true);
  } else {
    launch_gn(it_apass_, n_apass_, rw_);
    ++launches;
  }
  beta_kernel<<<pb, 128, 0, st_>>>(npairs, RS_, dp_.p, pairs_.p, part_.p, ne_part_.p,
                                   init ? 1 : 0);
  APL_LAUNCH_CHECK();
  launch_gt(it_gta_, n_gta_, cw_);
  // V = P^-1 g - cprev V
  launch_gt(it_gtq_, n_gtq_, cw_);
  launch_gt(it_gtv_, n_gtv_, cw_);
  launch_gn(it_gnv_, n_gnv_, 2);
  launch_gn(it_exp_, n_exp_, 2);
  // Z = P^-1 V
  launch_gt(it_gtqv_, n_gtqv_, cw_);
  launch_gt(it_gtv_, n_gtv_, cw_);
  launch_gn(it_gnv_, n_gnv_, 2);
  launch_gn(it_expz_, n_expz_, 2);
  APL_CUDA(cudaMemsetAsync(live_count_.p, 0, (1 + nprob()) * sizeof(int), st_));
  alpha_kernel<<<pb, 128, 0, st_>>>(npairs, RS_, dp_.p, pairs_.p, part_.p, init ? 1 : 0,
                                    live_count_.p + 1, live_count_.p);
  APL_LAUNCH_CHECK();
  if (n_vec_) {
    if (RS_ == 4) vec_kernel<4><<<n_vec_, BT, 0, st_>>>(it_vec_.p, dp_.p, pairs_.p);
    else vec_kernel<16><<<n_vec_, BT, 0, st_>>>(it_vec_.p, dp_.p, pairs_.p);
    APL_LAUNCH_CHECK();
  }
  launches += 12;
  if (!init) launches_per_iter_ = launches;
}

void BatchEngine::run_phase(const std::vector<char>& mask, const std::vector<double>& nu,
                            double eps, double tol, const std::vector<long long>& maxit,
                            std::vector<long long>& iters, std::vector<int>& reasons) {
  const int np = nprob();
  const size_t npairs = (size_t)np * RS_;
  iters.assign((size_t)np * R_, 0);
  reasons.assign((size_t)np * R_, 0);
  std::vector<int> plive(1 + np, 0);
  std::vector<BPair> hpairs(npairs);
  bool any = false;
  for (int p = 0; p < np; ++p) {
    int cnt = 0;
    for (int r = 0; r < RS_; ++r) {
      const size_t e = (size_t)p * RS_ + r, er = (size_t)p * R_ + r;
      BPair c{};
      c.live = (r < R_ && mask[er]) ? 1 : 0;
      c.nu = nu[p];
      c.sig_ell = sig_ell_[p];
      c.eps = eps;
      c.inner = 1e-4;
      // the device bound ||P|| ||Abar^T rbar|| / ||A^T b|| ends a phase early only well
      // below tol: its FP32 recurrences run ahead of the true residual, and a phase
      // stopped at tol would leave the refinement short of it
      c.tol = 0.1 * tol;
      c.normP = normP_[p];
      c.norm_ref = norm_ref_[e] > 0.0 ? norm_ref_[e] : 1.0;
      c.maxit = c.live ? maxit[er] : 0;
      cnt += c.live;
      hpairs[e] = c;
    }
    const int want = cnt > 0 ? 1 : 0;
    if (want != hp_[p].active) items_dirty_ = true;
    hp_[p].active = want;
    plive[1 + p] = cnt;
    any = any || cnt > 0;
  }
  if (!any) return;
  if (items_dirty_) build_items();
  upload_probs();
  APL_CUDA(cudaMemcpyAsync(pairs_.p, hpairs.data(), npairs * sizeof(BPair), cudaMemcpyHostToDevice, st_));
  APL_CUDA(cudaMemcpyAsync(live_count_.p, plive.data(), plive.size() * sizeof(int), cudaMemcpyHostToDevice, st_));
  launch_iteration(true);
  long long maxall = 0;
  for (size_t e = 0; e < npairs; ++e) if (hpairs[e].live) maxall = std::max(maxall, hpairs[e].maxit);
  const int G = 8;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  APL_CUDA(cudaStreamBeginCapture(st_, cudaStreamCaptureModeThreadLocal));
  {
    CaptureScope cs;
    try {
      for (int g = 0; g < G; ++g) launch_iteration(false);
    } catch (...) {
      cudaStreamEndCapture(st_, &graph);
      if (graph) cudaGraphDestroy(graph);
      throw;
    }
  }
  APL_CUDA(cudaStreamEndCapture(st_, &graph));
  cudaError_t ge = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  APL_CUDA(ge);
  struct Guard {
    cudaGraphExec_t e;
    ~Guard() { cudaGraphExecDestroy(e); }
  } guard{exec};
  int live = 1;
  for (long long done = 0; done < maxall && live > 0; done += G) {
    APL_CUDA(cudaGraphLaunch(exec, st_));
    add_launches(G * launches_per_iter_);
    APL_CUDA(cudaMemcpyAsync(&live, live_count_.p, sizeof(int), cudaMemcpyDeviceToHost, st_));
    APL_CUDA(cudaStreamSynchronize(st_));
  }
  APL_CUDA(cudaMemcpyAsync(hpairs.data(), pairs_.p, npairs * sizeof(BPair), cudaMemcpyDeviceToHost, st_));
  APL_CUDA(cudaStreamSynchronize(st_));
  for (int p = 0; p < np; ++p)
    for (int r = 0; r < R_; ++r) {
      iters[(size_t)p * R_ + r] = hpairs[(size_t)p * RS_ + r].it;
      reasons[(size_t)p * R_ + r] = hpairs[(size_t)p * RS_ + r].reason;
    }
}

void BatchEngine::ne_residual(const std::vector<char>& mask, std::vector<double>& ne) {
  const int np = nprob();
  const size_t npairs = (size_t)np * RS_;
  ne.assign((size_t)np * R_, 0.0);
  std::vector<int> plive(1 + np, 0);
  for (int p = 0; p < np; ++p) {
    int cnt = 0;
    for (int r = 0; r < R_; ++r) cnt += mask[(size_t)p * R_ + r] ? 1 : 0;
    const int want = cnt > 0 ? 1 : 0;
    if (want != hp_[p].active) items_dirty_ = true;
    hp_[p].active = want;
    plive[1 + p] = cnt;
  }
  if (items_dirty_) build_items();
  upload_probs();
  APL_CUDA(cudaMemcpyAsync(live_count_.p, plive.data(), plive.size() * sizeof(int), cudaMemcpyHostToDevice, st_));
  launch_residual(false);
  launch_gtr(false);
  DBuf<double> out;
  out.alloc(npairs, st_);
  ne_kernel<<<(unsigned)cdiv((int64_t)npairs, 128), 128, 0, st_>>>((int)npairs, RS_, dp_.p,
                                                                  ne_part_.p, out.p);
  APL_LAUNCH_CHECK();
  std::vector<double> h(npairs);
  APL_CUDA(cudaMemcpyAsync(h.data(), out.p, npairs * sizeof(double), cudaMemcpyDeviceToHost, st_));
  APL_CUDA(cudaStreamSynchronize(st_));
  for (int p = 0; p < np; ++p)
    for (int r = 0; r < R_; ++r) {
      const size_t er = (size_t)p * R_ + r, e = (size_t)p * RS_ + r;
      if (!mask[er]) continue;
      const double ref = norm_ref_[e];
      ne[er] = ref > 0.0 ? h[e] / ref : h[e];
    }
}

void BatchEngine::autotune() {
  // time the dense A pass (rows per warp) and A^T pass (columns per lane) candidates on
  // this batch with every problem active and zero coefficients (outputs stay zero)
  const int np = nprob();
  for (int p = 0; p < np; ++p) hp_[p].active = 1;
  std::vector<int> plive(1 + np, 1);
  std::vector<BPair> hpairs((size_t)np * RS_);
  for (auto& c : hpairs) c = BPair{};
  APL_CUDA(cudaMemcpyAsync(pairs_.p, hpairs.data(), hpairs.size() * sizeof(BPair), cudaMemcpyHostToDevice, st_));
  APL_CUDA(cudaMemcpyAsync(live_count_.p, plive.data(), plive.size() * sizeof(int), cudaMemcpyHostToDevice, st_));
  cudaEvent_t e0, e1;
  APL_CUDA(cudaEventCreate(&e0));
  APL_CUDA(cudaEventCreate(&e1));
  auto time_it = [&](auto&& f) {
    f();
    APL_CUDA(cudaEventRecord(e0, st_));
    for (int k = 0; k < 3; ++k) f();
    APL_CUDA(cudaEventRecord(e1, st_));
    APL_CUDA(cudaEventSynchronize(e1));
    float ms = 0;
    APL_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    return ms;
  };
  float best = INFINITY;
  int best_rw = rw_;
  for (int rw : {2, 4}) {
    build_items();
    upload_probs();
    const float ms = time_it([&]() { launch_gn(it_apass_, n_apass_, rw); });
    if (ms < best) { best = ms; best_rw = rw; }
  }
  rw_ = best_rw;
  best = INFINITY;
  int best_cw = cw_;
  for (int cw : {1, 2, 4}) {
    cw_ = cw;
    build_items();
    upload_probs();
    const float ms = time_it([&]() { launch_gt(it_gta_, n_gta_, cw); });
    if (ms < best) { best = ms; best_cw = cw; }
  }
  cw_ = best_cw;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  for (int p = 0; p < np; ++p) hp_[p].active = 0;
  items_dirty_ = true;
}

}  // namespace apl
