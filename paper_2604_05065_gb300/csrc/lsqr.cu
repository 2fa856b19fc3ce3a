// LSQR phase kernels.  One iteration is
//   K1  u' = A z - alpha u (rows of A) and u'_bot = delta z - alpha u_bot, beta = ||u'||
//   K2  g = (A^T u'_top + delta u'_bot) / beta, plus the deferred x/d update of the
//       previous iteration; without a preconditioner also v' = g - beta v, alpha = ||v'||
//   K3  t = Vhat^T g                    (preconditioned only)
//   K4  v' = g + Vhat (coef t) - beta v, z' = g + Vhat (coef2 t) - beta z, alpha = ||v'||
// Vectors v', z', u' are stored unnormalised with their scale (1/alpha, 1/beta) kept
// in the device-resident control block, so no extra pass rescales them.  The last
// block of each reducing kernel finishes the scalar recurrences (Givens rotation,
// Paige-Saunders and dynamic stopping tests) on the device.
//
// Products with A come in three modes:
//   0  FP64 products and sums (FP32-stored values are promoted exactly);
//   1  FP32 products and FP32 sums per thread (FP64 across threads);
//   2  compensated FP32: each operand vector is split into FP32 hi + lo parts once per
//      iteration; a * hi is made exact by an FMA residual, the running sum is kept as an
//      unevaluated pair (Knuth's TwoSum), so the result is accurate to about 2^-44
//      relative to sum |a_i z_i| while every instruction is an FP32 one.
#include <cstddef>
#include <mutex>
#include <vector>

#include "../../include/aplicur.h"
#include "lsqr.cuh"
#include "apass.cuh"
#include "df32.cuh"

namespace apl {

namespace {

constexpr int NT = 256;

__device__ __forceinline__ void split(double v, float* hi, float* lo, int64_t i) {
  const float h = __double2float_rn(v);
  hi[i] = h;
  lo[i] = __double2float_rn(v - (double)h);
}

__device__ __forceinline__ bool dyn_stop(double phibar_prev, double phibar, double rate1,
                                         double nu, double sig_ell) {
  if (!isfinite(nu)) return false;
  if (phibar_prev - phibar < sig_ell) return true;
  if (phibar <= 0.0) return false;
  const double rate = log(phibar_prev / phibar);
  if (rate <= 0.0) return true;
  return rate1 / rate > nu;
}

__device__ void finalize_alpha(LsqrCtl* c, double sumsq, int init) {
  const double alpha = sqrt(sumsq);
  if (init) {
    c->alpha = alpha;
    c->rhobar = alpha;
    c->zs = alpha > 0.0 ? 1.0 / alpha : 0.0;
    c->pending = 1;
    c->init = 0;
    c->it = 0;
    c->arnorm0 = alpha * c->beta1;
    if (alpha == 0.0) { c->done = 1; c->reason = R_EXACT; }
    return;
  }
  const double beta = c->beta;
  const double rho = sqrt(c->rhobar * c->rhobar + beta * beta);
  const double cc = c->rhobar / rho;
  const double s = beta / rho;
  const double theta = s * alpha;
  c->rhobar = -cc * alpha;
  const double phi = cc * c->phibar;
  const double phibar_prev = c->phibar;
  const double phibar = s * c->phibar;
  c->phibar = phibar;
  c->phibar_prev = phibar_prev;
  c->xc = phi / rho;
  c->dc = theta / rho;
  c->pending = 2;
  c->alpha = alpha;
  c->zs = alpha > 0.0 ? 1.0 / alpha : 0.0;
  c->cabs = fabs(cc);
  const int it = ++c->it;
  if (it == 1) c->rate1 = phibar > 0.0 ? log(phibar_prev / phibar) : INFINITY;
  int reason = R_NONE;
  if (c->fixed_len >= 0) {
    if (it >= c->fixed_len) reason = R_REPLAY;
  } else if (beta == 0.0 || alpha == 0.0) {
    reason = R_EXACT;
  } else if (alpha * fabs(cc) <= c->eps * sqrt(c->anorm2)) {
    reason = R_PS2;
  } else if (phibar <= c->eps * c->beta1) {
    reason = R_PS1;
  } else if (c->inner > 0.0 && phibar * alpha * fabs(cc) <= c->inner * c->arnorm0) {
    reason = R_INNER;
  } else if (dyn_stop(phibar_prev, phibar, c->rate1, c->nu, c->sig_ell)) {
    reason = R_DYNAMIC;
  } else if (c->tol > 0.0 && it >= c->next_check &&
             c->normP * phibar * alpha * fabs(cc) / c->norm_ref <= c->tol) {
    reason = R_CHECK;
  } else if ((long long)it >= c->maxit) {
    reason = R_MAXIT;
  }
  if (reason != R_NONE) { c->done = 1; c->reason = reason; }
}

// ---- per-element product helpers for the three modes ----------------------------------

template <int MODE>
struct Acc;
template <>
struct Acc<0> {
  double v = 0.0;
  __device__ __forceinline__ void add(double a, double x, float, float) { v = fma(a, x, v); }
  __device__ __forceinline__ double get() const { return v; }
};
template <>
struct Acc<1> {
  float v = 0.f;
  __device__ __forceinline__ void add(float a, double, float h, float) { v = fmaf(a, h, v); }
  __device__ __forceinline__ double get() const { return (double)v; }
};
template <>
struct Acc<2> {
  DF v{0.f, 0.f};
  __device__ __forceinline__ void add(float a, double, float h, float l) { df_fma(v, a, h, l); }
  __device__ __forceinline__ double get() const { return df_val(v); }
};

// ---- K1: rows of A, K1_RPW rows per warp ----------------------------------------------

// Rows per warp of the dense A z pass.  The grid gives every warp one group of rows
// (while the rows fit in one resident wave: FP32 A is held to 48 registers, five blocks
// per SM), so no warp streams a second group while the others idle, and each load of z
// serves all rows of the group.
constexpr int K1_RPW = 4;

template <typename TA, int MODE, bool VEC>
__global__ void __launch_bounds__(NT, sizeof(TA) == 4 ? 5 : 1) k1_dense(int64_t m, int64_t n, int64_t ld,
                                               const TA* __restrict__ A,
                                               const double* __restrict__ z,
                                               const float* __restrict__ zh,
                                               const float* __restrict__ zl,
                                               double* __restrict__ u, float* __restrict__ uh,
                                               float* __restrict__ ul, LsqrCtl* ctl,
                                               double* __restrict__ red, int init) {
  __shared__ double sh[NT / 32];
  if (ctl->done) return;
  const double ca = init ? -1.0 : ctl->zs;
  const double cu = init ? 1.0 : -ctl->alpha * ctl->us;
  const double delta = ctl->delta;
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * NT + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * NT) >> 5;
  // init == 2: z is known to be zero, so every row product is zero and A is not read
  const int64_t np = init == 2 ? 0 : n;
  double ss = 0.0;
  for (int64_t i0 = (int64_t)K1_RPW * warp; i0 < m; i0 += (int64_t)K1_RPW * nwarps) {
    const int nr = (int)(m - i0 < K1_RPW ? m - i0 : K1_RPW);
    const TA* ar[K1_RPW];
#pragma unroll
    for (int r = 0; r < K1_RPW; ++r) ar[r] = A + (i0 + (r < nr ? r : nr - 1)) * ld;
    Acc<MODE> s[K1_RPW];
    int64_t jt = 0;
    if constexpr (VEC && MODE != 0 && sizeof(TA) == 4) {
      const int64_t n4 = np >> 2;
      const float4* hv = reinterpret_cast<const float4*>(zh);
      const float4* lv = reinterpret_cast<const float4*>(zl);
      // one stretch of every row per pass, all loads issued first: 2 KB of A in flight per
      // warp, and each z load serves K1_RPW rows
#pragma unroll 1
      for (int64_t q = lane; q < n4; q += 32) {
        float4 x[K1_RPW];
#pragma unroll
        for (int r = 0; r < K1_RPW; ++r) x[r] = __ldcs(reinterpret_cast<const float4*>(ar[r]) + q);
        const float4 h = hv[q];
        const float4 l = MODE == 2 ? lv[q] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int r = 0; r < K1_RPW; ++r) {
          s[r].add(x[r].x, 0.0, h.x, l.x);
          s[r].add(x[r].y, 0.0, h.y, l.y);
          s[r].add(x[r].z, 0.0, h.z, l.z);
          s[r].add(x[r].w, 0.0, h.w, l.w);
        }
      }
      jt = n4 << 2;
    }
    for (int64_t j = jt + lane; j < np; j += 32) {
      if constexpr (MODE == 0) {
        const double zj = z[j];
#pragma unroll
        for (int r = 0; r < K1_RPW; ++r) s[r].add(widen(ar[r][j]), zj, 0.f, 0.f);
      } else {
        const float h = zh[j];
        const float l = MODE == 2 ? zl[j] : 0.f;
#pragma unroll
        for (int r = 0; r < K1_RPW; ++r) s[r].add((float)ar[r][j], 0.0, h, l);
      }
    }
    double d[K1_RPW];
#pragma unroll
    for (int r = 0; r < K1_RPW; ++r) d[r] = warp_sum(s[r].get());
    if (lane == 0) {
#pragma unroll
      for (int r = 0; r < K1_RPW; ++r) {
        if (r >= nr) break;
        const double v = ca * d[r] + cu * u[i0 + r];
        u[i0 + r] = v;
        ss += v * v;
        if (uh) split(v, uh, ul, i0 + r);
      }
    }
  }
  for (int64_t j = (int64_t)blockIdx.x * NT + threadIdx.x; j < n; j += (int64_t)gridDim.x * NT) {
    const double val = ca * delta * z[j] + cu * u[m + j];
    u[m + j] = val;
    ss += val * val;
  }
  const double b = block_sum(ss, sh);
  if (threadIdx.x == 0) red[blockIdx.x] = b;
  if (!last_block_done(&ctl->counter[0])) return;
  const double tot = block_sum_partials(red, gridDim.x, sh);
  if (threadIdx.x == 0) finalize_beta(ctl, tot, init);
}

template <typename TA, int MODE>
__global__ void __launch_bounds__(NT) k1_csr(int64_t m, int64_t n, const int* __restrict__ rowptr,
                                             const int* __restrict__ colidx,
                                             const TA* __restrict__ vals,
                                             const double* __restrict__ z,
                                             const float* __restrict__ zh,
                                             const float* __restrict__ zl,
                                             double* __restrict__ u, float* __restrict__ uh,
                                             float* __restrict__ ul, LsqrCtl* ctl,
                                             double* __restrict__ red, int init) {
  __shared__ double sh[NT / 32];
  if (ctl->done) return;
  const double ca = init ? -1.0 : ctl->zs;
  const double cu = init ? 1.0 : -ctl->alpha * ctl->us;
  const double delta = ctl->delta;
  double ss = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x; i < m + n;
       i += (int64_t)gridDim.x * NT) {
    double val;
    if (i < m) {
      Acc<MODE> acc;
      // init == 2: z is known to be zero (no product)
      const int e0 = rowptr[i];
      const int e1 = init == 2 ? e0 : rowptr[i + 1];
      for (int e = e0; e < e1; ++e) {
        const int c = colidx[e];
        if constexpr (MODE == 0) acc.add(widen(vals[e]), z[c], 0.f, 0.f);
        else acc.add((float)vals[e], 0.0, zh[c], MODE == 2 ? zl[c] : 0.f);
      }
      val = ca * acc.get() + cu * u[i];
      if (uh) split(val, uh, ul, i);
    } else {
      val = ca * delta * z[i - m] + cu * u[i];
    }
    u[i] = val;
    ss += val * val;
  }
  const double b = block_sum(ss, sh);
  if (threadIdx.x == 0) red[blockIdx.x] = b;
  if (!last_block_done(&ctl->counter[0])) return;
  const double tot = block_sum_partials(red, gridDim.x, sh);
  if (threadIdx.x == 0) finalize_beta(ctl, tot, init);
}

// ---- K2 -------------------------------------------------------------------------------

// Common per-column tail: g_j given; deferred x/d update; optionally v' = g - beta v.
// v and z are the same buffer when there is no preconditioner: no __restrict__ here.
__device__ __forceinline__ double k2_tail(int64_t j, double gj, const LsqrCtl* c, int init,
                                          int fused, double* g, double* v, double* z, double* d,
                                          double* x, float* zh, float* zl) {
  const int pend = c->pending;
  const double zs = c->zs;
  if (pend == 1) {
    d[j] = z[j] * zs;
  } else if (pend == 2) {
    const double dj = d[j];
    x[j] += c->xc * dj;
    d[j] = z[j] * zs - c->dc * dj;
  } else if (pend == 3) {
    d[j] = z[j] * zs - c->dc * d[j];
  }
  if (fused) {
    const double vn = init ? gj : gj - c->beta * (v[j] * zs);
    v[j] = vn;
    if (zh) split(vn, zh, zl, j);
    return vn * vn;
  }
  g[j] = gj;
  return 0.0;
}

template <typename TA, int MODE>
__global__ void __launch_bounds__(NT) k2_csr(int64_t m, int64_t n, const int* __restrict__ colptr,
                                             const int* __restrict__ rowidx,
                                             const TA* __restrict__ cvals,
                                             const double* __restrict__ u,
                                             const float* __restrict__ uh,
                                             const float* __restrict__ ul, double* g, double* v,
                                             double* z, double* d, double* x, float* zh, float* zl,
                                             LsqrCtl* ctl, double* __restrict__ red, int init,
                                             int fused) {
  __shared__ double sh[NT / 32];
  if (ctl->done) return;
  const double us = ctl->us, delta = ctl->delta;
  double ss = 0.0;
  for (int64_t j = (int64_t)blockIdx.x * NT + threadIdx.x; j < n; j += (int64_t)gridDim.x * NT) {
    Acc<MODE> acc;
    const int e1 = colptr[j + 1];
    for (int e = colptr[j]; e < e1; ++e) {
      const int r = rowidx[e];
      if constexpr (MODE == 0) acc.add(widen(cvals[e]), u[r], 0.f, 0.f);
      else acc.add((float)cvals[e], 0.0, uh[r], MODE == 2 ? ul[r] : 0.f);
    }
    const double gj = us * (acc.get() + delta * u[m + j]);
    ss += k2_tail(j, gj, ctl, init, fused, g, v, z, d, x, zh, zl);
  }
  if (!fused) return;
  const double b = block_sum(ss, sh);
  if (threadIdx.x == 0) red[blockIdx.x] = b;
  if (!last_block_done(&ctl->counter[0])) return;
  const double tot = block_sum_partials(red, gridDim.x, sh);
  if (threadIdx.x == 0) finalize_alpha(ctl, tot, init);
}

// Dense A^T u: per (column block, row chunk) partial sums; four columns per thread in
// the vector path.
template <typename TA, int MODE, bool VEC>
__global__ void __launch_bounds__(NT) k2a_dense(int64_t m, int64_t n, int64_t ld,
                                                const TA* __restrict__ A,
                                                const double* __restrict__ u,
                                                const float* __restrict__ uh,
                                                const float* __restrict__ ul,
                                                double* __restrict__ part, int64_t rows_per,
                                                const LsqrCtl* ctl) {
  if (ctl && ctl->done) return;
  const int64_t t = (int64_t)blockIdx.x * NT + threadIdx.x;
  const int64_t r0 = (int64_t)blockIdx.y * rows_per;
  const int64_t r1 = r0 + rows_per < m ? r0 + rows_per : m;
  double* out = part + (int64_t)blockIdx.y * n;
  if constexpr (VEC && MODE != 0 && sizeof(TA) == 4) {
    const int64_t j = 4 * t;
    if (j + 3 < n) {
      Acc<MODE> a0, a1, a2, a3;
      int64_t i = r0;
      // four rows per pass with their loads issued first (same summation order)
      for (; i + 3 < r1; i += 4) {
        float4 x[4];
        float h[4], l[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          x[u] = __ldcs(reinterpret_cast<const float4*>(A + (i + u) * ld + j));
          h[u] = uh[i + u];
          l[u] = MODE == 2 ? ul[i + u] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          a0.add(x[u].x, 0.0, h[u], l[u]);
          a1.add(x[u].y, 0.0, h[u], l[u]);
          a2.add(x[u].z, 0.0, h[u], l[u]);
          a3.add(x[u].w, 0.0, h[u], l[u]);
        }
      }
      for (; i < r1; ++i) {
        const float4 x = __ldcs(reinterpret_cast<const float4*>(A + i * ld + j));
        const float h = uh[i];
        const float l = MODE == 2 ? ul[i] : 0.f;
        a0.add(x.x, 0.0, h, l);
        a1.add(x.y, 0.0, h, l);
        a2.add(x.z, 0.0, h, l);
        a3.add(x.w, 0.0, h, l);
      }
      out[j] = a0.get();
      out[j + 1] = a1.get();
      out[j + 2] = a2.get();
      out[j + 3] = a3.get();
    } else {
      for (int64_t jj = j; jj < n; ++jj) {
        Acc<MODE> a;
        for (int64_t i = r0; i < r1; ++i)
          a.add((float)A[i * ld + jj], 0.0, uh[i], MODE == 2 ? ul[i] : 0.f);
        out[jj] = a.get();
      }
    }
  } else {
    const int64_t j = t;
    if (j >= n) return;
    Acc<MODE> a;
    for (int64_t i = r0; i < r1; ++i) {
      if constexpr (MODE == 0) a.add(widen(A[i * ld + j]), u[i], 0.f, 0.f);
      else a.add((float)A[i * ld + j], 0.0, uh[i], MODE == 2 ? ul[i] : 0.f);
    }
    out[j] = a.get();
  }
}

__global__ void __launch_bounds__(NT) k2b_dense(int64_t m, int64_t n, int rchunks,
                                                const double* __restrict__ part,
                                                const double* __restrict__ u, double* g,
                                                double* v, double* z, double* d, double* x,
                                                float* zh, float* zl, LsqrCtl* ctl,
                                                double* __restrict__ red, int init, int fused) {
  __shared__ double sh[NT / 32];
  if (ctl->done) return;
  const double us = ctl->us, delta = ctl->delta;
  double ss = 0.0;
  for (int64_t j = (int64_t)blockIdx.x * NT + threadIdx.x; j < n; j += (int64_t)gridDim.x * NT) {
    double acc = 0.0;
    for (int c = 0; c < rchunks; ++c) acc += part[(int64_t)c * n + j];
    const double gj = us * (acc + delta * u[m + j]);
    ss += k2_tail(j, gj, ctl, init, fused, g, v, z, d, x, zh, zl);
  }
  if (!fused) return;
  const double b = block_sum(ss, sh);
  if (threadIdx.x == 0) red[blockIdx.x] = b;
  if (!last_block_done(&ctl->counter[0])) return;
  const double tot = block_sum_partials(red, gridDim.x, sh);
  if (threadIdx.x == 0) finalize_alpha(ctl, tot, init);
}

// ---- preconditioner passes (FP64, Vhat = Q_R V_M implicit) -----------------------------

// Partial q1 = Q^T w: block (k, c) sums column k of Q over the row chunk c (QT_CHUNK
// rows), so ell x chunks blocks share the pass; pre_qsum adds the chunks in order.
constexpr int QT_CHUNK = 2048;
__global__ void __launch_bounds__(NT) pre_qt(int64_t n, int ell, int64_t ldq,
                                             const double* __restrict__ Q,
                                             const double* __restrict__ w,
                                             double* __restrict__ qpart, const LsqrCtl* ctl) {
  __shared__ double sh[NT / 32];
  if (ctl && ctl->done) return;
  const int64_t k = blockIdx.x, c = blockIdx.y;
  const double* qk = Q + k * ldq;
  const int64_t i1 = min(n, (c + 1) * (int64_t)QT_CHUNK);
  double s = 0.0;
  for (int64_t i = c * QT_CHUNK + threadIdx.x; i < i1; i += NT) s = fma(qk[i], w[i], s);
  s = block_sum(s, sh);
  if (threadIdx.x == 0) qpart[k * gridDim.y + c] = s;
}

__global__ void pre_qsum(int ell, int nch, const double* __restrict__ qpart,
                         double* __restrict__ q1, const LsqrCtl* ctl) {
  if (ctl && ctl->done) return;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= ell) return;
  double s = 0.0;
  for (int c = 0; c < nch; ++c) s += qpart[(int64_t)k * nch + c];
  q1[k] = s;
}

// ct = coef (V_M^T q1), c2t = coef2 (V_M^T q1): one warp per column of V_M.
__global__ void __launch_bounds__(NT) pre_vt(int ell, const double* __restrict__ VM,
                                             const double* __restrict__ q1,
                                             const double* __restrict__ coef,
                                             const double* __restrict__ coef2,
                                             double* __restrict__ ct, double* __restrict__ c2t,
                                             const LsqrCtl* ctl) {
  if (ctl && ctl->done) return;
  const int lane = threadIdx.x & 31;
  const int64_t k = ((int64_t)blockIdx.x * NT + threadIdx.x) >> 5;
  if (k >= ell) return;
  const double* vk = VM + k * (int64_t)ell;
  double s = 0.0;
  for (int i = lane; i < ell; i += 32) s = fma(vk[i], q1[i], s);
  s = warp_sum(s);
  if (lane == 0) {
    ct[k] = coef[k] * s;
    if (c2t) c2t[k] = coef2[k] * s;
  }
}

// q3 = V_M ct, q3b = V_M c2t: a block takes 32 rows (lanes, coalesced column reads of the
// column-major V_M) and its 8 warps split the k range; the partial sums meet in shared
// memory in warp order.
// SVD-free variant (sf = 1, 2; VM holds M^{-1}, sighat scales, q1 = Q_R^T w):
//  sf = 1: ct = sighat M^{-T} q1 (from pre_vt); q3 = ct - q1 and q3b = sighat M^{-1} ct - q1,
//          so the expansion gives P^{-T} w and P^{-1} P^{-T} w;
//  sf = 2: ct = q1; q3 = sighat M^{-1} q1 - q1, so the expansion gives P^{-1} w.
__global__ void __launch_bounds__(NT) pre_v(int ell, const double* __restrict__ VM,
                                            const double* __restrict__ ct,
                                            const double* __restrict__ c2t,
                                            double* __restrict__ q3, double* __restrict__ q3b,
                                            const double* __restrict__ q1, double sighat,
                                            int sf, const LsqrCtl* ctl) {
  __shared__ double r1[NT / 32][32], r2[NT / 32][32];
  if (ctl && ctl->done) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i = blockIdx.x * 32 + lane;
  double s1 = 0.0, s2 = 0.0;
  if (i < ell) {
    for (int k = warp; k < ell; k += NT / 32) {
      const double v = VM[i + (int64_t)k * ell];
      s1 = fma(v, ct[k], s1);
      if (q3b && c2t) s2 = fma(v, c2t[k], s2);
    }
  }
  r1[warp][lane] = s1;
  r2[warp][lane] = s2;
  __syncthreads();
  if (warp != 0 || i >= ell) return;
  double t1 = 0.0, t2 = 0.0;
  for (int w = 0; w < NT / 32; ++w) { t1 += r1[w][lane]; t2 += r2[w][lane]; }
  if (sf == 1) {
    q3[i] = ct[i] - q1[i];
    q3b[i] = sighat * t1 - q1[i];
  } else if (sf == 2) {
    q3[i] = sighat * t1 - q1[i];
  } else {
    q3[i] = t1;
    if (q3b) q3b[i] = t2;
  }
}

// out1 = w + Q q3, out2 = w + Q q3b.  A block takes 32 rows per pass (lanes: coalesced
// reads of the column-major Q) and its 8 warps split the k range; warp 0 combines the
// partial sums in warp order and writes the row.  In the LSQR phase also subtracts beta v /
// beta z, writes the FP32 split of z' and reduces ||v'||^2.
__global__ void __launch_bounds__(NT) pre_expand(int64_t n, int ell, int64_t ldq,
                                                 const double* __restrict__ Q,
                                                 const double* __restrict__ q3,
                                                 const double* __restrict__ q3b,
                                                 const double* __restrict__ w, double* out1,
                                                 double* out2, float* zh, float* zl,
                                                 LsqrCtl* ctl, double* __restrict__ red,
                                                 int init) {
  __shared__ double sh[NT / 32];
  __shared__ double r1[NT / 32][32], r2[NT / 32][32];
  if (ctl && ctl->done) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double beta = 0.0, zs = 0.0;
  if (ctl && !init) { beta = ctl->beta; zs = ctl->zs; }
  double ss = 0.0;
  for (int64_t r0 = (int64_t)blockIdx.x * 32; r0 < n; r0 += (int64_t)gridDim.x * 32) {
    const int64_t i = r0 + lane;
    double s1 = 0.0, s2 = 0.0;
    if (i < n) {
      for (int k = warp; k < ell; k += NT / 32) {
        const double q = Q[i + k * ldq];
        s1 = fma(q, q3[k], s1);
        if (out2) s2 = fma(q, q3b[k], s2);
      }
    }
    r1[warp][lane] = s1;
    r2[warp][lane] = s2;
    __syncthreads();
    if (warp == 0 && i < n) {
      double t1 = 0.0, t2 = 0.0;
      for (int v = 0; v < NT / 32; ++v) { t1 += r1[v][lane]; t2 += r2[v][lane]; }
      const double wi = w[i];
      double o1 = wi + t1;
      if (ctl && !init) o1 -= beta * (out1[i] * zs);
      out1[i] = o1;
      if (out2) {
        double o2 = wi + t2;
        if (ctl && !init) o2 -= beta * (out2[i] * zs);
        out2[i] = o2;
        if (zh) split(o2, zh, zl, i);
      }
      ss += o1 * o1;
    }
    __syncthreads();
  }
  if (!ctl) return;
  const double b = block_sum(ss, sh);
  if (threadIdx.x == 0) red[blockIdx.x] = b;
  if (!last_block_done(&ctl->counter[0])) return;
  const double tot = block_sum_partials(red, gridDim.x, sh);
  if (threadIdx.x == 0) finalize_alpha(ctl, tot, init);
}

// ---- misc -----------------------------------------------------------------------------

__global__ void flush_x_kernel(int64_t n, double* x, const double* d, const LsqrCtl* ctl) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) x[j] += ctl->xc * d[j];
}

__global__ void split_kernel(int64_t n, const double* v, float* hi, float* lo) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) split(v[i], hi, lo, i);
}

template <typename TA, int MODE>
__global__ void __launch_bounds__(NT) mv_dense_rows(int64_t m, int64_t n, int64_t ld,
                                                    const TA* __restrict__ A,
                                                    const double* __restrict__ x,
                                                    const float* __restrict__ xh,
                                                    const float* __restrict__ xl, double* y,
                                                    double alpha, double beta) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * NT + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * NT) >> 5;
  for (int64_t i = warp; i < m; i += nwarps) {
    const TA* a = A + i * ld;
    Acc<MODE> acc;
    for (int64_t j = lane; j < n; j += 32) {
      if constexpr (MODE == 0) acc.add(widen(a[j]), x[j], 0.f, 0.f);
      else acc.add((float)a[j], 0.0, xh[j], MODE == 2 ? xl[j] : 0.f);
    }
    const double s = warp_sum(acc.get());
    if (lane == 0) y[i] = beta == 0.0 ? alpha * s : alpha * s + beta * y[i];
  }
}

template <typename TA, int MODE>
__global__ void mv_csr_rows(int64_t m, const int* __restrict__ rowptr,
                            const int* __restrict__ colidx, const TA* __restrict__ vals,
                            const double* __restrict__ x, const float* __restrict__ xh,
                            const float* __restrict__ xl, double* y, double alpha, double beta) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  Acc<MODE> acc;
  for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
    const int c = colidx[e];
    if constexpr (MODE == 0) acc.add(widen(vals[e]), x[c], 0.f, 0.f);
    else acc.add((float)vals[e], 0.0, xh[c], MODE == 2 ? xl[c] : 0.f);
  }
  const double s = acc.get();
  y[i] = beta == 0.0 ? alpha * s : alpha * s + beta * y[i];
}

template <typename TA, int MODE>
__global__ void mv_csc_cols(int64_t n, const int* __restrict__ colptr,
                            const int* __restrict__ rowidx, const TA* __restrict__ cvals,
                            const double* __restrict__ x, const float* __restrict__ xh,
                            const float* __restrict__ xl, double* y) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  Acc<MODE> acc;
  for (int e = colptr[j]; e < colptr[j + 1]; ++e) {
    const int r = rowidx[e];
    if constexpr (MODE == 0) acc.add(widen(cvals[e]), x[r], 0.f, 0.f);
    else acc.add((float)cvals[e], 0.0, xh[r], MODE == 2 ? xl[r] : 0.f);
  }
  y[j] = acc.get();
}

__global__ void colsum_kernel(int64_t n, int rchunks, const double* part, double* y) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double acc = 0.0;
  for (int c = 0; c < rchunks; ++c) acc += part[(int64_t)c * n + j];
  y[j] = acc;
}

// q = q + delta * (rb - delta x)  (rb NULL = 0)
__global__ void ne_tail_kernel(int64_t n, double* q, const double* rb, const double* x,
                               double delta) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double r = (rb ? rb[j] : 0.0) - delta * x[j];
  q[j] += delta * r;
}

__global__ void scale_to_kernel(int64_t n, const double* v, double a, double* out) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) out[j] = a * v[j];
}

__global__ void norm2_kernel(int64_t n, const double* v, double* red, double* out,
                             unsigned int* counter) {
  __shared__ double sh[NT / 32];
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x; i < n; i += (int64_t)gridDim.x * NT)
    s += v[i] * v[i];
  const double b = block_sum(s, sh);
  if (threadIdx.x == 0) red[blockIdx.x] = b;
  if (!last_block_done(counter)) return;
  const double tot = block_sum_partials(red, gridDim.x, sh);
  if (threadIdx.x == 0) *out = sqrt(tot);
}

inline int sm_blocks() { return 152 * 8; }

// Launch helpers dispatching (format, dtype, mode, vector) to template instances.
template <int MODE>
void launch_k1_mode(cudaStream_t st, const MatView& A, bool vec, int blocks, const double* z,
                    const float* zh, const float* zl, double* u, float* uh, float* ul, LsqrCtl* c,
                    double* red, int init) {
  if (A.fmt == 0) {
    if (A.dtype == 0) {
      k1_dense<double, 0, false><<<blocks, NT, 0, st>>>(A.m, A.n, A.ld, (const double*)A.vals, z,
                                                        zh, zl, u, uh, ul, c, red, init);
    } else if (vec) {
      k1_dense<float, MODE, true><<<blocks, NT, 0, st>>>(A.m, A.n, A.ld, (const float*)A.vals, z,
                                                         zh, zl, u, uh, ul, c, red, init);
    } else {
      k1_dense<float, MODE, false><<<blocks, NT, 0, st>>>(A.m, A.n, A.ld, (const float*)A.vals, z,
                                                          zh, zl, u, uh, ul, c, red, init);
    }
  } else {
    if (A.dtype == 0)
      k1_csr<double, 0><<<blocks, NT, 0, st>>>(A.m, A.n, A.rowptr, A.colidx,
                                               (const double*)A.vals, z, zh, zl, u, uh, ul, c,
                                               red, init);
    else
      k1_csr<float, MODE><<<blocks, NT, 0, st>>>(A.m, A.n, A.rowptr, A.colidx,
                                                 (const float*)A.vals, z, zh, zl, u, uh, ul, c,
                                                 red, init);
  }
}

template <int MODE>
void launch_k2_mode(cudaStream_t st, const MatView& A, bool vec, int blocks, int rchunks,
                    double* part, const double* u, const float* uh, const float* ul, double* g,
                    double* v, double* z, double* d, double* x, float* zh, float* zl, LsqrCtl* c,
                    double* red, int init, int fused) {
  if (A.fmt == 0) {
    const int64_t rows_per = cdiv(A.m, rchunks);
    if (A.dtype == 0) {
      dim3 grid((unsigned)cdiv(A.n, NT), (unsigned)rchunks);
      k2a_dense<double, 0, false><<<grid, NT, 0, st>>>(A.m, A.n, A.ld, (const double*)A.vals, u,
                                                       uh, ul, part, rows_per, c);
    } else if (vec && MODE != 0) {
      dim3 grid((unsigned)cdiv(cdiv(A.n, 4), NT), (unsigned)rchunks);
      k2a_dense<float, MODE, true><<<grid, NT, 0, st>>>(A.m, A.n, A.ld, (const float*)A.vals, u,
                                                        uh, ul, part, rows_per, c);
    } else {
      dim3 grid((unsigned)cdiv(A.n, NT), (unsigned)rchunks);
      k2a_dense<float, MODE, false><<<grid, NT, 0, st>>>(A.m, A.n, A.ld, (const float*)A.vals, u,
                                                         uh, ul, part, rows_per, c);
    }
    APL_LAUNCH_CHECK();
    k2b_dense<<<blocks, NT, 0, st>>>(A.m, A.n, rchunks, part, u, g, v, z, d, x, zh, zl, c, red,
                                     init, fused);
  } else {
    if (A.dtype == 0)
      k2_csr<double, 0><<<blocks, NT, 0, st>>>(A.m, A.n, A.colptr, A.rowidx,
                                               (const double*)A.cvals, u, uh, ul, g, v, z, d, x,
                                               zh, zl, c, red, init, fused);
    else
      k2_csr<float, MODE><<<blocks, NT, 0, st>>>(A.m, A.n, A.colptr, A.rowidx,
                                                 (const float*)A.cvals, u, uh, ul, g, v, z, d, x,
                                                 zh, zl, c, red, init, fused);
  }
}

}  // namespace

// ======================================================================================

void LsqrEngine::setup(cudaStream_t st, const MatView& A, int mode, int graph_iters,
                       int dense_pass) {
  st_ = st;
  A_ = A;
  mode_ = A.dtype == 1 ? mode : 0;  // FP64-stored A always uses FP64 products
  graph_iters_ = graph_iters;
  m_ = A.m;
  n_ = A.n;
  ctl_.alloc(1, st);
  u_.alloc(m_ + n_, st);
  v_.alloc(n_, st);
  z_.alloc(n_, st);
  g_.alloc(n_, st);
  d_.alloc(n_, st);
  r_.alloc(m_, st);
  q_.alloc(n_, st);
  scal_.alloc(4, st);
  cnt_.alloc(1, st);
  cnt_.zero(st);
  if (mode_ != 0) {
    zh_.alloc(n_, st);
    zl_.alloc(n_, st);
    uh_.alloc(std::max(m_, n_), st);
    ul_.alloc(std::max(m_, n_), st);
  }
  vec_ = A.fmt == 0 && A.dtype == 1 && (A.ld % 4 == 0) &&
         ((reinterpret_cast<uintptr_t>(A.vals) & 15) == 0);
  if (A.fmt == 0) {
    k1_blocks_ = (int)std::min<int64_t>(cdiv(cdiv(m_, K1_RPW) * 32, NT), sm_blocks());
    const int64_t cb = vec_ ? cdiv(cdiv(n_, 4), NT) : cdiv(n_, NT);
    k2_rchunks_ = (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(4 * 152, cb), cdiv(m_, 32)));
    k2_blocks_ = (int)std::min<int64_t>(cdiv(n_, NT), sm_blocks());
    part_.alloc((size_t)k2_rchunks_ * n_, st);
  } else {
    // two rows per thread halve the FP64 block reductions (FP64 issues at 1/64 rate); the
    // CSC pass keeps one column per thread: splitting a column over lanes adds FP64
    // shuffle-reductions, which cost more than the latency they hide
    k1_blocks_ = (int)std::min<int64_t>(cdiv(m_ + n_, 2 * NT), sm_blocks());
    k2_blocks_ = (int)std::min<int64_t>(cdiv(n_, NT), sm_blocks());
  }
  red_cap_ = sm_blocks() + 64;
  red_.alloc(red_cap_, st);
  fused_ = FusedPlan();
  const bool want = dense_pass == 2 ? mode_ != 0 : (dense_pass == 0 && mode_ == 1);
  if (A.fmt == 0 && A.dtype == 1 && want) {
    fused_ = plan_fused_apass(m_, n_, A.ld, A.vals, mode_);
    if (fused_.ok && fused_.nclusters * fused_.C > red_cap_) fused_.ok = false;
  }
  if (fused_.ok) {
    part_.alloc((size_t)std::max<int64_t>(k2_rchunks_, fused_.nclusters) * n_, st);
    ferr_.alloc(1, st);
    ferr_.zero(st);
  }
}

void LsqrEngine::launch_fused(const double* z, bool fused_v) {
  launch_fused_apass(st_, fused_, mode_, A_, z, zh_.p, zl_.p, u_.p, ctl_.p, red_.p, part_.p,
                     ferr_.p);
  APL_CUDA(cudaGetLastError());
}

void LsqrEngine::launch_k1(bool init, const double* z) {
  // the residual that starts a phase is always formed with FP64 products (none when x0 is
  // known to be zero: the residual is then the right-hand side itself); in the FP32 modes
  // it also writes the split of u' for the following A^T pass
  float* uh = mode_ ? uh_.p : nullptr;
  float* ul = mode_ ? ul_.p : nullptr;
  const int md = init ? 0 : mode_;
  const int ik = init ? (x0_zero_ ? 2 : 1) : 0;
  if (md == 0)
    launch_k1_mode<0>(st_, A_, vec_, k1_blocks_, z, zh_.p, zl_.p, u_.p, uh, ul, ctl_.p, red_.p,
                      ik);
  else if (md == 1)
    launch_k1_mode<1>(st_, A_, vec_, k1_blocks_, z, zh_.p, zl_.p, u_.p, uh, ul, ctl_.p, red_.p,
                      ik);
  else
    launch_k1_mode<2>(st_, A_, vec_, k1_blocks_, z, zh_.p, zl_.p, u_.p, uh, ul, ctl_.p, red_.p,
                      ik);
  APL_LAUNCH_CHECK();
}

void LsqrEngine::launch_k2(bool init, bool fused) {
  // the stored z' lives in v_ when there is no preconditioner (z = v)
  double* zbuf = fused ? v_.p : z_.p;
  float* zh = (mode_ && fused) ? zh_.p : nullptr;
  float* zl = (mode_ && fused) ? zl_.p : nullptr;
  if (mode_ == 0)
    launch_k2_mode<0>(st_, A_, vec_, k2_blocks_, k2_rchunks_, part_.p, u_.p, uh_.p, ul_.p, g_.p,
                      v_.p, zbuf, d_.p, x_, zh, zl, ctl_.p, red_.p, init, fused);
  else if (mode_ == 1)
    launch_k2_mode<1>(st_, A_, vec_, k2_blocks_, k2_rchunks_, part_.p, u_.p, uh_.p, ul_.p, g_.p,
                      v_.p, zbuf, d_.p, x_, zh, zl, ctl_.p, red_.p, init, fused);
  else
    launch_k2_mode<2>(st_, A_, vec_, k2_blocks_, k2_rchunks_, part_.p, u_.p, uh_.p, ul_.p, g_.p,
                      v_.p, zbuf, d_.p, x_, zh, zl, ctl_.p, red_.p, init, fused);
  APL_LAUNCH_CHECK();
}

void LsqrEngine::launch_pre(const PrecondDev& P, const double* w, double* o1, double* o2,
                            bool in_phase, bool init) {
  const int ell = P.ell;
  q1_.alloc(ell, st_);
  ct_.alloc(ell, st_);
  c2t_.alloc(ell, st_);
  q3_.alloc(ell, st_);
  q3b_.alloc(ell, st_);
  const LsqrCtl* c = in_phase ? ctl_.p : nullptr;
  const unsigned wb = (unsigned)cdiv((int64_t)ell * 32, NT);
  const int nch = (int)cdiv(n_, (int64_t)QT_CHUNK);
  qpart_.alloc((size_t)ell * nch, st_);
  pre_qt<<<dim3((unsigned)ell, (unsigned)nch), NT, 0, st_>>>(n_, ell, P.ldq, P.Q, w, qpart_.p, c);
  APL_LAUNCH_CHECK();
  pre_qsum<<<(unsigned)cdiv(ell, NT), NT, 0, st_>>>(ell, nch, qpart_.p, q1_.p, c);
  APL_LAUNCH_CHECK();
  if (P.svdfree && o2) {
    // ct = sighat M^{-T} q1 (coef holds sighat), then q3, q3b for P^{-T} w, P^{-1} P^{-T} w
    pre_vt<<<wb, NT, 0, st_>>>(ell, P.VM, q1_.p, P.coef, nullptr, ct_.p, nullptr, c);
    APL_LAUNCH_CHECK();
    pre_v<<<(unsigned)cdiv(ell, 32), NT, 0, st_>>>(ell, P.VM, ct_.p, nullptr, q3_.p, q3b_.p,
                                                   q1_.p, P.sighat, 1, c);
  } else if (P.svdfree) {
    // P^{-1} w alone: q3 = sighat M^{-1} q1 - q1
    pre_v<<<(unsigned)cdiv(ell, 32), NT, 0, st_>>>(ell, P.VM, q1_.p, nullptr, q3_.p, nullptr,
                                                   q1_.p, P.sighat, 2, c);
  } else {
    pre_vt<<<wb, NT, 0, st_>>>(ell, P.VM, q1_.p, P.coef, P.coef2, ct_.p,
                               o2 ? c2t_.p : nullptr, c);
    APL_LAUNCH_CHECK();
    pre_v<<<(unsigned)cdiv(ell, 32), NT, 0, st_>>>(ell, P.VM, ct_.p, c2t_.p, q3_.p,
                                                   o2 ? q3b_.p : nullptr, nullptr, 0.0, 0, c);
  }
  APL_LAUNCH_CHECK();
  const int blocks = (int)std::min<int64_t>(cdiv(n_, 32), sm_blocks());
  LsqrCtl* cw = in_phase ? ctl_.p : nullptr;
  float* zh = (in_phase && mode_) ? zh_.p : nullptr;
  float* zl = (in_phase && mode_) ? zl_.p : nullptr;
  pre_expand<<<blocks, NT, 0, st_>>>(n_, ell, P.ldq, P.Q, q3_.p, q3b_.p, w, o1, o2, zh, zl, cw,
                                     red_.p, init);
  APL_LAUNCH_CHECK();
}

// Inside stream capture an event record only becomes a graph node when it is marked
// external; outside capture it is an ordinary record.
void LsqrEngine::record(int slot) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  APL_CUDA(cudaStreamIsCapturing(st_, &cs));
  if (cs == cudaStreamCaptureStatusActive)
    APL_CUDA(cudaEventRecordWithFlags(ev_[slot], st_, cudaEventRecordExternal));
  else
    APL_CUDA(cudaEventRecord(ev_[slot], st_));
}

void LsqrEngine::ensure_events(int n) {
  while ((int)ev_.size() < n) {
    cudaEvent_t e;
    APL_CUDA(cudaEventCreate(&e));
    ev_.push_back(e);
  }
}

void LsqrEngine::launch_iteration(const PrecondDev& P, bool init) {
  const bool pre = P.ell > 0;
  launch_k1(init, init ? x_ : (pre ? z_.p : v_.p));
  launch_k2(init, !pre);
  if (pre) launch_pre(P, g_.p, v_.p, z_.p, true, init);
}

void LsqrEngine::harvest(int iters, int ell) {
  for (int i = 0; i < iters; ++i) {
    float t[3];
    cudaError_t e = cudaEventElapsedTime(&t[0], ev_[4 * i], ev_[4 * i + 1]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t[1], ev_[4 * i + 1], ev_[4 * i + 2]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t[2], ev_[4 * i + 2], ev_[4 * i + 3]);
    if (e != cudaSuccess) {
      // timing unavailable: stop profiling rather than fail the solve
      (void)cudaGetLastError();
      profile_ = false;
      prof.broken = 1;
      return;
    }
    for (int k = 0; k < 3; ++k) {
      if (k == 2 && ell == 0) continue;
      prof.ms[k] += t[k];
      prof.launches[k] += 1;
      prof.bytes_total[k] += prof.bytes[k];
    }
  }
}

void LsqrEngine::flush_x() {
  flush_x_kernel<<<(unsigned)cdiv(n_, NT), NT, 0, st_>>>(n_, x_, d_.p, ctl_.p);
  APL_LAUNCH_CHECK();
  const int three = 3;
  APL_CUDA(cudaMemcpyAsync((char*)ctl_.p + offsetof(LsqrCtl, pending), &three, sizeof(int),
                           cudaMemcpyHostToDevice, st_));
}

PhaseResult LsqrEngine::run_phase(const PrecondDev& P, const PhaseArgs& a) {
  PhaseResult res;
  x_ = a.x;
  x0_zero_ = a.x_zero;
  const bool pre = P.ell > 0;
  if (pre) {
    q1_.alloc(P.ell, st_);
    ct_.alloc(P.ell, st_);
    c2t_.alloc(P.ell, st_);
    q3_.alloc(P.ell, st_);
    q3b_.alloc(P.ell, st_);
  }
  // In the FP32-sum mode each phase is the inner solve of an FP64 iterative refinement:
  // it stops once the estimate of ||Abar^T rbar|| fell by 1e-4 from its phase-start value
  // (FP32 products cannot resolve much more), and the next phase restarts from an
  // exactly formed residual.
  const double eps = a.eps;
  // state
  APL_CUDA(cudaMemcpyAsync(u_.p, a.rhs_top, m_ * sizeof(double), cudaMemcpyDeviceToDevice, st_));
  if (a.rhs_bot)
    APL_CUDA(cudaMemcpyAsync(u_.p + m_, a.rhs_bot, n_ * sizeof(double), cudaMemcpyDeviceToDevice,
                             st_));
  else
    APL_CUDA(cudaMemsetAsync(u_.p + m_, 0, n_ * sizeof(double), st_));
  v_.zero(st_);
  z_.zero(st_);
  d_.zero(st_);
  LsqrCtl h{};
  h.init = 1;
  h.delta = sqrt(a.mu);
  h.eps = eps;
  h.nu = a.nu;
  h.sig_ell = P.sig_ell;
  h.tol = a.tol;
  h.normP = P.normP;
  h.norm_ref = a.norm_ref;
  h.fixed_len = a.fixed_len;
  h.maxit = a.maxit;
  h.next_check = 0;
  h.use_p = pre ? 1 : 0;
  h.inner = (mode_ == 1 && a.fixed_len < 0) ? 1e-4 : 0.0;
  APL_CUDA(cudaMemcpyAsync(ctl_.p, &h, sizeof(LsqrCtl), cudaMemcpyHostToDevice, st_));
  launch_iteration(P, true);
  x0_zero_ = false;
  APL_CUDA(cudaMemcpyAsync(&h, ctl_.p, sizeof(LsqrCtl), cudaMemcpyDeviceToHost, st_));
  APL_CUDA(cudaStreamSynchronize(st_));
  if (h.done) {
    res.reason = h.reason;
    return res;
  }
  if (a.fixed_len == 0 || a.maxit <= 0) {
    res.reason = a.fixed_len == 0 ? R_REPLAY : R_MAXIT;
    return res;
  }
  cudaGraphExec_t exec = nullptr;
  const int G = graph_iters_;
  const int ell = P.ell;
  {
    // algorithmic bytes of one launch of each hot-loop kernel
    const double va = A_.dtype == 0 ? 8.0 : 4.0;
    const double sv = mode_ == 1 ? 4.0 : 8.0;  // operand vector bytes per element
    if (fused_.ok) {
      // the fused pass reads A once: A, z split and z (bottom rows), u read and written,
      // the column partials written; the column sums read them back
      const double pb = 8.0 * fused_.nclusters * n_;
      prof.bytes[0] = (double)m_ * n_ * va + sv * n_ + 8.0 * n_ + 16.0 * (m_ + n_) + pb;
      prof.bytes[1] = pb + 8.0 * n_ + 48.0 * n_;
    } else if (A_.fmt == 0) {
      prof.bytes[0] = (double)m_ * n_ * va + sv * n_ + 16.0 * (m_ + n_) + (mode_ ? 8.0 * m_ : 0);
      prof.bytes[1] = (double)m_ * n_ * va + sv * m_ + 8.0 * n_ + 48.0 * n_;
    } else {
      prof.bytes[0] = (double)A_.nnz * (va + 4) + 4.0 * (m_ + 1) + sv * n_ + 16.0 * (m_ + n_);
      prof.bytes[1] = (double)A_.nnz * (va + 4) + 4.0 * (n_ + 1) + sv * m_ + 8.0 * n_ + 48.0 * n_;
    }
    prof.bytes[2] = 2.0 * n_ * ell * 8.0 + 2.0 * ell * ell * 8.0 + 56.0 * n_;
  }
  kernels_per_iter_ = (A_.fmt == 0 ? (fused_.ok ? 2 : 3) : 2) + (ell > 0 ? 5 : 0);
  if (profile_) ensure_events(4 * std::max(G, 1));
  auto iteration = [&](int i) {
    if (profile_) record(4 * i);
    if (fused_.ok) {
      launch_fused(ell > 0 ? z_.p : v_.p, ell == 0);
      if (profile_) record(4 * i + 1);
      double* zbuf = ell == 0 ? v_.p : z_.p;
      float* zh = ell == 0 ? zh_.p : nullptr;
      float* zl = ell == 0 ? zl_.p : nullptr;
      k2b_dense<<<k2_blocks_, NT, 0, st_>>>(m_, n_, fused_.nclusters, part_.p, u_.p, g_.p, v_.p,
                                            zbuf, d_.p, x_, zh, zl, ctl_.p, red_.p, 0,
                                            ell == 0 ? 1 : 0);
      APL_LAUNCH_CHECK();
    } else {
      launch_k1(false, ell > 0 ? z_.p : v_.p);
      if (profile_) record(4 * i + 1);
      launch_k2(false, ell == 0);
    }
    if (profile_) record(4 * i + 2);
    if (ell > 0) launch_pre(P, g_.p, v_.p, z_.p, true, false);
    if (profile_) record(4 * i + 3);
  };
  if (G > 0) {
    cudaGraph_t graph = nullptr;
    APL_CUDA(cudaStreamBeginCapture(st_, cudaStreamCaptureModeThreadLocal));
    CaptureScope cs;
    try {
      for (int i = 0; i < G; ++i) iteration(i);
    } catch (...) {
      cudaStreamEndCapture(st_, &graph);
      if (graph) cudaGraphDestroy(graph);
      throw;
    }
    APL_CUDA(cudaStreamEndCapture(st_, &graph));
    cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    APL_CUDA(e);
  }
  struct GraphGuard {
    cudaGraphExec_t e;
    ~GraphGuard() { if (e) cudaGraphExecDestroy(e); }
  } guard{exec};
  const long long max_launch = a.maxit / std::max(G, 1) + 4;
  long long launches = 0;
  // FP32-sum mode: an explicit FP64 check every `periodic` iterations ends the phase when
  // the true residual stops falling (the recurrence can run ahead of it)
  const int periodic = 10 * a.check_gap;
  int next_periodic = periodic;
  double last_periodic = INFINITY;
  while (true) {
    const int it0 = h.it;
    if (G > 0) APL_CUDA(cudaGraphLaunch(exec, st_));
    else iteration(0);
    ++launches;
    APL_CUDA(cudaMemcpyAsync(&h, ctl_.p, sizeof(LsqrCtl), cudaMemcpyDeviceToHost, st_));
    APL_CUDA(cudaStreamSynchronize(st_));
    if (profile_) harvest(std::min(h.it - it0, std::max(G, 1)), ell);
    if (G > 0) add_launches((long long)kernels_per_iter_ * G);
    if (!h.done) {
      if (launches > max_launch) { res.reason = R_MAXIT; break; }
      if (mode_ == 1 && a.tol > 0.0 && a.fixed_len < 0 && h.it >= next_periodic) {
        if (h.pending == 2) { flush_x(); h.pending = 3; }
        const double ne = ne_residual(a.rhs_top, a.rhs_bot, x_, sqrt(a.mu), a.norm_ref, a.tol);
        res.checks++;
        res.ne_res = ne;
        if (ne <= a.tol) { res.reason = R_TOL; break; }
        if (ne > 0.5 * last_periodic) { res.reason = R_DRIFT; break; }
        last_periodic = ne;
        next_periodic = h.it + periodic;
      }
      continue;
    }
    if (h.reason == R_CHECK) {
      if (h.pending == 2) { flush_x(); h.pending = 3; }
      const double ne = ne_residual(a.rhs_top, a.rhs_bot, x_, sqrt(a.mu), a.norm_ref, a.tol);
      res.checks++;
      res.ne_res = ne;
      if (ne <= a.tol) { res.reason = R_TOL; break; }
      if ((long long)h.it >= a.maxit) { res.reason = R_MAXIT; break; }
      // FP32-sum mode: the recurrence passed tol but the FP64 residual did not; end the
      // phase so that the caller restarts from an exactly formed residual
      if (mode_ == 1) { res.reason = R_DRIFT; break; }
      const int zero = 0;
      const int nc = h.it + a.check_gap;
      APL_CUDA(cudaMemcpyAsync((char*)ctl_.p + offsetof(LsqrCtl, next_check), &nc, sizeof(int),
                               cudaMemcpyHostToDevice, st_));
      APL_CUDA(cudaMemcpyAsync((char*)ctl_.p + offsetof(LsqrCtl, done), &zero, sizeof(int),
                               cudaMemcpyHostToDevice, st_));
      continue;
    }
    res.reason = h.reason;
    break;
  }
  if (h.pending == 2) flush_x();
  res.iters = h.it;
  APL_CUDA(cudaStreamSynchronize(st_));
  if (fused_.ok) {
    int fe = 0;
    APL_CUDA(cudaMemcpyAsync(&fe, ferr_.p, sizeof(int), cudaMemcpyDeviceToHost, st_));
    APL_CUDA(cudaStreamSynchronize(st_));
    if (fe) throw Error(ST_ETIMEOUT, "fused A pass: a bounded wait ran past its bound");
  }
  return res;
}

void LsqrEngine::matvec(int trans, const double* x, double* y, double alpha, double beta,
                        bool fp64) {
  matvec_md(trans, x, y, alpha, beta, fp64 ? 0 : mode_);
}

void LsqrEngine::matvec_md(int trans, const double* x, double* y, double alpha, double beta,
                           int md) {
  if (A_.dtype == 0) md = 0;
  APL_REQUIRE(md == 0 || mode_ != 0, "matvec: FP32 products need the FP32 split buffers");
  const int64_t len = trans ? m_ : n_;
  if (md != 0) {
    split_kernel<<<(unsigned)cdiv(len, NT), NT, 0, st_>>>(len, x, uh_.p, ul_.p);
    APL_LAUNCH_CHECK();
  }
  const float* xh = uh_.p;
  const float* xl = ul_.p;
  if (!trans) {
    if (A_.fmt == 0) {
      const int blocks = (int)std::min<int64_t>(cdiv(m_ * 32, NT), sm_blocks());
      if (A_.dtype == 0)
        mv_dense_rows<double, 0><<<blocks, NT, 0, st_>>>(m_, n_, A_.ld, (const double*)A_.vals, x,
                                                         xh, xl, y, alpha, beta);
      else if (md == 0)
        mv_dense_rows<float, 0><<<blocks, NT, 0, st_>>>(m_, n_, A_.ld, (const float*)A_.vals, x,
                                                        xh, xl, y, alpha, beta);
      else if (md == 1)
        mv_dense_rows<float, 1><<<blocks, NT, 0, st_>>>(m_, n_, A_.ld, (const float*)A_.vals, x,
                                                        xh, xl, y, alpha, beta);
      else
        mv_dense_rows<float, 2><<<blocks, NT, 0, st_>>>(m_, n_, A_.ld, (const float*)A_.vals, x,
                                                        xh, xl, y, alpha, beta);
    } else {
      const unsigned g = (unsigned)cdiv(m_, NT);
      if (A_.dtype == 0)
        mv_csr_rows<double, 0><<<g, NT, 0, st_>>>(m_, A_.rowptr, A_.colidx, (const double*)A_.vals,
                                                  x, xh, xl, y, alpha, beta);
      else if (md == 0)
        mv_csr_rows<float, 0><<<g, NT, 0, st_>>>(m_, A_.rowptr, A_.colidx, (const float*)A_.vals,
                                                 x, xh, xl, y, alpha, beta);
      else if (md == 1)
        mv_csr_rows<float, 1><<<g, NT, 0, st_>>>(m_, A_.rowptr, A_.colidx, (const float*)A_.vals,
                                                 x, xh, xl, y, alpha, beta);
      else
        mv_csr_rows<float, 2><<<g, NT, 0, st_>>>(m_, A_.rowptr, A_.colidx, (const float*)A_.vals,
                                                 x, xh, xl, y, alpha, beta);
    }
    APL_LAUNCH_CHECK();
    return;
  }
  // y = A^T x (alpha = 1, beta = 0 only)
  APL_REQUIRE(alpha == 1.0 && beta == 0.0, "matvec: transposed product takes alpha=1, beta=0");
  if (A_.fmt == 0) {
    const int64_t rows_per = cdiv(m_, k2_rchunks_);
    dim3 grid((unsigned)cdiv(n_, NT), (unsigned)k2_rchunks_);
    if (A_.dtype == 0)
      k2a_dense<double, 0, false><<<grid, NT, 0, st_>>>(m_, n_, A_.ld, (const double*)A_.vals, x,
                                                        xh, xl, part_.p, rows_per, nullptr);
    else if (md == 0)
      k2a_dense<float, 0, false><<<grid, NT, 0, st_>>>(m_, n_, A_.ld, (const float*)A_.vals, x, xh,
                                                       xl, part_.p, rows_per, nullptr);
    else if (md == 1)
      k2a_dense<float, 1, false><<<grid, NT, 0, st_>>>(m_, n_, A_.ld, (const float*)A_.vals, x, xh,
                                                       xl, part_.p, rows_per, nullptr);
    else
      k2a_dense<float, 2, false><<<grid, NT, 0, st_>>>(m_, n_, A_.ld, (const float*)A_.vals, x, xh,
                                                       xl, part_.p, rows_per, nullptr);
    APL_LAUNCH_CHECK();
    colsum_kernel<<<(unsigned)cdiv(n_, NT), NT, 0, st_>>>(n_, k2_rchunks_, part_.p, y);
  } else {
    const unsigned g = (unsigned)cdiv(n_, NT);
    if (A_.dtype == 0)
      mv_csc_cols<double, 0><<<g, NT, 0, st_>>>(n_, A_.colptr, A_.rowidx, (const double*)A_.cvals,
                                                x, xh, xl, y);
    else if (md == 0)
      mv_csc_cols<float, 0><<<g, NT, 0, st_>>>(n_, A_.colptr, A_.rowidx, (const float*)A_.cvals, x,
                                               xh, xl, y);
    else if (md == 1)
      mv_csc_cols<float, 1><<<g, NT, 0, st_>>>(n_, A_.colptr, A_.rowidx, (const float*)A_.cvals, x,
                                               xh, xl, y);
    else
      mv_csc_cols<float, 2><<<g, NT, 0, st_>>>(n_, A_.colptr, A_.rowidx, (const float*)A_.cvals, x,
                                               xh, xl, y);
  }
  APL_LAUNCH_CHECK();
}

double LsqrEngine::norm2(const double* v, int64_t n) {
  const int blocks = (int)std::min<int64_t>(cdiv(n, NT), 1024);
  norm2_kernel<<<blocks, NT, 0, st_>>>(n, v, red_.p, scal_.p, cnt_.p);
  APL_LAUNCH_CHECK();
  double out = 0.0;
  APL_CUDA(cudaMemcpyAsync(&out, scal_.p, sizeof(double), cudaMemcpyDeviceToHost, st_));
  APL_CUDA(cudaStreamSynchronize(st_));
  return out;
}

double LsqrEngine::ne_residual_md(const double* rhs_top, const double* rhs_bot,
                                  const double* x, double delta, double norm_ref, int md) {
  APL_CUDA(cudaMemcpyAsync(r_.p, rhs_top, m_ * sizeof(double), cudaMemcpyDeviceToDevice, st_));
  matvec_md(0, x, r_.p, -1.0, 1.0, md);
  matvec_md(1, r_.p, q_.p, 1.0, 0.0, md);
  ne_tail_kernel<<<(unsigned)cdiv(n_, NT), NT, 0, st_>>>(n_, q_.p, rhs_bot, x, delta);
  APL_LAUNCH_CHECK();
  return norm2(q_.p, n_) / norm_ref;
}

double LsqrEngine::ne_residual(const double* rhs_top, const double* rhs_bot, const double* x,
                               double delta, double norm_ref, double screen_tol) {
  // FP32 values in an FP32-product form: a first evaluation with compensated FP32 products
  // (A read at FP32 speed, about 44 significant bits per sum instead of one FP64 FMA per
  // element at GB300's FP64 rate) settles every residual far above tol; one within
  // kScreen * tol of it is formed again with FP64 products, so every comparison with tol
  // is made on the FP64 value.
  constexpr double kScreen = 100.0;
  if (screen_tol > 0.0 && mode_ != 0) {
    const double est = ne_residual_md(rhs_top, rhs_bot, x, delta, norm_ref, 2);
    if (est > kScreen * screen_tol) return est;
  }
  return ne_residual_md(rhs_top, rhs_bot, x, delta, norm_ref, 0);
}

void LsqrEngine::correction_rhs(const double* b, const double* x, double delta,
                                double* rhs_bot) {
  APL_CUDA(cudaMemcpyAsync(r_.p, b, m_ * sizeof(double), cudaMemcpyDeviceToDevice, st_));
  matvec(0, x, r_.p, -1.0, 1.0, true);
  matvec(1, r_.p, q_.p, 1.0, 0.0, true);
  ne_tail_kernel<<<(unsigned)cdiv(n_, NT), NT, 0, st_>>>(n_, q_.p, nullptr, x, delta);
  APL_LAUNCH_CHECK();
  scale_to_kernel<<<(unsigned)cdiv(n_, NT), NT, 0, st_>>>(n_, q_.p, 1.0 / delta, rhs_bot);
  APL_LAUNCH_CHECK();
}

void LsqrEngine::apply_precond(const PrecondDev& P, const double* w, double* out, double* out2) {
  if (P.ell <= 0) {
    APL_CUDA(cudaMemcpyAsync(out, w, n_ * sizeof(double), cudaMemcpyDeviceToDevice, st_));
    if (out2)
      APL_CUDA(cudaMemcpyAsync(out2, w, n_ * sizeof(double), cudaMemcpyDeviceToDevice, st_));
    return;
  }
  launch_pre(P, w, out, out2, false, false);
}

}  // namespace apl

// ======================================================================================
// Allocation-free dense A^T x (aplicur_dense_atx_noalloc).
//
// Its only scratch, the row-chunk partial sums of the transposed product, lives in this
// file-scope device array; every GPU that loads the library holds it until the process
// exits.  Host code cannot use the symbol as a device address, so the address is looked
// up once per device with cudaGetSymbolAddress and cached.
// ======================================================================================

namespace {
constexpr int64_t kNoAllocDoubles = int64_t(1) << 19;  // 4 MiB
constexpr int kMaxDevices = 64;
}  // namespace

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

namespace {
std::mutex g_noalloc_mu;
double* g_noalloc_ptr[kMaxDevices] = {nullptr};

// Address of g_noalloc_scratch on the current device (looked up on first use).
cudaError_t noalloc_scratch(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}
}  // namespace

namespace apl {
void set_noalloc_error(const char* msg);
}

extern "C" aplicur_status aplicur_dense_atx_noalloc(const aplicur_matrix* A, const double* x,
                                                    double* y, void* stream) {
  using namespace apl;
  if (!A || !x || !y || !A->values) {
    set_noalloc_error("aplicur_dense_atx_noalloc: null argument");
    return APLICUR_EINVAL;
  }
  if (A->format != APLICUR_DENSE_ROWMAJOR || (A->dtype != APLICUR_F64 && A->dtype != APLICUR_F32) ||
      A->m < 1 || A->n < 1 || A->ld < A->n) {
    set_noalloc_error("aplicur_dense_atx_noalloc: need a dense row-major F64/F32 matrix, "
                      "m, n >= 1, ld >= n");
    return APLICUR_EINVAL;
  }
  if (A->n > kNoAllocDoubles) {
    set_noalloc_error("aplicur_dense_atx_noalloc: n exceeds the 524288-column limit of the "
                      "static scratch array");
    return APLICUR_EINVAL;
  }
  double* scratch = nullptr;
  cudaError_t e = noalloc_scratch(&scratch);
  if (e != cudaSuccess) {
    set_noalloc_error(cudaGetErrorString(e));
    return APLICUR_ECUDA;
  }
  const int64_t m = A->m, n = A->n;
  // row chunks: as many as the scratch holds, at most 64, at least 32 rows each; every
  // partial is written before it is read, so nothing needs clearing between calls
  const int64_t rchunks = std::max<int64_t>(
      1, std::min<int64_t>(std::min<int64_t>(kNoAllocDoubles / n, 64), cdiv(m, 32)));
  const int64_t rows_per = cdiv(m, rchunks);
  cudaStream_t st = (cudaStream_t)stream;
  dim3 grid((unsigned)cdiv(n, NT), (unsigned)rchunks);
  if (A->dtype == APLICUR_F64)
    k2a_dense<double, 0, false><<<grid, NT, 0, st>>>(m, n, A->ld, (const double*)A->values, x,
                                                     nullptr, nullptr, scratch, rows_per, nullptr);
  else
    k2a_dense<float, 0, false><<<grid, NT, 0, st>>>(m, n, A->ld, (const float*)A->values, x,
                                                    nullptr, nullptr, scratch, rows_per, nullptr);
  e = cudaGetLastError();
  if (e == cudaSuccess) {
    colsum_kernel<<<(unsigned)cdiv(n, NT), NT, 0, st>>>(n, (int)rchunks, scratch, y);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    set_noalloc_error(cudaGetErrorString(e));
    return APLICUR_ECUDA;
  }
  note_launch();
  note_launch();
  return APLICUR_OK;
}

