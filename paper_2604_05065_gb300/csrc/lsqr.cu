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
#include <cstddef>
#include <vector>

#include "lsqr.cuh"

namespace apl {

namespace {

constexpr int NT = 256;

__device__ __forceinline__ bool dyn_stop(double phibar_prev, double phibar, double rate1,
                                         double nu, double sig_ell) {
  if (!isfinite(nu)) return false;
  if (phibar_prev - phibar < sig_ell) return true;
  if (phibar <= 0.0) return false;
  const double rate = log(phibar_prev / phibar);
  if (rate <= 0.0) return true;
  return rate1 / rate > nu;
}

__device__ void finalize_beta(LsqrCtl* c, double sumsq, int init) {
  const double beta = sqrt(sumsq);
  c->beta = beta;
  c->us = beta > 0.0 ? 1.0 / beta : 0.0;
  if (init) {
    c->beta1 = beta;
    c->phibar = beta;
    if (beta == 0.0) { c->done = 1; c->reason = R_EXACT; }
  } else {
    c->anorm2 += c->alpha * c->alpha + beta * beta;
  }
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

// ---- K1 -------------------------------------------------------------------------------

template <typename TA, typename TAcc>
__global__ void __launch_bounds__(NT) k1_dense(int64_t m, int64_t n, int64_t ld,
                                               const TA* __restrict__ A,
                                               const double* __restrict__ z,
                                               double* __restrict__ u, LsqrCtl* ctl,
                                               double* __restrict__ red, int init) {
  __shared__ double sh[NT / 32];
  if (ctl->done) return;
  const double ca = init ? -1.0 : ctl->zs;
  const double cu = init ? 1.0 : -ctl->alpha * ctl->us;
  const double delta = ctl->delta;
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * NT + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * NT) >> 5;
  double ss = 0.0;
  for (int64_t i = warp; i < m; i += nwarps) {
    const TA* a = A + i * ld;
    TAcc acc = 0;
    int64_t j = lane;
    for (; j + 96 < n; j += 128) {
      acc += (TAcc)a[j] * (TAcc)z[j];
      acc += (TAcc)a[j + 32] * (TAcc)z[j + 32];
      acc += (TAcc)a[j + 64] * (TAcc)z[j + 64];
      acc += (TAcc)a[j + 96] * (TAcc)z[j + 96];
    }
    for (; j < n; j += 32) acc += (TAcc)a[j] * (TAcc)z[j];
    const double s = warp_sum((double)acc);
    if (lane == 0) {
      const double val = ca * s + cu * u[i];
      u[i] = val;
      ss += val * val;
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

template <typename TA, typename TAcc>
__global__ void __launch_bounds__(NT) k1_csr(int64_t m, int64_t n, const int* __restrict__ rowptr,
                                             const int* __restrict__ colidx,
                                             const TA* __restrict__ vals,
                                             const double* __restrict__ z,
                                             double* __restrict__ u, LsqrCtl* ctl,
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
      TAcc acc = 0;
      const int e1 = rowptr[i + 1];
      for (int e = rowptr[i]; e < e1; ++e) acc += (TAcc)vals[e] * (TAcc)z[colidx[e]];
      val = ca * (double)acc + cu * u[i];
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
                                          double* x) {
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
    return vn * vn;
  }
  g[j] = gj;
  return 0.0;
}

template <typename TA, typename TAcc>
__global__ void __launch_bounds__(NT) k2_csr(int64_t m, int64_t n, const int* __restrict__ colptr,
                                             const int* __restrict__ rowidx,
                                             const TA* __restrict__ cvals,
                                             const double* __restrict__ u, double* g, double* v,
                                             double* z, double* d, double* x, LsqrCtl* ctl,
                                             double* __restrict__ red, int init, int fused) {
  __shared__ double sh[NT / 32];
  if (ctl->done) return;
  const double us = ctl->us, delta = ctl->delta;
  double ss = 0.0;
  for (int64_t j = (int64_t)blockIdx.x * NT + threadIdx.x; j < n; j += (int64_t)gridDim.x * NT) {
    TAcc acc = 0;
    const int e1 = colptr[j + 1];
    for (int e = colptr[j]; e < e1; ++e) acc += (TAcc)cvals[e] * (TAcc)u[rowidx[e]];
    const double gj = us * ((double)acc + delta * u[m + j]);
    ss += k2_tail(j, gj, ctl, init, fused, g, v, z, d, x);
  }
  if (!fused) return;
  const double b = block_sum(ss, sh);
  if (threadIdx.x == 0) red[blockIdx.x] = b;
  if (!last_block_done(&ctl->counter[0])) return;
  const double tot = block_sum_partials(red, gridDim.x, sh);
  if (threadIdx.x == 0) finalize_alpha(ctl, tot, init);
}

// Dense A^T u: per (column block, row chunk) partial sums.
template <typename TA, typename TAcc>
__global__ void __launch_bounds__(NT) k2a_dense(int64_t m, int64_t n, int64_t ld,
                                                const TA* __restrict__ A,
                                                const double* __restrict__ u,
                                                double* __restrict__ part, int64_t rows_per,
                                                const LsqrCtl* ctl) {
  if (ctl && ctl->done) return;
  const int64_t j = (int64_t)blockIdx.x * NT + threadIdx.x;
  if (j >= n) return;
  const int64_t r0 = (int64_t)blockIdx.y * rows_per;
  const int64_t r1 = r0 + rows_per < m ? r0 + rows_per : m;
  TAcc acc = 0;
  for (int64_t i = r0; i < r1; ++i) acc += (TAcc)A[i * ld + j] * (TAcc)u[i];
  part[(int64_t)blockIdx.y * n + j] = (double)acc;
}

__global__ void __launch_bounds__(NT) k2b_dense(int64_t m, int64_t n, int rchunks,
                                                const double* __restrict__ part,
                                                const double* __restrict__ u, double* g,
                                                double* v, double* z, double* d, double* x,
                                                LsqrCtl* ctl, double* __restrict__ red, int init,
                                                int fused) {
  __shared__ double sh[NT / 32];
  if (ctl->done) return;
  const double us = ctl->us, delta = ctl->delta;
  double ss = 0.0;
  for (int64_t j = (int64_t)blockIdx.x * NT + threadIdx.x; j < n; j += (int64_t)gridDim.x * NT) {
    double acc = 0.0;
    for (int c = 0; c < rchunks; ++c) acc += part[(int64_t)c * n + j];
    const double gj = us * (acc + delta * u[m + j]);
    ss += k2_tail(j, gj, ctl, init, fused, g, v, z, d, x);
  }
  if (!fused) return;
  const double b = block_sum(ss, sh);
  if (threadIdx.x == 0) red[blockIdx.x] = b;
  if (!last_block_done(&ctl->counter[0])) return;
  const double tot = block_sum_partials(red, gridDim.x, sh);
  if (threadIdx.x == 0) finalize_alpha(ctl, tot, init);
}

// ---- preconditioner passes ------------------------------------------------------------

template <typename TV, typename TAcc>
__global__ void __launch_bounds__(128) k3_partial(int64_t n, int ell, int64_t ldv,
                                                  const TV* __restrict__ V,
                                                  const double* __restrict__ w,
                                                  double* __restrict__ tpart, int64_t rows_per,
                                                  const LsqrCtl* ctl) {
  if (ctl && ctl->done) return;
  const int k = blockIdx.x * 128 + threadIdx.x;
  if (k >= ell) return;
  const int64_t r0 = (int64_t)blockIdx.y * rows_per;
  const int64_t r1 = r0 + rows_per < n ? r0 + rows_per : n;
  TAcc acc = 0;
  for (int64_t i = r0; i < r1; ++i) acc += (TAcc)V[i * ldv + k] * (TAcc)w[i];
  tpart[(int64_t)blockIdx.y * ell + k] = (double)acc;
}

__global__ void k3_reduce(int ell, int chunks, const double* __restrict__ tpart,
                          const double* __restrict__ coef, const double* __restrict__ coef2,
                          double* __restrict__ ct, double* __restrict__ c2t, const LsqrCtl* ctl) {
  if (ctl && ctl->done) return;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= ell) return;
  double t = 0.0;
  for (int c = 0; c < chunks; ++c) t += tpart[(int64_t)c * ell + k];
  ct[k] = coef[k] * t;
  if (c2t) c2t[k] = coef2[k] * t;
}

// Expansion, one warp per row: out1 = w + V ct, out2 = w + V c2t.  In the LSQR phase
// also subtracts beta v / beta z and reduces ||v'||^2.
template <typename TV, typename TAcc>
__global__ void __launch_bounds__(NT) k4_expand(int64_t n, int ell, int64_t ldv,
                                                const TV* __restrict__ V,
                                                const double* __restrict__ ct,
                                                const double* __restrict__ c2t,
                                                const double* __restrict__ w, double* out1,
                                                double* out2, LsqrCtl* ctl,
                                                double* __restrict__ red, int init) {
  __shared__ double sh[NT / 32];
  if (ctl && ctl->done) return;
  double beta = 0.0, zs = 0.0;
  if (ctl && !init) { beta = ctl->beta; zs = ctl->zs; }
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * NT + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * NT) >> 5;
  double ss = 0.0;
  for (int64_t i = warp; i < n; i += nwarps) {
    const TV* vr = V + i * ldv;
    TAcc s1 = 0, s2 = 0;
    for (int k = lane; k < ell; k += 32) {
      const TAcc vv = (TAcc)vr[k];
      s1 += vv * (TAcc)ct[k];
      if (out2) s2 += vv * (TAcc)c2t[k];
    }
    const double a1 = warp_sum((double)s1);
    const double a2 = out2 ? warp_sum((double)s2) : 0.0;
    if (lane == 0) {
      const double wi = w[i];
      double o1 = wi + a1;
      if (ctl && !init) o1 -= beta * (out1[i] * zs);
      out1[i] = o1;
      if (out2) {
        double o2 = wi + a2;
        if (ctl && !init) o2 -= beta * (out2[i] * zs);
        out2[i] = o2;
      }
      ss += o1 * o1;
    }
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

template <typename TA, typename TAcc>
__global__ void __launch_bounds__(NT) mv_dense_rows(int64_t m, int64_t n, int64_t ld,
                                                    const TA* __restrict__ A,
                                                    const double* __restrict__ x, double* y,
                                                    double alpha, double beta) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * NT + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * NT) >> 5;
  for (int64_t i = warp; i < m; i += nwarps) {
    const TA* a = A + i * ld;
    TAcc acc = 0;
    for (int64_t j = lane; j < n; j += 32) acc += (TAcc)a[j] * (TAcc)x[j];
    const double s = warp_sum((double)acc);
    if (lane == 0) y[i] = beta == 0.0 ? alpha * s : alpha * s + beta * y[i];
  }
}

template <typename TA, typename TAcc>
__global__ void mv_csr_rows(int64_t m, const int* __restrict__ rowptr,
                            const int* __restrict__ colidx, const TA* __restrict__ vals,
                            const double* __restrict__ x, double* y, double alpha, double beta) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  TAcc acc = 0;
  for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) acc += (TAcc)vals[e] * (TAcc)x[colidx[e]];
  y[i] = beta == 0.0 ? alpha * (double)acc : alpha * (double)acc + beta * y[i];
}

template <typename TA, typename TAcc>
__global__ void mv_csc_cols(int64_t n, const int* __restrict__ colptr,
                            const int* __restrict__ rowidx, const TA* __restrict__ cvals,
                            const double* __restrict__ x, double* y) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  TAcc acc = 0;
  for (int e = colptr[j]; e < colptr[j + 1]; ++e) acc += (TAcc)cvals[e] * (TAcc)x[rowidx[e]];
  y[j] = (double)acc;
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

}  // namespace

// ======================================================================================

void LsqrEngine::setup(cudaStream_t st, const MatView& A, int mixed, int graph_iters) {
  st_ = st;
  A_ = A;
  mixed_ = mixed;
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
  if (A.fmt == 0) {
    k1_blocks_ = (int)std::min<int64_t>(cdiv(m_ * 32, NT), sm_blocks());
    const int64_t cb = cdiv(n_, NT);
    k2_rchunks_ = (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(4 * 152, cb), cdiv(m_, 32)));
    k2_blocks_ = (int)std::min<int64_t>(cdiv(n_, NT), sm_blocks());
    part_.alloc((size_t)k2_rchunks_ * n_, st);
  } else {
    k1_blocks_ = (int)std::min<int64_t>(cdiv(m_ + n_, NT), sm_blocks());
    k2_blocks_ = (int)std::min<int64_t>(cdiv(n_, NT), sm_blocks());
  }
  red_cap_ = sm_blocks() + 64;
  red_.alloc(red_cap_, st);
}

void LsqrEngine::launch_k1(bool init, const double* z) {
  LsqrCtl* c = ctl_.p;
  // the residual that starts a phase is always formed with FP64 products (in the mixed
  // form this makes every warm restart one step of FP64 iterative refinement)
  const bool f32 = mixed_ && !init;
  if (A_.fmt == 0) {
    if (A_.dtype == 0)
      k1_dense<double, double><<<k1_blocks_, NT, 0, st_>>>(m_, n_, A_.ld, (const double*)A_.vals, z,
                                                           u_.p, c, red_.p, init);
    else if (f32)
      k1_dense<float, float><<<k1_blocks_, NT, 0, st_>>>(m_, n_, A_.ld, (const float*)A_.vals, z,
                                                         u_.p, c, red_.p, init);
    else
      k1_dense<float, double><<<k1_blocks_, NT, 0, st_>>>(m_, n_, A_.ld, (const float*)A_.vals, z,
                                                          u_.p, c, red_.p, init);
  } else {
    if (A_.dtype == 0)
      k1_csr<double, double><<<k1_blocks_, NT, 0, st_>>>(m_, n_, A_.rowptr, A_.colidx,
                                                         (const double*)A_.vals, z, u_.p, c,
                                                         red_.p, init);
    else if (f32)
      k1_csr<float, float><<<k1_blocks_, NT, 0, st_>>>(m_, n_, A_.rowptr, A_.colidx,
                                                       (const float*)A_.vals, z, u_.p, c, red_.p,
                                                       init);
    else
      k1_csr<float, double><<<k1_blocks_, NT, 0, st_>>>(m_, n_, A_.rowptr, A_.colidx,
                                                        (const float*)A_.vals, z, u_.p, c, red_.p,
                                                        init);
  }
  APL_LAUNCH_CHECK();
}

void LsqrEngine::launch_k2(bool init, bool fused) {
  LsqrCtl* c = ctl_.p;
  // the stored z' lives in v_ when there is no preconditioner (z = v)
  double* zbuf = fused ? v_.p : z_.p;
  if (A_.fmt == 0) {
    dim3 grid((unsigned)cdiv(n_, NT), (unsigned)k2_rchunks_);
    const int64_t rows_per = cdiv(m_, k2_rchunks_);
    if (A_.dtype == 0)
      k2a_dense<double, double><<<grid, NT, 0, st_>>>(m_, n_, A_.ld, (const double*)A_.vals, u_.p,
                                                      part_.p, rows_per, c);
    else if (mixed_)
      k2a_dense<float, float><<<grid, NT, 0, st_>>>(m_, n_, A_.ld, (const float*)A_.vals, u_.p,
                                                    part_.p, rows_per, c);
    else
      k2a_dense<float, double><<<grid, NT, 0, st_>>>(m_, n_, A_.ld, (const float*)A_.vals, u_.p,
                                                     part_.p, rows_per, c);
    APL_LAUNCH_CHECK();
    k2b_dense<<<k2_blocks_, NT, 0, st_>>>(m_, n_, k2_rchunks_, part_.p, u_.p, g_.p, v_.p, zbuf,
                                          d_.p, x_, c, red_.p, init, fused);
  } else {
    if (A_.dtype == 0)
      k2_csr<double, double><<<k2_blocks_, NT, 0, st_>>>(m_, n_, A_.colptr, A_.rowidx,
                                                         (const double*)A_.cvals, u_.p, g_.p,
                                                         v_.p, zbuf, d_.p, x_, c, red_.p, init,
                                                         fused);
    else if (mixed_)
      k2_csr<float, float><<<k2_blocks_, NT, 0, st_>>>(m_, n_, A_.colptr, A_.rowidx,
                                                       (const float*)A_.cvals, u_.p, g_.p, v_.p,
                                                       zbuf, d_.p, x_, c, red_.p, init, fused);
    else
      k2_csr<float, double><<<k2_blocks_, NT, 0, st_>>>(m_, n_, A_.colptr, A_.rowidx,
                                                        (const float*)A_.cvals, u_.p, g_.p, v_.p,
                                                        zbuf, d_.p, x_, c, red_.p, init, fused);
  }
  APL_LAUNCH_CHECK();
}

void LsqrEngine::launch_pre(const PrecondDev& P, const double* w, double* o1, double* o2,
                            bool in_phase, bool init) {
  const int ell = P.ell;
  const int kb = (int)cdiv(ell, 128);
  const int64_t rows_per = cdiv(n_, tchunks_);
  dim3 grid((unsigned)kb, (unsigned)tchunks_);
  const LsqrCtl* c = in_phase ? ctl_.p : nullptr;
  if (P.fp32)
    k3_partial<float, float><<<grid, 128, 0, st_>>>(n_, ell, P.ldv, P.V32, w, tpart_.p, rows_per,
                                                    c);
  else
    k3_partial<double, double><<<grid, 128, 0, st_>>>(n_, ell, P.ldv, P.V64, w, tpart_.p,
                                                      rows_per, c);
  APL_LAUNCH_CHECK();
  k3_reduce<<<(unsigned)cdiv(ell, 128), 128, 0, st_>>>(ell, tchunks_, tpart_.p, P.coef, P.coef2,
                                                       ct_.p, o2 ? c2t_.p : nullptr, c);
  APL_LAUNCH_CHECK();
  const int blocks = (int)std::min<int64_t>(cdiv(n_ * 32, NT), sm_blocks());
  LsqrCtl* cw = in_phase ? ctl_.p : nullptr;
  if (P.fp32)
    k4_expand<float, float><<<blocks, NT, 0, st_>>>(n_, ell, P.ldv, P.V32, ct_.p, c2t_.p, w, o1,
                                                    o2, cw, red_.p, init);
  else
    k4_expand<double, double><<<blocks, NT, 0, st_>>>(n_, ell, P.ldv, P.V64, ct_.p, c2t_.p, w, o1,
                                                      o2, cw, red_.p, init);
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

// Iteration i of a captured graph records events 4i..4i+3 around K1, K2 and the
// preconditioner passes.
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
  const bool pre = P.ell > 0;
  if (pre) {
    tchunks_ = (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(4 * 152, cdiv(P.ell, 128)),
                                                          cdiv(n_, 32)));
    tpart_.alloc((size_t)tchunks_ * P.ell, st_);
    ct_.alloc(P.ell, st_);
    c2t_.alloc(P.ell, st_);
  }
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
  h.eps = a.eps;
  h.nu = a.nu;
  h.sig_ell = P.sig_ell;
  h.tol = a.tol;
  h.normP = P.normP;
  h.norm_ref = a.norm_ref;
  h.fixed_len = a.fixed_len;
  h.maxit = a.maxit;
  h.next_check = 0;
  h.use_p = pre ? 1 : 0;
  APL_CUDA(cudaMemcpyAsync(ctl_.p, &h, sizeof(LsqrCtl), cudaMemcpyHostToDevice, st_));
  launch_iteration(P, true);
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
    if (A_.fmt == 0) {
      prof.bytes[0] = (double)m_ * n_ * va + 8.0 * n_ + 16.0 * (m_ + n_);
      prof.bytes[1] = (double)m_ * n_ * va + 8.0 * (m_ + n_) + 48.0 * n_;
    } else {
      prof.bytes[0] = (double)A_.nnz * (va + 4) + 4.0 * (m_ + 1) + 8.0 * n_ + 16.0 * (m_ + n_);
      prof.bytes[1] = (double)A_.nnz * (va + 4) + 4.0 * (n_ + 1) + 8.0 * (m_ + n_) + 48.0 * n_;
    }
    const double vv = P.fp32 ? 4.0 : 8.0;
    prof.bytes[2] = 2.0 * n_ * ell * vv + 56.0 * n_;
  }
  kernels_per_iter_ = (A_.fmt == 0 ? 3 : 2) + (ell > 0 ? 3 : 0);
  if (profile_) ensure_events(4 * std::max(G, 1));
  auto iteration = [&](int i) {
    if (profile_) record(4 * i);
    launch_k1(false, ell > 0 ? z_.p : v_.p);
    if (profile_) record(4 * i + 1);
    launch_k2(false, ell == 0);
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
      continue;
    }
    if (h.reason == R_CHECK) {
      if (h.pending == 2) { flush_x(); h.pending = 3; }
      const double ne = ne_residual(a.rhs_top, a.rhs_bot, x_, sqrt(a.mu), a.norm_ref);
      res.checks++;
      res.ne_res = ne;
      if (ne <= a.tol) { res.reason = R_TOL; break; }
      if ((long long)h.it >= a.maxit) { res.reason = R_MAXIT; break; }
      // mixed form: the recurrence passed tol but the FP64 residual did not; end the phase
      // so that the caller restarts from an exactly formed residual
      if (mixed_) { res.reason = R_DRIFT; break; }
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
  return res;
}

void LsqrEngine::matvec(int trans, const double* x, double* y, double alpha, double beta,
                        bool fp64) {
  const bool f32acc = !fp64 && mixed_ && A_.dtype == 1;
  if (!trans) {
    if (A_.fmt == 0) {
      const int blocks = (int)std::min<int64_t>(cdiv(m_ * 32, NT), sm_blocks());
      if (A_.dtype == 0)
        mv_dense_rows<double, double><<<blocks, NT, 0, st_>>>(m_, n_, A_.ld, (const double*)A_.vals,
                                                              x, y, alpha, beta);
      else if (f32acc)
        mv_dense_rows<float, float><<<blocks, NT, 0, st_>>>(m_, n_, A_.ld, (const float*)A_.vals, x,
                                                            y, alpha, beta);
      else
        mv_dense_rows<float, double><<<blocks, NT, 0, st_>>>(m_, n_, A_.ld, (const float*)A_.vals,
                                                             x, y, alpha, beta);
    } else {
      const unsigned g = (unsigned)cdiv(m_, NT);
      if (A_.dtype == 0)
        mv_csr_rows<double, double><<<g, NT, 0, st_>>>(m_, A_.rowptr, A_.colidx,
                                                       (const double*)A_.vals, x, y, alpha, beta);
      else if (f32acc)
        mv_csr_rows<float, float><<<g, NT, 0, st_>>>(m_, A_.rowptr, A_.colidx,
                                                     (const float*)A_.vals, x, y, alpha, beta);
      else
        mv_csr_rows<float, double><<<g, NT, 0, st_>>>(m_, A_.rowptr, A_.colidx,
                                                      (const float*)A_.vals, x, y, alpha, beta);
    }
    APL_LAUNCH_CHECK();
    return;
  }
  // y = A^T x (alpha = 1, beta = 0 only)
  APL_REQUIRE(alpha == 1.0 && beta == 0.0, "matvec: transposed product takes alpha=1, beta=0");
  if (A_.fmt == 0) {
    dim3 grid((unsigned)cdiv(n_, NT), (unsigned)k2_rchunks_);
    const int64_t rows_per = cdiv(m_, k2_rchunks_);
    if (A_.dtype == 0)
      k2a_dense<double, double><<<grid, NT, 0, st_>>>(m_, n_, A_.ld, (const double*)A_.vals, x,
                                                      part_.p, rows_per, nullptr);
    else if (f32acc)
      k2a_dense<float, float><<<grid, NT, 0, st_>>>(m_, n_, A_.ld, (const float*)A_.vals, x,
                                                    part_.p, rows_per, nullptr);
    else
      k2a_dense<float, double><<<grid, NT, 0, st_>>>(m_, n_, A_.ld, (const float*)A_.vals, x,
                                                     part_.p, rows_per, nullptr);
    APL_LAUNCH_CHECK();
    colsum_kernel<<<(unsigned)cdiv(n_, NT), NT, 0, st_>>>(n_, k2_rchunks_, part_.p, y);
  } else {
    const unsigned g = (unsigned)cdiv(n_, NT);
    if (A_.dtype == 0)
      mv_csc_cols<double, double><<<g, NT, 0, st_>>>(n_, A_.colptr, A_.rowidx,
                                                     (const double*)A_.cvals, x, y);
    else if (f32acc)
      mv_csc_cols<float, float><<<g, NT, 0, st_>>>(n_, A_.colptr, A_.rowidx,
                                                   (const float*)A_.cvals, x, y);
    else
      mv_csc_cols<float, double><<<g, NT, 0, st_>>>(n_, A_.colptr, A_.rowidx,
                                                    (const float*)A_.cvals, x, y);
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

double LsqrEngine::ne_residual(const double* rhs_top, const double* rhs_bot, const double* x,
                               double delta, double norm_ref) {
  APL_CUDA(cudaMemcpyAsync(r_.p, rhs_top, m_ * sizeof(double), cudaMemcpyDeviceToDevice, st_));
  matvec(0, x, r_.p, -1.0, 1.0, true);
  matvec(1, r_.p, q_.p, 1.0, 0.0, true);
  ne_tail_kernel<<<(unsigned)cdiv(n_, NT), NT, 0, st_>>>(n_, q_.p, rhs_bot, x, delta);
  APL_LAUNCH_CHECK();
  return norm2(q_.p, n_) / norm_ref;
}

void LsqrEngine::apply_precond(const PrecondDev& P, const double* w, double* out, double* out2) {
  if (P.ell <= 0) {
    APL_CUDA(cudaMemcpyAsync(out, w, n_ * sizeof(double), cudaMemcpyDeviceToDevice, st_));
    if (out2)
      APL_CUDA(cudaMemcpyAsync(out2, w, n_ * sizeof(double), cudaMemcpyDeviceToDevice, st_));
    return;
  }
  tchunks_ = (int)std::max<int64_t>(1, std::min<int64_t>(cdiv(4 * 152, cdiv(P.ell, 128)),
                                                        cdiv(n_, 32)));
  tpart_.alloc((size_t)tchunks_ * P.ell, st_);
  ct_.alloc(P.ell, st_);
  c2t_.alloc(P.ell, st_);
  launch_pre(P, w, out, out2, false, false);
}

}  // namespace apl
