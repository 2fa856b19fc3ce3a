// Preconditioned LSQR phase on the GPU (Section 2.2, warm start of Section 3.2, stopping
// rules of Section 5.3.2): Golub-Kahan bidiagonalisation of [A; delta I] P^{-1} with an
// explicit (m+n)-vector u, all scalars resident in device memory.
#pragma once
#include "cur.cuh"

namespace apl {

// Plan of the fused dense A pass (apass.cu).
struct FusedPlan {
  bool ok = false;      // the fused pass applies to this matrix
  int C = 1;            // CTAs per thread-block cluster (column panels of A)
  int W = 0;            // panel width in columns (multiple of 4)
  int R = 1;            // rows of A per pipeline stage
  int S = 2;            // pipeline stages
  int KQ = 1;           // float4 columns per consumer thread and row
  int nclusters = 0;    // clusters of the persistent grid
  int64_t rows_per_cluster = 0;
  int ucap = 0;         // rows of u held in shared memory (>= rows_per_cluster)
  size_t smem = 0;      // dynamic shared memory per CTA
};

enum StopReason { R_NONE = 0, R_EXACT = 1, R_REPLAY = 2, R_PS2 = 3, R_PS1 = 4, R_DYNAMIC = 5,
                  R_TOL = 6, R_MAXIT = 7, R_CHECK = 8, R_DRIFT = 9, R_INNER = 10 };

// Per-kernel device time of the hot loop, collected with CUDA events recorded inside the
// captured iteration graphs when profiling is on.
struct KernelProfile {
  double ms[3] = {0, 0, 0};        // 0: A z pass (K1), 1: A^T u pass (K2), 2: Vhat passes
  long long launches[3] = {0, 0, 0};
  double bytes[3] = {0, 0, 0};     // algorithmic bytes of one launch (current phase)
  double bytes_total[3] = {0, 0, 0};  // summed over the timed launches
  int broken = 0;                    // event timing failed; numbers incomplete
};

// Device-resident LSQR state and phase parameters.
struct LsqrCtl {
  double alpha, beta, rhobar, phibar, phibar_prev, beta1, anorm2, rate1;
  double us;        // scale of the stored u (1/beta)
  double zs;        // scale of the stored v' and z' (1/alpha)
  double xc, dc;    // pending update x += xc d ; d = z - dc d
  double cabs;
  int pending;      // 0 none, 1 d = z, 2 x and d update, 3 d update only
  int it, done, reason, init;
  int next_check, fixed_len, use_p, pad;
  double delta, eps, nu, sig_ell, tol, normP, norm_ref;
  double inner;     // > 0: stop when ||Abar^T rbar|| estimate <= inner * its phase-start value
  double arnorm0;   // alpha_1 beta_1 = ||Abar^T rbar_0||
  long long maxit;
  unsigned int counter[8];
};

// beta = ||u'|| from its squared norm: the scale of the stored u' and, after the first
// step of a phase, the running ||Abar||_F^2 estimate of the Paige-Saunders test 2.
__device__ __forceinline__ void finalize_beta(LsqrCtl* c, double sumsq, int init) {
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

// The preconditioner P^{-1} = I + Vhat diag(coef) Vhat^T (Eq. preconditioner2) with Vhat
// kept implicit as Q_R V_M: Q (n x ell, column-major, ld ldq) and VM (ell x ell,
// column-major).  coef2 gives P^{-2} = I + Vhat diag(coef2) Vhat^T.
struct PrecondDev {
  int ell = 0;
  int64_t ldq = 0;
  const double* Q = nullptr;
  const double* VM = nullptr;
  const double* coef = nullptr;
  const double* coef2 = nullptr;
  double normP = 1.0;    // ||P||_2
  double sig_ell = 0.0;  // smallest CUR singular value
  // SVD-free variant: VM holds M^{-1} (ell x ell), coef the constant sighat; the passes
  // form P^{-T} w and P^{-1} P^{-T} w (P is not symmetric)
  int svdfree = 0;
  double sighat = 0.0;
};

struct PhaseArgs {
  const double* rhs_top = nullptr;  // m
  const double* rhs_bot = nullptr;  // n, NULL = zeros
  double* x = nullptr;              // n, in: x0, out: x
  double eps = 1e-10, nu = INFINITY, tol = 0.0, norm_ref = 1.0, mu = 0.0;
  int fixed_len = -1;
  long long maxit = 1000000;
  int check_gap = 10;
  bool x_zero = false;  // x0 is zero: the phase-start residual is the right-hand side
};

struct PhaseResult {
  long long iters = 0;
  int reason = R_NONE;
  int checks = 0;
  double ne_res = -1.0;  // last explicit check, -1 if none
};

class LsqrEngine {
 public:
  // mode: 0 FP64 products, 1 FP32 products and sums, 2 compensated FP32 (see lsqr.cu)
  // dense_pass: 0 the fused single-read A pass where it applies with FP32 products
  // (mode 1), 1 always the two-pass form, 2 the fused pass where it applies (modes 1, 2)
  void setup(cudaStream_t st, const MatView& A, int mode, int graph_iters, int dense_pass = 0);
  bool fused_pass() const { return fused_.ok; }
  const FusedPlan& fused_plan() const { return fused_; }
  void set_profile(bool on) { profile_ = on; }
  KernelProfile prof;
  PhaseResult run_phase(const PrecondDev& P, const PhaseArgs& a);
  // ||A_delta^T (rhs - A_delta x)|| / norm_ref in FP64 (rhs_bot NULL = 0).  With
  // screen_tol > 0 and FP32 values in an FP32-product form, a value above 100 screen_tol
  // may come from compensated FP32 products; every value at or below it is FP64.
  double ne_residual(const double* rhs_top, const double* rhs_bot, const double* x, double delta,
                     double norm_ref, double screen_tol = 0.0);
  // y = alpha A x + beta y (trans 0) or y = A^T x (trans 1), FP64 or mixed products.
  void matvec(int trans, const double* x, double* y, double alpha, double beta, bool fp64);
  double norm2(const double* v, int64_t n);
  // Right-hand side of the correction form at x: rhs_bot = g / delta with
  // g = A^T (b - A x) - mu x formed with FP64 products.
  void correction_rhs(const double* b, const double* x, double delta, double* rhs_bot);
  // out = P^{-1} w (and P^{-2} w in out2 when not NULL)
  void apply_precond(const PrecondDev& P, const double* w, double* out, double* out2);
  cudaStream_t stream() const { return st_; }

 private:
  void launch_iteration(const PrecondDev& P, bool init);
  void launch_k1(bool init, const double* z);
  void launch_k2(bool init, bool fused_v);
  // fused dense A pass (one read of A) followed by the column sums; non-init steps only
  void launch_fused(const double* z, bool fused_v);
  void launch_pre(const PrecondDev& P, const double* w, double* o1, double* o2, bool in_phase,
                  bool init);
  void flush_x();
  void matvec_md(int trans, const double* x, double* y, double alpha, double beta, int md);
  double ne_residual_md(const double* rhs_top, const double* rhs_bot, const double* x,
                        double delta, double norm_ref, int md);

  cudaStream_t st_ = nullptr;
  MatView A_;
  int mode_ = 0, graph_iters_ = 16;
  bool vec_ = false;  // dense rows 16-byte aligned: vector loads
  int64_t m_ = 0, n_ = 0;
  int k1_blocks_ = 0, k2_blocks_ = 0, k2_rchunks_ = 1, red_cap_ = 0;
  DBuf<LsqrCtl> ctl_;
  DBuf<double> u_, v_, z_, g_, d_, red_, part_, q1_, ct_, c2t_, q3_, q3b_, r_, q_, qpart_;
  DBuf<float> zh_, zl_, uh_, ul_;  // FP32 hi/lo splits of z' and u' (modes 1, 2)
  DBuf<double> scal_;
  DBuf<unsigned int> cnt_;
  FusedPlan fused_;
  DBuf<int> ferr_;  // set by the fused pass when a bounded wait gave up
  double* x_ = nullptr;
  bool x0_zero_ = false;  // the phase being started has x0 = 0
  bool profile_ = false;
  std::vector<cudaEvent_t> ev_;
  int kernels_per_iter_ = 0;
  void record(int slot);
  void ensure_events(int n);
  void harvest(int iters, int ell);
};

}  // namespace apl
