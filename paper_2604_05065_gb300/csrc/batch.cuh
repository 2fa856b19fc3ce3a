// Grouped multi-right-hand-side LSQR for a batch of independent problems.
//
// Every problem p has its own A_p (FP32 values, dense row-major or CSR with a CSC copy),
// its own CUR preconditioner and R right-hand sides that share it.  One launch of each
// kernel covers all problems of the batch: the launch walks a work list of
// (problem, tile) items, so problems of uneven m and n share the GPU, and products with
// A become products with an n x R block (SpMM / tall-skinny GEMM) whose A tile is read
// once for all R right-hand sides.  A, the preconditioner factors and the Krylov
// vectors are FP32 with FP32 products; the bidiagonalisation scalars, x and its search
// direction are FP64.  Every phase starts from the normal-equation residual
// g = A^T (b - A x) - mu x formed with compensated FP32 products (about 2^-44 relative)
// and solves for the correction with the right-hand side [0; g / delta], which has the
// same normal equations (and, in exact arithmetic, the same iterates) as the paper's warm
// start but shrinks with g, so the phases form an FP64-accurate iterative refinement;
// the convergence test uses the same residual.
#pragma once
#include <memory>
#include <vector>

#include "common.cuh"
#include "cur.cuh"
#include "lsqr.cuh"

namespace apl {

constexpr int BATCH_MAX_RHS = 16;

// One problem as the grouped kernels see it (device array, rebuilt at phase start).
struct BProb {
  int64_t m = 0, n = 0, lda = 0;
  int fmt = 0;      // 0 dense row-major FP32, 1 CSR FP32 (+ CSC)
  int ell = 0;      // rank of the preconditioner in use (0: none)
  int active = 0;   // has a pair in the running phase that is not done
  int vec4 = 0;     // dense rows 16-byte aligned: float4 loads
  double delta = 0, mu = 0;
  const float* A = nullptr;
  const int* rowptr = nullptr;
  const int* colidx = nullptr;
  const float* vals = nullptr;
  const int* colptr = nullptr;
  const int* rowidx = nullptr;
  const float* cvals = nullptr;
  const float* Q = nullptr;   // n x ell, row-major
  const float* VM = nullptr;  // ell x ell, row-major, VM[k * ell + j] = V_M(k, j)
  const float* c1 = nullptr;  // ell: coefficients c of P^-1 = I + Vhat diag(c) Vhat^T
  float* U = nullptr;   // (m + n) x RS, unnormalised u (top m rows: A part)
  float* V = nullptr;   // n x RS unnormalised v
  float* Z = nullptr;   // n x RS unnormalised z = P^-1 v (formed from V each iteration)
  float* G = nullptr;   // n x RS, g = A^T u_top + delta u_bot
  float* q = nullptr;   // ell x RS, Q^T w
  float* t = nullptr;   // ell x RS, c (VM^T q)
  float* s = nullptr;   // ell x RS, VM t
  double* X = nullptr;  // n x RS solution
  double* D = nullptr;  // n x RS search direction in x space
  const double* B = nullptr;  // m x RS right-hand sides (NULL: zero, the adjoint solves)
  const double* Gx = nullptr; // n x RS forcing added to A^T (b - A x) - mu x (adjoint: the
                              // incoming gradient), or NULL
  float* Xh = nullptr;  // n x RS hi/lo FP32 split of X
  float* Xl = nullptr;
  float* Rh = nullptr;  // m x RS hi/lo FP32 split of the residual
  float* Rl = nullptr;
  int b0 = 0, b1 = 0;   // item range of the A-pass list (beta^2 partial sums)
  int a0 = 0, a1 = 0;   // item range of the expansion list (alpha^2 partial sums)
  int g0 = 0, g1 = 0;   // item range of the residual A^T list (norm partial sums)
  int q0 = 0, q1 = 0;   // item range of the residual list (beta^2 partial sums at init)
};

// LSQR state of one (problem, right-hand side) pair; all FP64.
struct BPair {
  double alpha, beta, rhobar, phibar, phibar_prev, beta1, anorm2, rate1, arnorm0;
  double su, sv;      // u = su U, v = sv V, z = sv Z
  double ca, cb;      // A pass: U <- ca A Z - cb U
  double cprev;       // expansion: V <- g + Q s1 - cprev V (likewise Z)
  double xc, dc;      // x += xc D ; D <- sv Z - dc D
  double nu, sig_ell, eps, inner, tol, normP, norm_ref;
  long long it, maxit;
  int live;           // takes part in the running phase and has not stopped
  int upd;            // 0 none, 1 D = sv Z (phase start), 2 x and D update
  int reason, pad;
};

struct BItem {
  int p, kind;
  int64_t r0, r1;
};

struct BatchSrc {
  MatView A;          // FP32 values; CSR views carry the CSC copy
  const double* b;    // m x R, column-major
};

class BatchEngine {
 public:
  ~BatchEngine();
  void setup(cudaStream_t st, const std::vector<BatchSrc>& src, int R, double mu);
  int nprob() const { return (int)hp_.size(); }
  int rhs() const { return R_; }
  // Preconditioner of problem p from the FP64 factors of the single-problem build:
  // Q (n x ell, column-major, ld ldq), VM (ell x ell, column-major), coefficients.
  void set_precond(int p, const PrecondDev& P);
  void clear_precond(int p);
  void zero_x();
  // One phase for the pairs with mask[p * R + r] != 0; nu[p] per problem, maxit per
  // pair.  Returns the iterations and stop reasons per pair (index p * R + r).
  void run_phase(const std::vector<char>& mask, const std::vector<double>& nu, double eps,
                 double tol, const std::vector<long long>& maxit, std::vector<long long>& iters,
                 std::vector<int>& reasons);
  // ||A^T (b - A x) - mu x|| / ||A^T b|| for the masked pairs (index p * R + r; others 0).
  void ne_residual(const std::vector<char>& mask, std::vector<double>& ne);
  double norm_ref(int p, int r) const { return norm_ref_[(size_t)p * RS_ + r]; }
  void get_x(int p, double* x_out) const;  // n x R column-major, device
  // Adjoint mode: the phases solve (A^T A + mu I) lambda = g for the incoming gradients
  // g of every problem (gx[p]: n x R column-major FP64, device) with the preconditioners
  // in place: b is taken as zero, g is added to the normal-equation residual, x restarts
  // at zero and the residuals are relative to ||g||.  end_adjoint restores the forward
  // right-hand sides, solutions and references.
  void begin_adjoint(const std::vector<const double*>& gx);
  void end_adjoint();
  // Picks the dense tile shapes by timing the candidates on this batch.
  void autotune();
  int tuned_rw() const { return rw_; }
  int tuned_cw() const { return cw_; }
  int64_t launches_per_iter() const { return launches_per_iter_; }

 private:
  void build_items();
  void upload_probs();
  void launch_iteration(bool init);
  void launch_gn(const DBuf<BItem>& items, int nitems, int rw);
  void launch_gt(const DBuf<BItem>& items, int nitems, int cw);
  void launch_residual(bool init);
  void launch_gtr(bool init);
  cudaStream_t st_ = nullptr;
  int R_ = 0, RS_ = 0;
  double mu_ = 0, delta_ = 0;
  std::vector<BProb> hp_;
  std::unique_ptr<DBuf<float>[]> qf_, vmf_, c1f_, fvec_;
  std::unique_ptr<DBuf<double>[]> dvec_;
  DBuf<BProb> dp_;
  DBuf<BPair> pairs_;
  DBuf<double> part_, ne_part_;
  DBuf<int> live_count_;
  // work lists
  DBuf<BItem> it_apass_, it_gta_, it_gtq_, it_gtqv_, it_gtv_, it_gnv_, it_exp_, it_expz_,
      it_vec_, it_res_, it_gtr_;
  int n_apass_ = 0, n_gta_ = 0, n_gtq_ = 0, n_gtqv_ = 0, n_gtv_ = 0, n_gnv_ = 0, n_exp_ = 0,
      n_expz_ = 0, n_vec_ = 0, n_res_ = 0, n_gtr_ = 0;
  std::vector<double> norm_ref_;    // per pair, index p * RS + r
  std::vector<double> saved_ref_;   // forward references during the adjoint
  std::unique_ptr<DBuf<double>[]> adj_;  // per problem: saved X (n x RS), then g (n x RS)
  std::vector<const double*> saved_b_;
  std::vector<double> normP_, sig_ell_;  // per problem
  int rw_ = 4, cw_ = 2;
  size_t gn_smem_ = 0;
  int64_t launches_per_iter_ = 0;
  bool items_dirty_ = true;
};

}  // namespace apl
