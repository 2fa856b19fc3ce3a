// Small dense FP64 linear algebra used by the CUR and preconditioner steps.
// All matrices here are column-major with explicit leading dimensions.
#pragma once
#include "common.cuh"

namespace apl {

// C = alpha op(A) op(B) + beta C  (op = transpose when trans != 0), C is M x N.
void dgemm(cudaStream_t st, int transA, int transB, int64_t M, int64_t N, int64_t K,
           double alpha, const double* A, int64_t lda, const double* B, int64_t ldb,
           double beta, double* C, int64_t ldc);

// hi[r + c rows] = fl32(A(r, c)), lo = fl32(A(r, c) - hi): the compensated-FP32 operand
// split of a rows x cols block of A (leading dimension ld) into compact arrays.
void split_hilo(cudaStream_t st, int64_t rows, int64_t cols, const double* A, int64_t ld,
                float* hi, float* lo);

// Solve op(A) X = B (left) or X op(A) = B (right) in place of B (M x N).
// uplo: 'L' or 'U' as stored; unit: unit diagonal assumed.
void dtrsm(cudaStream_t st, bool left, char uplo, bool trans, bool unit, int64_t M, int64_t N,
           const double* A, int64_t lda, double* B, int64_t ldb);

// In-place upper Cholesky of the n x n matrix A (upper triangle read, lower part
// zeroed).  Writes 0 to *info_dev on success, k+1 when pivot k is not positive.
void dpotrf_upper(cudaStream_t st, int64_t n, double* A, int64_t lda, int* info_dev);

// Thin QR of E (n x k) by Cholesky QR twice: E <- Q, R (k x k, ldr) upper.
// Returns false if a Cholesky step broke down.
bool cholqr2(cudaStream_t st, int64_t n, int64_t k, double* E, int64_t lde, double* R,
             int64_t ldr, double* work, int* info_dev);

// One-sided Jacobi on the columns of the square B (l x l, in place, destroyed).
// sigma receives the singular values of B in descending order and U (l x l, ldu) the
// matching left singular vectors (normalised columns).  With B = M^T these are the
// singular values and right singular vectors of M.  flag_dev is device scratch of at
// least 3 ints.  Warm start: W0 (l0 x l0, ld l0, orthogonal, l0 <= l) pre-rotates the first
// l0 columns of B (the FP32 stage then starts from them nearly orthogonal when B's leading
// block is close to the matrix W0 came from).  Wout (l x l, ld l), when given, receives
// the FP32 stage's whole rotation (orthogonal to FP64 accuracy) and *wout_l its order, or
// 0 when that stage did not run.  Returns the sweep count; throws ST_ETIMEOUT when a
// bounded wait of a sweep kernel gave up.
int jacobi_left(cudaStream_t st, int64_t l, double* B, int64_t ldb, double* U, int64_t ldu,
                double* sigma, int* flag_dev, const double* W0 = nullptr, int64_t l0 = 0,
                double* Wout = nullptr, int64_t* wout_l = nullptr);

// sigma_min(M) = 1 / ||M^{-1}||_2 for M^{-1} (L x L, column-major, ld ldm) by `iters` steps
// of power iteration on M^{-T} M^{-1} from a fixed start vector; work holds 3 L + 1
// doubles.  Converges from above.
double power_sigma_min(cudaStream_t st, int64_t L, const double* Minv, int64_t ldm, double* work,
                       int iters);

// Elementwise helpers.
void dcopy2d(cudaStream_t st, int64_t rows, int64_t cols, const double* src, int64_t lds,
             double* dst, int64_t ldd, bool transpose);
void dset2d(cudaStream_t st, int64_t rows, int64_t cols, double v, double* dst, int64_t ldd);
void dzero_lower(cudaStream_t st, int64_t n, double* A, int64_t lda);
void dset_diag(cudaStream_t st, int64_t n, double v, double* A, int64_t lda);
void dadd_diag(cudaStream_t st, int64_t n, double v, double* A, int64_t lda);
void dgather_cols(cudaStream_t st, int64_t rows, const double* src, int64_t lds,
                  const int* idx, int64_t k, double* dst, int64_t ldd);

}  // namespace apl
