// Kernels of the sketch and of the incremental CUR refinement (Section 5.1,
// Algorithms IterativeCUR and augmentCUR).
#pragma once
#include "common.cuh"

namespace apl {

// The problem matrix as the kernels see it.  Dense: row-major `vals` (m x n, ld).
// CSR: rowptr/colidx/vals plus the library's CSC copy colptr/rowidx/cvals.
struct MatView {
  int fmt = 0;     // 0 dense row-major, 1 CSR
  int dtype = 0;   // 0 f64, 1 f32
  int64_t m = 0, n = 0, ld = 0, nnz = 0;
  const void* vals = nullptr;
  const int* rowptr = nullptr;
  const int* colidx = nullptr;
  const int* colptr = nullptr;
  const int* rowidx = nullptr;
  const void* cvals = nullptr;
};

// Y = S A (s x n column-major) in canonical order: Y(r, j) sums sign * A(i, j) over the
// rows i of A mapped to r, in ascending i, in FP64, then scales by `scale` once.
// tptr/ti/tsgn: for every sketch row r, the ascending list of rows i of A with S(r,i)
// nonzero (tptr has s+1 entries).  srows (m x xi) maps row i to its sketch rows.
void sketch(cudaStream_t st, const MatView& A, int s, int xi, const int* tptr, const int* ti,
            const signed char* tsgn, const int* srows, const signed char* ssign, double scale,
            double* Y);

// Y = S A (s x n column-major FP64) for a dense sketching operator S (s x m column-major
// FP64, device): CSR A by its CSC copy (FP64 products in ascending row order), dense A by
// row chunks through dgemm (the dense routines' products: compensated FP32 by default).
// Needs the calling context's dense workspace installed.
void operator_sketch(cudaStream_t st, const MatView& A, int s, const double* S, double* Y,
                     DBuf<double>& chunk);

// Partial-pivoting selection on X (N x K) in place: X(i, c) = X[i * rs + c * cs].
// Performs k elimination steps; piv_host receives the pivot rows (original indices),
// the return value is the number of nonzero pivots taken, *margin the smallest
// relative gap between the best and second-best candidate magnitudes.
struct LuppWork {
  DBuf<int> pos_of, row_at, piv;
  DBuf<double> pval, psec;
  DBuf<int> ppos;
  DBuf<long long> cv, cs;  // cooperative form: partial candidates, two buffers
  DBuf<int> cp, cr;
  DBuf<unsigned int> counter;  // [0] arrivals / last-block counter, [1] barrier generation
  DBuf<double> scal;   // [0] margin
  DBuf<int> iscal;     // [0] nz, [1] stopped, [2] a barrier wait gave up
  // all steps in one cooperative launch; owners that run selections concurrently on
  // several streams keep this off (one launch per step)
  bool cooperative = true;
};
int lupp_select(cudaStream_t st, int64_t N, int64_t K, double* X, int64_t rs, int64_t cs, int k,
                LuppWork& w, std::vector<int>& piv_host, double* margin);

// Column gathers of A into an FP64 column-major block (rows x k, ld ldo).
void gather_cols(cudaStream_t st, const MatView& A, const int* idx, int k, const int* colmap,
                 double* out, int64_t ldo);
// Row gathers of A transposed: out (n x k column-major) holds A(idx, :)^T.
void gather_rows_T(cudaStream_t st, const MatView& A, const int* idx, int k, double* out,
                   int64_t ldo);
// Append rows A(idx, :) to R (column-major, ld ldr) starting at row r0 (dense A only).
void append_rows(cudaStream_t st, const MatView& A, const int* idx, int k, double* R, int64_t ldr,
                 int64_t r0);
// Cross A(rI, cJ) as dense |rI| x |cJ| column-major (ld ldo).  colmap maps a column of A
// to its position in cJ (or -1); it is used for CSR.
void gather_cross(cudaStream_t st, const MatView& A, const int* rI, int nI, const int* cJ, int nJ,
                  const int* colmap, double* out, int64_t ldo);
// out (k x ncols) = rows idx of the column-major block B (ld ldb).
void gather_rows_cm(cudaStream_t st, const double* B, int64_t ldb, int64_t ncols, const int* idx,
                    int k, double* out, int64_t ldo);

// E_col = A(:, J+) - C X for CSR A (X: ell x kb column-major).  Rows in I are zeroed.
void ecol_csr(cudaStream_t st, const MatView& A, const int* colpos, const int* colpos_plus,
              const int* rowpos, const double* X, int64_t ldx, int kb, double* out);
// E_row = Y - Z A(I, :) for CSR A (Z: s x ell column-major).
void erow_csr(cudaStream_t st, const MatView& A, const int* rowpos, const double* Z, int s,
              const double* Y, double* E);
// G (nq x kb, ld ldg) = A(:, Jall)^T Cp for CSR A, Cp dense m x kb column-major.
void gram_csr(cudaStream_t st, const MatView& A, const int* Jall, int nq, const double* Cp,
              int kb, double* G, int64_t ldg);

void zero_cols_cm(cudaStream_t st, double* E, int64_t ldE, int64_t rows, const int* cols, int k);
void zero_rows_cm(cudaStream_t st, double* E, int64_t ldE, int64_t ncols, const int* rows, int k);
// rho = factor * max_q ||T(:, q)||  (T: s x r column-major), written to *out (device).
void colnorm_max(cudaStream_t st, const double* T, int s, int r, double factor, double* out);
// map[idx[q]] = base + q
void set_map(cudaStream_t st, int* map, const int* idx, int k, int base);
void fill_int(cudaStream_t st, int* p, int64_t n, int v);

}  // namespace apl
