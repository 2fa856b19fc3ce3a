// APLICUR driver (Algorithm "APLICUR: detailed implementation") and the C ABI.
// The host keeps the state machine (rank steps, rebuild decisions, phases); every
// operation with an m- or n-sized extent runs in the library's kernels.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <exception>
#include <mutex>
#include <thread>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/aplicur.h"
#include "batch.cuh"
#include "dense.cuh"
#include "lsqr.cuh"
#include "tcsketch.cuh"

using namespace apl;

namespace {

// ---- project random generator (SplitMix64, Steele, Lea & Flood 2014) ------------------
constexpr uint64_t GOLDEN = 0x9E3779B97F4A7C15ULL;
inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
inline uint64_t stream_state(uint64_t seed, uint64_t t, uint64_t i) {
  return mix64(seed ^ ((t & 0xFFULL) << 56) ^ (i & ((1ULL << 56) - 1)));
}

// Sparse sign embedding (Section 5.1): column i holds xi distinct rows in [0, s).
void draw_sketch(uint64_t seed, int s, int64_t m, int xi, std::vector<int>& rows,
                 std::vector<int8_t>& signs) {
  rows.assign((size_t)m * xi, 0);
  signs.assign((size_t)m * xi, 1);
  for (int64_t i = 0; i < m; ++i) {
    uint64_t st = stream_state(seed, 1, (uint64_t)i);
    int cnt = 0;
    int* r = rows.data() + i * xi;
    while (cnt < xi) {
      st += GOLDEN;
      const uint64_t z = mix64(st);
      const int v = (int)(((z >> 32) * (uint64_t)s) >> 32);
      bool taken = false;
      for (int k = 0; k < cnt; ++k) taken = taken || r[k] == v;
      if (!taken) r[cnt++] = v;
    }
    uint64_t ss = stream_state(seed, 2, (uint64_t)i);
    for (int k = 0; k < xi; ++k) {
      ss += GOLDEN;
      signs[i * xi + k] = (mix64(ss) >> 63) == 0 ? 1 : -1;
    }
  }
}

// Dense sketching operators of the appendix "Sketch comparison", s x m column-major.
// Gaussian embedding: entry (r, c) from stream (4, c s + r) by Box-Muller, divided by
// sqrt(s).  Subsampled randomized Hadamard transform: column signs d_c from the first draw
// of stream (5, c) (bit 63 clear: +1), s distinct rows p_r of the m' x m' Walsh-Hadamard
// matrix (m' the power of two >= m) drawn in turn from stream (6, 0) as
// ((z >> 32) m') >> 32, entry (-1)^popcount(p_r & c) d_c / sqrt(s).
void draw_gaussian_sketch(uint64_t seed, int s, int64_t m, std::vector<double>& S) {
  S.resize((size_t)s * m);
  const double two_pi = 2.0 * M_PI, sc = 1.0 / std::sqrt((double)s);
  for (int64_t idx = 0; idx < (int64_t)s * m; ++idx) {
    const uint64_t st = stream_state(seed, 4, (uint64_t)idx);
    const uint64_t z1 = mix64(st + GOLDEN);
    const uint64_t z2 = mix64(st + 2 * GOLDEN);
    const double u1 = (double)((z1 >> 11) + 1) * 0x1.0p-53;
    const double u2 = (double)(z2 >> 11) * 0x1.0p-53;
    S[idx] = std::sqrt(-2.0 * std::log(u1)) * std::cos(two_pi * u2) * sc;
  }
}

void draw_srht_sketch(uint64_t seed, int s, int64_t m, std::vector<double>& S) {
  uint64_t mp = 1;
  while ((int64_t)mp < m) mp <<= 1;
  APL_REQUIRE((uint64_t)s <= mp, "SRHT: sketch rows exceed the padded length");
  std::vector<uint64_t> rows;
  uint64_t st = stream_state(seed, 6, 0);
  while ((int)rows.size() < s) {
    st += GOLDEN;
    const uint64_t p = ((mix64(st) >> 32) * mp) >> 32;
    if (std::find(rows.begin(), rows.end(), p) == rows.end()) rows.push_back(p);
  }
  S.resize((size_t)s * m);
  const double sc = 1.0 / std::sqrt((double)s);
  for (int64_t c = 0; c < m; ++c) {
    const double d = (mix64(stream_state(seed, 5, (uint64_t)c) + GOLDEN) >> 63) == 0 ? 1.0 : -1.0;
    for (int r = 0; r < s; ++r)
      S[(size_t)c * s + r] = (__builtin_popcountll(rows[r] & (uint64_t)c) & 1) ? -d * sc : d * sc;
  }
}

// Gaussian n x r matrix (column-major) by Box-Muller on the generator's uniforms.
void draw_gaussian(uint64_t seed, int64_t n, int r, std::vector<double>& W) {
  W.resize((size_t)n * r);
  const double two_pi = 2.0 * M_PI;
  for (int64_t idx = 0; idx < n * r; ++idx) {
    const uint64_t st = stream_state(seed, 3, (uint64_t)idx);
    const uint64_t z1 = mix64(st + GOLDEN);
    const uint64_t z2 = mix64(st + 2 * GOLDEN);
    const double u1 = (double)((z1 >> 11) + 1) * 0x1.0p-53;
    const double u2 = (double)(z2 >> 11) * 0x1.0p-53;
    W[idx] = std::sqrt(-2.0 * std::log(u1)) * std::cos(two_pi * u2);
  }
}

// ---- small kernels local to the driver --------------------------------------------------
__global__ void add2d_kernel(int64_t rows, int64_t cols, const double* src, int64_t lds,
                             double* dst, int64_t ldd) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= rows * cols) return;
  const int64_t r = e % rows, c = e / rows;
  dst[r + c * ldd] += src[r + c * lds];
}
__global__ void axpy_kernel(int64_t n, double a, const double* x, double* y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] += a * x[i];
}

__global__ void scale_kernel(int64_t n, const double* s, double a, double* d) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) d[i] = a * s[i];
}
__global__ void dot_kernel(int64_t n, const double* a, const double* b, double* out) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s = fma(a[i], b[i], s);
  s = block_sum(s, sh);
  if (threadIdx.x == 0) *out = s;
}
// grad_A(i, j) = r_i lambda_j - (A lambda)_i x_j, row-major, ld n.
template <typename T>
__global__ void rank2_kernel(int64_t m, int64_t n, const double* r, const double* lam,
                             const double* al, const double* x, T* G) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m * n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / n, j = e - i * n;
    G[e] = (T)(r[i] * lam[j] - al[i] * x[j]);
  }
}

struct StepRec { int ell; double rho; int rebuilt; double margin; };
struct PhaseRec { int ell; long long iters; int reason; double ne; };

}  // namespace

struct aplicur_ctx {
  cudaStream_t st = nullptr;
  bool own_stream = false;
  MatView A;
  DBuf<int> colptr, rowidx;
  DBuf<double> cv64;
  DBuf<float> cv32;
  // The matrix the CUR is taken of: A itself, or A_mu = [A; delta I] ((m + n) x n, values
  // in A's type) for the SVD-free variant with mu > 0.  cm is its row count.
  MatView CA;
  int64_t cm = 0;
  DBuf<int> ca_rowptr, ca_colidx, ca_colptr, ca_rowidx;
  DBuf<double> ca_v64, ca_cv64;
  DBuf<float> ca_v32, ca_cv32;
  const double* b = nullptr;
  double mu = 0, delta = 0, eps_cur = 0;
  int bsize = 0, s = 0, xi = 0, r = 0;
  int64_t m = 0, n = 0, kmax = 0;
  aplicur_options opt{};
  std::vector<int> rp_phases;
  std::vector<int8_t> rp_rebuild;
  bool replay = false;
  // sketch
  DBuf<int> srows, tptr, ti;
  DBuf<signed char> ssign, tsgn;
  DBuf<double> Y, E, Et, W, T, scal;
  // CUR state
  int ell = 0, cap = 0;
  std::vector<int> I, J;
  DBuf<int> I_d, J_d, Jp_d, Ip_d, colpos, colpos_plus, rowpos;
  DBuf<double> LU, QR, TR, TC, Cbuf, Rbuf;
  DBuf<double> Ecol, Xb, U12, L21, Gb, Cp, Zb, P2b, work;
  DBuf<int> info;
  LuppWork lw;
  // preconditioner
  DBuf<double> Mb, VM, sigma, coef, coef2;
  DBuf<double> Wprev, Wnext;  // rotation of the last build's FP32 Jacobi stage (warm start)
  int64_t wl = 0;             // its order (0: none)
  PrecondDev P;
  double sighat = 1.0;
  std::vector<double> sig_host;
  // solve
  LsqrEngine eng;
  DBuf<double> x, tmp_m, tmp_n, tmp_n2, lam;
  DBuf<double> dx, rbot, zm;  // correction-form phases (FP32 products): dx, g / delta, 0
  double norm_Atb = 0;
  bool solved = false;
  std::vector<StepRec> steps;
  std::vector<PhaseRec> phases;
  aplicur_stats stats{};
  std::string err;
  float setup_ms = 0;
  ProfSink sink;
  DenseWork dw;  // scratch of the dense routines, used on st only
  Allocator alloc_;       // caller's device allocator (empty: cudaMallocAsync)
  bool poisoned = false;  // a bounded device wait gave up: buffers undefined
  TcSketchWork tcw;       // tensor-core sketch (dense operators in bfloat16)
};

namespace {

void ctx_grow(aplicur_ctx* h, int need) {
  if (need <= h->cap) return;
  cudaStream_t st = h->st;
  const int64_t kmax = h->kmax;
  int nc = (int)std::min<int64_t>(kmax, std::max<int64_t>(std::max(2 * h->cap, need), 64));
  const int64_t oc = h->cap;
  auto regrow_sq = [&](DBuf<double>& B) {
    DBuf<double> nb;
    nb.alloc((size_t)nc * nc, st);
    nb.zero(st);
    if (oc > 0 && B.p) dcopy2d(st, oc, oc, B.p, oc, nb.p, nc, false);
    B.swap(nb);
  };
  regrow_sq(h->LU);
  regrow_sq(h->TR);
  regrow_sq(h->TC);
  auto regrow_cols = [&](DBuf<double>& B, int64_t rows) {
    DBuf<double> nb;
    nb.alloc((size_t)rows * nc, st);
    if (oc > 0 && B.p)
      APL_CUDA(cudaMemcpyAsync(nb.p, B.p, (size_t)rows * oc * sizeof(double),
                               cudaMemcpyDeviceToDevice, st));
    B.swap(nb);
  };
  const double* oldQ = h->QR.p;
  regrow_cols(h->QR, h->n);
  // the preconditioner reads the leading columns of Q_R in place
  if (h->P.Q == oldQ) h->P.Q = h->QR.p;
  if (h->CA.fmt == 0) {
    regrow_cols(h->Cbuf, h->cm);
    DBuf<double> nb;
    nb.alloc((size_t)nc * h->n, st);
    if (oc > 0 && h->Rbuf.p) dcopy2d(st, oc, h->n, h->Rbuf.p, oc, nb.p, nc, false);
    h->Rbuf.swap(nb);
  }
  const int bs = h->bsize;
  h->Xb.alloc((size_t)nc * bs, st);
  h->U12.alloc((size_t)nc * bs, st);
  h->L21.alloc((size_t)nc * bs, st);
  h->Gb.alloc((size_t)nc * bs, st);
  h->P2b.alloc((size_t)nc * bs, st);
  h->Zb.alloc((size_t)h->s * nc, st);
  h->cap = nc;
  APL_CUDA(cudaStreamSynchronize(st));
}

// CSC copy (colptr, rowidx, values) of the CSR matrix V (m rows), attached to V.
void build_csc(cudaStream_t st, MatView& V, int64_t m, DBuf<int>& colptr_b, DBuf<int>& rowidx_b,
               DBuf<double>& cv64_b, DBuf<float>& cv32_b) {
  const int64_t n = V.n, nnz = V.nnz;
  std::vector<int> rp(m + 1), ci(nnz);
  APL_CUDA(cudaMemcpyAsync(rp.data(), V.rowptr, (m + 1) * sizeof(int), cudaMemcpyDeviceToHost, st));
  if (nnz)
    APL_CUDA(cudaMemcpyAsync(ci.data(), V.colidx, nnz * sizeof(int), cudaMemcpyDeviceToHost, st));
  const size_t vs = V.dtype == 0 ? 8 : 4;
  std::vector<char> vals(nnz * vs), cvals(nnz * vs);
  if (nnz)
    APL_CUDA(cudaMemcpyAsync(vals.data(), V.vals, nnz * vs, cudaMemcpyDeviceToHost, st));
  APL_CUDA(cudaStreamSynchronize(st));
  APL_REQUIRE(rp[0] == 0 && rp[m] == nnz, "CSR rowptr inconsistent with nnz");
  std::vector<int> cp(n + 1, 0), ri(nnz);
  for (int64_t e = 0; e < nnz; ++e) {
    APL_REQUIRE(ci[e] >= 0 && ci[e] < n, "CSR column index out of range");
    cp[ci[e] + 1]++;
  }
  for (int64_t j = 0; j < n; ++j) cp[j + 1] += cp[j];
  std::vector<int> cur(cp.begin(), cp.end() - 1);
  for (int64_t i = 0; i < m; ++i) {
    APL_REQUIRE(rp[i + 1] >= rp[i], "CSR rowptr not monotone");
    for (int e = rp[i]; e < rp[i + 1]; ++e) {
      const int p = cur[ci[e]]++;
      ri[p] = (int)i;
      std::memcpy(&cvals[p * vs], &vals[e * vs], vs);
    }
  }
  colptr_b.alloc(n + 1, st);
  rowidx_b.alloc(std::max<int64_t>(nnz, 1), st);
  APL_CUDA(cudaMemcpyAsync(colptr_b.p, cp.data(), (n + 1) * sizeof(int), cudaMemcpyHostToDevice, st));
  if (nnz)
    APL_CUDA(cudaMemcpyAsync(rowidx_b.p, ri.data(), nnz * sizeof(int), cudaMemcpyHostToDevice, st));
  if (V.dtype == 0) {
    cv64_b.alloc(std::max<int64_t>(nnz, 1), st);
    if (nnz) APL_CUDA(cudaMemcpyAsync(cv64_b.p, cvals.data(), nnz * vs, cudaMemcpyHostToDevice, st));
    V.cvals = cv64_b.p;
  } else {
    cv32_b.alloc(std::max<int64_t>(nnz, 1), st);
    if (nnz) APL_CUDA(cudaMemcpyAsync(cv32_b.p, cvals.data(), nnz * vs, cudaMemcpyHostToDevice, st));
    V.cvals = cv32_b.p;
  }
  V.colptr = colptr_b.p;
  V.rowidx = rowidx_b.p;
  APL_CUDA(cudaStreamSynchronize(st));
}

void build_csc(aplicur_ctx* h) {
  build_csc(h->st, h->A, h->m, h->colptr, h->rowidx, h->cv64, h->cv32);
}

template <typename T>
__global__ void amu_diag_kernel(int64_t m, int64_t n, T delta, T* V) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) V[(m + j) * n + j] = delta;
}

// A_mu = [A; delta I] ((m + n) x n, delta rounded to A's value type) as the CUR matrix:
// dense row-major with ld n, or CSR with one entry delta in each appended row (and its CSC).
void build_amu(aplicur_ctx* h) {
  cudaStream_t st = h->st;
  const int64_t m = h->m, n = h->n;
  const MatView& A = h->A;
  MatView V = A;
  V.m = m + n;
  V.colptr = nullptr; V.rowidx = nullptr; V.cvals = nullptr;
  const size_t es = A.dtype == 0 ? 8 : 4;
  if (A.fmt == 0) {
    void* buf;
    if (A.dtype == 0) { h->ca_v64.alloc((size_t)(m + n) * n, st); buf = h->ca_v64.p; }
    else { h->ca_v32.alloc((size_t)(m + n) * n, st); buf = h->ca_v32.p; }
    APL_CUDA(cudaMemcpy2DAsync(buf, n * es, A.vals, A.ld * es, n * es, m, cudaMemcpyDeviceToDevice, st));
    APL_CUDA(cudaMemsetAsync((char*)buf + (size_t)m * n * es, 0, (size_t)n * n * es, st));
    const unsigned g = (unsigned)cdiv(n, 256);
    if (A.dtype == 0) amu_diag_kernel<double><<<g, 256, 0, st>>>(m, n, h->delta, (double*)buf);
    else amu_diag_kernel<float><<<g, 256, 0, st>>>(m, n, (float)h->delta, (float*)buf);
    APL_LAUNCH_CHECK();
    V.ld = n;
    V.nnz = (m + n) * n;
    V.vals = buf;
  } else {
    const int64_t nnz = A.nnz;
    APL_REQUIRE(nnz + n < (1LL << 31), "A_mu: nnz + n exceeds int32 indexing");
    std::vector<int> rp(m + n + 1), ci(nnz + n);
    std::vector<char> vals((nnz + n) * es);
    APL_CUDA(cudaMemcpyAsync(rp.data(), A.rowptr, (m + 1) * sizeof(int), cudaMemcpyDeviceToHost, st));
    if (nnz) {
      APL_CUDA(cudaMemcpyAsync(ci.data(), A.colidx, nnz * sizeof(int), cudaMemcpyDeviceToHost, st));
      APL_CUDA(cudaMemcpyAsync(vals.data(), A.vals, nnz * es, cudaMemcpyDeviceToHost, st));
    }
    APL_CUDA(cudaStreamSynchronize(st));
    const double d64 = h->delta;
    const float d32 = (float)h->delta;
    for (int64_t j = 0; j < n; ++j) {
      rp[m + j + 1] = (int)(nnz + j + 1);
      ci[nnz + j] = (int)j;
      std::memcpy(&vals[(nnz + j) * es], A.dtype == 0 ? (const void*)&d64 : (const void*)&d32, es);
    }
    h->ca_rowptr.alloc(m + n + 1, st);
    h->ca_colidx.alloc(nnz + n, st);
    APL_CUDA(cudaMemcpyAsync(h->ca_rowptr.p, rp.data(), (m + n + 1) * sizeof(int), cudaMemcpyHostToDevice, st));
    APL_CUDA(cudaMemcpyAsync(h->ca_colidx.p, ci.data(), (nnz + n) * sizeof(int), cudaMemcpyHostToDevice, st));
    void* vb;
    if (A.dtype == 0) { h->ca_v64.alloc(nnz + n, st); vb = h->ca_v64.p; }
    else { h->ca_v32.alloc(nnz + n, st); vb = h->ca_v32.p; }
    APL_CUDA(cudaMemcpyAsync(vb, vals.data(), (nnz + n) * es, cudaMemcpyHostToDevice, st));
    V.rowptr = h->ca_rowptr.p;
    V.colidx = h->ca_colidx.p;
    V.vals = vb;
    V.nnz = nnz + n;
    build_csc(st, V, m + n, h->ca_colptr, h->ca_rowidx, h->ca_cv64, h->ca_cv32);
  }
  APL_CUDA(cudaStreamSynchronize(st));
  h->CA = V;
  h->cm = m + n;
}

void upload_sketch(aplicur_ctx* h, const std::vector<int>& rows, const std::vector<int8_t>& sg) {
  const int64_t m = h->cm;
  const int xi = h->xi, s = h->s;
  cudaStream_t st = h->st;
  for (size_t e = 0; e < rows.size(); ++e)
    APL_REQUIRE(rows[e] >= 0 && rows[e] < s, "sketch row index out of range");
  // transposed lists: rows i of A for each sketch row r, ascending i
  std::vector<int> tp(s + 1, 0), tl((size_t)m * xi);
  std::vector<int8_t> ts((size_t)m * xi);
  for (size_t e = 0; e < rows.size(); ++e) tp[rows[e] + 1]++;
  for (int r = 0; r < s; ++r) tp[r + 1] += tp[r];
  std::vector<int> cur(tp.begin(), tp.end() - 1);
  for (int64_t i = 0; i < m; ++i)
    for (int k = 0; k < xi; ++k) {
      const int r = rows[i * xi + k];
      const int p = cur[r]++;
      tl[p] = (int)i;
      ts[p] = sg[i * xi + k];
    }
  h->srows.alloc(rows.size(), st);
  h->ssign.alloc(rows.size(), st);
  h->tptr.alloc(s + 1, st);
  h->ti.alloc(rows.size(), st);
  h->tsgn.alloc(rows.size(), st);
  APL_CUDA(cudaMemcpyAsync(h->srows.p, rows.data(), rows.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  APL_CUDA(cudaMemcpyAsync(h->ssign.p, sg.data(), sg.size(), cudaMemcpyHostToDevice, st));
  APL_CUDA(cudaMemcpyAsync(h->tptr.p, tp.data(), (s + 1) * sizeof(int), cudaMemcpyHostToDevice, st));
  APL_CUDA(cudaMemcpyAsync(h->ti.p, tl.data(), tl.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  APL_CUDA(cudaMemcpyAsync(h->tsgn.p, ts.data(), ts.size(), cudaMemcpyHostToDevice, st));
  APL_CUDA(cudaStreamSynchronize(st));
}

void reset_cur(aplicur_ctx* h) {
  cudaStream_t st = h->st;
  h->ell = 0;
  h->I.clear();
  h->J.clear();
  fill_int(st, h->colpos.p, h->n, -1);
  fill_int(st, h->colpos_plus.p, h->n, -1);
  fill_int(st, h->rowpos.p, h->cm, -1);
  APL_CUDA(cudaMemcpyAsync(h->E.p, h->Y.p, (size_t)h->s * h->n * sizeof(double),
                           cudaMemcpyDeviceToDevice, st));
  if (h->LU.p) h->LU.zero(st);
  if (h->TR.p) h->TR.zero(st);
  if (h->TC.p) h->TC.zero(st);
  h->wl = 0;
  h->P = PrecondDev{};
  h->steps.clear();
  h->phases.clear();
}

// One rank step (Part 1 and Part 2 of the driver).  Returns the number of new indices;
// *exhausted is set when LUPP met a zero pivot before the block was complete.
int rank_step(aplicur_ctx* h, double* rho_out, bool* exhausted, double* margin) {
  DenseWorkScope dws(&h->dw);
  cudaStream_t st = h->st;
  const int64_t m = h->cm, n = h->n;
  const int s = h->s;
  const int ell = h->ell;
  const int kj = (int)std::min<int64_t>(h->bsize, h->kmax - ell);
  // capacity for the whole step before any ell-sized block is written
  ctx_grow(h, (int)std::min<int64_t>(h->kmax, ell + std::max(kj, 1)));
  // ---- column selection: LUPP on E_row^T with the chosen columns zeroed
  zero_cols_cm(st, h->E.p, s, s, h->J_d.p, ell);
  // E_row^T as an n x s column-major block: the elimination then reads columns
  // contiguously across threads
  dcopy2d(st, s, n, h->E.p, s, h->Et.p, n, true);
  std::vector<int> Jp, Ip;
  double mJ = INFINITY, mI = INFINITY;
  const int nzJ = lupp_select(st, n, s, h->Et.p, 1, n, kj, h->lw, Jp, &mJ);
  int k = 0;
  if (nzJ > 0) {
    APL_CUDA(cudaMemcpyAsync(h->Jp_d.p, Jp.data(), nzJ * sizeof(int), cudaMemcpyHostToDevice, st));
    set_map(st, h->colpos_plus.p, h->Jp_d.p, nzJ, 0);
    // ---- column residual E_col = A(:, J+) - C U R(:, J+)
    if (ell > 0) {
      gather_cross(st, h->CA, h->I_d.p, ell, h->Jp_d.p, nzJ, h->colpos_plus.p, h->U12.p, h->cap);
      dtrsm(st, true, 'L', false, true, ell, nzJ, h->LU.p, h->cap, h->U12.p, h->cap);
      dcopy2d(st, ell, nzJ, h->U12.p, h->cap, h->Xb.p, h->cap, false);
      dtrsm(st, true, 'U', false, false, ell, nzJ, h->LU.p, h->cap, h->Xb.p, h->cap);
    }
    if (h->CA.fmt == 0) {
      gather_cols(st, h->CA, h->Jp_d.p, nzJ, nullptr, h->Ecol.p, m);
      if (ell > 0) {
        dgemm(st, 0, 0, m, nzJ, ell, -1.0, h->Cbuf.p, m, h->Xb.p, h->cap, 1.0, h->Ecol.p, m);
        zero_rows_cm(st, h->Ecol.p, m, nzJ, h->I_d.p, ell);
      }
    } else {
      ecol_csr(st, h->CA, h->colpos.p, h->colpos_plus.p, h->rowpos.p, h->Xb.p, h->cap, nzJ,
               h->Ecol.p);
    }
    // ---- row selection: LUPP on E_col
    const int nzI = lupp_select(st, m, nzJ, h->Ecol.p, 1, m, nzJ, h->lw, Ip, &mI);
    k = std::min(nzJ, nzI);
    if (k < nzJ) {
      // drop the columns whose rows could not be matched
      fill_int(st, h->colpos_plus.p, n, -1);
      set_map(st, h->colpos_plus.p, h->Jp_d.p, k, 0);
      Jp.resize(k);
    }
  }
  *exhausted = k < std::min<int64_t>(h->bsize, h->kmax - ell);
  *margin = std::min(mJ, mI);
  if (k > 0) {
    const int cap = h->cap;
    APL_CUDA(cudaMemcpyAsync(h->Ip_d.p, Ip.data(), k * sizeof(int), cudaMemcpyHostToDevice, st));
    // ---- bordered LU of A(I, J): [L11 0; L21 L22][U11 U12; 0 U22]
    if (ell > 0) {
      dcopy2d(st, ell, k, h->U12.p, cap, h->LU.p + (int64_t)ell * cap, cap, false);
      if (h->CA.fmt == 0) gather_rows_cm(st, h->Cbuf.p, m, ell, h->Ip_d.p, k, h->L21.p, k);
      else gather_cross(st, h->CA, h->Ip_d.p, k, h->J_d.p, ell, h->colpos.p, h->L21.p, k);
      dtrsm(st, false, 'U', false, false, k, ell, h->LU.p, cap, h->L21.p, k);
      dcopy2d(st, k, ell, h->L21.p, k, h->LU.p + ell, cap, false);
    }
    // the pivot rows of the E_col elimination hold L22 \ U22
    gather_rows_cm(st, h->Ecol.p, m, k, h->Ip_d.p, k, h->LU.p + ell + (int64_t)ell * cap, cap);
    // ---- Gram of the new columns for T_C (before the maps change)
    APL_CUDA(cudaMemcpyAsync(h->J_d.p + ell, Jp.data(), k * sizeof(int), cudaMemcpyHostToDevice, st));
    APL_CUDA(cudaMemcpyAsync(h->I_d.p + ell, Ip.data(), k * sizeof(int), cudaMemcpyHostToDevice, st));
    const int ln = ell + k;
    if (h->CA.fmt == 0) {
      gather_cols(st, h->CA, h->Jp_d.p, k, nullptr, h->Cbuf.p + (int64_t)ell * m, m);
      append_rows(st, h->CA, h->Ip_d.p, k, h->Rbuf.p, cap, ell);
    } else {
      gather_cols(st, h->CA, h->Jp_d.p, k, h->colpos_plus.p, h->Cp.p, m);
    }
    set_map(st, h->rowpos.p, h->Ip_d.p, k, ell);
    set_map(st, h->colpos.p, h->Jp_d.p, k, ell);
    fill_int(st, h->colpos_plus.p, n, -1);
    // ---- T_C: Gram of the new columns and bordered Cholesky of C^T C.  C^T C squares
    // the condition of C: when the compensated-FP32 products leave a non-positive pivot
    // the update is redone with FP64 products (a breakdown then is the FP64 one).
    double* T22 = h->TC.p + ell + (int64_t)ell * cap;
    auto tc_update = [&]() -> int {
      if (h->CA.fmt == 0)
        dgemm(st, 1, 0, ln, k, m, 1.0, h->Cbuf.p, m, h->Cbuf.p + (int64_t)ell * m, m, 0.0,
              h->Gb.p, cap);
      else
        gram_csr(st, h->CA, h->J_d.p, ln, h->Cp.p, k, h->Gb.p, cap);
      if (ell > 0) {
        dtrsm(st, true, 'U', true, false, ell, k, h->TC.p, cap, h->Gb.p, cap);
        dcopy2d(st, ell, k, h->Gb.p, cap, h->TC.p + (int64_t)ell * cap, cap, false);
        dgemm(st, 1, 0, k, k, ell, -1.0, h->Gb.p, cap, h->Gb.p, cap, 1.0, h->Gb.p + ell, cap);
      }
      dcopy2d(st, k, k, h->Gb.p + ell, cap, T22, cap, false);
      dpotrf_upper(st, k, T22, cap, h->info.p);
      int inf = 0;
      APL_CUDA(cudaMemcpyAsync(&inf, h->info.p, sizeof(int), cudaMemcpyDeviceToHost, st));
      APL_CUDA(cudaStreamSynchronize(st));
      return inf;
    };
    int info = tc_update();
    if (info && !dense_work().fp64_gemm) {
      Fp64Scope f64;
      info = tc_update();
    }
    if (info) throw Error(ST_EBREAKDOWN, "Cholesky of C^T C met a non-positive pivot");
    // ---- augmentQR(Q_R, T_R, A(I+, :)^T) with two Gram-Schmidt passes
    double* Cn = h->QR.p + (int64_t)ell * n;
    gather_rows_T(st, h->CA, h->Ip_d.p, k, Cn, n);
    if (ell > 0) {
      double* P1 = h->TR.p + (int64_t)ell * cap;
      dgemm(st, 1, 0, ell, k, n, 1.0, h->QR.p, n, Cn, n, 0.0, P1, cap);
      dgemm(st, 0, 0, n, k, ell, -1.0, h->QR.p, n, P1, cap, 1.0, Cn, n);
      dgemm(st, 1, 0, ell, k, n, 1.0, h->QR.p, n, Cn, n, 0.0, h->P2b.p, cap);
      dgemm(st, 0, 0, n, k, ell, -1.0, h->QR.p, n, h->P2b.p, cap, 1.0, Cn, n);
      add2d_kernel<<<(unsigned)cdiv((int64_t)ell * k, 256), 256, 0, st>>>(ell, k, h->P2b.p, cap, P1, cap);
      APL_LAUNCH_CHECK();
    }
    h->work.alloc((size_t)3 * k * k + 16, st);
    if (!cholqr2(st, n, k, Cn, n, h->TR.p + ell + (int64_t)ell * cap, cap, h->work.p, h->info.p))
      throw Error(ST_EBREAKDOWN, "Cholesky QR of the new rows of R met a non-positive pivot");
    h->I.insert(h->I.end(), Ip.begin(), Ip.begin() + k);
    h->J.insert(h->J.end(), Jp.begin(), Jp.begin() + k);
    h->ell = ln;
  }
  // ---- sketched residual E_row = Y - Y(:, J) A(I, J)^{-1} A(I, :)
  const int L = h->ell;
  if (L > 0) {
    const int cap = h->cap;
    dgather_cols(st, s, h->Y.p, s, h->J_d.p, L, h->Zb.p, s);
    dtrsm(st, false, 'U', false, false, s, L, h->LU.p, cap, h->Zb.p, s);
    dtrsm(st, false, 'L', false, true, s, L, h->LU.p, cap, h->Zb.p, s);
    if (h->CA.fmt == 0) {
      APL_CUDA(cudaMemcpyAsync(h->E.p, h->Y.p, (size_t)s * n * sizeof(double),
                               cudaMemcpyDeviceToDevice, st));
      dgemm(st, 0, 0, s, n, L, -1.0, h->Zb.p, s, h->Rbuf.p, cap, 1.0, h->E.p, s);
    } else {
      erow_csr(st, h->CA, h->rowpos.p, h->Zb.p, s, h->Y.p, h->E.p);
    }
  } else {
    APL_CUDA(cudaMemcpyAsync(h->E.p, h->Y.p, (size_t)s * n * sizeof(double),
                             cudaMemcpyDeviceToDevice, st));
  }
  // ---- rho = 10 sqrt(2/pi) max_i ||E_row w_i||  (Eq. 2normestimate)
  dgemm(st, 0, 0, s, h->r, n, 1.0, h->E.p, s, h->W.p, n, 0.0, h->T.p, s);
  colnorm_max(st, h->T.p, s, h->r, 10.0 * std::sqrt(2.0 / M_PI), h->scal.p);
  APL_CUDA(cudaMemcpyAsync(rho_out, h->scal.p, sizeof(double), cudaMemcpyDeviceToHost, st));
  APL_CUDA(cudaStreamSynchronize(st));
  return k;
}

// CURPreconditioner Part 2: M = T_C U T_R^T, SVD of M, coefficients.  Vhat = Q_R V_M is
// kept implicit (applied as two matrix-vector products per use).
// SVD-free variant (Eq. preconditioner_svdfree, Algorithm SVD-free CURPreconditioner,
// mu = 0): the core is kept as M^{-1} = T_R^{-T} A(I,J) T_C^{-1}, formed once here by two
// triangular solves (no SVD); the passes apply P^{-T} and P^{-1} P^{-T} from it.  The
// target level is sigma_min(M) from power iteration on M^{-T} M^{-1}.
void build_svdfree_preconditioner(aplicur_ctx* h) {
  DenseWorkScope dws(&h->dw);
  cudaStream_t st = h->st;
  const int L = h->ell, cap = h->cap;
  h->VM.alloc((size_t)L * L, st);
  h->sigma.alloc(L, st);
  h->work.alloc((size_t)3 * L + 16, st);
  double* Minv = h->VM.p;
  // A(I, J): rows I of C = A(:, J) (dense), or gathered from the CSR matrix
  if (h->CA.fmt == 0) gather_rows_cm(st, h->Cbuf.p, h->cm, L, h->I_d.p, L, Minv, L);
  else gather_cross(st, h->CA, h->I_d.p, L, h->J_d.p, L, h->colpos.p, Minv, L);
  dtrsm(st, false, 'U', false, false, L, L, h->TC.p, cap, Minv, L);  // A(I,J) T_C^{-1}
  dtrsm(st, true, 'U', true, false, L, L, h->TR.p, cap, Minv, L);   // T_R^{-T} (...)
  const double smin = power_sigma_min(st, L, Minv, L, h->work.p, 50);
  const double sighat = smin > 0.0 ? smin : 1.0;
  h->sighat = sighat;
  h->sig_host.assign(L, 0.0);  // this variant computes no singular values
  APL_CUDA(cudaMemsetAsync(h->sigma.p, 0, L * sizeof(double), st));
  std::vector<double> c1(L, sighat);
  h->coef.alloc(L, st);
  APL_CUDA(cudaMemcpyAsync(h->coef.p, c1.data(), L * sizeof(double), cudaMemcpyHostToDevice, st));
  PrecondDev P;
  P.ell = L;
  P.Q = h->QR.p;
  P.ldq = h->n;
  P.VM = Minv;
  P.coef = h->coef.p;
  P.coef2 = nullptr;
  P.svdfree = 1;
  P.sighat = sighat;
  P.normP = 1.0;
  P.sig_ell = sighat;
  h->P = P;
  APL_CUDA(cudaStreamSynchronize(st));
}

void build_preconditioner(aplicur_ctx* h) {
  if (h->opt.variant == APLICUR_VARIANT_SVDFREE) {
    build_svdfree_preconditioner(h);
    return;
  }
  DenseWorkScope dws(&h->dw);
  cudaStream_t st = h->st;
  const int L = h->ell, cap = h->cap;
  h->Mb.alloc((size_t)L * L, st);
  h->VM.alloc((size_t)L * L, st);
  h->sigma.alloc(L, st);
  h->work.alloc((size_t)L * L + 16, st);
  double* X = h->work.p;
  // X = A(I,J)^{-1} T_R^T
  dcopy2d(st, L, L, h->TR.p, cap, X, L, true);
  dtrsm(st, true, 'L', false, true, L, L, h->LU.p, cap, X, L);
  dtrsm(st, true, 'U', false, false, L, L, h->LU.p, cap, X, L);
  // M^T = X^T T_C^T; the Jacobi sweep on the columns of M^T gives the singular values
  // and right singular vectors of M
  dgemm(st, 1, 1, L, L, L, 1.0, X, L, h->TC.p, cap, 0.0, h->Mb.p, L);
  // the leading block of this M is close to the last build's M (the same leading
  // columns of Q_C and Q_R, both CURs accurate there): its Jacobi rotation warm-starts
  // this one
  h->Wnext.alloc((size_t)L * L, st);
  int64_t wl_new = 0;
  jacobi_left(st, L, h->Mb.p, L, h->VM.p, L, h->sigma.p, h->info.p,
              h->wl > 0 ? h->Wprev.p : nullptr, h->wl, h->Wnext.p, &wl_new);
  h->Wprev.swap(h->Wnext);
  h->wl = wl_new;
  h->sig_host.resize(L);
  APL_CUDA(cudaMemcpyAsync(h->sig_host.data(), h->sigma.p, L * sizeof(double),
                           cudaMemcpyDeviceToHost, st));
  APL_CUDA(cudaStreamSynchronize(st));
  const double d2 = h->delta * h->delta;
  const double sl = h->sig_host[L - 1];
  h->sighat = std::sqrt(sl * sl + d2);
  std::vector<double> c1(L), c2(L);
  for (int k = 0; k < L; ++k) {
    const double lam2 = h->sig_host[k] * h->sig_host[k] + d2;
    const double lam = std::sqrt(lam2);
    c1[k] = h->sighat / lam - 1.0;
    c2[k] = (h->sighat * h->sighat) / lam2 - 1.0;
  }
  h->coef.alloc(L, st);
  h->coef2.alloc(L, st);
  APL_CUDA(cudaMemcpyAsync(h->coef.p, c1.data(), L * sizeof(double), cudaMemcpyHostToDevice, st));
  APL_CUDA(cudaMemcpyAsync(h->coef2.p, c2.data(), L * sizeof(double), cudaMemcpyHostToDevice, st));
  PrecondDev P;
  P.ell = L;
  P.Q = h->QR.p;
  P.ldq = h->n;
  P.VM = h->VM.p;
  P.coef = h->coef.p;
  P.coef2 = h->coef2.p;
  P.normP = std::sqrt(h->sig_host[0] * h->sig_host[0] + d2) / h->sighat;
  P.sig_ell = sl;
  h->P = P;
  APL_CUDA(cudaStreamSynchronize(st));
}

double run_phase(aplicur_ctx* h, double nu, double tol, long long maxit, int fixed, long long* it,
                 int* reason) {
  PhaseArgs a;
  a.rhs_top = h->b;
  a.x = h->x.p;
  a.eps = h->opt.eps_lsqr;
  a.nu = nu;
  a.tol = h->replay ? 0.0 : tol;
  // the solve starts from x = 0, so the first phase needs no product for its residual
  a.x_zero = h->phases.empty();
  a.norm_ref = h->norm_Atb;
  a.mu = h->mu;
  a.fixed_len = fixed;
  a.maxit = maxit;
  a.check_gap = h->opt.check_gap;
  // FP32 products (MIXED): a final phase (no dynamic stop) is one step of an FP64
  // iterative refinement in correction form.  With g = A^T (b - A x) - mu x formed with
  // FP64 products, LSQR on [A; delta I] P^{-1} with right-hand side [0; g / delta] has the
  // normal equations (A^T A + mu I) dx = g of the paper's warm start (Section 3.2), but
  // all its vectors shrink with g, so FP32 products keep their relative accuracy and the
  // refinement is not held at the FP32 floor u32 ||A|| ||b - A x|| of the warm-start form.
  // Phases with the dynamic stop keep the warm-start form: the stopping rule reads the
  // paper's residual estimate, which the correction form cannot recover accurately when
  // ||g|| / delta is far above the residual.
  const bool corr = h->opt.precision == APLICUR_PREC_MIXED && h->A.dtype == APLICUR_F32 &&
                    h->mu > 0.0 && !std::isfinite(nu);
  if (corr) {
    cudaStream_t st = h->st;
    h->dx.alloc(h->n, st);
    h->rbot.alloc(h->n, st);
    h->zm.alloc(h->m, st);
    h->dx.zero(st);
    h->zm.zero(st);
    h->eng.correction_rhs(h->b, h->x.p, h->delta, h->rbot.p);
    a.rhs_top = h->zm.p;
    a.rhs_bot = h->rbot.p;
    a.x = h->dx.p;
    a.x_zero = true;
    // the Paige-Saunders tests must not end a phase short of tol
    if (a.tol > 0.0) a.eps = std::min(a.eps, a.tol / 100.0);
  }
  PhaseResult r = h->eng.run_phase(h->P, a);
  if (corr) {
    axpy_kernel<<<(unsigned)cdiv(h->n, 256), 256, 0, h->st>>>(h->n, 1.0, h->dx.p, h->x.p);
    APL_LAUNCH_CHECK();
  }
  const double ne = h->eng.ne_residual(h->b, nullptr, h->x.p, h->delta, h->norm_Atb, a.tol);
  h->phases.push_back(PhaseRec{h->P.ell, r.iters, r.reason == R_CHECK ? R_TOL : r.reason, ne});
  *it = r.iters;
  *reason = r.reason;
  return ne;
}

int do_solve(aplicur_ctx* h, double tol, long long maxit) {
  cudaStream_t st = h->st;
  reset_cur(h);
  h->x.zero(st);
  long long total = 0;
  size_t rp_ph = 0, rp_rb = 0;
  auto next_fixed = [&]() -> int {
    if (!h->replay) return -1;
    return rp_ph < h->rp_phases.size() ? h->rp_phases[rp_ph++] : 0;
  };
  double ne = INFINITY;
  auto finish = [&](double ne_) {
    h->stats.iters = total;
    h->stats.ell = h->ell;
    h->stats.nphases = (int)h->phases.size();
    h->stats.nsteps = (int)h->steps.size();
    h->stats.ne_res = ne_;
    h->stats.converged = ne_ <= tol ? 1 : 0;
    h->solved = true;
    return (ne_ <= tol || h->replay) ? ST_OK : ST_ENOTCONV;
  };
  if (h->norm_Atb == 0.0) return finish(0.0);
  double d_cur = INFINITY;
  using clk = std::chrono::steady_clock;
  auto ms_since = [](clk::time_point t0) {
    return std::chrono::duration<double, std::milli>(clk::now() - t0).count();
  };
  h->stats.time_rank_ms = h->stats.time_build_ms = h->stats.time_lsqr_ms = 0.0;
  h->stats.rank_breakdown = 0;
  while (true) {
    double rho = 0, margin = INFINITY;
    bool exhausted = false;
    auto t0 = clk::now();
    try {
      rank_step(h, &rho, &exhausted, &margin);
    } catch (const Error& e) {
      // numerically dependent new indices: rank growth ends at the current rank (the
      // step's partial writes lie beyond it), and the solve goes on with the last
      // preconditioner built
      if (e.code != ST_EBREAKDOWN) throw;
      h->stats.rank_breakdown = 1;
      h->stats.time_rank_ms += ms_since(t0);
      break;
    }
    h->stats.time_rank_ms += ms_since(t0);
    h->stats.rho = rho;
    const bool full = h->ell >= h->kmax;
    const double rho_eff = exhausted ? 0.0 : rho;
    const bool last = rho_eff <= h->eps_cur || full || exhausted;
    bool rebuild;
    if (h->replay) {
      rebuild = rp_rb < h->rp_rebuild.size() ? h->rp_rebuild[rp_rb++] != 0 : last;
    } else {
      // single-shot schedule: one build, when rank growth ends
      const double gap = rho_eff - h->eps_cur;
      rebuild = last || (h->opt.schedule == APLICUR_SCHEDULE_ADAPTIVE && gap > 0.0 &&
                         d_cur / gap >= h->opt.nu_prec);
    }
    h->steps.push_back(StepRec{h->ell, rho, rebuild ? 1 : 0, margin});
    if (rebuild && h->ell > 0) {
      t0 = clk::now();
      build_preconditioner(h);
      h->stats.time_build_ms += ms_since(t0);
      long long it = 0;
      int reason = 0;
      t0 = clk::now();
      ne = run_phase(h, last ? INFINITY : h->opt.nu_lsqr, tol, std::max(0LL, maxit - total),
                     next_fixed(), &it, &reason);
      h->stats.time_lsqr_ms += ms_since(t0);
      total += it;
      if (!h->replay && ne <= tol) return finish(ne);
      d_cur = rho_eff - h->eps_cur;
    }
    if (last) break;
    if (total >= maxit) return finish(h->eng.ne_residual(h->b, nullptr, h->x.p, h->delta, h->norm_Atb));
  }
  if (!h->phases.empty()) ne = h->phases.back().ne;
  else ne = h->eng.ne_residual(h->b, nullptr, h->x.p, h->delta, h->norm_Atb);
  int extra = 0;
  while ((h->replay && rp_ph < h->rp_phases.size()) ||
         (!h->replay && ne > tol && total < maxit && extra < h->opt.max_extra_phases)) {
    const double prev = ne;
    long long it = 0;
    int reason = 0;
    auto t1 = clk::now();
    ne = run_phase(h, INFINITY, tol, std::max(0LL, maxit - total), next_fixed(), &it, &reason);
    h->stats.time_lsqr_ms += ms_since(t1);
    total += it;
    ++extra;
    if (!h->replay && (it == 0 || ne > 0.5 * prev)) break;
  }
  return finish(ne);
}

// Validation, sketch draws, the one-time sketch Y = S A and buffers of one problem; with
// with_lsqr also the single-right-hand-side LSQR engine and ||A^T b||.  Throws Error.
void ctx_init(aplicur_ctx* h, const aplicur_matrix* A, const double* b, double mu,
              int32_t sketch_dim, const aplicur_options* opt, void* stream, bool with_lsqr) {
  APL_REQUIRE(A->format == APLICUR_DENSE_ROWMAJOR || A->format == APLICUR_CSR, "bad format");
  APL_REQUIRE(A->dtype == APLICUR_F64 || A->dtype == APLICUR_F32, "bad dtype");
  APL_REQUIRE(A->m >= 1 && A->n >= 1 && A->m >= A->n, "need m >= n >= 1");
  APL_REQUIRE(A->m < (1LL << 31) && A->n < (1LL << 31), "dimensions exceed int32 indexing");
  APL_REQUIRE(A->values != nullptr, "A values NULL");
  APL_REQUIRE(mu >= 0.0 && std::isfinite(mu), "mu must be finite and >= 0");
  APL_REQUIRE(sketch_dim >= 1 && sketch_dim <= A->n, "need 1 <= sketch_dim <= n");
  if (A->format == APLICUR_DENSE_ROWMAJOR) APL_REQUIRE(A->ld >= A->n, "ld < n");
  else APL_REQUIRE(A->rowptr && A->colidx && A->nnz >= 0 && A->nnz < (1LL << 31), "bad CSR");
  if (opt) h->opt = *opt; else aplicur_options_default(&h->opt);
  if (h->opt.replay_phases && h->opt.replay_nphases > 0)
    h->rp_phases.assign(h->opt.replay_phases, h->opt.replay_phases + h->opt.replay_nphases);
  else h->opt.replay_nphases = 0;
  if (h->opt.replay_rebuild && h->opt.replay_nsteps > 0)
    h->rp_rebuild.assign(h->opt.replay_rebuild, h->opt.replay_rebuild + h->opt.replay_nsteps);
  else h->opt.replay_nsteps = 0;
  APL_REQUIRE(h->opt.xi >= 1 && h->opt.normest_r >= 1 && h->opt.check_gap >= 1, "bad options");
  APL_REQUIRE(h->opt.graph_iters >= 0 && h->opt.graph_iters <= 4096, "bad graph_iters");
  APL_REQUIRE(h->opt.precision >= APLICUR_PREC_FP64 && h->opt.precision <= APLICUR_PREC_DF32,
              "bad precision");
  APL_REQUIRE(h->opt.variant == APLICUR_VARIANT_SVD || h->opt.variant == APLICUR_VARIANT_SVDFREE,
              "bad variant");
  APL_REQUIRE(h->opt.schedule == APLICUR_SCHEDULE_ADAPTIVE ||
                  h->opt.schedule == APLICUR_SCHEDULE_SINGLE_SHOT,
              "bad schedule");
  APL_REQUIRE(h->opt.sketch_kind >= APLICUR_SKETCH_SPARSE_SIGN &&
                  h->opt.sketch_kind <= APLICUR_SKETCH_SRHT,
              "bad sketch_kind");
  APL_REQUIRE(h->opt.sketch_tc >= 0 && h->opt.sketch_tc <= 3, "sketch_tc: 0 to 3 terms");
  APL_REQUIRE(!h->opt.sketch_tc || (h->opt.sketch_kind != APLICUR_SKETCH_SPARSE_SIGN &&
                                    A->format == APLICUR_DENSE_ROWMAJOR),
              "sketch_tc needs a dense operator (Gaussian or SRHT) and a dense A");
  if (stream) h->st = (cudaStream_t)stream;
  else { APL_CUDA(cudaStreamCreateWithFlags(&h->st, cudaStreamNonBlocking)); h->own_stream = true; }
  cudaStream_t st = h->st;
  h->m = A->m; h->n = A->n; h->kmax = std::min(h->m, h->n);
  APL_REQUIRE(h->opt.max_rank >= 0, "max_rank must be >= 0");
  if (h->opt.max_rank > 0) h->kmax = std::min<int64_t>(h->kmax, h->opt.max_rank);
  h->A.fmt = A->format; h->A.dtype = A->dtype; h->A.m = A->m; h->A.n = A->n; h->A.ld = A->ld;
  h->A.nnz = A->format == APLICUR_CSR ? A->nnz : A->m * A->n;
  h->A.vals = A->values; h->A.rowptr = A->rowptr; h->A.colidx = A->colidx;
  h->b = b;
  h->mu = mu;
  h->delta = std::sqrt(mu);
  h->eps_cur = h->opt.eps_cur_factor * h->delta;
  h->bsize = sketch_dim;
  h->s = (11 * sketch_dim + 9) / 10;
  h->xi = std::min(h->opt.xi, h->s);
  APL_REQUIRE(!h->opt.sketch_tc || h->s <= TC_SKETCH_MAX_S,
              "sketch_tc: the tensor-core sketch takes s = ceil(1.1 sketch_dim) <= 512");
  h->dw.fp64_gemm = h->opt.fp64_dense != 0;
  h->r = h->opt.normest_r;
  if (h->A.fmt == 1) build_csc(h);
  // the CUR matrix: A, or A_mu = [A; delta I] for the SVD-free variant with mu > 0
  // (section "SVD-free variant": a CUR of the regularised matrix)
  h->CA = h->A;
  h->cm = h->m;
  if (h->opt.variant == APLICUR_VARIANT_SVDFREE && mu > 0.0) {
    APL_REQUIRE(h->m + h->n < (1LL << 31), "A_mu: m + n exceeds int32 indexing");
    build_amu(h);
  }
  h->kmax = std::min(h->cm, h->n);
  if (h->opt.max_rank > 0) h->kmax = std::min<int64_t>(h->kmax, h->opt.max_rank);
  // sketch and norm-estimate draws
  std::vector<int> rows;
  std::vector<int8_t> sg;
  if (h->opt.sketch_rows && h->opt.sketch_signs) {
    rows.assign(h->opt.sketch_rows, h->opt.sketch_rows + h->cm * h->xi);
    sg.assign(h->opt.sketch_signs, h->opt.sketch_signs + h->cm * h->xi);
  } else {
    draw_sketch(h->opt.seed, h->s, h->cm, h->xi, rows, sg);
  }
  upload_sketch(h, rows, sg);
  std::vector<double> W;
  if (h->opt.normest_w) W.assign(h->opt.normest_w, h->opt.normest_w + h->n * h->r);
  else draw_gaussian(h->opt.seed, h->n, h->r, W);
  h->W.alloc(W.size(), st);
  APL_CUDA(cudaMemcpyAsync(h->W.p, W.data(), W.size() * sizeof(double), cudaMemcpyHostToDevice, st));
  h->opt.sketch_rows = nullptr; h->opt.sketch_signs = nullptr; h->opt.normest_w = nullptr;
  h->opt.replay_phases = nullptr; h->opt.replay_rebuild = nullptr;
  // buffers
  const int64_t m = h->m, n = h->n;
  h->Y.alloc((size_t)h->s * n, st);
  h->E.alloc((size_t)h->s * n, st);
  h->Et.alloc((size_t)h->s * n, st);
  h->T.alloc((size_t)h->s * h->r, st);
  h->scal.alloc(4, st);
  h->info.alloc(4, st);
  h->I_d.alloc(h->kmax, st); h->J_d.alloc(h->kmax, st);
  h->Jp_d.alloc(h->bsize, st); h->Ip_d.alloc(h->bsize, st);
  h->colpos.alloc(n, st); h->colpos_plus.alloc(n, st); h->rowpos.alloc(h->cm, st);
  h->Ecol.alloc((size_t)h->cm * h->bsize, st);
  if (h->A.fmt == 1) h->Cp.alloc((size_t)h->cm * h->bsize, st);
  if (with_lsqr) {
    h->x.alloc(n, st); h->tmp_m.alloc(m, st); h->tmp_n.alloc(n, st); h->tmp_n2.alloc(n, st);
    h->lam.alloc(n, st);
  }
  // the one-time sketch Y = S A
  cudaEvent_t e0, e1;
  APL_CUDA(cudaEventCreate(&e0));
  APL_CUDA(cudaEventCreate(&e1));
  APL_CUDA(cudaEventRecord(e0, st));
  if (h->opt.sketch_kind == APLICUR_SKETCH_SPARSE_SIGN) {
    sketch(st, h->CA, h->s, h->xi, h->tptr.p, h->ti.p, h->tsgn.p, h->srows.p, h->ssign.p,
           1.0 / std::sqrt((double)h->xi), h->Y.p);
  } else {
    // a dense operator drawn on the host (the draw is not part of the timed product)
    APL_CUDA(cudaEventRecord(e1, st));
    APL_CUDA(cudaEventSynchronize(e1));
    std::vector<double> S;
    if (h->opt.sketch_kind == APLICUR_SKETCH_GAUSSIAN) draw_gaussian_sketch(h->opt.seed, h->s, h->cm, S);
    else draw_srht_sketch(h->opt.seed, h->s, h->cm, S);
    if (h->opt.sketch_tc) {
      tc_sketch_upload(st, S.data(), h->s, h->cm, h->n, h->tcw);
      tc_sketch_apply(st, h->CA, h->tcw, h->Y.p, h->opt.sketch_tc, e0, e1);
    } else {
      DBuf<double> Sd, chunk;
      Sd.alloc(S.size(), st);
      APL_CUDA(cudaMemcpyAsync(Sd.p, S.data(), S.size() * sizeof(double), cudaMemcpyHostToDevice, st));
      APL_CUDA(cudaEventRecord(e0, st));
      DenseWorkScope dws(&h->dw);
      operator_sketch(st, h->CA, h->s, Sd.p, h->Y.p, chunk);
      APL_CUDA(cudaEventRecord(e1, st));
      APL_CUDA(cudaEventSynchronize(e1));
    }
  }
  if (!(h->opt.sketch_kind != APLICUR_SKETCH_SPARSE_SIGN && h->opt.sketch_tc))
    APL_CUDA(cudaEventRecord(e1, st));
  APL_CUDA(cudaEventSynchronize(e1));
  APL_CUDA(cudaEventElapsedTime(&h->setup_ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->stats.time_setup_ms = h->setup_ms;
  if (!with_lsqr) return;
  APL_REQUIRE(h->opt.dense_pass >= APLICUR_DENSE_PASS_AUTO &&
                  h->opt.dense_pass <= APLICUR_DENSE_PASS_FUSED,
              "bad dense_pass");
  h->eng.setup(st, h->A, h->opt.precision, h->opt.graph_iters, h->opt.dense_pass);
  h->stats.fused_pass = h->eng.fused_pass() ? 1 : 0;
  h->stats.cluster_size = h->eng.fused_pass() ? h->eng.fused_plan().C : 0;
  h->eng.set_profile(h->opt.profile != 0);
  // ||A^T b|| in FP64
  h->eng.matvec(1, b, h->tmp_n.p, 1.0, 0.0, true);
  h->norm_Atb = h->eng.norm2(h->tmp_n.p, n);
}

aplicur_status fail(aplicur_ctx* h, const Error& e) {
  if (h) h->err = e.what();
  return (aplicur_status)e.code;
}

template <typename F>
aplicur_status guarded(aplicur_ctx* h, F&& f) {
  if (h && h->poisoned) {
    h->err = "an earlier call of this handle returned ETIMEOUT: a bounded device wait gave up, "
             "so the handle's device buffers are undefined; destroy the handle";
    return APLICUR_ETIMEOUT;
  }
  AllocScope as(h && h->alloc_.alloc ? &h->alloc_ : nullptr);
  try {
    return (aplicur_status)f();
  } catch (const Error& e) {
    if (h && e.code == ST_ETIMEOUT) h->poisoned = true;
    return fail(h, e);
  } catch (const std::exception& e) {
    if (h) h->err = e.what();
    return APLICUR_ECUDA;
  } catch (...) {
    if (h) h->err = "unknown failure";
    return APLICUR_ECUDA;
  }
}

}  // namespace

// ======================================================================================
// C ABI
// ======================================================================================
extern "C" {

void aplicur_options_default(aplicur_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->seed = 1;
  o->eps_cur_factor = 30.0;
  o->nu_prec = 10.0;
  o->nu_lsqr = 100.0;
  o->eps_lsqr = 1e-10;
  o->xi = 8;
  o->normest_r = 10;
  o->check_gap = 10;
  o->max_extra_phases = 8;
  o->precision = APLICUR_PREC_FP64;
  o->graph_iters = 16;
}

static thread_local std::string g_create_err;

}  // extern "C"

namespace apl {
void set_noalloc_error(const char* msg) { g_create_err = msg; }
}  // namespace apl

extern "C" {

aplicur_status aplicur_create(aplicur_handle* out, const aplicur_matrix* A, const double* b,
                              double mu, int32_t sketch_dim, const aplicur_options* opt,
                              void* stream) {
  if (!out || !A || !b) { g_create_err = "null argument"; return APLICUR_EINVAL; }
  *out = nullptr;
  if (opt && ((opt->alloc != nullptr) != (opt->free_ != nullptr))) {
    g_create_err = "options: set both alloc and free_, or neither";
    return APLICUR_EINVAL;
  }
  aplicur_ctx* h = new (std::nothrow) aplicur_ctx();
  if (!h) return APLICUR_ENOMEM;
  if (opt) h->alloc_ = Allocator{opt->alloc, opt->free_, opt->alloc_ctx};
  aplicur_status stt = guarded(h, [&]() -> int {
    ctx_init(h, A, b, mu, sketch_dim, opt, stream, true);
    return ST_OK;
  });
  if (stt != APLICUR_OK) {
    g_create_err = h->err;
    aplicur_destroy(h);
    return stt;
  }
  *out = h;
  return APLICUR_OK;
}

static void load_replay(aplicur_ctx* h) {
  h->replay = h->opt.replay_nphases > 0 || h->opt.replay_nsteps > 0;
}

aplicur_status aplicur_solve(aplicur_handle h, double tol, int64_t maxit, double* x_out) {
  if (!h) return APLICUR_EINVAL;
  return guarded(h, [&]() -> int {
    APL_REQUIRE(x_out != nullptr, "x_out NULL");
    APL_REQUIRE(tol >= 0.0 && maxit >= 0, "tol and maxit must be >= 0");
    load_replay(h);
    auto t0 = std::chrono::steady_clock::now();
    struct SinkScope {
      explicit SinkScope(aplicur_ctx* c) : h(c) { if (h->opt.profile) prof_set_sink(&h->sink); }
      ~SinkScope() { prof_set_sink(nullptr); }
      aplicur_ctx* h;
    } scope(h);
    const int rc = do_solve(h, tol, maxit);
    if (h->opt.profile) h->sink.harvest();
    APL_CUDA(cudaMemcpyAsync(x_out, h->x.p, h->n * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
    APL_CUDA(cudaStreamSynchronize(h->st));
    h->stats.time_solve_ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return rc;
  });
}

aplicur_status aplicur_set_replay(aplicur_handle h, int32_t nph, const int32_t* ph, int32_t nst,
                                  const int8_t* rb) {
  if (!h) return APLICUR_EINVAL;
  h->rp_phases.assign(ph, ph + (ph ? nph : 0));
  h->rp_rebuild.assign(rb, rb + (rb ? nst : 0));
  h->opt.replay_nphases = nph;
  h->opt.replay_nsteps = nst;
  return APLICUR_OK;
}

aplicur_status aplicur_plain_lsqr(aplicur_handle h, double tol, int64_t maxit, double* x_out) {
  if (!h) return APLICUR_EINVAL;
  return guarded(h, [&]() -> int {
    APL_REQUIRE(x_out != nullptr, "x_out NULL");
    auto t0 = std::chrono::steady_clock::now();
    // no CUR state: a later aplicur_backward runs the adjoint solve unpreconditioned too
    reset_cur(h);
    h->x.zero(h->st);
    h->phases.clear();
    PrecondDev I;
    PhaseArgs a;
    a.rhs_top = h->b;
    a.x = h->x.p;
    a.eps = 0.0;
    a.nu = INFINITY;
    a.tol = tol;
    a.norm_ref = h->norm_Atb;
    a.mu = h->mu;
    a.maxit = maxit;
    a.check_gap = h->opt.check_gap;
    long long total = 0;
    double ne = INFINITY;
    for (int rep = 0; rep <= h->opt.max_extra_phases && total < maxit; ++rep) {
      a.maxit = maxit - total;
      a.x_zero = rep == 0;
      PhaseResult r = h->eng.run_phase(I, a);
      total += r.iters;
      ne = h->eng.ne_residual(h->b, nullptr, h->x.p, h->delta, h->norm_Atb, tol);
      h->phases.push_back(PhaseRec{0, r.iters, r.reason == R_CHECK ? R_TOL : r.reason, ne});
      if ((r.reason != R_DRIFT && r.reason != R_INNER) || ne <= tol) break;
    }
    h->stats.iters = total;
    h->stats.ne_res = ne;
    h->stats.converged = ne <= tol;
    h->stats.nphases = (int)h->phases.size();
    h->stats.ell = 0;
    h->stats.nsteps = 0;
    h->stats.rank_breakdown = 0;
    h->solved = true;
    APL_CUDA(cudaMemcpyAsync(x_out, h->x.p, h->n * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
    APL_CUDA(cudaStreamSynchronize(h->st));
    h->stats.time_solve_ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return ne <= tol ? ST_OK : ST_ENOTCONV;
  });
}

aplicur_status aplicur_backward(aplicur_handle h, const double* grad_x, double tol, int64_t maxit,
                                double* grad_b, double* grad_mu, void* grad_A) {
  if (!h) return APLICUR_EINVAL;
  return guarded(h, [&]() -> int {
    APL_REQUIRE(grad_x != nullptr, "grad_x NULL");
    APL_REQUIRE(h->solved, "aplicur_backward needs a previous aplicur_solve");
    APL_REQUIRE(h->mu > 0.0, "aplicur_backward needs mu > 0");
    APL_REQUIRE(!grad_A || h->A.fmt == 0, "grad_A is only produced for dense A");
    cudaStream_t st = h->st;
    const int64_t m = h->m, n = h->n;
    // rhs = [0; g / delta];  A_delta^T rhs = g
    scale_kernel<<<(unsigned)cdiv(n, 256), 256, 0, st>>>(n, grad_x, 1.0 / h->delta, h->tmp_n2.p);
    APL_LAUNCH_CHECK();
    APL_CUDA(cudaMemsetAsync(h->tmp_m.p, 0, m * sizeof(double), st));
    const double gnorm = h->eng.norm2(grad_x, n);
    h->lam.zero(st);
    double ne = 0.0;
    if (gnorm > 0.0) {
      PhaseArgs a;
      a.rhs_top = h->tmp_m.p;
      a.rhs_bot = h->tmp_n2.p;
      a.x = h->lam.p;
      a.eps = h->opt.eps_lsqr;
      a.nu = INFINITY;
      a.tol = tol;
      a.norm_ref = gnorm;
      a.mu = h->mu;
      a.check_gap = h->opt.check_gap;
      long long total = 0;
      ne = INFINITY;
      for (int rep = 0; rep <= h->opt.max_extra_phases && total < maxit; ++rep) {
        a.maxit = maxit - total;
        a.x_zero = rep == 0;
        PhaseResult r = h->eng.run_phase(h->P, a);
        total += r.iters;
        const double prev = ne;
        ne = h->eng.ne_residual(h->tmp_m.p, h->tmp_n2.p, h->lam.p, h->delta, gnorm, tol);
        if (ne <= tol || r.iters == 0 || ne > 0.5 * prev) break;
      }
    }
    // grad_b = A lambda ; grad_mu = -lambda^T x ; grad_A = r lambda^T - (A lambda) x^T
    h->eng.matvec(0, h->lam.p, h->tmp_m.p, 1.0, 0.0, true);
    if (grad_b)
      APL_CUDA(cudaMemcpyAsync(grad_b, h->tmp_m.p, m * sizeof(double), cudaMemcpyDeviceToDevice, st));
    if (grad_mu) {
      dot_kernel<<<1, 256, 0, st>>>(n, h->lam.p, h->x.p, h->scal.p);
      APL_LAUNCH_CHECK();
      double v = 0.0;
      APL_CUDA(cudaMemcpyAsync(&v, h->scal.p, sizeof(double), cudaMemcpyDeviceToHost, st));
      APL_CUDA(cudaStreamSynchronize(st));
      *grad_mu = -v;
    }
    if (grad_A) {
      DBuf<double> r;
      r.alloc(m, st);
      APL_CUDA(cudaMemcpyAsync(r.p, h->b, m * sizeof(double), cudaMemcpyDeviceToDevice, st));
      h->eng.matvec(0, h->x.p, r.p, -1.0, 1.0, true);
      const unsigned grid = (unsigned)std::min<int64_t>(cdiv(m * n, 256), 152 * 16);
      if (h->A.dtype == 0)
        rank2_kernel<double><<<grid, 256, 0, st>>>(m, n, r.p, h->lam.p, h->tmp_m.p, h->x.p,
                                                   (double*)grad_A);
      else
        rank2_kernel<float><<<grid, 256, 0, st>>>(m, n, r.p, h->lam.p, h->tmp_m.p, h->x.p,
                                                  (float*)grad_A);
      APL_LAUNCH_CHECK();
    }
    APL_CUDA(cudaStreamSynchronize(st));
    return ne <= tol ? ST_OK : ST_ENOTCONV;
  });
}

aplicur_status aplicur_get_indices(aplicur_handle h, int32_t* I, int32_t* J, int32_t* ell) {
  if (!h) return APLICUR_EINVAL;
  if (ell) *ell = h->ell;
  if (I && h->ell) std::memcpy(I, h->I.data(), h->ell * sizeof(int));
  if (J && h->ell) std::memcpy(J, h->J.data(), h->ell * sizeof(int));
  return APLICUR_OK;
}

aplicur_status aplicur_get_sketch(aplicur_handle h, double* y_out, int32_t* s_out) {
  if (!h) return APLICUR_EINVAL;
  return guarded(h, [&]() -> int {
    if (s_out) *s_out = h->s;
    if (y_out) {
      APL_CUDA(cudaMemcpyAsync(y_out, h->Y.p, (size_t)h->s * h->n * sizeof(double),
                               cudaMemcpyDeviceToDevice, h->st));
      APL_CUDA(cudaStreamSynchronize(h->st));
    }
    return ST_OK;
  });
}

aplicur_status aplicur_get_stats(aplicur_handle h, aplicur_stats* st) {
  if (!h || !st) return APLICUR_EINVAL;
  *st = h->stats;
  return APLICUR_OK;
}

aplicur_status aplicur_get_phase(aplicur_handle h, int32_t k, int32_t* ell, int64_t* iters,
                                 int32_t* reason, double* ne_res) {
  if (!h || k < 0 || k >= (int)h->phases.size()) return APLICUR_EINVAL;
  const PhaseRec& p = h->phases[k];
  if (ell) *ell = p.ell;
  if (iters) *iters = p.iters;
  if (reason) *reason = p.reason;
  if (ne_res) *ne_res = p.ne;
  return APLICUR_OK;
}

aplicur_status aplicur_get_step(aplicur_handle h, int32_t k, int32_t* ell, double* rho,
                                int32_t* rebuilt, double* margin) {
  if (!h || k < 0 || k >= (int)h->steps.size()) return APLICUR_EINVAL;
  const StepRec& s = h->steps[k];
  if (ell) *ell = s.ell;
  if (rho) *rho = s.rho;
  if (rebuilt) *rebuilt = s.rebuilt;
  if (margin) *margin = s.margin;
  return APLICUR_OK;
}

aplicur_status aplicur_get_preconditioner(aplicur_handle h, int32_t* ell, double* sigma,
                                          double* sighat) {
  if (!h) return APLICUR_EINVAL;
  return guarded(h, [&]() -> int {
    if (ell) *ell = h->P.ell;
    if (sighat) *sighat = h->P.ell ? h->sighat : 1.0;
    if (sigma && h->P.ell) {
      APL_CUDA(cudaMemcpyAsync(sigma, h->sigma.p, h->P.ell * sizeof(double),
                               cudaMemcpyDeviceToDevice, h->st));
      APL_CUDA(cudaStreamSynchronize(h->st));
    }
    return ST_OK;
  });
}

aplicur_status aplicur_apply_preconditioner(aplicur_handle h, const double* w, double* out) {
  if (!h || !w || !out) return APLICUR_EINVAL;
  return guarded(h, [&]() -> int {
    h->eng.apply_precond(h->P, w, out, nullptr);
    APL_CUDA(cudaStreamSynchronize(h->st));
    return ST_OK;
  });
}

aplicur_status aplicur_matvec(aplicur_handle h, int32_t trans, const double* x, double* y) {
  if (!h || !x || !y) return APLICUR_EINVAL;
  return guarded(h, [&]() -> int {
    h->eng.matvec(trans ? 1 : 0, x, y, 1.0, 0.0, h->opt.precision == APLICUR_PREC_FP64);
    APL_CUDA(cudaStreamSynchronize(h->st));
    return ST_OK;
  });
}

static_assert(sizeof(aplicur_profile::ms) / sizeof(double) == PROF_NCAT,
              "aplicur_profile must hold one entry per kernel family");

aplicur_status aplicur_get_profile(aplicur_handle h, aplicur_profile* out) {
  if (!h || !out) return APLICUR_EINVAL;
  for (int k = 0; k < 3; ++k) {
    out->ms[k] = h->eng.prof.ms[k];
    out->launches[k] = h->eng.prof.launches[k];
    out->work[k] = h->eng.prof.bytes_total[k];
  }
  for (int k = 3; k < PROF_NCAT; ++k) {
    out->ms[k] = h->sink.ms[k];
    out->launches[k] = h->sink.n[k];
    out->work[k] = h->sink.work[k];
  }
  out->kernel_launches = launch_count();
  return APLICUR_OK;
}

int64_t aplicur_launch_count(void) { return launch_count(); }

int64_t aplicur_internal_alloc_count(void) { return internal_alloc_count(); }

aplicur_status aplicur_reset_profile(aplicur_handle h) {
  if (!h) return APLICUR_EINVAL;
  for (int k = 0; k < 3; ++k) {
    h->eng.prof.ms[k] = 0;
    h->eng.prof.launches[k] = 0;
    h->eng.prof.bytes_total[k] = 0;
  }
  for (int k = 0; k < PROF_NCAT; ++k) {
    h->sink.ms[k] = 0;
    h->sink.work[k] = 0;
    h->sink.n[k] = 0;
  }
  return APLICUR_OK;
}

const char* aplicur_last_error(aplicur_handle h) {
  if (!h) return g_create_err.c_str();
  return h->err.c_str();
}

const char* aplicur_status_string(aplicur_status s) {
  switch (s) {
    case APLICUR_OK: return "ok";
    case APLICUR_EINVAL: return "invalid argument";
    case APLICUR_ENOMEM: return "out of memory";
    case APLICUR_ECUDA: return "CUDA error";
    case APLICUR_ENOTCONV: return "not converged within maxit";
    case APLICUR_EBREAKDOWN: return "factorisation breakdown";
    case APLICUR_ETIMEOUT: return "device wait timed out";
  }
  return "unknown status";
}

void aplicur_destroy(aplicur_handle h) {
  if (!h) return;
  cudaStream_t st = h->st;
  bool own = h->own_stream;
  if (st) cudaStreamSynchronize(st);
  delete h;
  if (own && st) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
}

}  // extern "C"

// ======================================================================================
// Batched solves: per-problem CUR state machines (the driver of do_solve, in lock step
// over the problems) around one grouped multi-right-hand-side LSQR engine.
// ======================================================================================

struct aplicur_batch_ctx {
  cudaStream_t st = nullptr;
  bool own_stream = false;
  int device = 0;
  int np = 0, R = 0;
  double mu = 0;
  std::vector<aplicur_ctx*> pc;
  apl::BatchEngine eng;
  std::vector<long long> iters;  // per pair p * R + r
  std::vector<double> ne;
  std::vector<char> conv;
  std::vector<char> broke;       // per problem: a rank step or build broke down
  bool solved = false;           // a solve has left forward solutions in the engine
  std::vector<const double*> bsrc;  // right-hand sides (m_p x R column-major, borrowed)
  Allocator alloc_;              // caller's device allocator (empty: cudaMallocAsync)
  aplicur_batch_stats stats{};
  std::string err;
  int nthreads = 1;
  ~aplicur_batch_ctx() {
    for (aplicur_ctx* c : pc) aplicur_destroy(c);
  }
};

namespace {

// Run f(i) for i < n on up to nthreads host threads (each bound to `device`); the first
// exception is rethrown after all threads finished.
template <typename F>
void parallel_for(int n, int nthreads, int device, F&& f) {
  std::atomic<int> next{0};
  std::exception_ptr first;
  std::mutex mtx;
  const Allocator* alloc = current_allocator();
  auto work = [&]() {
    cudaSetDevice(device);
    AllocScope as(alloc);
    while (true) {
      const int i = next.fetch_add(1);
      if (i >= n) break;
      try {
        f(i);
      } catch (...) {
        std::lock_guard<std::mutex> g(mtx);
        if (!first) first = std::current_exception();
      }
    }
  };
  const int nt = std::max(1, std::min(nthreads, n));
  std::vector<std::thread> th;
  for (int t = 1; t < nt; ++t) th.emplace_back(work);
  work();
  for (auto& t : th) t.join();
  if (first) std::rethrow_exception(first);
}

template <typename F>
aplicur_status bguarded(aplicur_batch_ctx* h, F&& f) {
  AllocScope as(h->alloc_.alloc ? &h->alloc_ : nullptr);
  try {
    return (aplicur_status)f();
  } catch (const Error& e) {
    h->err = e.what();
    return (aplicur_status)e.code;
  } catch (const std::exception& e) {
    h->err = e.what();
    return APLICUR_ECUDA;
  } catch (...) {
    h->err = "unknown failure";
    return APLICUR_ECUDA;
  }
}

// Convergence bookkeeping shared by the preconditioned and plain batched solves.
struct PairBook {
  std::vector<char> stopped;   // no further phases (converged, stagnated, out of budget)
  std::vector<double> prev;
};

void batch_phase(aplicur_batch_ctx* h, const std::vector<char>& mask, const std::vector<double>& nu,
                 double tol, long long maxit, std::vector<long long>& it_out) {
  const size_t npairs = (size_t)h->np * h->R;
  std::vector<long long> budget(npairs, 0);
  for (size_t e = 0; e < npairs; ++e) budget[e] = std::max(0LL, maxit - h->iters[e]);
  std::vector<int> reasons;
  // the Paige-Saunders tests must not end a phase before the refinement can reach tol:
  // with FP32 recurrences a phase stopped at eps_lsqr ~ tol leaves the pair just short
  const double eps = std::min(h->pc[0]->opt.eps_lsqr, 0.01 * tol);
  h->eng.run_phase(mask, nu, eps, tol, budget, it_out, reasons);
  for (size_t e = 0; e < npairs; ++e) h->iters[e] += it_out[e];
  std::vector<double> ne;
  h->eng.ne_residual(mask, ne);
  for (size_t e = 0; e < npairs; ++e) {
    if (!mask[e]) continue;
    h->ne[e] = ne[e];
    h->conv[e] = ne[e] <= tol ? 1 : 0;
  }
}

void refine_pairs(aplicur_batch_ctx* h, double tol, long long maxit, PairBook& bk, bool plain);

int batch_solve(aplicur_batch_ctx* h, double tol, long long maxit, bool plain) {
  using clk = std::chrono::steady_clock;
  auto ms_since = [](clk::time_point t0) {
    return std::chrono::duration<double, std::milli>(clk::now() - t0).count();
  };
  const int np = h->np, R = h->R;
  const size_t npairs = (size_t)np * R;
  h->iters.assign(npairs, 0);
  h->ne.assign(npairs, INFINITY);
  h->conv.assign(npairs, 0);
  h->broke.assign(np, 0);
  h->stats.time_rank_ms = h->stats.time_build_ms = h->stats.time_lsqr_ms = 0.0;
  h->stats.time_check_ms = 0.0;
  h->eng.zero_x();
  for (int p = 0; p < np; ++p) {
    h->eng.clear_precond(p);
    for (int r = 0; r < R; ++r)
      if (h->eng.norm_ref(p, r) == 0.0) { h->ne[(size_t)p * R + r] = 0.0; h->conv[(size_t)p * R + r] = 1; }
  }
  PairBook bk;
  bk.stopped.assign(npairs, 0);
  bk.prev.assign(npairs, INFINITY);
  for (size_t e = 0; e < npairs; ++e) bk.stopped[e] = h->conv[e];
  auto problem_done = [&](int p) {
    for (int r = 0; r < R; ++r)
      if (!bk.stopped[(size_t)p * R + r]) return false;
    return true;
  };
  std::vector<long long> it;
  const aplicur_options& o = h->pc[0]->opt;
  if (!plain) {
    std::vector<double> d_cur(np, INFINITY), rho(np, 0.0), margin(np, 0.0);
    std::vector<char> last(np, 0), rank_done(np, 0), rebuild(np, 0);
    std::vector<char> exhausted(np, 0);
    parallel_for(np, h->nthreads, h->device, [&](int p) { reset_cur(h->pc[p]); });
    while (true) {
      std::vector<int> act;
      for (int p = 0; p < np; ++p)
        if (!rank_done[p] && !problem_done(p)) act.push_back(p);
      if (act.empty()) break;
      auto t0 = clk::now();
      parallel_for((int)act.size(), h->nthreads, h->device, [&](int k) {
        const int p = act[k];
        aplicur_ctx* c = h->pc[p];
        double rh = 0, mg = INFINITY;
        bool ex = false;
        try {
          rank_step(c, &rh, &ex, &mg);
        } catch (const Error& e) {
          // a breakdown ends this problem's rank growth; its pairs finish with the last
          // preconditioner it built (or none)
          if (e.code != ST_EBREAKDOWN) throw;
          h->broke[p] = 1;
          last[p] = 1;
          rebuild[p] = 0;
          return;
        }
        const bool full = c->ell >= c->kmax;
        const double rho_eff = ex ? 0.0 : rh;
        last[p] = (rho_eff <= c->eps_cur || full || ex) ? 1 : 0;
        const double gap = rho_eff - c->eps_cur;
        rebuild[p] = (last[p] || (gap > 0.0 && d_cur[p] / gap >= c->opt.nu_prec)) ? 1 : 0;
        rho[p] = rh;
        exhausted[p] = ex ? 1 : 0;
        c->steps.push_back(StepRec{c->ell, rh, rebuild[p], mg});
      });
      h->stats.time_rank_ms += ms_since(t0);
      std::vector<int> reb;
      for (int p : act)
        if (rebuild[p] && h->pc[p]->ell > 0) reb.push_back(p);
      t0 = clk::now();
      parallel_for((int)reb.size(), h->nthreads, h->device, [&](int k) {
        try {
          build_preconditioner(h->pc[reb[k]]);
        } catch (const Error& e) {
          if (e.code != ST_EBREAKDOWN) throw;
          h->broke[reb[k]] = 1;
          last[reb[k]] = 1;
        }
      });
      {
        std::vector<int> ok;
        for (int p : reb)
          if (!h->broke[p]) ok.push_back(p);
        reb.swap(ok);
      }
      for (int p : reb) h->eng.set_precond(p, h->pc[p]->P);
      h->stats.time_build_ms += ms_since(t0);
      std::vector<char> mask(npairs, 0);
      std::vector<double> nu(np, INFINITY);
      bool any = false;
      for (int p : reb) {
        nu[p] = last[p] ? INFINITY : h->pc[p]->opt.nu_lsqr;
        for (int r = 0; r < R; ++r) {
          const size_t e = (size_t)p * R + r;
          if (!bk.stopped[e] && h->iters[e] < maxit) { mask[e] = 1; any = true; }
        }
      }
      if (any) {
        t0 = clk::now();
        batch_phase(h, mask, nu, tol, maxit, it);
        h->stats.time_lsqr_ms += ms_since(t0);
        for (int p : reb) {
          long long mx = 0;
          for (int r = 0; r < R; ++r) mx = std::max(mx, it[(size_t)p * R + r]);
          double nmax = 0;
          for (int r = 0; r < R; ++r) nmax = std::max(nmax, h->ne[(size_t)p * R + r]);
          h->pc[p]->phases.push_back(PhaseRec{h->pc[p]->ell, mx, 0, nmax});
        }
        for (size_t e = 0; e < npairs; ++e) {
          if (!mask[e]) continue;
          bk.prev[e] = h->ne[e];
          if (h->conv[e] || h->iters[e] >= maxit) bk.stopped[e] = 1;
        }
      }
      for (int p : reb) d_cur[p] = (exhausted[p] ? 0.0 : rho[p]) - h->pc[p]->eps_cur;
      for (int p : act)
        if (last[p]) rank_done[p] = 1;
    }
  }
  // final phases without the dynamic test (the last phase of the driver continued, or
  // the plain solve).  FP32 recurrences end each phase after a smaller true gain than the
  // FP64 driver's (the estimate runs ahead of the residual), so the batch allows 4x the
  // phases
  refine_pairs(h, tol, maxit, bk, plain);
  h->solved = true;
  int nconv = 0;
  long long imax = 0, isum = 0;
  double nmax = 0;
  for (size_t e = 0; e < npairs; ++e) {
    nconv += h->conv[e];
    imax = std::max(imax, h->iters[e]);
    isum += h->iters[e];
    nmax = std::max(nmax, h->ne[e]);
  }
  h->stats.pairs = (int32_t)npairs;
  h->stats.converged = nconv;
  h->stats.iters_max = imax;
  h->stats.iters_sum = isum;
  h->stats.ne_max = nmax;
  h->stats.rows_per_warp = h->eng.tuned_rw();
  h->stats.cols_per_lane = h->eng.tuned_cw();
  h->stats.launches_per_iter = h->eng.launches_per_iter();
  return nconv == (int)npairs ? ST_OK : ST_ENOTCONV;
}

// Y (m x R, column-major) = A X (X: n x R column-major) with FP64 sums of the stored
// FP32 values, or, with Bsub, Y = Bsub - A X; one warp per row.
__global__ void batch_ax_kernel(int fmt, int64_t m, int64_t n, int64_t ld, const float* vals,
                                const int* rowptr, const int* colidx, const double* X, int R,
                                const double* Bsub, double* Y) {
  const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= m) return;
  double acc[16];
#pragma unroll
  for (int r = 0; r < 16; ++r) acc[r] = 0.0;
  if (fmt == 0) {
    for (int64_t j = lane; j < n; j += 32) {
      const double a = (double)vals[i * ld + j];
#pragma unroll
      for (int r = 0; r < 16; ++r)
        if (r < R) acc[r] = fma(a, X[j + (int64_t)r * n], acc[r]);
    }
  } else {
    for (int e = rowptr[i] + lane; e < rowptr[i + 1]; e += 32) {
      const double a = (double)vals[e];
      const int64_t j = colidx[e];
#pragma unroll
      for (int r = 0; r < 16; ++r)
        if (r < R) acc[r] = fma(a, X[j + (int64_t)r * n], acc[r]);
    }
  }
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    if (r >= R) break;
    double v = acc[r];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) Y[i + (int64_t)r * m] = Bsub ? Bsub[i + (int64_t)r * m] - v : v;
  }
}

// out[r] = -lambda_r^T x_r  (the gradient in mu of each pair), one block per pair
__global__ void batch_gmu_kernel(int64_t n, const double* lam, const double* x, double* out) {
  __shared__ double sh[32];
  const int r = blockIdx.x;
  double s = 0.0;
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x)
    s = fma(lam[j + (int64_t)r * n], x[j + (int64_t)r * n], s);
  s = block_sum(s, sh);
  if (threadIdx.x == 0) out[r] = -s;
}

// G(i, j) = sum_r res(i, r) lambda(j, r) - (A lambda)(i, r) x(j, r), FP32 row-major ld n
__global__ void batch_gA_kernel(int64_t m, int64_t n, int R, const double* res,
                                const double* al, const double* lam, const double* x, float* G) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m * n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / n, j = e - i * n;
    double g = 0.0;
    for (int r = 0; r < R; ++r)
      g += res[i + (int64_t)r * m] * lam[j + (int64_t)r * n] -
           al[i + (int64_t)r * m] * x[j + (int64_t)r * n];
    G[e] = (float)g;
  }
}

// Phases without the dynamic test (nu = infinity) for every pair not stopped, until tol,
// the iteration budget, or a phase that no longer gains 10% (the final phases of the
// driver, and the adjoint solves).
void refine_pairs(aplicur_batch_ctx* h, double tol, long long maxit, PairBook& bk, bool plain) {
  using clk = std::chrono::steady_clock;
  const size_t npairs = (size_t)h->np * h->R;
  const aplicur_options& o = h->pc[0]->opt;
  std::vector<long long> it;
  for (int rep = 0; rep <= 4 * o.max_extra_phases; ++rep) {
    std::vector<char> mask(npairs, 0);
    bool any = false;
    for (size_t e = 0; e < npairs; ++e)
      if (!bk.stopped[e] && h->iters[e] < maxit) { mask[e] = 1; any = true; }
    if (!any) break;
    std::vector<double> nu(h->np, INFINITY);
    auto t0 = clk::now();
    batch_phase(h, mask, nu, tol, maxit, it);
    h->stats.time_lsqr_ms += std::chrono::duration<double, std::milli>(clk::now() - t0).count();
    for (size_t e = 0; e < npairs; ++e) {
      if (!mask[e]) continue;
      const bool stag = !plain || rep > 0 ? (it[e] == 0 || h->ne[e] > 0.9 * bk.prev[e]) : false;
      if (h->conv[e] || h->iters[e] >= maxit || stag) bk.stopped[e] = 1;
      bk.prev[e] = h->ne[e];
    }
  }
}

// Adjoint of the batched solves: lambda_{p,r} = (A_p^T A_p + mu I)^{-1} g_{p,r} with the
// preconditioners of the last solve, then d/db = A lambda, d/dmu = -lambda^T x and, for
// dense problems, d/dA = r lambda^T - (A lambda) x^T summed over the right-hand sides.
int batch_backward(aplicur_batch_ctx* h, const double* const* gx, double tol, long long maxit,
                   double* const* gb, double* gmu, float* const* gA) {
  APL_REQUIRE(h->solved, "batched backward: run aplicur_batch_solve first");
  const int np = h->np, R = h->R;
  const size_t npairs = (size_t)np * R;
  cudaStream_t st = h->st;
  for (int p = 0; p < np; ++p) {
    APL_REQUIRE(gx[p] != nullptr, "batched backward: grad_x[p] NULL");
    APL_REQUIRE(!(gA && gA[p]) || h->pc[p]->A.fmt == 0, "grad_A is only produced for dense A");
  }
  std::vector<DBuf<double>> xs(np), lam(np);
  for (int p = 0; p < np; ++p) {
    xs[p].alloc((size_t)h->pc[p]->n * R, st);
    h->eng.get_x(p, xs[p].p);
  }
  h->eng.begin_adjoint(std::vector<const double*>(gx, gx + np));
  h->iters.assign(npairs, 0);
  h->ne.assign(npairs, INFINITY);
  h->conv.assign(npairs, 0);
  h->stats.time_lsqr_ms = 0.0;
  PairBook bk;
  bk.stopped.assign(npairs, 0);
  bk.prev.assign(npairs, INFINITY);
  for (int p = 0; p < np; ++p)
    for (int r = 0; r < R; ++r)
      if (h->eng.norm_ref(p, r) == 0.0) {
        const size_t e = (size_t)p * R + r;
        h->ne[e] = 0.0; h->conv[e] = 1; bk.stopped[e] = 1;
      }
  try {
    refine_pairs(h, tol, maxit, bk, false);
    for (int p = 0; p < np; ++p) {
      lam[p].alloc((size_t)h->pc[p]->n * R, st);
      h->eng.get_x(p, lam[p].p);
    }
  } catch (...) {
    h->eng.end_adjoint();
    throw;
  }
  h->eng.end_adjoint();
  for (int p = 0; p < np; ++p) {
    const aplicur_ctx* c = h->pc[p];
    const MatView& A = c->A;
    const int64_t m = c->m, n = c->n;
    const unsigned rows_blocks = (unsigned)cdiv(m * 32, 256);
    DBuf<double> al;
    double* alp = gb ? gb[p] : nullptr;
    if (!alp) { al.alloc((size_t)m * R, st); alp = al.p; }
    batch_ax_kernel<<<rows_blocks, 256, 0, st>>>(A.fmt, m, n, A.ld, (const float*)A.vals, A.rowptr,
                                                 A.colidx, lam[p].p, R, nullptr, alp);
    APL_LAUNCH_CHECK();
    if (gmu) {
      batch_gmu_kernel<<<R, 256, 0, st>>>(n, lam[p].p, xs[p].p, gmu + (size_t)p * R);
      APL_LAUNCH_CHECK();
    }
    if (gA && gA[p]) {
      DBuf<double> res;
      res.alloc((size_t)m * R, st);
      batch_ax_kernel<<<rows_blocks, 256, 0, st>>>(A.fmt, m, n, A.ld, (const float*)A.vals,
                                                   A.rowptr, A.colidx, xs[p].p, R, h->bsrc[p],
                                                   res.p);
      APL_LAUNCH_CHECK();
      batch_gA_kernel<<<(unsigned)std::min<int64_t>(cdiv(m * n, 256), 4096), 256, 0, st>>>(
          m, n, R, res.p, alp, lam[p].p, xs[p].p, gA[p]);
      APL_LAUNCH_CHECK();
    }
  }
  APL_CUDA(cudaStreamSynchronize(st));
  int nconv = 0;
  long long imax = 0, isum = 0;
  double nmax = 0;
  for (size_t e = 0; e < npairs; ++e) {
    nconv += h->conv[e];
    imax = std::max(imax, h->iters[e]);
    isum += h->iters[e];
    nmax = std::max(nmax, h->ne[e]);
  }
  h->stats.pairs = (int32_t)npairs;
  h->stats.converged = nconv;
  h->stats.iters_max = imax;
  h->stats.iters_sum = isum;
  h->stats.ne_max = nmax;
  return nconv == (int)npairs ? ST_OK : ST_ENOTCONV;
}

}  // namespace

static thread_local std::string g_batch_err;

extern "C" {

aplicur_status aplicur_batch_create(aplicur_batch_handle* out, int32_t nprob,
                                    const aplicur_matrix* A, const double* const* b,
                                    int32_t nrhs, double mu, int32_t sketch_dim,
                                    const aplicur_options* opt, void* stream) {
  if (!out || !A || !b || nprob < 1) { g_batch_err = "null argument or nprob < 1"; return APLICUR_EINVAL; }
  *out = nullptr;
  if (opt && ((opt->alloc != nullptr) != (opt->free_ != nullptr))) {
    g_batch_err = "options: set both alloc and free_, or neither";
    return APLICUR_EINVAL;
  }
  aplicur_batch_ctx* h = new (std::nothrow) aplicur_batch_ctx();
  if (!h) return APLICUR_ENOMEM;
  if (opt) h->alloc_ = Allocator{opt->alloc, opt->free_, opt->alloc_ctx};
  aplicur_status stt = bguarded(h, [&]() -> int {
    auto t0 = std::chrono::steady_clock::now();
    APL_REQUIRE(nrhs >= 1 && nrhs <= BATCH_MAX_RHS, "nrhs must be 1..16");
    APL_REQUIRE(mu > 0.0 && std::isfinite(mu), "batched solves need mu > 0");
    APL_REQUIRE(!opt || opt->variant == APLICUR_VARIANT_SVD,
                "batched solves use the SVD-based preconditioner");
    APL_REQUIRE(!opt || opt->schedule == APLICUR_SCHEDULE_ADAPTIVE,
                "batched solves use the fully adaptive schedule");
    for (int p = 0; p < nprob; ++p) {
      APL_REQUIRE(A[p].dtype == APLICUR_F32, "batched solves take FP32 matrices");
      APL_REQUIRE(b[p] != nullptr, "b[p] NULL");
    }
    APL_CUDA(cudaGetDevice(&h->device));
    if (stream) h->st = (cudaStream_t)stream;
    else { APL_CUDA(cudaStreamCreateWithFlags(&h->st, cudaStreamNonBlocking)); h->own_stream = true; }
    h->np = nprob;
    h->R = nrhs;
    h->mu = mu;
    // worker threads mostly wait on their problem's stream, so more threads than cores
    // keep more problems' small kernels in flight
    h->nthreads = (int)std::max(4u, std::min(32u, 2 * std::thread::hardware_concurrency()));
    aplicur_options o;
    if (opt) o = *opt; else aplicur_options_default(&o);
    o.replay_nphases = 0; o.replay_phases = nullptr;
    o.replay_nsteps = 0; o.replay_rebuild = nullptr;
    o.sketch_rows = nullptr; o.sketch_signs = nullptr; o.normest_w = nullptr;
    o.profile = 0;
    h->pc.assign(nprob, nullptr);
    for (int p = 0; p < nprob; ++p) {
      h->pc[p] = new (std::nothrow) aplicur_ctx();
      APL_REQUIRE(h->pc[p] != nullptr, "out of host memory");
      // the problems' selections run concurrently on several streams: one launch per
      // LUPP step rather than grid-resident cooperative launches
      h->pc[p]->lw.cooperative = false;
    }
    parallel_for(nprob, h->nthreads, h->device, [&](int p) {
      aplicur_options op = o;
      op.seed = o.seed + (uint64_t)p;
      ctx_init(h->pc[p], &A[p], nullptr, mu, sketch_dim, &op, nullptr, false);
    });
    std::vector<BatchSrc> src(nprob);
    for (int p = 0; p < nprob; ++p) src[p] = BatchSrc{h->pc[p]->A, b[p]};
    h->bsrc.assign(b, b + nprob);
    h->eng.setup(h->st, src, nrhs, mu);
    h->eng.autotune();
    h->stats.time_setup_ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    h->stats.rows_per_warp = h->eng.tuned_rw();
    h->stats.cols_per_lane = h->eng.tuned_cw();
    return ST_OK;
  });
  if (stt != APLICUR_OK) {
    g_batch_err = h->err;
    aplicur_batch_destroy(h);
    return stt;
  }
  *out = h;
  return APLICUR_OK;
}

static aplicur_status batch_run(aplicur_batch_handle h, double tol, int64_t maxit,
                                double* const* x_out, bool plain) {
  if (!h || !x_out) return APLICUR_EINVAL;
  return bguarded(h, [&]() -> int {
    APL_REQUIRE(tol >= 0.0 && maxit >= 0, "need tol >= 0 and maxit >= 0");
    for (int p = 0; p < h->np; ++p) APL_REQUIRE(x_out[p] != nullptr, "x_out[p] NULL");
    const int st = batch_solve(h, tol, maxit, plain);
    for (int p = 0; p < h->np; ++p) h->eng.get_x(p, x_out[p]);
    APL_CUDA(cudaStreamSynchronize(h->st));
    return st;
  });
}

aplicur_status aplicur_batch_solve(aplicur_batch_handle h, double tol, int64_t maxit,
                                   double* const* x_out) {
  return batch_run(h, tol, maxit, x_out, false);
}

aplicur_status aplicur_batch_plain_lsqr(aplicur_batch_handle h, double tol, int64_t maxit,
                                        double* const* x_out) {
  return batch_run(h, tol, maxit, x_out, true);
}

aplicur_status aplicur_batch_backward(aplicur_batch_handle h, const double* const* grad_x,
                                     double tol, int64_t maxit, double* const* grad_b,
                                     double* grad_mu, float* const* grad_A) {
  if (!h || !grad_x) return APLICUR_EINVAL;
  return bguarded(h, [&]() -> int {
    cudaSetDevice(h->device);
    return batch_backward(h, grad_x, tol, maxit, grad_b, grad_mu, grad_A);
  });
}

aplicur_status aplicur_batch_get_pair(aplicur_batch_handle h, int32_t p, int32_t r,
                                      int64_t* iters, double* ne_res, int32_t* converged) {
  if (!h || p < 0 || p >= h->np || r < 0 || r >= h->R) return APLICUR_EINVAL;
  if (h->iters.empty()) { h->err = "no solve yet"; return APLICUR_EINVAL; }
  const size_t e = (size_t)p * h->R + r;
  if (iters) *iters = h->iters[e];
  if (ne_res) *ne_res = h->ne[e];
  if (converged) *converged = h->conv[e];
  return APLICUR_OK;
}

aplicur_status aplicur_batch_get_problem(aplicur_batch_handle h, int32_t p, int32_t* ell,
                                         int32_t* nsteps, int32_t* nphases, int32_t* broke,
                                         int32_t* I, int32_t* J) {
  if (!h || p < 0 || p >= h->np) return APLICUR_EINVAL;
  const aplicur_ctx* c = h->pc[p];
  if (broke) *broke = h->broke.empty() ? 0 : h->broke[p];
  if (ell) *ell = c->ell;
  if (nsteps) *nsteps = (int32_t)c->steps.size();
  if (nphases) *nphases = (int32_t)c->phases.size();
  if (I) std::copy(c->I.begin(), c->I.end(), I);
  if (J) std::copy(c->J.begin(), c->J.end(), J);
  return APLICUR_OK;
}

aplicur_status aplicur_batch_get_stats(aplicur_batch_handle h, aplicur_batch_stats* st) {
  if (!h || !st) return APLICUR_EINVAL;
  *st = h->stats;
  return APLICUR_OK;
}

const char* aplicur_batch_last_error(aplicur_batch_handle h) {
  if (!h) return g_batch_err.c_str();
  return h->err.c_str();
}

void aplicur_batch_destroy(aplicur_batch_handle h) {
  if (!h) return;
  cudaStream_t st = h->st;
  const bool own = h->own_stream;
  if (st) cudaStreamSynchronize(st);
  delete h;
  if (own && st) cudaStreamDestroy(st);
}

}  // extern "C"
