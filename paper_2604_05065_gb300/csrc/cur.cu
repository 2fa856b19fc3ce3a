// Sketch and CUR-refinement kernels.
#include <algorithm>
#include <climits>

#include "cur.cuh"
#include "dense.cuh"
#include "df32.cuh"

namespace apl {

namespace {

template <typename T>
__device__ __forceinline__ double ld_val(const void* p, int64_t i) {
  return (double)(reinterpret_cast<const T*>(p)[i]);
}

// ---- sketch ---------------------------------------------------------------------------

// Dense: thread (r, j) sums the rows of A listed for sketch row r, ascending.  The sign is
// applied before widening (negation is exact), so each term costs one FP64 add.
template <typename T>
__global__ void sketch_dense_kernel(int64_t n, int64_t ld, const T* __restrict__ A, int s,
                                    const int* __restrict__ tptr, const int* __restrict__ ti,
                                    const signed char* __restrict__ tsgn, double scale,
                                    double* __restrict__ Y) {
  const int64_t j = (int64_t)blockIdx.y * blockDim.x + threadIdx.x;
  const int r = blockIdx.x;
  if (j >= n) return;
  double acc = 0.0;
  const int e0 = tptr[r], e1 = tptr[r + 1];
  for (int e = e0; e < e1; ++e) {
    const T a = A[(int64_t)ti[e] * ld + j];
    acc += widen(tsgn[e] > 0 ? a : -a);
  }
  Y[r + j * (int64_t)s] = acc * scale;
}

// CSR: thread (r, j) walks column j (ascending rows) and keeps entries whose row maps to r.
template <typename T>
__global__ void sketch_csc_kernel(int64_t n, const int* __restrict__ colptr,
                                  const int* __restrict__ rowidx, const T* __restrict__ cvals,
                                  int s, int xi, const int* __restrict__ srows,
                                  const signed char* __restrict__ ssign, double scale,
                                  double* __restrict__ Y) {
  const int64_t j = (int64_t)blockIdx.y * blockDim.x + threadIdx.x;
  const int r = blockIdx.x;
  if (j >= n) return;
  double acc = 0.0;
  for (int e = colptr[j]; e < colptr[j + 1]; ++e) {
    const int64_t i = rowidx[e];
    const int* rr = srows + i * xi;
    for (int k = 0; k < xi; ++k) {
      if (rr[k] == r) {
        const double a = (double)cvals[e];
        acc = ssign[i * xi + k] > 0 ? acc + a : acc - a;
      }
    }
  }
  Y[r + j * (int64_t)s] = acc * scale;
}

// ---- LUPP -----------------------------------------------------------------------------

// A pivot candidate.  |value| is carried as its IEEE bit pattern: for non-negative
// doubles the patterns order like the values, so every comparison and maximum of the
// argmax reduction is an integer operation (GB300 issues FP64 compares at 1/64 of the
// integer rate).  -1 marks "no candidate".
struct Cand {
  long long v;    // bits of |value| of the best candidate, -1 if none
  int pos;        // its position in the current row order
  long long sec;  // bits of the second-best |value|, -1 if none
  int row;        // its row index (-1 if none)
};

__device__ __forceinline__ long long abs_key(double x) {
  return __double_as_longlong(x) & 0x7fffffffffffffffLL;
}

__device__ __forceinline__ bool cand_better(long long v1, int p1, long long v2, int p2) {
  return v1 > v2 || (v1 == v2 && p1 < p2);
}

__device__ __forceinline__ Cand cand_merge(Cand a, Cand b) {
  Cand r;
  if (cand_better(a.v, a.pos, b.v, b.pos)) {
    r.v = a.v; r.pos = a.pos; r.sec = a.sec > b.v ? a.sec : b.v; r.row = a.row;
  } else {
    r.v = b.v; r.pos = b.pos; r.sec = b.sec > a.v ? b.sec : a.v; r.row = b.row;
  }
  return r;
}

__device__ __forceinline__ Cand warp_cand(Cand c) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    Cand d;
    d.v = __shfl_down_sync(0xffffffffu, c.v, o);
    d.pos = __shfl_down_sync(0xffffffffu, c.pos, o);
    d.sec = __shfl_down_sync(0xffffffffu, c.sec, o);
    d.row = __shfl_down_sync(0xffffffffu, c.row, o);
    c = cand_merge(c, d);
  }
  return c;
}

__device__ Cand block_cand(Cand c) {
  __shared__ long long sv[32], ss[32];
  __shared__ int sp[32], sr[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  c = warp_cand(c);
  if (lane == 0) { sv[wid] = c.v; sp[wid] = c.pos; ss[wid] = c.sec; sr[wid] = c.row; }
  __syncthreads();
  Cand r{-1, INT_MAX, -1, -1};
  if (wid == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    if (lane < nw) { r.v = sv[lane]; r.pos = sp[lane]; r.sec = ss[lane]; r.row = sr[lane]; }
    r = warp_cand(r);
  }
  return r;
}

// One elimination step j.  A block owns 32 consecutive rows (lane = row) and its 8 warps
// split the columns j-1.. K-1 (warp w takes columns j + w, j + w + 8, ...), so every
// access X(i, c) is coalesced when rs = 1.  Step j applies the elimination of column
// j-1 by the pivot row chosen at step j-1, then looks for the pivot of column j.
constexpr int LUPP_U = 8;

__global__ void __launch_bounds__(256) lupp_step_kernel(
    int64_t N, int64_t K, double* __restrict__ X, int64_t rs, int64_t cs, int j,
    int* __restrict__ pos_of, int* __restrict__ row_at, int* __restrict__ piv,
    double* __restrict__ pval, int* __restrict__ ppos, double* __restrict__ psec,
    unsigned int* counter, double* margin, int* iscal) {
  extern __shared__ double prow[];  // pivot row values for columns j-1 .. K-1
  if (iscal[1]) return;             // selection already stopped at a zero pivot
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  const int p = j > 0 ? piv[j - 1] : -1;
  if (j > 0) {
    for (int64_t c = j - 1 + threadIdx.x; c < K; c += blockDim.x)
      prow[c - (j - 1)] = X[(int64_t)p * rs + c * cs];
  }
  const int64_t i = (int64_t)blockIdx.x * 32 + lane;
  const bool live = i < N && pos_of[i] >= j;  // not yet a pivot row
  double* xi = X + i * rs;
  double l = 0.0;
  __syncthreads();
  // multipliers by the pivot's reciprocal, formed once per block (as LAPACK's getf2
  // scales the column by 1 / pivot)
  if (j > 0 && threadIdx.x == 0) prow[K - (j - 1)] = 1.0 / prow[0];
  __syncthreads();
  if (live && j > 0) l = xi[(int64_t)(j - 1) * cs] * prow[K - (j - 1)];
  __syncthreads();  // every warp has read X(i, j-1) before it is overwritten
  Cand mine{-1, INT_MAX, -1, -1};
  if (live) {
    if (j > 0 && wid == 0) xi[(int64_t)(j - 1) * cs] = l;
    // LUPP_U columns per warp are loaded before any is updated and stored, so their L2
    // round trips overlap instead of following one another
    for (int64_t c0 = j + wid; c0 < K; c0 += (int64_t)nw * LUPP_U) {
      double v[LUPP_U];
#pragma unroll
      for (int u = 0; u < LUPP_U; ++u) {
        const int64_t c = c0 + (int64_t)u * nw;
        v[u] = c < K ? xi[c * cs] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < LUPP_U; ++u) {
        const int64_t c = c0 + (int64_t)u * nw;
        if (c >= K) continue;
        if (j > 0) {
          v[u] = v[u] - l * prow[c - (j - 1)];
          xi[c * cs] = v[u];
        }
        if (c == j) {
          Cand cd{abs_key(v[u]), pos_of[i], -1, (int)i};
          mine = cd;
        }
      }
    }
  }
  Cand b = block_cand(mine);
  if (threadIdx.x == 0) {
    pval[blockIdx.x] = __longlong_as_double(b.v);
    ppos[blockIdx.x] = b.pos;
    psec[blockIdx.x] = __longlong_as_double(b.sec);
  }
  if (!last_block_done(counter)) return;
  Cand t{-1, INT_MAX, -1, -1};
  for (int q = threadIdx.x; q < (int)gridDim.x; q += blockDim.x) {
    Cand c{__double_as_longlong(__ldcg(pval + q)), __ldcg(ppos + q),
           __double_as_longlong(__ldcg(psec + q)), -1};
    t = cand_merge(t, c);
  }
  t = block_cand(t);
  if (threadIdx.x == 0) {
    if (!(t.v > 0)) {
      iscal[1] = 1;  // zero pivot (or no candidates): rank exhausted
    } else {
      const int pr = row_at[t.pos];
      const int q = row_at[j];
      row_at[t.pos] = q;
      pos_of[q] = t.pos;
      row_at[j] = pr;
      pos_of[pr] = j;
      piv[j] = pr;
      iscal[0] = j + 1;
      if (t.sec >= 0) {
        const double tv = __longlong_as_double(t.v), ts = __longlong_as_double(t.sec);
        *margin = fmin(*margin, (tv - ts) / tv);
      }
    }
  }
}

__global__ void lupp_init_kernel(int64_t N, int* pos_of, int* row_at, double* margin, int* iscal,
                                 unsigned int* counter) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) { pos_of[i] = (int)i; row_at[i] = (int)i; }
  if (i == 0) {
    *margin = INFINITY;
    iscal[0] = 0;
    iscal[1] = 0;
    iscal[2] = 0;
    counter[0] = 0u;
    counter[1] = 0u;
  }
}

// ---- LUPP as one cooperative launch ----------------------------------------------------
//
// All k elimination steps in one kernel whose blocks are resident together (cooperative
// launch).  Block b owns the 32-row tiles b, b + G, b + 2G, ... (G blocks); a step updates
// the owned rows and finds each block's best candidate (phase A), the blocks meet at a
// grid barrier, and every block merges the G partial candidates itself (phase B), so all
// of them know the pivot without a second barrier.  The positions of a block's rows live
// in its shared memory: the swap of step j (pivot row to position j, the row that held
// position j to the pivot's old position) is applied by the owners when they read the
// positions in step j + 1.  Column j of the owned rows, found while forming the
// candidates, stays in shared memory for step j + 1's multipliers.  Partial candidates alternate between two buffers by step
// parity: a block can run at most one step ahead of the slowest.

constexpr long long kLuppSpin = 1LL << 22;  // polls of the grid barrier before it gives up

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid-wide barrier: bar[0] counts arrivals, bar[1] is the generation.  Returns false
// (and sets *err) when the wait ran past its bound or another block already gave up;
// every later barrier then gives up too, so the launch ends in bounded time.
__device__ bool lupp_grid_sync(unsigned* bar, int* err) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    const unsigned gen = ld_acquire_u32(bar + 1);
    __threadfence();  // this block's writes are visible before its arrival
    if (atomicAdd(bar, 1u) == gridDim.x - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      long long it = 0;
      while (ld_acquire_u32(bar + 1) == gen) {
        if (++it > kLuppSpin || *(volatile int*)err) {
          atomicExch(err, 1);
          ok = 0;
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

__global__ void __launch_bounds__(256) lupp_coop_kernel(
    int64_t N, int64_t K, double* __restrict__ X, int64_t rs, int64_t cs, int k, int tpb,
    int* __restrict__ piv, long long* __restrict__ pv, int* __restrict__ pp,
    long long* __restrict__ ps, int* __restrict__ pr, unsigned* bar, double* margin,
    int* iscal) {
  // dynamic shared memory: the pivot row for columns j-1 .. K-1 and 1/pivot (K + 1), then
  // column j-1 / j of the owned rows by step parity (2 x tpb x 32), then the owned rows'
  // positions (tpb x 32 ints); tpb bounds the tiles a block owns
  extern __shared__ double prow[];
  double* xcol = prow + (K + 1);
  int* spos = reinterpret_cast<int*>(xcol + 2 * (int64_t)tpb * 32);
  __shared__ long long s_v, s_sec;
  __shared__ int s_pos, s_row;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  const int64_t ntiles = (N + 31) / 32;
  for (int e = threadIdx.x; e < tpb * 32; e += blockDim.x) {
    const int64_t i = (blockIdx.x + (int64_t)(e / 32) * gridDim.x) * 32 + (e % 32);
    spos[e] = i < N ? (int)i : -1;
  }
  __syncthreads();
  int p = -1;     // pivot row of the previous step
  int ppos = -1;  // its position before that step's swap
  for (int j = 0; j < k; ++j) {
    if (j > 0) {
      // written by the pivot row's owner before the last barrier: read through L2
      for (int64_t c = j - 1 + threadIdx.x; c < K; c += blockDim.x)
        prow[c - (j - 1)] = __ldcg(X + (int64_t)p * rs + c * cs);
      __syncthreads();
      if (threadIdx.x == 0) prow[K - (j - 1)] = 1.0 / prow[0];
      __syncthreads();
    }
    const double* xprev = xcol + (int64_t)((j + 1) & 1) * tpb * 32;  // column j - 1
    double* xnext = xcol + (int64_t)(j & 1) * tpb * 32;               // column j
    Cand mine{-1, INT_MAX, -1, -1};
    int lt = 0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++lt) {
      const int64_t i = tile * 32 + lane;
      const int slot = lt * 32 + lane;
      int pi = -1;
      if (i < N) {
        pi = spos[slot];
        if (j > 0) {
          // the swap of step j - 1 (idempotent, so every warp may apply it)
          const int q = (i == p) ? j - 1 : (pi == j - 1 ? ppos : pi);
          if (q != pi) {
            pi = q;
            if (wid == 0) spos[slot] = q;
          }
        }
      }
      const bool live = i < N && pi >= j;
      double* xi = X + i * rs;
      if (live) {
        // X(i, j - 1) was kept from the previous step, so no warp reads it from memory
        // and warp 0 may overwrite it with the multiplier at once
        const double l = j > 0 ? xprev[slot] * prow[K - (j - 1)] : 0.0;
        if (j > 0 && wid == 0) xi[(int64_t)(j - 1) * cs] = l;
        for (int64_t c0 = j + wid; c0 < K; c0 += (int64_t)nw * LUPP_U) {
          double v[LUPP_U];
#pragma unroll
          for (int u = 0; u < LUPP_U; ++u) {
            const int64_t c = c0 + (int64_t)u * nw;
            v[u] = c < K ? xi[c * cs] : 0.0;
          }
#pragma unroll
          for (int u = 0; u < LUPP_U; ++u) {
            const int64_t c = c0 + (int64_t)u * nw;
            if (c >= K) continue;
            if (j > 0) {
              v[u] = v[u] - l * prow[c - (j - 1)];
              xi[c * cs] = v[u];
            }
            if (c == j) {
              mine = cand_merge(mine, Cand{abs_key(v[u]), pi, -1, (int)i});
              xnext[slot] = v[u];
            }
          }
        }
      }
    }
    const Cand b = block_cand(mine);
    const int64_t base = (int64_t)(j & 1) * gridDim.x;
    if (threadIdx.x == 0) {
      pv[base + blockIdx.x] = b.v;
      pp[base + blockIdx.x] = b.pos;
      ps[base + blockIdx.x] = b.sec;
      pr[base + blockIdx.x] = b.row;
    }
    if (!lupp_grid_sync(bar, iscal + 2)) return;
    Cand t{-1, INT_MAX, -1, -1};
    for (int q = threadIdx.x; q < (int)gridDim.x; q += blockDim.x)
      t = cand_merge(t, Cand{__ldcg(pv + base + q), __ldcg(pp + base + q),
                             __ldcg(ps + base + q), __ldcg(pr + base + q)});
    t = block_cand(t);
    if (threadIdx.x == 0) { s_v = t.v; s_pos = t.pos; s_sec = t.sec; s_row = t.row; }
    __syncthreads();
    const long long tv_bits = s_v, ts_bits = s_sec;
    const int tpos = s_pos, trow = s_row;
    if (!(tv_bits > 0)) {  // zero pivot (or no candidates): rank exhausted
      if (blockIdx.x == 0 && threadIdx.x == 0) iscal[1] = 1;
      break;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      piv[j] = trow;
      iscal[0] = j + 1;
      if (ts_bits >= 0) {
        const double tv = __longlong_as_double(tv_bits), ts = __longlong_as_double(ts_bits);
        *margin = fmin(*margin, (tv - ts) / tv);
      }
    }
    p = trow;
    ppos = tpos;
  }
}

// ---- gathers --------------------------------------------------------------------------

template <typename T>
__global__ void gather_cols_dense_kernel(int64_t m, int64_t ld, const T* __restrict__ A,
                                         const int* __restrict__ idx, int k, double* out,
                                         int64_t ldo) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m * k) return;
  const int64_t q = e / m, i = e % m;
  out[i + q * ldo] = (double)A[i * ld + idx[q]];
}

template <typename T>
__global__ void gather_cols_csr_kernel(int64_t m, const int* __restrict__ rowptr,
                                       const int* __restrict__ colidx, const T* __restrict__ v,
                                       const int* __restrict__ colmap, int k, double* out,
                                       int64_t ldo) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  for (int q = 0; q < k; ++q) out[i + q * ldo] = 0.0;
  for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
    const int q = colmap[colidx[e]];
    if (q >= 0 && q < k) out[i + q * ldo] = (double)v[e];
  }
}

template <typename T>
__global__ void gather_rows_T_dense_kernel(int64_t n, int64_t ld, const T* __restrict__ A,
                                           const int* __restrict__ idx, int k, double* out,
                                           int64_t ldo) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * k) return;
  const int64_t q = e / n, j = e % n;
  out[j + q * ldo] = (double)A[(int64_t)idx[q] * ld + j];
}

template <typename T>
__global__ void gather_rows_T_csr_kernel(int64_t n, const int* __restrict__ rowptr,
                                         const int* __restrict__ colidx, const T* __restrict__ v,
                                         const int* __restrict__ idx, double* out, int64_t ldo) {
  const int q = blockIdx.x;
  const int64_t i = idx[q];
  for (int e = rowptr[i] + threadIdx.x; e < rowptr[i + 1]; e += blockDim.x)
    out[(int64_t)colidx[e] + q * ldo] = (double)v[e];
}

template <typename T>
__global__ void append_rows_kernel(int64_t n, int64_t ld, const T* __restrict__ A,
                                   const int* __restrict__ idx, int k, double* R, int64_t ldr,
                                   int64_t r0) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * k) return;
  const int64_t q = e / n, j = e % n;
  R[(r0 + q) + j * ldr] = (double)A[(int64_t)idx[q] * ld + j];
}

template <typename T>
__global__ void cross_dense_kernel(int64_t ld, const T* __restrict__ A, const int* rI, int nI,
                                   const int* cJ, int nJ, double* out, int64_t ldo) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)nI * nJ) return;
  const int64_t a = e % nI, c = e / nI;
  out[a + c * ldo] = (double)A[(int64_t)rI[a] * ld + cJ[c]];
}

template <typename T>
__global__ void cross_csr_kernel(const int* __restrict__ rowptr, const int* __restrict__ colidx,
                                 const T* __restrict__ v, const int* rI, int nI,
                                 const int* __restrict__ colmap, int nJ, double* out,
                                 int64_t ldo) {
  const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= nI) return;
  for (int c = 0; c < nJ; ++c) out[a + c * ldo] = 0.0;
  const int64_t i = rI[a];
  for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
    const int c = colmap[colidx[e]];
    if (c >= 0 && c < nJ) out[a + c * ldo] = (double)v[e];
  }
}

__global__ void gather_rows_cm_kernel(const double* B, int64_t ldb, int64_t ncols,
                                      const int* idx, int k, double* out, int64_t ldo) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ncols * k) return;
  const int64_t a = e % k, c = e / k;
  out[a + c * ldo] = B[(int64_t)idx[a] + c * ldb];
}

// ---- residuals for CSR ----------------------------------------------------------------

template <typename T>
__global__ void ecol_csr_kernel(int64_t m, const int* __restrict__ rowptr,
                                const int* __restrict__ colidx, const T* __restrict__ v,
                                const int* __restrict__ colpos,
                                const int* __restrict__ colpos_plus,
                                const int* __restrict__ rowpos, const double* __restrict__ X,
                                int64_t ldx, int kb, double* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  for (int k = 0; k < kb; ++k) out[i + k * m] = 0.0;
  if (rowpos[i] >= 0) return;
  for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
    const int c = colidx[e];
    const double a = (double)v[e];
    const int jp = colpos_plus[c];
    if (jp >= 0) out[i + jp * m] += a;
    const int q = colpos[c];
    if (q >= 0) {
      for (int k = 0; k < kb; ++k) out[i + k * m] -= a * X[q + k * ldx];
    }
  }
}

template <typename T>
__global__ void erow_csr_kernel(int64_t n, const int* __restrict__ colptr,
                                const int* __restrict__ rowidx, const T* __restrict__ cv,
                                const int* __restrict__ rowpos, const double* __restrict__ Z,
                                int s, const double* __restrict__ Y, double* __restrict__ E) {
  const int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (j >= n) return;
  for (int r = lane; r < s; r += 32) {
    double e = Y[r + j * s];
    for (int p = colptr[j]; p < colptr[j + 1]; ++p) {
      const int q = rowpos[rowidx[p]];
      if (q >= 0) e -= (double)cv[p] * Z[r + (int64_t)q * s];
    }
    E[r + j * s] = e;
  }
}

template <typename T>
__global__ void gram_csr_kernel(int64_t m, const int* __restrict__ colptr,
                                const int* __restrict__ rowidx, const T* __restrict__ cv,
                                const int* __restrict__ Jall, int nq, const double* __restrict__ Cp,
                                int kb, double* __restrict__ G, int64_t ldg) {
  const int q = blockIdx.x;
  if (q >= nq) return;
  const int64_t col = Jall[q];
  for (int k = threadIdx.x; k < kb; k += blockDim.x) {
    double acc = 0.0;
    for (int p = colptr[col]; p < colptr[col + 1]; ++p)
      acc += (double)cv[p] * Cp[(int64_t)rowidx[p] + (int64_t)k * m];
    G[q + k * ldg] = acc;
  }
}

// ---- small helpers --------------------------------------------------------------------

__global__ void zero_cols_kernel(double* E, int64_t ldE, int64_t rows, const int* cols, int k) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= rows * k) return;
  E[e % rows + (int64_t)cols[e / rows] * ldE] = 0.0;
}
__global__ void zero_rows_kernel(double* E, int64_t ldE, int64_t ncols, const int* rows, int k) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ncols * k) return;
  E[(int64_t)rows[e % k] + (e / k) * ldE] = 0.0;
}
__global__ void colnorm_max_kernel(const double* T, int s, int r, double factor, double* out) {
  __shared__ double sh[32];
  double best = 0.0;
  for (int q = 0; q < r; ++q) {
    double v = 0.0;
    for (int i = threadIdx.x; i < s; i += blockDim.x) v = fma(T[i + q * s], T[i + q * s], v);
    v = block_sum(v, sh);
    if (threadIdx.x == 0) best = fmax(best, sqrt(v));
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = factor * best;
}
__global__ void set_map_kernel(int* map, const int* idx, int k, int base) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < k) map[idx[q]] = base + q;
}
__global__ void fill_int_kernel(int* p, int64_t n, int v) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

}  // namespace

// ------------------------------------------------------------------------------------

void sketch(cudaStream_t st, const MatView& A, int s, int xi, const int* tptr, const int* ti,
            const signed char* tsgn, const int* srows, const signed char* ssign, double scale,
            double* Y) {
  // sketch rows vary fastest across blocks: the blocks resident together cover every
  // sketch row of a few 128-column strips of A, so a strip is read from HBM about once and
  // its other reads (one per nonzero of the sketch column) hit L2
  APL_REQUIRE(cdiv(A.n, 128) <= 65535, "sketch: n too large");
  dim3 grid((unsigned)s, (unsigned)cdiv(A.n, 128));
  if (A.fmt == 0) {
    if (A.dtype == 0)
      sketch_dense_kernel<double><<<grid, 128, 0, st>>>(A.n, A.ld, (const double*)A.vals, s, tptr,
                                                        ti, tsgn, scale, Y);
    else
      sketch_dense_kernel<float><<<grid, 128, 0, st>>>(A.n, A.ld, (const float*)A.vals, s, tptr,
                                                       ti, tsgn, scale, Y);
  } else {
    if (A.dtype == 0)
      sketch_csc_kernel<double><<<grid, 128, 0, st>>>(A.n, A.colptr, A.rowidx,
                                                      (const double*)A.cvals, s, xi, srows,
                                                      ssign, scale, Y);
    else
      sketch_csc_kernel<float><<<grid, 128, 0, st>>>(A.n, A.colptr, A.rowidx,
                                                     (const float*)A.cvals, s, xi, srows, ssign,
                                                     scale, Y);
  }
  APL_LAUNCH_CHECK();
}

int lupp_select(cudaStream_t st, int64_t N, int64_t K, double* X, int64_t rs, int64_t cs, int k,
                LuppWork& w, std::vector<int>& piv_host, double* margin) {
  piv_host.clear();
  *margin = INFINITY;
  if (k <= 0 || N <= 0) return 0;
  const int threads = 256;
  const int64_t blocks64 = cdiv(N, 32);
  APL_REQUIRE(blocks64 < (1LL << 31), "lupp_select: too many rows");
  const int blocks = (int)blocks64;
  w.pos_of.alloc(N, st);
  w.row_at.alloc(N, st);
  w.piv.alloc(k, st);
  w.pval.alloc(blocks, st);
  w.psec.alloc(blocks, st);
  w.ppos.alloc(blocks, st);
  w.counter.alloc(2, st);
  w.scal.alloc(1, st);
  w.iscal.alloc(3, st);
  lupp_init_kernel<<<(unsigned)cdiv(N, 256), 256, 0, st>>>(N, w.pos_of.p, w.row_at.p, w.scal.p,
                                                          w.iscal.p, w.counter.p);
  APL_LAUNCH_CHECK();
  const size_t shm = (size_t)(K + 1) * sizeof(double);
  // one cooperative launch when the device offers it and the caller runs no concurrent
  // selections; one launch per step otherwise
  int coop_grid = 0, tpb = 0;
  size_t coop_shm = 0;
  if (w.cooperative) {
    int dev = 0, coop = 0, nsm = 0, per_sm = 0;
    APL_CUDA(cudaGetDevice(&dev));
    APL_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
    APL_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    // shared memory for the most tiles a block can own (one block per SM)
    const int64_t tpb_max = cdiv(blocks64, (int64_t)nsm);
    coop_shm = shm + (size_t)tpb_max * 32 * (2 * sizeof(double) + sizeof(int));
    if (coop && coop_shm <= 200 * 1024) {
      APL_CUDA(cudaFuncSetAttribute(lupp_coop_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    200 * 1024));
      APL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lupp_coop_kernel, threads,
                                                             coop_shm));
    }
    if (per_sm > 0) {
      // as few blocks as give the same number of tiles to the busiest block
      const int64_t per_block = cdiv(blocks64, (int64_t)per_sm * nsm);
      coop_grid = (int)cdiv(blocks64, per_block);
      tpb = (int)cdiv(blocks64, (int64_t)coop_grid);
    }
  }
  const int tok = prof_begin(st);
  if (coop_grid > 0) {
    w.cv.alloc(2 * (size_t)coop_grid, st);
    w.cs.alloc(2 * (size_t)coop_grid, st);
    w.cp.alloc(2 * (size_t)coop_grid, st);
    w.cr.alloc(2 * (size_t)coop_grid, st);
    int* piv = w.piv.p;
    long long* pv = w.cv.p;
    int* pp = w.cp.p;
    long long* ps = w.cs.p;
    int* pr = w.cr.p;
    unsigned* bar = w.counter.p;
    double* mg = w.scal.p;
    int* isc = w.iscal.p;
    void* args[] = {(void*)&N, (void*)&K, (void*)&X, (void*)&rs, (void*)&cs, (void*)&k,
                    (void*)&tpb, (void*)&piv, (void*)&pv, (void*)&pp, (void*)&ps,
                    (void*)&pr, (void*)&bar, (void*)&mg, (void*)&isc};
    APL_CUDA(cudaLaunchCooperativeKernel((const void*)lupp_coop_kernel, dim3(coop_grid),
                                         dim3(threads), args, coop_shm, st));
    APL_LAUNCH_CHECK();
  } else {
    for (int j = 0; j < k; ++j) {
      lupp_step_kernel<<<blocks, threads, shm, st>>>(N, K, X, rs, cs, j, w.pos_of.p, w.row_at.p,
                                                     w.piv.p, w.pval.p, w.ppos.p, w.psec.p,
                                                     w.counter.p, w.scal.p, w.iscal.p);
      APL_LAUNCH_CHECK();
    }
  }
  {
    // algorithmic bytes: step j reads and writes the N x (K - j) trailing block
    double bytes = 0.0;
    for (int j = 0; j < k; ++j) bytes += 16.0 * (double)N * (double)(K - j);
    prof_end(st, tok, PROF_LUPP, bytes);
  }
  int isc[3];
  APL_CUDA(cudaMemcpyAsync(isc, w.iscal.p, 3 * sizeof(int), cudaMemcpyDeviceToHost, st));
  APL_CUDA(cudaMemcpyAsync(margin, w.scal.p, sizeof(double), cudaMemcpyDeviceToHost, st));
  APL_CUDA(cudaStreamSynchronize(st));
  if (isc[2]) throw Error(ST_ETIMEOUT, "LUPP: a grid barrier wait ran past its bound");
  const int nz = isc[0];
  piv_host.resize(nz);
  if (nz)
    APL_CUDA(cudaMemcpyAsync(piv_host.data(), w.piv.p, nz * sizeof(int), cudaMemcpyDeviceToHost,
                             st));
  APL_CUDA(cudaStreamSynchronize(st));
  return nz;
}

void gather_cols(cudaStream_t st, const MatView& A, const int* idx, int k, const int* colmap,
                 double* out, int64_t ldo) {
  if (k <= 0) return;
  if (A.fmt == 0) {
    const unsigned g = (unsigned)cdiv(A.m * k, 256);
    if (A.dtype == 0)
      gather_cols_dense_kernel<double><<<g, 256, 0, st>>>(A.m, A.ld, (const double*)A.vals, idx,
                                                          k, out, ldo);
    else
      gather_cols_dense_kernel<float><<<g, 256, 0, st>>>(A.m, A.ld, (const float*)A.vals, idx, k,
                                                         out, ldo);
  } else {
    const unsigned g = (unsigned)cdiv(A.m, 256);
    if (A.dtype == 0)
      gather_cols_csr_kernel<double><<<g, 256, 0, st>>>(A.m, A.rowptr, A.colidx,
                                                        (const double*)A.vals, colmap, k, out,
                                                        ldo);
    else
      gather_cols_csr_kernel<float><<<g, 256, 0, st>>>(A.m, A.rowptr, A.colidx,
                                                       (const float*)A.vals, colmap, k, out, ldo);
  }
  APL_LAUNCH_CHECK();
}

void gather_rows_T(cudaStream_t st, const MatView& A, const int* idx, int k, double* out,
                   int64_t ldo) {
  if (k <= 0) return;
  if (A.fmt == 0) {
    const unsigned g = (unsigned)cdiv(A.n * k, 256);
    if (A.dtype == 0)
      gather_rows_T_dense_kernel<double><<<g, 256, 0, st>>>(A.n, A.ld, (const double*)A.vals, idx,
                                                            k, out, ldo);
    else
      gather_rows_T_dense_kernel<float><<<g, 256, 0, st>>>(A.n, A.ld, (const float*)A.vals, idx,
                                                           k, out, ldo);
  } else {
    for (int q = 0; q < k; ++q)
      APL_CUDA(cudaMemsetAsync(out + q * ldo, 0, A.n * sizeof(double), st));
    if (A.dtype == 0)
      gather_rows_T_csr_kernel<double><<<k, 128, 0, st>>>(A.n, A.rowptr, A.colidx,
                                                          (const double*)A.vals, idx, out, ldo);
    else
      gather_rows_T_csr_kernel<float><<<k, 128, 0, st>>>(A.n, A.rowptr, A.colidx,
                                                         (const float*)A.vals, idx, out, ldo);
  }
  APL_LAUNCH_CHECK();
}

void append_rows(cudaStream_t st, const MatView& A, const int* idx, int k, double* R, int64_t ldr,
                 int64_t r0) {
  if (k <= 0) return;
  const unsigned g = (unsigned)cdiv(A.n * k, 256);
  if (A.dtype == 0)
    append_rows_kernel<double><<<g, 256, 0, st>>>(A.n, A.ld, (const double*)A.vals, idx, k, R,
                                                  ldr, r0);
  else
    append_rows_kernel<float><<<g, 256, 0, st>>>(A.n, A.ld, (const float*)A.vals, idx, k, R, ldr,
                                                 r0);
  APL_LAUNCH_CHECK();
}

void gather_cross(cudaStream_t st, const MatView& A, const int* rI, int nI, const int* cJ, int nJ,
                  const int* colmap, double* out, int64_t ldo) {
  if (nI <= 0 || nJ <= 0) return;
  if (A.fmt == 0) {
    const unsigned g = (unsigned)cdiv((int64_t)nI * nJ, 256);
    if (A.dtype == 0)
      cross_dense_kernel<double><<<g, 256, 0, st>>>(A.ld, (const double*)A.vals, rI, nI, cJ, nJ,
                                                    out, ldo);
    else
      cross_dense_kernel<float><<<g, 256, 0, st>>>(A.ld, (const float*)A.vals, rI, nI, cJ, nJ, out,
                                                   ldo);
  } else {
    const unsigned g = (unsigned)cdiv(nI, 128);
    if (A.dtype == 0)
      cross_csr_kernel<double><<<g, 128, 0, st>>>(A.rowptr, A.colidx, (const double*)A.vals, rI,
                                                  nI, colmap, nJ, out, ldo);
    else
      cross_csr_kernel<float><<<g, 128, 0, st>>>(A.rowptr, A.colidx, (const float*)A.vals, rI, nI,
                                                 colmap, nJ, out, ldo);
  }
  APL_LAUNCH_CHECK();
}

void gather_rows_cm(cudaStream_t st, const double* B, int64_t ldb, int64_t ncols, const int* idx,
                    int k, double* out, int64_t ldo) {
  if (k <= 0 || ncols <= 0) return;
  gather_rows_cm_kernel<<<(unsigned)cdiv(ncols * k, 256), 256, 0, st>>>(B, ldb, ncols, idx, k,
                                                                        out, ldo);
  APL_LAUNCH_CHECK();
}

void ecol_csr(cudaStream_t st, const MatView& A, const int* colpos, const int* colpos_plus,
              const int* rowpos, const double* X, int64_t ldx, int kb, double* out) {
  const unsigned g = (unsigned)cdiv(A.m, 128);
  if (A.dtype == 0)
    ecol_csr_kernel<double><<<g, 128, 0, st>>>(A.m, A.rowptr, A.colidx, (const double*)A.vals,
                                               colpos, colpos_plus, rowpos, X, ldx, kb, out);
  else
    ecol_csr_kernel<float><<<g, 128, 0, st>>>(A.m, A.rowptr, A.colidx, (const float*)A.vals,
                                              colpos, colpos_plus, rowpos, X, ldx, kb, out);
  APL_LAUNCH_CHECK();
}

void erow_csr(cudaStream_t st, const MatView& A, const int* rowpos, const double* Z, int s,
              const double* Y, double* E) {
  const unsigned g = (unsigned)cdiv(A.n * 32, 256);
  if (A.dtype == 0)
    erow_csr_kernel<double><<<g, 256, 0, st>>>(A.n, A.colptr, A.rowidx, (const double*)A.cvals,
                                               rowpos, Z, s, Y, E);
  else
    erow_csr_kernel<float><<<g, 256, 0, st>>>(A.n, A.colptr, A.rowidx, (const float*)A.cvals,
                                              rowpos, Z, s, Y, E);
  APL_LAUNCH_CHECK();
}

void gram_csr(cudaStream_t st, const MatView& A, const int* Jall, int nq, const double* Cp, int kb,
              double* G, int64_t ldg) {
  if (nq <= 0 || kb <= 0) return;
  if (A.dtype == 0)
    gram_csr_kernel<double><<<nq, 128, 0, st>>>(A.m, A.colptr, A.rowidx, (const double*)A.cvals,
                                                Jall, nq, Cp, kb, G, ldg);
  else
    gram_csr_kernel<float><<<nq, 128, 0, st>>>(A.m, A.colptr, A.rowidx, (const float*)A.cvals,
                                               Jall, nq, Cp, kb, G, ldg);
  APL_LAUNCH_CHECK();
}

void zero_cols_cm(cudaStream_t st, double* E, int64_t ldE, int64_t rows, const int* cols, int k) {
  if (k <= 0 || rows <= 0) return;
  zero_cols_kernel<<<(unsigned)cdiv(rows * k, 256), 256, 0, st>>>(E, ldE, rows, cols, k);
  APL_LAUNCH_CHECK();
}
void zero_rows_cm(cudaStream_t st, double* E, int64_t ldE, int64_t ncols, const int* rows, int k) {
  if (k <= 0 || ncols <= 0) return;
  zero_rows_kernel<<<(unsigned)cdiv(ncols * k, 256), 256, 0, st>>>(E, ldE, ncols, rows, k);
  APL_LAUNCH_CHECK();
}
void colnorm_max(cudaStream_t st, const double* T, int s, int r, double factor, double* out) {
  colnorm_max_kernel<<<1, 256, 0, st>>>(T, s, r, factor, out);
  APL_LAUNCH_CHECK();
}
void set_map(cudaStream_t st, int* map, const int* idx, int k, int base) {
  if (k <= 0) return;
  set_map_kernel<<<(unsigned)cdiv(k, 256), 256, 0, st>>>(map, idx, k, base);
  APL_LAUNCH_CHECK();
}
void fill_int(cudaStream_t st, int* p, int64_t n, int v) {
  if (n <= 0) return;
  fill_int_kernel<<<(unsigned)cdiv(n, 256), 256, 0, st>>>(p, n, v);
  APL_LAUNCH_CHECK();
}

}  // namespace apl

// ---- dense sketching operators (Gaussian, SRHT) with FP64-level products -------------

namespace apl {
namespace {

template <typename T>
__global__ void widen_rows_kernel(int64_t rows, int64_t n, int64_t ld, const T* __restrict__ A,
                                  double* __restrict__ out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= rows * n) return;
  const int64_t i = e / n, j = e - i * n;
  out[e] = (double)A[i * ld + j];
}

// Y(:, j) = sum over the nonzeros a_ij of column j, in ascending i, of a_ij S(:, i); one
// warp per column, lanes over the sketch rows.
template <typename T>
__global__ void opsketch_csc_kernel(int s, int64_t n, const int* __restrict__ colptr,
                                    const int* __restrict__ rowidx, const T* __restrict__ cvals,
                                    const double* __restrict__ S, double* __restrict__ Y) {
  const int lane = threadIdx.x & 31;
  const int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (j >= n) return;
  const int e0 = colptr[j], e1 = colptr[j + 1];
  for (int r0 = 0; r0 < s; r0 += 32) {
    const int r = r0 + lane;
    double acc = 0.0;
    if (r < s)
      for (int e = e0; e < e1; ++e) acc = fma((double)cvals[e], S[r + (int64_t)s * rowidx[e]], acc);
    if (r < s) Y[r + (int64_t)s * j] = acc;
  }
}

}  // namespace

void operator_sketch(cudaStream_t st, const MatView& A, int s, const double* S, double* Y,
                     DBuf<double>& chunk) {
  if (A.fmt == 1) {
    const unsigned blocks = (unsigned)cdiv(A.n * 32, 256);
    if (A.dtype == 0)
      opsketch_csc_kernel<double><<<blocks, 256, 0, st>>>(s, A.n, A.colptr, A.rowidx,
                                                          (const double*)A.cvals, S, Y);
    else
      opsketch_csc_kernel<float><<<blocks, 256, 0, st>>>(s, A.n, A.colptr, A.rowidx,
                                                         (const float*)A.cvals, S, Y);
    APL_LAUNCH_CHECK();
    return;
  }
  // dense: Y = sum over row chunks of S(:, chunk) A(chunk, :), the chunk viewed column-major
  // as its n x rows transpose
  const int64_t rows = std::max<int64_t>(1, std::min<int64_t>(A.m, (int64_t)(1 << 25) / A.n));
  for (int64_t i0 = 0; i0 < A.m; i0 += rows) {
    const int64_t mc = std::min(rows, A.m - i0);
    const double* blk;
    int64_t ldb;
    if (A.dtype == 0) {
      blk = (const double*)A.vals + i0 * A.ld;
      ldb = A.ld;
    } else {
      chunk.alloc((size_t)rows * A.n, st);
      widen_rows_kernel<float><<<(unsigned)cdiv(mc * A.n, 256), 256, 0, st>>>(
          mc, A.n, A.ld, (const float*)A.vals + i0 * A.ld, chunk.p);
      APL_LAUNCH_CHECK();
      blk = chunk.p;
      ldb = A.n;
    }
    dgemm(st, 0, 1, s, A.n, mc, 1.0, S + (int64_t)s * i0, s, blk, ldb, i0 == 0 ? 0.0 : 1.0, Y, s);
  }
}

}  // namespace apl
