// Fused dense A pass of one LSQR iteration: u' = ca A z + cu u and the column partial
// sums of A^T u' from one read of A (FP32, row-major).
//
// Layout.  A persistent grid of thread-block clusters; a cluster of C CTAs owns a
// contiguous range of rows of A, and CTA c of the cluster owns the column panel
// [c W, c W + W).  A producer warp streams row segments of its panel into a ring of S
// shared-memory stages with bulk (TMA) copies completing on mbarriers.  Per tile of R
// rows, the compute warps form the partial dot products of the rows with z over the
// panel; a sender warp adds them and stores them into every CTA of the cluster with
// st.async (distributed shared memory, completing transaction bytes on the receiver's
// mbarrier); one step later a u' warp adds the C partials in rank order (every CTA gets
// the same u'_i), and one step after that the compute warps accumulate A(i, panel)^T u'_i
// from the tile still in shared memory.  Each CTA ends with the column partials of its
// panel over its cluster's rows; the column-sum kernel adds them in cluster order.  Every
// wait is bounded in time; a wait that gives up sets the error flag and the kernel
// finishes its protocol without data (no barrier is skipped, no copy is left in flight
// at exit).
#include <cuda_runtime.h>

#include <algorithm>

#include "apass.cuh"
#include "df32.cuh"

namespace apl {

namespace {

// Compute warps per CTA: compensated products issue about eleven FP32 instructions per
// product, so that mode takes more warps to hide the latency of its dependent chains.
__host__ __device__ constexpr int ncw_for(int mode) { return mode == 2 ? 12 : 8; }
// threads of a CTA: compute warps, then a sender, a u' and a producer warp
__host__ __device__ constexpr int nthr_for(int mode) { return ncw_for(mode) * 32 + 96; }
constexpr int RMAX = 8;            // rows per stage
constexpr int SMAX = 8;            // stages
constexpr int CMAX = 8;            // CTAs per cluster
constexpr int LAG = 1;             // steps between sending a tile's partials and using them
constexpr int XSLOTS = 2 * LAG + 2;  // exchange slots: a slot is rewritten only after its
                                     // receiver has read it (needs XSLOTS >= 2 LAG + 2)
constexpr int KQMAX = 6;           // float4 columns per consumer thread (7, 8 spill)
constexpr size_t kSmemBytes = 220 * 1024;  // dynamic shared memory of a CTA at most
// Rows per stage that the register arrays of an instance hold: wide panels (large KQ)
// take few rows per 40 KB stage anyway, and the row accumulators must not spill.
__host__ __device__ constexpr int rows_cap(int kq) {
  return kq <= 1 ? 8 : kq == 2 ? 5 : kq == 3 ? 4 : kq == 4 ? 3 : 2;
}
// Bound of one wait in SM clock cycles (about 2 s at the 2.07 GHz maximum clock; the
// cycle counter is read at full rate, unlike the global timer).
constexpr long long kWaitCycles = 4000000000ll;

__device__ __forceinline__ uint32_t saddr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ unsigned cta_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned cluster_index() {
  unsigned r;
  asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n"
               "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ void mb_init(uint64_t* b, unsigned cnt) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(b)), "r"(cnt) : "memory");
}
__device__ __forceinline__ void mb_arrive_expect(uint64_t* b, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(b)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mb_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(b)) : "memory");
}
__device__ __forceinline__ bool mb_try(uint64_t* b, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(saddr(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// acquire at cluster scope: the data of the phase was written by other CTAs
__device__ __forceinline__ bool mb_try_cluster(uint64_t* b, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(saddr(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// shared::cluster address of the variable at local address p in CTA `rank`
__device__ __forceinline__ uint32_t map_rank(const void* p, unsigned rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr(p)), "r"(rank));
  return r;
}
__device__ __forceinline__ void st_remote_f2(uint32_t addr, float a, float b) {
  asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(addr), "f"(a), "f"(b)
               : "memory");
}
// Asynchronous store of two floats into another CTA's shared memory that completes
// 8 transaction bytes on that CTA's mbarrier (no fence on the sending side).
__device__ __forceinline__ void st_async_f2(uint32_t addr, float a, float b, uint32_t mbar) {
  asm volatile(
      "st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f32 [%0], {%1, %2}, [%3];" ::
          "r"(addr),
      "f"(a), "f"(b), "r"(mbar)
      : "memory");
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes,
                                          uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(saddr(dst)),
      "l"(src), "r"(bytes), "r"(saddr(bar))
      : "memory");
}
// the per-step barrier of the compute, sender and u' warps
template <int NSYNC>
__device__ __forceinline__ void step_sync() {
  asm volatile("bar.sync 1, %0;" ::"n"(NSYNC) : "memory");
}

// Waits for the phase of the given parity.  Returns early (false) once `abort` is set;
// sets it (and the global error flag) when the wait runs past its bound.
template <bool CLUSTER>
__device__ bool wait_phase(uint64_t* b, unsigned parity, volatile int* abort, int* err) {
  if (CLUSTER ? mb_try_cluster(b, parity) : mb_try(b, parity)) return true;
  const long long t0 = clock64();
  while (true) {
    if (CLUSTER ? mb_try_cluster(b, parity) : mb_try(b, parity)) return true;
    if (*abort) return false;
    if (clock64() - t0 > kWaitCycles) {
      *abort = 1;
      atomicExch(err, 1);
      return false;
    }
  }
}
// Bounded wait that ignores `abort` (copies in flight must land before the CTA exits).
__device__ void wait_drain(uint64_t* b, unsigned parity, int* err) {
  const long long t0 = clock64();
  while (!mb_try(b, parity)) {
    if (clock64() - t0 > kWaitCycles) {
      atomicExch(err, 1);
      return;
    }
  }
}

__device__ __forceinline__ DF df_add(DF a, DF b) {
  float s, e;
  df_two_sum(a.s, b.s, s, e);
  return DF{s, __fadd_rn(__fadd_rn(a.c, b.c), e)};
}
__device__ __forceinline__ DF warp_sum_df(DF v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    DF w;
    w.s = __shfl_down_sync(0xffffffffu, v.s, o);
    w.c = __shfl_down_sync(0xffffffffu, v.c, o);
    v = df_add(v, w);
  }
  return v;
}

// Accumulators: mode 1 FP32 products and sums, mode 2 compensated FP32.
template <int MODE>
struct FAcc;
template <>
struct FAcc<1> {
  float v = 0.f;
  __device__ __forceinline__ void add(float a, float h, float) { v = fmaf(a, h, v); }
  __device__ __forceinline__ DF df() const { return DF{v, 0.f}; }
};
template <>
struct FAcc<2> {
  DF v{0.f, 0.f};
  __device__ __forceinline__ void add(float a, float h, float l) { df_fma(v, a, h, l); }
  __device__ __forceinline__ DF df() const { return v; }
};

// Warp roles: eight compute warps (dot products of tile t, then the column partials of
// tile t - LAG - 1); a sender warp (sums the compute warps' row partials of tile t and
// stores them into every CTA of the cluster with st.async, which completes transaction
// bytes on the receiver's mbarrier); a u' warp (forms u' of tile t - LAG from the C
// partials it received and re-arms that exchange slot); a producer warp (bulk copies).
// Compute, sender and u' warps meet once per step at a named barrier; the sender's and
// the u' warp's serial work of a step overlaps the compute warps' column partials and
// next dot products.
template <int MODE, int KQ>
__global__ void __launch_bounds__(nthr_for(MODE), 1)
    fused_apass_kernel(int64_t m, int64_t n, int64_t ld, const float* __restrict__ A, int W,
                       int R, int S, int C, int64_t rpc, int ucap,
                       const double* __restrict__ z,
                       const float* __restrict__ zh, const float* __restrict__ zl,
                       double* __restrict__ u, LsqrCtl* ctl, double* __restrict__ red,
                       double* __restrict__ part, int* err) {
  constexpr int NCW = ncw_for(MODE), NCT = NCW * 32, NTHR = nthr_for(MODE);
  constexpr int SWARP = NCW, UWARP = NCW + 1, PWARP = NCW + 2, NSYNC = NCT + 64;
  extern __shared__ __align__(128) unsigned char fsm[];
  float* tiles = reinterpret_cast<float*>(fsm);  // S x R rows of W floats
  // u of the cluster's rows before the update (read once at the start: every CTA of the
  // cluster has its copy before rank 0 writes u' of any of these rows)
  double* uall = reinterpret_cast<double*>(fsm + (size_t)S * R * W * sizeof(float));
  // per-thread row partials of the dot products, two slots: [slot][row][thread]
  float2* wpart = reinterpret_cast<float2*>(uall + ucap);
  __shared__ __align__(8) uint64_t full[SMAX], empty[SMAX], xbar[XSLOTS];
  __shared__ __align__(8) float2 xch[XSLOTS][CMAX][RMAX];  // [slot][sender rank][row]
  __shared__ float2 ush[2][RMAX];                           // u'_i split into hi + lo
  __shared__ double shr[nthr_for(2) / 32];
  __shared__ int abort_flag;
  if (ctl->done) return;  // the same decision in every CTA of the grid
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const unsigned rank = cta_rank();
  const int64_t cl = cluster_index();
  const int64_t r0 = cl * rpc, r1 = r0 + rpc < m ? r0 + rpc : m;
  const int64_t nrows = r1 > r0 ? r1 - r0 : 0;
  const int T = (int)((nrows + R - 1) / R);
  const int64_t c0 = (int64_t)rank * W;
  const int Wc = (int)(n - c0 < W ? n - c0 : W);  // > 0 by the plan
  const int Wc4 = Wc >> 2;
  const double ca = ctl->zs, cu = -ctl->alpha * ctl->us, delta = ctl->delta;
  auto tile_rows = [&](int t) {
    const int64_t left = r1 - (r0 + (int64_t)t * R);
    return (int)(left < R ? left : R);
  };
  if (tid == 0) {
    abort_flag = 0;
    for (int s = 0; s < S; ++s) {
      mb_init(&full[s], 1);
      mb_init(&empty[s], NCW);
    }
    for (int k = 0; k < XSLOTS; ++k) mb_init(&xbar[k], 1u);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    // arm the first exchange slots: one arrival of this CTA and the bytes of C senders
    for (int k = 0; k < XSLOTS && k < T; ++k)
      mb_arrive_expect(&xbar[k], (unsigned)(tile_rows(k) * C) * (unsigned)sizeof(float2));
  }
  __syncthreads();
  cluster_sync();  // every barrier of the cluster exists before the first remote arrive
  for (int64_t i = tid; i < nrows; i += NTHR) uall[i] = u[r0 + i];
  __syncthreads();
  cluster_sync();  // every CTA of the cluster holds u before rank 0 may overwrite it
  double ss = 0.0;
  // rows of delta I: u'_bot = ca delta z + cu u_bot, spread over the whole grid
  for (int64_t j = (int64_t)blockIdx.x * NTHR + tid; j < n; j += (int64_t)gridDim.x * NTHR) {
    const double v = ca * delta * z[j] + cu * u[m + j];
    u[m + j] = v;
    ss += v * v;
  }
  const int NSTEP = T + LAG + 1;
  if (warp == PWARP) {
    // producer: one lane streams the panel rows of every tile into the stage ring
    if (lane == 0) {
      int issued = 0;
      for (int t = 0; t < T; ++t) {
        const int s = t % S;
        if (t >= S) wait_phase<false>(&empty[s], (unsigned)((t / S) - 1) & 1u, &abort_flag, err);
        if (abort_flag) break;
        const int64_t row0 = r0 + (int64_t)t * R;
        const int nr = tile_rows(t);
        mb_arrive_expect(&full[s], (unsigned)nr * (unsigned)Wc * 4u);
        for (int r = 0; r < nr; ++r)
          bulk_load(tiles + ((size_t)s * R + r) * W, A + (row0 + r) * ld + c0,
                    (unsigned)Wc * 4u, &full[s]);
        issued = t + 1;
      }
      // the last use of every stage: no copy may still target this CTA at exit
      for (int t = issued - S > 0 ? issued - S : 0; t < issued; ++t)
        wait_drain(&full[t % S], (unsigned)(t / S) & 1u, err);
    }
  } else if (warp == SWARP) {
    // sender: row sums of tile t to every CTA of the cluster
    for (int t = 0; t < NSTEP; ++t) {
      step_sync<NSYNC>();
      if (t < T) {
        const int nr = tile_rows(t);
        // row sums over the compute threads' partials, in a fixed order
        float vs[RMAX], vc[RMAX];
#pragma unroll
        for (int r = 0; r < RMAX; ++r) {
          DF a{0.f, 0.f};
          if (r < nr) {
            const float2* wp = wpart + ((size_t)(t & 1) * R + r) * NCT;
            if (MODE == 1) {
              float f = 0.f;
#pragma unroll
              for (int j = 0; j < NCT / 32; ++j) f += wp[lane + 32 * j].x;
#pragma unroll
              for (int o = 16; o > 0; o >>= 1) f += __shfl_down_sync(0xffffffffu, f, o);
              a = DF{f, 0.f};
            } else {
#pragma unroll
              for (int j = 0; j < NCT / 32; ++j) {
                const float2 w = wp[lane + 32 * j];
                a = df_add(a, DF{w.x, w.y});
              }
              a = warp_sum_df(a);
            }
          }
          vs[r] = __shfl_sync(0xffffffffu, a.s, 0);
          vc[r] = __shfl_sync(0xffffffffu, a.c, 0);
        }
        if (lane < C) {
          const int slot = t % XSLOTS;
          const uint32_t bar = map_rank(&xbar[slot], (unsigned)lane);
#pragma unroll
          for (int r = 0; r < RMAX; ++r)
            if (r < nr) st_async_f2(map_rank(&xch[slot][rank][r], (unsigned)lane), vs[r], vc[r], bar);
        }
      }
    }
  } else if (warp == UWARP) {
    // u' of tile t - LAG: add the C exchanged partials in rank order
    for (int t = 0; t < NSTEP; ++t) {
      step_sync<NSYNC>();
      const int tp = t - LAG;
      if (tp >= 0 && tp < T) {
        const int slot = tp % XSLOTS;
        wait_phase<true>(&xbar[slot], (unsigned)(tp / XSLOTS) & 1u, &abort_flag, err);
        const int64_t row0 = r0 + (int64_t)tp * R;
        const int nr = tile_rows(tp);
        if (lane < nr) {
          const float2 p0 = xch[slot][0][lane];
          DF acc{p0.x, p0.y};
          for (int c = 1; c < C; ++c) {
            const float2 pc = xch[slot][c][lane];
            acc = df_add(acc, DF{pc.x, pc.y});
          }
          const double d = (double)acc.s + (double)acc.c;
          const double v = ca * d + cu * uall[row0 - r0 + lane];
          if (rank == 0) {
            u[row0 + lane] = v;
            ss += v * v;
          }
          const float h = __double2float_rn(v);
          ush[tp & 1][lane] = make_float2(h, __double2float_rn(v - (double)h));
        }
        __syncwarp();
        // the slot was read: arm it for tile tp + XSLOTS
        if (lane == 0 && tp + XSLOTS < T)
          mb_arrive_expect(&xbar[slot],
                           (unsigned)(tile_rows(tp + XSLOTS) * C) * (unsigned)sizeof(float2));
      }
    }
  } else {
    float4 zhv[KQ], zlv[KQ];
#pragma unroll
    for (int k = 0; k < KQ; ++k) {
      const int q = tid + NCT * k;
      zhv[k] = make_float4(0.f, 0.f, 0.f, 0.f);
      zlv[k] = zhv[k];
      if (q < Wc4) {
        zhv[k] = reinterpret_cast<const float4*>(zh + c0)[q];
        if (MODE == 2) zlv[k] = reinterpret_cast<const float4*>(zl + c0)[q];
      }
    }
    FAcc<MODE> col[KQ][4];
    constexpr int RC = rows_cap(KQ);
    for (int t = 0; t < NSTEP; ++t) {
      // (a) partial dot products of the rows of tile t with z over this panel (two
      // accumulators per row keep independent chains); the sender adds the partials
      if (t < T) {
        const int s = t % S;
        wait_phase<false>(&full[s], (unsigned)(t / S) & 1u, &abort_flag, err);
        const int nr = tile_rows(t);
        FAcc<MODE> dot[RC][2];
        const float* base = tiles + (size_t)s * R * W;
#pragma unroll
        for (int k = 0; k < KQ; ++k) {
          const int q = tid + NCT * k;
          if (q < Wc4) {
#pragma unroll
            for (int r = 0; r < RC; ++r) {
              if (r < nr) {
                const float4 x = reinterpret_cast<const float4*>(base + (size_t)r * W)[q];
                dot[r][0].add(x.x, zhv[k].x, zlv[k].x);
                dot[r][1].add(x.y, zhv[k].y, zlv[k].y);
                dot[r][0].add(x.z, zhv[k].z, zlv[k].z);
                dot[r][1].add(x.w, zhv[k].w, zlv[k].w);
              }
            }
          }
        }
#pragma unroll
        for (int r = 0; r < RC; ++r) {
          if (r < nr) {
            DF v;
            if (MODE == 1) v = DF{dot[r][0].df().s + dot[r][1].df().s, 0.f};
            else v = df_add(dot[r][0].df(), dot[r][1].df());
            wpart[((size_t)(t & 1) * R + r) * NCT + tid] = make_float2(v.s, v.c);
          }
        }
      }
      step_sync<NSYNC>();
      // (d) column partials with tile t - LAG - 1 (its u' was formed by the reducer in
      // the previous step), then release its stage
      const int tq = t - LAG - 1;
      if (tq >= 0) {
        const int sp = tq % S;
        const int nr = tile_rows(tq);
        const float* base = tiles + (size_t)sp * R * W;
#pragma unroll
        for (int r = 0; r < RC; ++r) {
          if (r < nr) {
            const float2 hl = ush[tq & 1][r];
#pragma unroll
            for (int k = 0; k < KQ; ++k) {
              const int q = tid + NCT * k;
              if (q < Wc4) {
                const float4 x = reinterpret_cast<const float4*>(base + (size_t)r * W)[q];
                col[k][0].add(x.x, hl.x, hl.y);
                col[k][1].add(x.y, hl.x, hl.y);
                col[k][2].add(x.z, hl.x, hl.y);
                col[k][3].add(x.w, hl.x, hl.y);
              }
            }
          }
        }
        __syncwarp();
        if (lane == 0) mb_arrive(&empty[sp]);
      }
    }
    double* out = part + cl * n + c0;
#pragma unroll
    for (int k = 0; k < KQ; ++k) {
      const int q = tid + NCT * k;
      if (q < Wc4) {
#pragma unroll
        for (int e = 0; e < 4; ++e) out[4 * q + e] = df_val(col[k][e].df());
      }
    }
  }
  // ||u'||^2: block partials, the last block of the grid finishes beta
  const double b = block_sum(ss, shr);
  if (tid == 0) red[blockIdx.x] = b;
  const bool last = last_block_done(&ctl->counter[0]);
  if (last) {
    const double tot = block_sum_partials(red, gridDim.x, shr);
    if (tid == 0) finalize_beta(ctl, tot, 0);
  }
  cluster_sync();  // no CTA leaves while a peer may still address its shared memory
}

using KernFn = void (*)(int64_t, int64_t, int64_t, const float*, int, int, int, int, int64_t, int,
                        const double*, const float*, const float*, double*, LsqrCtl*, double*,
                        double*, int*);

template <int MODE>
KernFn kernel_for_mode(int kq) {
  switch (kq) {
    case 1: return fused_apass_kernel<MODE, 1>;
    case 2: return fused_apass_kernel<MODE, 2>;
    case 3: return fused_apass_kernel<MODE, 3>;
    case 4: return fused_apass_kernel<MODE, 4>;
    case 5: return fused_apass_kernel<MODE, 5>;
    default: return fused_apass_kernel<MODE, 6>;
  }
}
KernFn kernel_for(int mode, int kq) {
  return mode == 1 ? kernel_for_mode<1>(kq) : kernel_for_mode<2>(kq);
}

}  // namespace

FusedPlan plan_fused_apass(int64_t m, int64_t n, int64_t ld, const void* vals, int mode) {
  FusedPlan best;
  if (m < 1 || n < 4 || n % 4 != 0 || ld % 4 != 0 ||
      (reinterpret_cast<uintptr_t>(vals) & 15) != 0)
    return best;
  int best_sms = 0;
  const int nct = ncw_for(mode) * 32;
  for (int C = 1; C <= CMAX; C *= 2) {
    const int64_t W = ((n + C - 1) / C + 3) / 4 * 4;
    if ((int64_t)(C - 1) * W >= n) continue;  // every panel holds columns
    const int KQ = (int)((W / 4 + nct - 1) / nct);
    if (KQ > (mode == 2 ? KQMAX - 1 : KQMAX)) continue;  // mode 2 at six spills
    const int64_t rowb = W * 4;
    if (rowb > 48 * 1024) continue;
    const int R = (int)std::max<int64_t>(
        1, std::min<int64_t>(std::min(RMAX, rows_cap(KQ)), 40 * 1024 / rowb));
    const int64_t wpb = 2LL * R * nct * (int64_t)sizeof(float2);
    KernFn fn = kernel_for(mode, KQ);
    // The attribute is the largest size of any plan, so that planning another shape
    // (which shares this kernel instance) never lowers it below a plan already made.
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kSmemBytes) != cudaSuccess) {
      (void)cudaGetLastError();
      continue;
    }
    // rows per cluster: first for one CTA per SM, then for the grid the occupancy query
    // gives with that shared memory (the u copy is sized for it)
    int64_t rpc = (m + std::max(1, 152 / C) - 1) / std::max(1, 152 / C);
    int S = 0, nact = 0;
    int64_t ncl = 0, ucap = 0;
    size_t smem = 0;
    for (int pass = 0; pass < 2; ++pass) {
      ucap = (rpc + 15) / 16 * 16;
      const int64_t fixed = ucap * (int64_t)sizeof(double) + wpb;
      S = (int)std::min<int64_t>(SMAX, ((int64_t)kSmemBytes - fixed) / (R * rowb));
      if (S < LAG + 4) break;  // LAG + 2 stages held by the compute warps, two loading
      smem = (size_t)S * R * rowb + (size_t)fixed;
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3((unsigned)C * 152u);
      cfg.blockDim = dim3(nthr_for(mode));
      cfg.dynamicSmemBytes = smem;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = (unsigned)C;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      nact = 0;
      if (cudaOccupancyMaxActiveClusters(&nact, fn, &cfg) != cudaSuccess || nact <= 0) {
        (void)cudaGetLastError();
        nact = 0;
        break;
      }
      ncl = std::min<int64_t>(nact, (m + R - 1) / R);
      const int64_t need = (m + ncl - 1) / ncl;
      if (need <= ucap) { rpc = need; break; }
      rpc = need;
      nact = 0;  // a second pass sizes the u copy for this grid
    }
    if (nact <= 0 || S < LAG + 4 || rpc > ucap) continue;
    // the smallest cluster that keeps nearly every SM busy: fewer panels give longer
    // row segments per copy and fewer exchanges
    const int sms = nact * C;
    if (sms > best_sms + best_sms / 16) {
      best_sms = sms;
      best.ok = true;
      best.C = C;
      best.W = (int)W;
      best.R = R;
      best.S = S;
      best.KQ = KQ;
      best.smem = smem;
      best.ucap = (int)ucap;
      best.nclusters = (int)ncl;
      best.rows_per_cluster = rpc;
    }
  }
  return best;
}

void launch_fused_apass(cudaStream_t st, const FusedPlan& p, int mode, const MatView& A,
                        const double* z, const float* zh, const float* zl, double* u,
                        LsqrCtl* ctl, double* red, double* part, int* err) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(p.nclusters * p.C));
  cfg.blockDim = dim3(nthr_for(mode));
  cfg.dynamicSmemBytes = p.smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)p.C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  KernFn fn = kernel_for(mode, p.KQ);
  APL_CUDA(cudaLaunchKernelEx(&cfg, fn, A.m, A.n, A.ld, (const float*)A.vals, p.W, p.R, p.S,
                              p.C, p.rows_per_cluster, p.ucap, z, zh, zl, u, ctl, red, part,
                              err));
  note_launch();
}

}  // namespace apl
