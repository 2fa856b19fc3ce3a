// Dense sketch Y = S A on the tensor cores (appendix "Sketch comparison": Gaussian and
// SRFT embeddings; their cost is a dense product with A).
//
// Operands: S rounded to bfloat16 (S~ is the sketching operator: the rounding of a
// Gaussian or SRHT matrix is again a valid embedding) and A as a sum of 1 to 3 bfloat16
// terms of its FP32 value (A = A_0 + A_1 + A_2 exactly with three terms), each term one
// more MMA into the same FP32 accumulator.  One term rounds A to 8 significant bits, which
// puts a noise floor of about 2^-9 |A| under the sketched spectrum; two terms lower it to
// 2^-17, three leave only the FP32 accumulation.
//
// The product is D (n x s) = A^T S^T in tcgen05 terms: the MMA's M dimension runs over
// the columns of A (tiles of 128), its N dimension over the sketch rows (s rounded up to
// 16, one or two MMAs of at most 256 columns), its K dimension over the rows of A (blocks
// of 64).  Both operands are bfloat16 tiles in shared memory with the 128-byte swizzle:
// S K-major, pre-arranged in that layout in global memory (one bulk copy per K-block);
// A MN-major, so that a row of A is a row of the tile.  A stager warp bulk-copies the
// rows of A (as stored) into a ring of staging units, eight converter warps round them to
// bfloat16 terms and write the swizzled tiles.  One thread issues the MMAs (FP32
// accumulation in tensor memory) and commits them to mbarriers that free the A slot and
// the S tile and, at the end of an output tile, hand the accumulator to the converter
// warps, which copy it out with tcgen05.ld.
//
// Work split ("stream-K"): the tiles x K-blocks of the product are cut into one
// contiguous range per CTA of a persistent grid, so every SM gets the same number of
// K-blocks; a CTA's range covers the ends of at most a few output tiles, whose FP32
// partial sums it writes to a partial buffer, and a second kernel adds the partials of
// every tile in CTA order (FP64) into Y.
//
// Every wait is bounded in time (a wait that gives up sets the error flag and the kernel
// finishes its protocol without data); tensor memory is released only after the MMA
// thread's last commit has completed.
#include <cuda.h>  // CUtensorMap (the encoder is reached through the runtime's entry point)
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "tcsketch.cuh"

namespace apl {

namespace {

constexpr int BM = 128;        // columns of A per output tile (MMA M)
constexpr int BK = 64;         // rows of A per K-block (one 128-byte swizzle atom)
constexpr int MAX_A = 4;  // ring of bfloat16 A tiles (all terms of a K-block per slot)
constexpr int MAX_S = 8;  // ring of S tiles
constexpr int SMEM_LIMIT = 227 * 1024;  // opt-in shared memory per CTA
constexpr int NCV = 16;        // converter / epilogue warps
constexpr int RPW = 64 / NCV;  // rows of a K-block per converter warp
constexpr int PRODUCER = NCV;  // warp issuing the bulk copies of S
constexpr int ISSUER = NCV + 1;  // warp holding tensor memory and issuing the MMAs
constexpr int STAGER = NCV + 2;  // warp issuing the bulk copies of A's rows
constexpr int NTH = (NCV + 3) * 32;
constexpr int UNIT_ROWS = 32;  // rows of A per staging unit (half a K-block)
constexpr int MAX_UNITS = 8;   // staging ring length
constexpr int A_TILE_BYTES = BM * BK * 2;  // 16 KB
constexpr long long kWaitCycles = 4000000000ll;  // about 2 s at 2.07 GHz

__device__ __forceinline__ uint32_t saddr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mb_init(uint64_t* b, unsigned cnt) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(b)), "r"(cnt) : "memory");
}
__device__ __forceinline__ void mb_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(b)) : "memory");
}
__device__ __forceinline__ void mb_arrive_expect(uint64_t* b, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(b)),
               "r"(bytes)
               : "memory");
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
// Waits for the phase of the given parity; returns early once `abort` is set, and sets it
// (and the error flag) when the wait runs past its bound.
__device__ bool wait_phase(uint64_t* b, unsigned parity, volatile int* abort, int* err) {
  if (mb_try(b, parity)) return true;
  const long long t0 = clock64();
  while (true) {
    if (mb_try(b, parity)) return true;
    if (*abort) return false;
    if (clock64() - t0 > kWaitCycles) {
      *abort = 1;
      atomicExch(err, 1);
      return false;
    }
  }
}
// Bounded wait that ignores `abort` (asynchronous work must land before release).
__device__ void wait_drain(uint64_t* b, unsigned parity, int* err) {
  const long long t0 = clock64();
  while (!mb_try(b, parity)) {
    if (clock64() - t0 > kWaitCycles) {
      atomicExch(err, 1);
      return;
    }
  }
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes,
                                          uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(saddr(dst)),
      "l"(src), "r"(bytes), "r"(saddr(bar))
      : "memory");
}
// 2-D tensor copy of one box at (x, y) = (column, row) of the tensor map into shared
// memory, completing transaction bytes on the mbarrier (x is a multiple of 128 elements)
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, "
      "{%2, %3}], [%4];" ::"r"(saddr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(saddr(bar))
      : "memory");
}
// generic-proxy writes to shared memory become visible to the tensor cores (async proxy)
__device__ __forceinline__ void fence_async_shared() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// Shared-memory matrix descriptor of a K-major tile with the 128-byte swizzle: rows of
// 128 bytes, 8-row groups 1024 bytes apart (stride byte offset), start address in 16-byte
// units; the leading byte offset is not used by this layout (one swizzle atom spans the
// K extent of an instruction).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of the 5th-generation tensor cores
  d |= (uint64_t)2 << 61;  // 128-byte swizzle
  return d;
}
// Descriptor of an MN-major tile with the 128-byte swizzle: atoms of 64 MN elements (one
// 128-byte row) by 8 K rows (1 KB); the leading byte offset steps between atoms along MN,
// the stride byte offset between 8-row K groups.
__device__ __forceinline__ uint64_t sw128_mn_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}
// Instruction descriptor of kind::f16: FP32 accumulator, bfloat16 A and B, A MN-major
// (transposed), B K-major, N and M encoded as N / 8 and M / 16.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accum)
      : "memory");
}
// arrive on the mbarrier once every tcgen05 operation issued so far by this thread is done
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          saddr(bar))
      : "memory");
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
  uint32_t r[8];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int k = 0; k < 8; ++k) v[k] = __uint_as_float(r[k]);
}

__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(double v) { return __double2float_rn(v); }
// four consecutive values from the staging ring (shared memory)
__device__ __forceinline__ void read4(const float* p, float (&v)[4]) {
  const float4 q = *reinterpret_cast<const float4*>(p);
  v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
__device__ __forceinline__ void read4(const double* p, float (&v)[4]) {
  const double2 a = reinterpret_cast<const double2*>(p)[0];
  const double2 b = reinterpret_cast<const double2*>(p)[1];
  v[0] = __double2float_rn(a.x); v[1] = __double2float_rn(a.y);
  v[2] = __double2float_rn(b.x); v[3] = __double2float_rn(b.y);
}
// four consecutive values of a row, 16-byte aligned (read once: evict-first)
__device__ __forceinline__ void load4(const float* p, float (&v)[4]) {
  const float4 q = __ldcs(reinterpret_cast<const float4*>(p));
  v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
__device__ __forceinline__ void load4(const double* p, float (&v)[4]) {
  const double2 a = __ldcs(reinterpret_cast<const double2*>(p));
  const double2 b = __ldcs(reinterpret_cast<const double2*>(p) + 1);
  v[0] = __double2float_rn(a.x); v[1] = __double2float_rn(a.y);
  v[2] = __double2float_rn(b.x); v[3] = __double2float_rn(b.y);
}

// Grid: one CTA per SM; CTA c owns the K-blocks [c L, (c + 1) L) of the tiles x KB blocks.
// Dynamic shared memory: nA slots of NPC A tiles (128 rows x 128 B, one per bfloat16 term
// of A), nS S tiles (Np rows x 128 B), all 1024-byte aligned, and nstg staging units of
// 32 rows of A as stored.  The MMA of a K-block frees its A slot and its S tile (one
// commit to each ring), so S tiles are fetched ahead independently of the conversion.
// Nineteen warps spread five, five, five and four over the SM's four register partitions
// of 16K registers: at most 96 registers a thread.
template <typename TA, int NPC>
__global__ void __launch_bounds__(NTH, 1)
    tc_sketch_kernel(int64_t m, int64_t n, int64_t ld, const TA* __restrict__ A,
                     const uint16_t* __restrict__ St, int Np, int nsplit, int nch, int KB, int nA,
                     int nS,
                     int vec, int nstg,
                     int64_t KT, int64_t L, int QMAX, uint32_t tmem_cols,
                     float* __restrict__ part, int* err, const __grid_constant__ CUtensorMap tmA) {
  extern __shared__ unsigned char dsm[];
  __shared__ __align__(8) uint64_t a_full[MAX_A], a_free[MAX_A], s_full[MAX_S], s_free[MAX_S];
  __shared__ __align__(8) uint64_t acc_full, acc_empty, done_bar;
  __shared__ __align__(8) uint64_t stg_full[MAX_UNITS], stg_empty[MAX_UNITS];
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // 1024-byte aligned tile area (the swizzle pattern is anchored at 1024-byte boundaries)
  const uint32_t raw = saddr(dsm);
  unsigned char* base = dsm + (((raw + 1023u) & ~1023u) - raw);
  unsigned char* a_tiles = base;
  unsigned char* s_tiles = base + nA * NPC * A_TILE_BYTES;
  const int s_tile_bytes = Np * 128;
  // staging ring of A's rows (FP32 or FP64 as stored) behind the stages
  constexpr int ROW_BYTES = BM * (int)sizeof(TA);
  constexpr int UNIT_BYTES = UNIT_ROWS * ROW_BYTES;
  unsigned char* stg = s_tiles + nS * s_tile_bytes;
  const int64_t k_lo = (int64_t)blockIdx.x * L;
  const int64_t k_hi = k_lo + L < KT ? k_lo + L : KT;
  const int nk = k_hi > k_lo ? (int)(k_hi - k_lo) : 0;
  const int64_t t0 = k_lo / KB;
  if (tid == 0) {
    abort_flag = 0;
    for (int s = 0; s < nA; ++s) {
      mb_init(&a_full[s], NCV);
      mb_init(&a_free[s], 1);
    }
    for (int s = 0; s < nS; ++s) {
      mb_init(&s_full[s], 1);
      mb_init(&s_free[s], 1);
    }
    for (int u = 0; u < nstg; ++u) {
      mb_init(&stg_full[u], 1);
      mb_init(&stg_empty[u], UNIT_ROWS / RPW);
    }
    mb_init(&acc_full, 1);
    mb_init(&acc_empty, NCV);
    mb_init(&done_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == ISSUER) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     saddr(&tmem_slot)),
                 "r"(tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tmem_slot;

  if (warp < NCV) {
    // ---- converters: A (FP32 / FP64, row-major) -> bfloat16 MN-major swizzled tiles.
    // Warp w owns the rows RPW w .. RPW w + RPW - 1 of the K-block, lane l the four
    // columns 4l .. 4l + 3 of the tile: one 16-byte read per row (FP32) and one 8-byte
    // store per row and term, conflict-free (the 16 lanes of a 64-column atom fill one
    // 128-byte row).  Element (c, k) of the tile sits in atom c / 64 (8 KB apart), K-group
    // k / 8 (1 KB apart), row k % 8 (128 B apart), 16-byte chunk ((c % 64) / 8) ^ (k % 8).
    // K-blocks come from the staging ring (rows copied by the stager warp; the warps of
    // the first 32 rows read the first unit of a K-block, the others the second); rows
    // that are not 16-byte aligned are read from global memory.  The converters also run
    // the epilogue: accumulator rows 32 (warp % 4) .. + 31, a quarter of the columns each.
    const int k0 = RPW * warp;  // first row of the warp in the K-block
    const int st_off = (((lane >> 4) * 8 + (k0 >> 3)) << 10) + ((lane & 1) << 3);
    const int chunk = (lane & 15) >> 1;
    int sg = 0, sidx = 0;
    const int cw = 16 * ((Np + 16 * (NCV / 4) - 1) / (16 * (NCV / 4)));  // columns per part
    const int c_lo = (warp >> 2) * cw;
    const int c_hi = c_lo + cw < Np ? c_lo + cw : Np;
    int64_t cv_tt = k_lo / KB;
    int cv_kk = (int)(k_lo % KB);
    for (int li = 0; li < nk; ++li) {
      const int kk = cv_kk;
      const int64_t j0 = cv_tt * BM + 4 * lane;
      const int64_t i0 = (int64_t)kk * BK + k0;
      const int64_t rows = m - i0;
      float cur[RPW][4];
      if (nstg > 0) {
        const int uidx = 2 * sidx + k0 / UNIT_ROWS;
        const int b = uidx % nstg, u = uidx / nstg;
        wait_phase(&stg_full[b], (unsigned)u & 1u, &abort_flag, err);
        const unsigned char* src = stg + b * UNIT_BYTES + (k0 % UNIT_ROWS) * ROW_BYTES +
                                   lane * 4 * (int)sizeof(TA);
#pragma unroll
        for (int t = 0; t < RPW; ++t) {
          if (t < rows) {
            read4(reinterpret_cast<const TA*>(src + t * ROW_BYTES), cur[t]);
          } else {
            cur[t][0] = cur[t][1] = cur[t][2] = cur[t][3] = 0.f;
          }
        }
        __syncwarp();
        if (lane == 0) mb_arrive(&stg_empty[b]);
        ++sidx;
      } else {
        const int64_t rem = n - j0;
        const TA* p = A + i0 * ld + j0;
#pragma unroll
        for (int t = 0; t < RPW; ++t) {
          if (t < rows && rem >= 4 && vec) {
            load4(p + t * ld, cur[t]);
          } else {
#pragma unroll
            for (int c = 0; c < 4; ++c)
              cur[t][c] = (t < rows && c < rem) ? to_f(p[t * ld + c]) : 0.f;
          }
        }
      }
      const int s = li % nA, u = li / nA;
      if (li >= nA) wait_phase(&a_free[s], (unsigned)(u - 1) & 1u, &abort_flag, err);
      unsigned char* at = a_tiles + s * NPC * A_TILE_BYTES + st_off;
#pragma unroll
      for (int t = 0; t < RPW; ++t) {
        const int r8 = (k0 + t) & 7;
        const int off = (r8 << 7) + ((chunk ^ r8) << 4);
        // term pc of the bfloat16 expansion: round the FP32 remainder, subtract (exact)
#pragma unroll
        for (int pc = 0; pc < NPC; ++pc) {
          const __nv_bfloat162 h0 = __floats2bfloat162_rn(cur[t][0], cur[t][1]);
          const __nv_bfloat162 h1 = __floats2bfloat162_rn(cur[t][2], cur[t][3]);
          if (pc + 1 < NPC) {
            cur[t][0] -= __low2float(h0);
            cur[t][1] -= __high2float(h0);
            cur[t][2] -= __low2float(h1);
            cur[t][3] -= __high2float(h1);
          }
          uint2 q;
          memcpy(&q.x, &h0, 4);
          memcpy(&q.y, &h1, 4);
          *reinterpret_cast<uint2*>(at + pc * A_TILE_BYTES + off) = q;
        }
      }
      fence_async_shared();
      __syncwarp();
      if (lane == 0) mb_arrive(&a_full[s]);
      if (kk == KB - 1 || li == nk - 1) {
        // end of an output tile segment: copy the accumulator out
        wait_phase(&acc_full, (unsigned)sg & 1u, &abort_flag, err);
        __syncwarp();  // tcgen05.ld is warp-collective
        tc_fence_after();
        const int64_t q = cv_tt - t0;
        const int row = 32 * (warp & 3) + lane;
        float* out = part + (((int64_t)blockIdx.x * QMAX + q) * BM + row) * Np;
        for (int col = c_lo; col < c_hi; col += 8) {
          float v[8];
          tmem_ld8(tbase + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)col, v);
#pragma unroll
          for (int k = 0; k < 8; k += 4)
            *reinterpret_cast<float4*>(out + col + k) = make_float4(v[k], v[k + 1], v[k + 2], v[k + 3]);
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mb_arrive(&acc_empty);
        ++sg;
      }
      if (++cv_kk == KB) { cv_kk = 0; ++cv_tt; }
    }
  } else if (warp == STAGER) {
    // ---- stager: each K-block of A (as stored) into the staging ring, two tensor copies
    // of 32 rows x 128 columns (rows and columns outside A arrive as zeros)
    if (lane == 0 && nstg > 0) {
      int issued = 0;
      int64_t tt = k_lo / KB;
      int kk = (int)(k_lo % KB);
      for (int li = 0; li < nk; ++li) {
        for (int h = 0; h < 2; ++h) {
          const int b = issued % nstg, u = issued / nstg;
          if (issued >= nstg) wait_phase(&stg_empty[b], (unsigned)(u - 1) & 1u, &abort_flag, err);
          if (abort_flag) break;
          mb_arrive_expect(&stg_full[b], (unsigned)UNIT_BYTES);
          tma_load_2d(stg + b * UNIT_BYTES, &tmA, (int)(tt * BM), kk * BK + UNIT_ROWS * h,
                      &stg_full[b]);
          ++issued;
        }
        if (abort_flag) break;
        if (++kk == KB) { kk = 0; ++tt; }
      }
      // the copies in flight land before the CTA's shared memory is released
      for (int x = issued - nstg > 0 ? issued - nstg : 0; x < issued; ++x)
        wait_drain(&stg_full[x % nstg], (unsigned)(x / nstg) & 1u, err);
    }
  } else if (warp == PRODUCER) {
    // ---- producer: the K-block of the pre-swizzled S into the S ring
    if (lane == 0) {
      int issued = 0;
      int kk = (int)(k_lo % KB);
      for (int li = 0; li < nk; ++li, kk = kk + 1 == KB ? 0 : kk + 1) {
        const int s = li % nS, u = li / nS;
        if (li >= nS) wait_phase(&s_free[s], (unsigned)(u - 1) & 1u, &abort_flag, err);
        if (abort_flag) break;
        mb_arrive_expect(&s_full[s], (unsigned)s_tile_bytes);
        bulk_load(s_tiles + s * s_tile_bytes, St + kk * (int64_t)Np * BK, (unsigned)s_tile_bytes,
                  &s_full[s]);
        issued = li + 1;
      }
      for (int li = issued - nS > 0 ? issued - nS : 0; li < issued; ++li)
        wait_drain(&s_full[li % nS], (unsigned)(li / nS) & 1u, err);
    }
  } else {
    // ---- MMA issuer
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(BM, nch);
      int sg = 0;
      for (int li = 0; li < nk; ++li) {
        const int64_t g = k_lo + li;
        const int64_t kk = g % KB;
        const int sa = li % nA, ua = li / nA;
        const int ss = li % nS, us = li / nS;
        const bool first = li == 0 || kk == 0;
        if (first && sg > 0) {
          wait_phase(&acc_empty, (unsigned)(sg - 1) & 1u, &abort_flag, err);
          tc_fence_after();
        }
        wait_phase(&a_full[sa], (unsigned)ua & 1u, &abort_flag, err);
        wait_phase(&s_full[ss], (unsigned)us & 1u, &abort_flag, err);
        tc_fence_after();
        const uint32_t a0 = saddr(a_tiles + sa * NPC * A_TILE_BYTES);
        const uint32_t b0 = saddr(s_tiles + ss * s_tile_bytes);
#pragma unroll
        for (int pc = 0; pc < NPC; ++pc)
#pragma unroll
          for (int ks = 0; ks < BK / 16; ++ks) {
            for (int ch = 0; ch < nsplit; ++ch) {
              mma_bf16(tbase + (uint32_t)(ch * nch),
                       sw128_mn_desc(a0 + pc * A_TILE_BYTES + ks * 2048, 8192, 1024),
                       sw128_desc(b0 + ch * nch * 128 + ks * 32), idesc,
                       (first && pc == 0 && ks == 0) ? 0u : 1u);
            }
          }
        mma_commit(&a_free[sa]);
        mma_commit(&s_free[ss]);
        if (kk == KB - 1 || li == nk - 1) {
          mma_commit(&acc_full);
          ++sg;
        }
      }
      // every MMA of this thread complete before tensor memory is released
      mma_commit(&done_bar);
      wait_drain(&done_bar, 0u, err);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == ISSUER) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase),
                 "r"(tmem_cols)
                 : "memory");
  }
}

// Y(r, j) = sum over the CTAs whose K range met tile j / BM of their partials, in CTA order.
__global__ void tc_reduce_kernel(int s, int Np, int64_t n, int KB, int64_t L, int QMAX,
                                 const float* __restrict__ part, double* __restrict__ Y) {
  const int64_t t = blockIdx.x;
  const int64_t c_lo = (t * KB) / L, c_hi = ((t + 1) * KB - 1) / L;
  for (int64_t idx = threadIdx.x; idx < (int64_t)BM * s; idx += blockDim.x) {
    const int jl = (int)(idx / s), r = (int)(idx % s);
    const int64_t j = t * BM + jl;
    if (j >= n) continue;
    double acc = 0.0;
    for (int64_t c = c_lo; c <= c_hi; ++c) {
      const int64_t q = t - (c * L) / KB;
      acc += (double)part[((c * QMAX + q) * BM + jl) * Np + r];
    }
    Y[r + (int64_t)s * j] = acc;
  }
}

uint16_t bf16_bits(double v) {
  // through FP32, then to the nearest bfloat16 (ties to even); sketch values are finite
  const float f = (float)v;
  uint32_t u;
  std::memcpy(&u, &f, 4);
  u = (u + 0x7FFFu + ((u >> 16) & 1u)) >> 16;
  return (uint16_t)u;
}

}  // namespace

void tc_sketch_upload(cudaStream_t st, const double* S, int s, int64_t m, int64_t n,
                      TcSketchWork& w) {
  APL_REQUIRE(s >= 1 && s <= TC_SKETCH_MAX_S, "tensor-core sketch: 1 <= s <= 512");
  // rows of the S tile: s rounded up to 16, or to 32 above 256 so that the two MMAs of
  // an output tile take halves of a multiple of 16
  const int Np = s <= 256 ? (s + 15) / 16 * 16 : (s + 31) / 32 * 32;
  const int KB = (int)cdiv(m, BK);
  // K-block kb, row r, element k: at kb Np 64 + r 64 + ((k / 8) ^ (r % 8)) 8 + k % 8, the
  // 128-byte swizzle of a K-major tile with 128-byte rows
  std::vector<uint16_t> h((size_t)KB * Np * BK, 0);
  for (int kb = 0; kb < KB; ++kb)
    for (int r = 0; r < s; ++r)
      for (int k = 0; k < BK; ++k) {
        const int64_t i = (int64_t)kb * BK + k;
        if (i >= m) break;
        const size_t off = ((size_t)kb * Np + r) * BK + (size_t)(((k >> 3) ^ (r & 7)) << 3) +
                           (size_t)(k & 7);
        h[off] = bf16_bits(S[r + (size_t)s * i]);
      }
  w.st.alloc(h.size(), st);
  APL_CUDA(cudaMemcpyAsync(w.st.p, h.data(), h.size() * sizeof(uint16_t), cudaMemcpyHostToDevice, st));
  int dev = 0, nsm = 0;
  APL_CUDA(cudaGetDevice(&dev));
  APL_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int64_t KT = cdiv(n, BM) * KB;
  w.G = std::min<int64_t>(nsm, KT);
  w.L = cdiv(KT, w.G);
  w.QMAX = (int)((w.L - 1) / KB) + 2;
  w.part.alloc((size_t)w.G * w.QMAX * BM * Np, st);
  w.err.alloc(1, st);
  APL_CUDA(cudaStreamSynchronize(st));
  w.s = s;
  w.Np = Np;
  w.KB = KB;
  w.n = n;
}

namespace {

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                 const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                 const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                 CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encoder() {
  static EncodeTiled fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return reinterpret_cast<EncodeTiled>(p);
  }();
  return fn;
}

// Tensor map of A (row-major, m rows of n values, row stride ld) with boxes of 32 rows x
// 128 values, no swizzle, zeros outside A.  Needs 16-byte aligned rows.
bool encode_rows_map(const MatView& A, CUtensorMap* map) {
  EncodeTiled enc = encoder();
  if (!enc) return false;
  const size_t es = A.dtype == 0 ? 8 : 4;
  const cuuint64_t dims[2] = {(cuuint64_t)A.n, (cuuint64_t)A.m};
  const cuuint64_t strides[1] = {(cuuint64_t)(A.ld * es)};
  const cuuint32_t box[2] = {(cuuint32_t)BM, (cuuint32_t)UNIT_ROWS};
  const cuuint32_t estr[2] = {1, 1};
  return enc(map, A.dtype == 0 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
             2, const_cast<void*>(A.vals), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <typename TA, int NPC>
void launch_tc(cudaStream_t st, const MatView& A, TcSketchWork& w, int64_t G, int nsplit, int nch,
               int64_t KT, int64_t L, int QMAX, uint32_t cols, cudaEvent_t e0) {
  // shared memory: two slots of bfloat16 A tiles, two S tiles and four staging units of
  // A's rows, then one more of each in turn while they fit (up to 4 A slots, 8 S tiles, 8
  // units); the static shared memory of the kernel is under 512 bytes
  const int a_bytes = NPC * A_TILE_BYTES;
  const int s_bytes = w.Np * 128;
  const int unit_bytes = UNIT_ROWS * BM * (int)sizeof(TA);
  const int avail = SMEM_LIMIT - 1024 - 512;
  // 16-byte row loads and the tensor copies need 16-byte aligned rows
  const int vec = ((uintptr_t)A.vals % 16 == 0 && (A.ld * (int64_t)sizeof(TA)) % 16 == 0) ? 1 : 0;
  CUtensorMap tmA;
  std::memset(&tmA, 0, sizeof(tmA));
  const bool staged = vec && encode_rows_map(A, &tmA);
  int nA = 2, nS = 2, nstg = 0;
  APL_REQUIRE(nA * a_bytes + nS * s_bytes <= avail, "tensor-core sketch: shared memory");
  auto used = [&]() { return nA * a_bytes + nS * s_bytes + nstg * unit_bytes; };
  if (staged)
    while (nstg < 4 && used() + unit_bytes <= avail) ++nstg;
  for (bool grew = true; grew;) {
    grew = false;
    if (nA < MAX_A && used() + a_bytes <= avail) { ++nA; grew = true; }
    if (nS < MAX_S && used() + s_bytes <= avail) { ++nS; grew = true; }
    if (staged && nstg < MAX_UNITS && used() + unit_bytes <= avail) { ++nstg; grew = true; }
  }
  if (nstg < 2) nstg = 0;  // too few units to overlap: every K-block read directly
  const size_t smem = (size_t)used() + 1024;
  APL_CUDA(cudaFuncSetAttribute(tc_sketch_kernel<TA, NPC>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  // the timed region starts after the host-side preparation
  if (e0) APL_CUDA(cudaEventRecord(e0, st));
  tc_sketch_kernel<TA, NPC><<<(unsigned)G, NTH, smem, st>>>(
      A.m, A.n, A.ld, (const TA*)A.vals, w.st.p, w.Np, nsplit, nch, w.KB, nA, nS, vec, nstg, KT,
      L, QMAX, cols, w.part.p, w.err.p, tmA);
  APL_LAUNCH_CHECK();
}

}  // namespace

void tc_sketch_apply(cudaStream_t st, const MatView& A, TcSketchWork& w, double* Y, int terms,
                     cudaEvent_t e0, cudaEvent_t e1) {
  APL_REQUIRE(A.fmt == 0, "tensor-core sketch: dense A only");
  APL_REQUIRE(w.st.p && w.KB == (int)cdiv(A.m, BK) && w.n == A.n,
              "tensor-core sketch: S not uploaded for this shape");
  APL_REQUIRE(terms >= 1 && terms <= 3, "tensor-core sketch: 1 to 3 bfloat16 terms of A");
  const int Np = w.Np, KB = w.KB;
  const int nsplit = Np > 256 ? 2 : 1;
  const int nch = Np / nsplit;
  APL_REQUIRE(nch * nsplit == Np && nch % 16 == 0 && nch <= 256, "tensor-core sketch: bad N split");
  const int64_t tiles = cdiv(A.n, BM);
  const int64_t KT = tiles * KB;
  const int64_t G = w.G, L = w.L;
  const int QMAX = w.QMAX;
  uint32_t cols = 32;
  while ((int)cols < Np) cols <<= 1;
  w.err.zero(st);
  if (A.dtype == 0) {
    if (terms == 1) launch_tc<double, 1>(st, A, w, G, nsplit, nch, KT, L, QMAX, cols, e0);
    else if (terms == 2) launch_tc<double, 2>(st, A, w, G, nsplit, nch, KT, L, QMAX, cols, e0);
    else launch_tc<double, 3>(st, A, w, G, nsplit, nch, KT, L, QMAX, cols, e0);
  } else {
    if (terms == 1) launch_tc<float, 1>(st, A, w, G, nsplit, nch, KT, L, QMAX, cols, e0);
    else if (terms == 2) launch_tc<float, 2>(st, A, w, G, nsplit, nch, KT, L, QMAX, cols, e0);
    else launch_tc<float, 3>(st, A, w, G, nsplit, nch, KT, L, QMAX, cols, e0);
  }
  tc_reduce_kernel<<<(unsigned)tiles, 256, 0, st>>>(w.s, Np, A.n, KB, L, QMAX, w.part.p, Y);
  APL_LAUNCH_CHECK();
  if (e1) APL_CUDA(cudaEventRecord(e1, st));
  int e = 0;
  APL_CUDA(cudaMemcpyAsync(&e, w.err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  APL_CUDA(cudaStreamSynchronize(st));
  if (e) throw Error(ST_ETIMEOUT, "tensor-core sketch: a bounded wait ran past its bound");
}

}  // namespace apl
