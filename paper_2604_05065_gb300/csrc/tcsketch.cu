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
// of 64).  Both operands are K-major bfloat16 tiles in shared memory with the 128-byte
// swizzle: S is pre-arranged in that layout in global memory (one bulk copy per K-block),
// A is read from global memory by eight converter warps, rounded to bfloat16 and written
// transposed into the swizzled tile.  One thread issues the MMAs (FP32 accumulation in
// tensor memory) and commits them to mbarriers that free the stage and, at the end of an
// output tile, hand the accumulator to the converter warps, which copy it out with
// tcgen05.ld.
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
constexpr int MAX_STAGES = 4;
constexpr int SMEM_LIMIT = 227 * 1024;  // opt-in shared memory per CTA
constexpr int NCV = 8;         // converter / epilogue warps
constexpr int PRODUCER = NCV;  // warp issuing the bulk copies of S
constexpr int ISSUER = NCV + 1;  // warp holding tensor memory and issuing the MMAs
constexpr int NTH = (NCV + 2) * 32;
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
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}

__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(double v) { return __double2float_rn(v); }
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
// Dynamic shared memory: nst stages of NPC A tiles (128 rows x 128 B, one per bfloat16 term
// of A) and nst S tiles (Np rows x 128 B), all 1024-byte aligned.
// Ten warps spread three, three, two and two over the SM's four register partitions of
// 16K registers: at most 168 registers a thread.
template <typename TA, int NPC>
__global__ void __launch_bounds__(NTH, 1)
    tc_sketch_kernel(int64_t m, int64_t n, int64_t ld, const TA* __restrict__ A,
                     const uint16_t* __restrict__ St, int Np, int nsplit, int nch, int KB, int nst,
                     int vec,
                     int64_t KT, int64_t L, int QMAX, uint32_t tmem_cols,
                     float* __restrict__ part, int* err) {
  extern __shared__ unsigned char dsm[];
  __shared__ __align__(8) uint64_t a_full[MAX_STAGES], s_full[MAX_STAGES], stage_free[MAX_STAGES];
  __shared__ __align__(8) uint64_t acc_full, acc_empty, done_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // 1024-byte aligned tile area (the swizzle pattern is anchored at 1024-byte boundaries)
  const uint32_t raw = saddr(dsm);
  unsigned char* base = dsm + (((raw + 1023u) & ~1023u) - raw);
  unsigned char* a_tiles = base;
  unsigned char* s_tiles = base + nst * NPC * A_TILE_BYTES;
  const int s_tile_bytes = Np * 128;
  const int64_t k_lo = (int64_t)blockIdx.x * L;
  const int64_t k_hi = k_lo + L < KT ? k_lo + L : KT;
  const int nk = k_hi > k_lo ? (int)(k_hi - k_lo) : 0;
  const int64_t t0 = k_lo / KB;
  if (tid == 0) {
    abort_flag = 0;
    for (int s = 0; s < nst; ++s) {
      mb_init(&a_full[s], NCV);
      mb_init(&s_full[s], 1);
      mb_init(&stage_free[s], 1);
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
    // Warp w owns the K-group w (rows 8w .. 8w + 7 of the K-block), lane l the four columns
    // 4l .. 4l + 3 of the tile: one 16-byte load per row (FP32) and one 8-byte store per
    // row and term, conflict-free (the 16 lanes of a 64-column atom fill one 128-byte
    // row).  Element (c, k) of the tile sits in atom c / 64 (8 KB apart), K-group k / 8
    // (1 KB apart), row k % 8 (128 B apart), 16-byte chunk ((c % 64) / 8) ^ (k % 8).
    // The next K-block is in flight in registers while one is converted.  The converters
    // also run the epilogue: accumulator rows 32 (warp % 4) .. + 31, half the columns each.
    const int st_off = (((lane >> 4) * 8 + warp) << 10) + ((lane & 1) << 3);
    const int chunk = (lane & 15) >> 1;
    // K-block positions advance one at a time (no 64-bit divisions in the loop): the
    // load position runs one K-block ahead of the conversion position
    int64_t ld_tt = k_lo / KB;
    int ld_kk = (int)(k_lo % KB);
    auto load = [&](float (&v)[8][4]) {
      const int64_t j0 = ld_tt * BM + 4 * lane;
      const int64_t rem = n - j0;
      const int64_t i0 = (int64_t)ld_kk * BK + 8 * warp;
      const int64_t rows = m - i0;
      const TA* p = A + i0 * ld + j0;
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        if (t < rows && rem >= 4 && vec) {
          load4(p + t * ld, v[t]);
        } else {
#pragma unroll
          for (int c = 0; c < 4; ++c) v[t][c] = (t < rows && c < rem) ? to_f(p[t * ld + c]) : 0.f;
        }
      }
      if (++ld_kk == KB) { ld_kk = 0; ++ld_tt; }
    };
    int sg = 0;
    const int nph = 16 * ((Np + 31) / 32);  // columns of the first half (multiple of 16)
    const int c_lo = (warp >> 2) ? nph : 0;
    const int c_hi = (warp >> 2) ? Np : (nph < Np ? nph : Np);
    int64_t cv_tt = k_lo / KB;
    int cv_kk = (int)(k_lo % KB);
    auto body = [&](int li, float (&cur)[8][4], float (&ahead)[8][4]) {
      const int kk = cv_kk;
      if (li + 1 < nk) load(ahead);
      const int s = li % nst, u = li / nst;
      if (li >= nst) wait_phase(&stage_free[s], (unsigned)(u - 1) & 1u, &abort_flag, err);
      unsigned char* at = a_tiles + s * NPC * A_TILE_BYTES + st_off;
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const int off = (t << 7) + ((chunk ^ t) << 4);
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
        for (int col = c_lo; col < c_hi; col += 16) {
          float v[16];
          tmem_ld16(tbase + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)col, v);
#pragma unroll
          for (int k = 0; k < 16; k += 4)
            *reinterpret_cast<float4*>(out + col + k) = make_float4(v[k], v[k + 1], v[k + 2], v[k + 3]);
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mb_arrive(&acc_empty);
        ++sg;
      }
      if (++cv_kk == KB) { cv_kk = 0; ++cv_tt; }
    };
    float b0[8][4], b1[8][4];
    if (nk > 0) load(b0);
    for (int li = 0; li < nk; li += 2) {
      body(li, b0, b1);
      if (li + 1 < nk) body(li + 1, b1, b0);
    }
  } else if (warp == PRODUCER) {
    // ---- producer: the K-block of the pre-swizzled S into the stage ring
    if (lane == 0) {
      int issued = 0;
      for (int li = 0; li < nk; ++li) {
        const int64_t kk = (k_lo + li) % KB;
        const int s = li % nst, u = li / nst;
        if (li >= nst) wait_phase(&stage_free[s], (unsigned)(u - 1) & 1u, &abort_flag, err);
        if (abort_flag) break;
        mb_arrive_expect(&s_full[s], (unsigned)s_tile_bytes);
        bulk_load(s_tiles + s * s_tile_bytes, St + kk * (int64_t)Np * BK, (unsigned)s_tile_bytes,
                  &s_full[s]);
        issued = li + 1;
      }
      for (int li = issued - nst > 0 ? issued - nst : 0; li < issued; ++li)
        wait_drain(&s_full[li % nst], (unsigned)(li / nst) & 1u, err);
    }
  } else {
    // ---- MMA issuer
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(BM, nch);
      int sg = 0;
      for (int li = 0; li < nk; ++li) {
        const int64_t g = k_lo + li;
        const int64_t kk = g % KB;
        const int s = li % nst, u = li / nst;
        const bool first = li == 0 || kk == 0;
        if (first && sg > 0) {
          wait_phase(&acc_empty, (unsigned)(sg - 1) & 1u, &abort_flag, err);
          tc_fence_after();
        }
        wait_phase(&a_full[s], (unsigned)u & 1u, &abort_flag, err);
        wait_phase(&s_full[s], (unsigned)u & 1u, &abort_flag, err);
        tc_fence_after();
        const uint32_t a0 = saddr(a_tiles + s * NPC * A_TILE_BYTES);
        const uint32_t b0 = saddr(s_tiles + s * s_tile_bytes);
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
        mma_commit(&stage_free[s]);
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

template <typename TA, int NPC>
void launch_tc(cudaStream_t st, const MatView& A, TcSketchWork& w, int64_t G, int nsplit, int nch,
               int64_t KT, int64_t L, int QMAX, uint32_t cols) {
  // as many stages as fit (the static shared memory of the kernel is under 256 bytes)
  const int stage_bytes = NPC * A_TILE_BYTES + w.Np * 128;
  const int nst = std::min(MAX_STAGES, (SMEM_LIMIT - 1024 - 256) / stage_bytes);
  APL_REQUIRE(nst >= 2, "tensor-core sketch: shared memory");
  const size_t smem = (size_t)nst * stage_bytes + 1024;
  // 16-byte row loads need 16-byte aligned rows
  const int vec = ((uintptr_t)A.vals % 16 == 0 && (A.ld * (int64_t)sizeof(TA)) % 16 == 0) ? 1 : 0;
  APL_CUDA(cudaFuncSetAttribute(tc_sketch_kernel<TA, NPC>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  tc_sketch_kernel<TA, NPC><<<(unsigned)G, NTH, smem, st>>>(
      A.m, A.n, A.ld, (const TA*)A.vals, w.st.p, w.Np, nsplit, nch, w.KB, nst, vec, KT, L, QMAX,
      cols,
      w.part.p, w.err.p);
  APL_LAUNCH_CHECK();
}

}  // namespace

void tc_sketch_apply(cudaStream_t st, const MatView& A, TcSketchWork& w, double* Y, int terms) {
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
    if (terms == 1) launch_tc<double, 1>(st, A, w, G, nsplit, nch, KT, L, QMAX, cols);
    else if (terms == 2) launch_tc<double, 2>(st, A, w, G, nsplit, nch, KT, L, QMAX, cols);
    else launch_tc<double, 3>(st, A, w, G, nsplit, nch, KT, L, QMAX, cols);
  } else {
    if (terms == 1) launch_tc<float, 1>(st, A, w, G, nsplit, nch, KT, L, QMAX, cols);
    else if (terms == 2) launch_tc<float, 2>(st, A, w, G, nsplit, nch, KT, L, QMAX, cols);
    else launch_tc<float, 3>(st, A, w, G, nsplit, nch, KT, L, QMAX, cols);
  }
  tc_reduce_kernel<<<(unsigned)tiles, 256, 0, st>>>(w.s, Np, A.n, KB, L, QMAX, w.part.p, Y);
  APL_LAUNCH_CHECK();
  int e = 0;
  APL_CUDA(cudaMemcpyAsync(&e, w.err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  APL_CUDA(cudaStreamSynchronize(st));
  if (e) throw Error(ST_ETIMEOUT, "tensor-core sketch: a bounded wait ran past its bound");
}

}  // namespace apl
