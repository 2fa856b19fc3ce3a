// Dense sketching operators (Gaussian embedding, subsampled randomized Hadamard
// transform) applied to a dense A on the 5th-generation tensor cores: Y = S A with S and A
// rounded to bfloat16 and FP32 accumulation (tcgen05.mma, accumulator in tensor memory).
#pragma once
#include "cur.cuh"

namespace apl {

// Largest sketch dimension of the tensor-core path (the accumulator of an output tile is
// 128 x roundup16(s) FP32 columns of tensor memory, at most 512).
constexpr int TC_SKETCH_MAX_S = 512;

struct TcSketchWork {
  DBuf<uint16_t> st;     // S as bfloat16, pre-arranged in swizzled K-blocks (see tcsketch.cu)
  DBuf<float> part;      // per-CTA partial output tiles
  DBuf<int> err;         // a bounded wait gave up
  int s = 0, Np = 0, KB = 0;
  int64_t n = 0, G = 0, L = 0;  // columns of A; grid and K-blocks per CTA
  int QMAX = 0;                 // output tiles a CTA's range can meet
};

// Round S (s x m, column-major FP64, host) to bfloat16 (through FP32, round to nearest
// even at both steps), upload it in the layout the kernel's bulk copies expect, and
// allocate the work buffers of a product with an m x n A.
void tc_sketch_upload(cudaStream_t st, const double* S_host, int s, int64_t m, int64_t n,
                      TcSketchWork& w);

// Y (s x n column-major FP64, device) = S~ A~ for a dense row-major A (FP32 or FP64
// values, FP64 rounded to FP32 first): S~ the bfloat16 S, A~ the sum of the first `terms`
// (1 to 3) terms of the bfloat16 expansion of A, FP32 accumulation.  Throws ST_ETIMEOUT
// when a bounded wait gave up (the work buffers are then undefined).  e0 / e1, when given,
// are recorded on st just before the product's first kernel and after its last.
void tc_sketch_apply(cudaStream_t st, const MatView& A, TcSketchWork& w, double* Y, int terms,
                     cudaEvent_t e0 = nullptr, cudaEvent_t e1 = nullptr);

}  // namespace apl
