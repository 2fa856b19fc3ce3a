// Fused dense A pass of one LSQR iteration (Section 2.2, Golub-Kahan step): for an FP32
// row-major A it forms u' = ca A z + cu u (rows of A) and the column partial sums of
// A^T u' from a single read of A.  The product is linear, so the normalisation by
// beta = ||u'|| is applied afterwards (by the column-sum kernel k2b_dense).
#pragma once
#include "lsqr.cuh"

namespace apl {

// Plan the fused pass (mode 1 or 2, as for the launch) for an m x n FP32 row-major A (leading dimension ld, base address
// `vals`): panels, stages and the largest persistent grid of clusters that fits the GPU.
// ok = false when A does not qualify (alignment, n % 4, panel width).
FusedPlan plan_fused_apass(int64_t m, int64_t n, int64_t ld, const void* vals, int mode);

// One launch of the fused pass on stream st.  mode 1: FP32 products and sums; mode 2:
// compensated FP32 (z split into zh + zl).  u (m + n, unnormalised u' of the previous
// iteration, overwritten), z and its split, part (nclusters x n column partial sums),
// red (per-CTA partial sums of ||u'||^2), err (set when a bounded wait gave up).
void launch_fused_apass(cudaStream_t st, const FusedPlan& p, int mode, const MatView& A,
                        const double* z, const float* zh, const float* zl, double* u,
                        LsqrCtl* ctl, double* red, double* part, int* err);

}  // namespace apl
