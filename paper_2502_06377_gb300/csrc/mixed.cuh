// Mixed-precision sweep state (tcgen05 split-BF16 products), internal.
#pragma once
#include "plan.cuh"

namespace ibmi {
ibmi_status mixed_create(ibmi_plan_s* P);
void mixed_destroy(ibmi_plan_s* P);
// Splits the FP64 invariants and the initial iterate into tensor-core operands.
ibmi_status mixed_prepare(ibmi_plan_s* P, const double* H, int64_t ldh, cudaStream_t st);
// a3 + a4 for set k on the mixed-precision iterate.
ibmi_status mixed_sweep_step(ibmi_plan_s* P, int k, cudaStream_t st);
// Writes the mixed iterate into the caller's FP64 H.
ibmi_status mixed_export(ibmi_plan_s* P, double* H, int64_t ldh, cudaStream_t st);
// Sweeps (tcgen05 BF16x3), hand-over test on a BF16x3 residual, then the
// Newton-Schulz tail with FP64-accurate residuals (sliced error-free products)
// and tensor-core updates.  Invariants must be computed and H initialised.
ibmi_status mixed_run(ibmi_plan_s* P, const double* A, int64_t lda, double* H, int64_t ldh, cudaStream_t st,
                      ibmi_result* res, double* flops);
}  // namespace ibmi
