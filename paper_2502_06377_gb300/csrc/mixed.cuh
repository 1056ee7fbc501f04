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
// The whole mixed pipeline: FP64 block factorisations and W on tensor cores,
// sweeps (tcgen05 BF16 slices), hand-over test on a BF16x3 residual, then the
// Newton-Schulz tail with FP64-accurate residuals (sliced error-free
// products) and tensor-core updates.
// Graph mode: every phase is captured once as a CUDA graph (for the A and H
// pointers of that run) and replayed; used by the batched executor, whose
// workers run each plan on its own staging buffers.
void mixed_enable_graphs(ibmi_plan_s* P, bool on);

ibmi_status mixed_run(ibmi_plan_s* P, const double* A, int64_t lda, double* H, int64_t ldh, cudaStream_t st,
                      ibmi_result* res, double* flops);
}  // namespace ibmi
