#include "mixed.cuh"
namespace ibmi {
ibmi_status mixed_create(ibmi_plan_s*) { return IBMI_ERR_INVALID_ARG; }
void mixed_destroy(ibmi_plan_s*) {}
ibmi_status mixed_prepare(ibmi_plan_s*, const double*, int64_t, cudaStream_t) { return IBMI_ERR_INVALID_ARG; }
ibmi_status mixed_sweep_step(ibmi_plan_s*, int, cudaStream_t) { return IBMI_ERR_INVALID_ARG; }
ibmi_status mixed_export(ibmi_plan_s*, double*, int64_t, cudaStream_t) { return IBMI_ERR_INVALID_ARG; }
}  // namespace ibmi
