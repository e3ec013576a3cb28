// Instantiations of the step kernel, mixed-precision path (see qp_step.cuh).
// This unit is compiled with -prec-div=false: FP32 quotients use the
// hardware reciprocal (2 ulp), well inside the path's FP32 error budget.
#include "qp_step.cuh"

namespace qp {

const void *step_kernel_mixed(int field_kind, bool batch)
{
    return batch ? step_kernel_of<kMixed, true>(field_kind) : step_kernel_of<kMixed, false>(field_kind);
}

size_t step_smem_mixed() { return sizeof(Smem<float>); }

const void *fused_kernel_mixed(int field_kind) { return fused_kernel_of<kMixed>(field_kind); }
const void *fused_photons_mixed() { return (const void *)k_fused_photons<kMixed>; }

}  // namespace qp
