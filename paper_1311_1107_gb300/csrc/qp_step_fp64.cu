// Instantiations of the step kernel, FP64 path (see qp_step.cuh).
#include "qp_step.cuh"

namespace qp {

const void *step_kernel_fp64(int field_kind, bool batch)
{
    return batch ? step_kernel_of<kFP64, true>(field_kind) : step_kernel_of<kFP64, false>(field_kind);
}

size_t step_smem_fp64() { return sizeof(Smem<double>); }

const void *fused_kernel_fp64(int field_kind) { return fused_kernel_of<kFP64>(field_kind); }
const void *fused_photons_fp64() { return (const void *)k_fused_photons<kFP64>; }

}  // namespace qp
