// ark_step_phi_split.cu -- FP32-split step kernels for a caller-supplied
// potential that depends on the gravity (last) axis only: the base state is
// one row per level as with uniform gravity, its FP64 tables formed from the
// caller's row potential; the kernel reads the potential per cell (the
// column kernel of ark_step2.cuh with a potential array).
#include "ark_step2_inst.cuh"

namespace ark {

StepKernelInfo step_kernel_phi_split(int dim, int visc)
{
    if (dim == 2)
        return visc ? step2_info<2, float, true, true, 256, 1, true>() : step2_info<2, float, true, false, 256, 1, true>();
    return visc ? step2_info<3, float, true, true, 32, 16, true>() : step2_info<3, float, true, false, 32, 16, true>();
}

}  // namespace ark
