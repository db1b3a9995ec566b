// ark_step_phi.cu -- step kernels for a caller-supplied potential array
// (ark_gravity.phi): the FP32 column kernel with the potential read per cell
// and the gravity source on every face.
#include "ark_step2_inst.cuh"

namespace ark {

StepKernelInfo step_kernel_phi(int dim, int prec, int visc)
{
    (void)prec;   // ARK_F32 (validated by ark_create)
    if (dim == 2)
        return visc ? step2_info<2, float, false, true, 256, 1, true>() : step2_info<2, float, false, false, 256, 1, true>();
    return visc ? step2_info<3, float, false, true, 32, 16, true>() : step2_info<3, float, false, false, 32, 16, true>();
}

}  // namespace ark
