// ark_step_na_f64.cu -- step kernels for the Noble-Abel stiffened gas (a
// covolume b in the equation of state): the FP64 instances here, the FP32
// forms in ark_step_na_f32.cu, with the tiles of the stiffened-gas kernels.
#include "ark_step_inst.cuh"

namespace ark {

StepKernelInfo step_kernel_noble_abel_f32(int dim, int split, int visc);

StepKernelInfo step_kernel_noble_abel(int dim, int prec, int visc)
{
    if (prec != P_F64) return step_kernel_noble_abel_f32(dim, prec == P_F32_SPLIT, visc);
    if (dim == 2)
        return visc ? step_info<2, double, false, true, 256, 1, false, true>()
                    : step_info<2, double, false, false, 256, 1, false, true>();
    return visc ? step_info<3, double, false, true, 16, 16, false, true>()
                : step_info<3, double, false, false, 16, 16, false, true>();
}

}  // namespace ark
