// ark_step_na_f32_3d.cu -- 3D FP32 and FP32-split step kernels (column form)
// for the Noble-Abel stiffened gas.
#include "ark_step2_inst.cuh"

namespace ark {

StepKernelInfo step_kernel_noble_abel_f32_3d(int split, int visc)
{
    if (split)
        return visc ? step2_info<3, float, true, true, 32, 16, false, true>()
                    : step2_info<3, float, true, false, 32, 16, false, true>();
    return visc ? step2_info<3, float, false, true, 32, 16, false, true>()
                : step2_info<3, float, false, false, 32, 16, false, true>();
}

}  // namespace ark
