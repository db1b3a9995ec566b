// ark_step_na_f32.cu -- FP32 and FP32-split step kernels (column form) for the
// Noble-Abel stiffened gas: the 2D instances here, the 3D ones in
// ark_step_na_f32_3d.cu (separate translation units build in parallel).
#include "ark_step2_inst.cuh"

namespace ark {

StepKernelInfo step_kernel_noble_abel_f32_3d(int split, int visc);

StepKernelInfo step_kernel_noble_abel_f32(int dim, int split, int visc)
{
    if (dim == 3) return step_kernel_noble_abel_f32_3d(split, visc);
    if (split)
        return visc ? step2_info<2, float, true, true, 128, 1, false, true>()
                    : step2_info<2, float, true, false, 128, 1, false, true>();
    return visc ? step2_info<2, float, false, true, 128, 1, false, true>()
                : step2_info<2, float, false, false, 128, 1, false, true>();
}

}  // namespace ark
