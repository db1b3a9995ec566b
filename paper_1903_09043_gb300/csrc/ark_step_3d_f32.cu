// ark_step_3d_f32.cu -- 3D FP32 and FP32-split step kernels: 28 x 12 output
// tiles, one thread per column of the 32 x 16 tile-plus-halo (ark_step2.cuh),
// marching along z.
#include "ark_step2_inst.cuh"

namespace ark {

StepKernelInfo step_kernel_3d_f64(int visc);

StepKernelInfo step_kernel_3d(int prec, int visc)
{
    if (prec == P_F64) return step_kernel_3d_f64(visc);
    if (prec == P_F32) return visc ? step2_info<3, float, false, true, 32, 16>() : step2_info<3, float, false, false, 32, 16>();
    return visc ? step2_info<3, float, true, true, 32, 16>() : step2_info<3, float, true, false, 32, 16>();
}

}  // namespace ark
