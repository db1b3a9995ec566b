// ark_step_3d_f32.cu -- 3D FP32 and FP32-split step-kernel instances: 16 x 16 tiles marching along z.
#include "ark_step_inst.cuh"

namespace ark {

StepKernelInfo step_kernel_3d_f64(int visc);

StepKernelInfo step_kernel_3d(int prec, int visc)
{
    if (prec == P_F64) return step_kernel_3d_f64(visc);
    if (prec == P_F32) return visc ? step_info<3, float, false, true, 16, 16>() : step_info<3, float, false, false, 16, 16>();
    return visc ? step_info<3, float, true, true, 16, 16>() : step_info<3, float, true, false, 16, 16>();
}

}  // namespace ark
