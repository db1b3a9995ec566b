// ark_step_3d_f64.cu -- 3D FP64 step-kernel instances: 16 x 16 tiles marching along z.
#include "ark_step_inst.cuh"

namespace ark {

StepKernelInfo step_kernel_3d_f64(int visc)
{
    return visc ? step_info<3, double, false, true, 16, 16>() : step_info<3, double, false, false, 16, 16>();
}

}  // namespace ark
