// ark_step_2d.cu -- 2D step-kernel instances: tile of 256 x 1 cells marching along y.
#include "ark_step_inst.cuh"

namespace ark {

StepKernelInfo step_kernel_2d(int prec, int visc)
{
    if (prec == P_F64) return visc ? step_info<2, double, false, true, 256, 1>() : step_info<2, double, false, false, 256, 1>();
    if (prec == P_F32) return visc ? step_info<2, float, false, true, 256, 1>() : step_info<2, float, false, false, 256, 1>();
    return visc ? step_info<2, float, true, true, 256, 1>() : step_info<2, float, true, false, 256, 1>();
}

}  // namespace ark
