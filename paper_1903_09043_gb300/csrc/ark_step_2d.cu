// ark_step_2d.cu -- 2D step-kernel instances.  FP64: 256 x 1 tiles with
// strided phases (ark_step.cuh); FP32 forms: 252 x 1 tiles, one thread per
// column of the tile and halo (ark_step2.cuh).  Both march along y.
#include "ark_step2_inst.cuh"
#include "ark_step_inst.cuh"

namespace ark {

StepKernelInfo step_kernel_2d(int prec, int visc)
{
    if (prec == P_F64) return visc ? step_info<2, double, false, true, 256, 1>() : step_info<2, double, false, false, 256, 1>();
    if (prec == P_F32) return visc ? step2_info<2, float, false, true, 256, 1>() : step2_info<2, float, false, false, 256, 1>();
    return visc ? step2_info<2, float, true, true, 256, 1>() : step2_info<2, float, true, false, 256, 1>();
}

}  // namespace ark
