// ark_step_2d.cu -- 2D step-kernel instances.  FP64: 256 x 1 tiles with
// strided phases (ark_step.cuh); FP32 forms: 124 x 1 tiles, one thread per
// column of the tile and halo (ark_step2.cuh), four 128-thread blocks per SM
// so that each barrier holds four warps rather than eight.  Both march along y.
#include "ark_step2_inst.cuh"
#include "ark_step_inst.cuh"

namespace ark {

StepKernelInfo step_kernel_2d(int prec, int visc)
{
    if (prec == P_F64) return visc ? step_info<2, double, false, true, 256, 1>() : step_info<2, double, false, false, 256, 1>();
    if (prec == P_F32) return visc ? step2_info<2, float, false, true, 128, 1>() : step2_info<2, float, false, false, 128, 1>();
    return visc ? step2_info<2, float, true, true, 128, 1>() : step2_info<2, float, true, false, 128, 1>();
}

}  // namespace ark
