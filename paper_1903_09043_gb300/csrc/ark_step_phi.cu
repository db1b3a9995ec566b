// ark_step_phi.cu -- step kernels for a caller-supplied potential array
// (ark_gravity.phi): the potential is read per cell and the gravity source
// acts on every face.  FP32: the column kernel; FP64: the plane-ring kernel.
#include "ark_step2_inst.cuh"
#include "ark_step_inst.cuh"

namespace ark {

StepKernelInfo step_kernel_phi_split(int dim, int visc);

StepKernelInfo step_kernel_phi(int dim, int prec, int visc)
{
    if (prec == P_F32_SPLIT) return step_kernel_phi_split(dim, visc);
    if (prec == P_F64) {
        if (dim == 2)
            return visc ? step_info<2, double, false, true, 256, 1, true>() : step_info<2, double, false, false, 256, 1, true>();
        return visc ? step_info<3, double, false, true, 16, 16, true>() : step_info<3, double, false, false, 16, 16, true>();
    }
    if (dim == 2)   // ARK_F32
        return visc ? step2_info<2, float, false, true, 256, 1, true>() : step2_info<2, float, false, false, 256, 1, true>();
    return visc ? step2_info<3, float, false, true, 32, 16, true>() : step2_info<3, float, false, false, 32, 16, true>();
}

}  // namespace ark
