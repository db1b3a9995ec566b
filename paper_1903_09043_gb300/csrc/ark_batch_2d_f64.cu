// ark_batch_2d_f64.cu -- batched 2D FP64 step kernels (ensembles of independent runs).
#include "ark_batch_inst.cuh"

namespace ark {

BatchKernelInfo batch_kernel_2d_f64(int visc, int width)
{
    if (width == 64) return visc ? batch_info<double, false, true, 64>() : batch_info<double, false, false, 64>();
    if (width == 128) return visc ? batch_info<double, false, true, 128>() : batch_info<double, false, false, 128>();
    if (width == 256) return visc ? batch_info<double, false, true, 256>() : batch_info<double, false, false, 256>();
    return BatchKernelInfo{nullptr, 0, 0, 0};
}

}  // namespace ark
