// ark_batch_2d_f32s.cu -- batched 2D FP32-split step kernels (ensembles of
// independent runs): one thread per column of a 64-, 128- or 256-wide
// tile-plus-halo (ark_step2.cuh).
#include "ark_step2_inst.cuh"

namespace ark {

BatchKernelInfo batch_kernel_2d_f64(int visc, int width);

BatchKernelInfo batch_kernel_2d(int prec, int visc, int width)
{
    if (prec == P_F64) return batch_kernel_2d_f64(visc, width);
    if (prec == P_F32_SPLIT) {
        if (width == 64) return visc ? batch2_info<float, true, true, 64>() : batch2_info<float, true, false, 64>();
        if (width == 128) return visc ? batch2_info<float, true, true, 128>() : batch2_info<float, true, false, 128>();
        if (width == 256) return visc ? batch2_info<float, true, true, 256>() : batch2_info<float, true, false, 256>();
    }
    return BatchKernelInfo{nullptr, 0, 0, 0};
}

}  // namespace ark
