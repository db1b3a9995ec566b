// ark_batch_2d_f32s.cu -- batched 2D FP32-split step kernels (ensembles of independent runs).
#include "ark_batch_inst.cuh"

namespace ark {

BatchKernelInfo batch_kernel_2d_f64(int visc, int tx);

BatchKernelInfo batch_kernel_2d(int prec, int visc, int tx)
{
    if (prec == P_F64) return batch_kernel_2d_f64(visc, tx);
    if (prec == P_F32_SPLIT) {
        if (tx == 64) return visc ? batch_info<float, true, true, 64>() : batch_info<float, true, false, 64>();
        if (tx == 128) return visc ? batch_info<float, true, true, 128>() : batch_info<float, true, false, 128>();
        if (tx == 256) return visc ? batch_info<float, true, true, 256>() : batch_info<float, true, false, 256>();
    }
    return BatchKernelInfo{nullptr, 0, 0, 0};
}

}  // namespace ark
