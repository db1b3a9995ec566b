// ark_step_inst.cuh -- launcher of one step-kernel instance.
#pragma once

#include "ark_aux.cuh"
#include "ark_step.cuh"

namespace ark {

template <int DIM, typename Real, bool SPLIT, bool VISC, int TX, int TY, bool PHIA = false, bool NA = false>
cudaError_t launch_step_impl(const StepArgs& a, dim3 grid, cudaStream_t s)
{
    using C = StepCfg<DIM, Real, SPLIT, VISC, TX, TY, PHIA>;
    static int attr_device = -1;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (attr_device != dev) {
        e = cudaFuncSetAttribute(ark_step_kernel<DIM, Real, SPLIT, VISC, TX, TY, PHIA, NA>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM_BYTES);
        if (e != cudaSuccess) return e;
        attr_device = dev;
    }
    ark_step_kernel<DIM, Real, SPLIT, VISC, TX, TY, PHIA, NA><<<grid, C::NT, C::SMEM_BYTES, s>>>(a);
    return cudaGetLastError();
}

template <int DIM, typename Real, bool SPLIT, bool VISC, int TX, int TY, bool PHIA = false, bool NA = false>
StepKernelInfo step_info()
{
    using C = StepCfg<DIM, Real, SPLIT, VISC, TX, TY, PHIA>;
    StepKernelInfo k;
    k.launch = &launch_step_impl<DIM, Real, SPLIT, VISC, TX, TY, PHIA, NA>;
    k.tx = TX;
    k.ty = TY;
    k.threads = C::NT;
    k.smem = C::SMEM_BYTES;
    const size_t per_sm = 228 * 1024;
    int b = (int)(per_sm / (C::SMEM_BYTES + 1024));
    if (b < 1) b = 1;
    if (b * C::NT > 2048) b = 2048 / C::NT;
    // Registers can leave room for fewer blocks than shared memory does (the 2D
    // FP64 kernel: two blocks' rings fit, one block's registers): take the
    // runtime's count when no earlier error is pending, else the estimate.
    if (cudaPeekAtLastError() == cudaSuccess) {
        const auto f = ark_step_kernel<DIM, Real, SPLIT, VISC, TX, TY, PHIA, NA>;
        int occ = 0;
        if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM_BYTES) == cudaSuccess &&
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, f, C::NT, C::SMEM_BYTES) == cudaSuccess) {
            if (occ >= 1) b = occ;
        } else {
            cudaGetLastError();   // the query's own error; nothing else was pending
        }
    }
    k.blocks_per_sm = b;
    k.balanced = true;
    return k;
}

}  // namespace ark
