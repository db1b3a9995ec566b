// ark_step2_inst.cuh -- launchers of the column-per-thread step kernels.
#pragma once

#include "ark_aux.cuh"
#include "ark_step2.cuh"

namespace ark {

template <int DIM, typename Real, bool SPLIT, bool VISC, int R2X, int R2Y, bool PHIA = false, bool NA = false>
cudaError_t launch_step2_impl(const StepArgs& a, dim3 grid, cudaStream_t s)
{
    using C = Step2Cfg<DIM, Real, SPLIT, VISC, R2X, R2Y, PHIA>;
    static int attr_device = -1;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (attr_device != dev) {
        e = cudaFuncSetAttribute(ark_step2_kernel<DIM, Real, SPLIT, VISC, R2X, R2Y, PHIA, NA>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM_BYTES);
        if (e != cudaSuccess) return e;
        attr_device = dev;
    }
    ark_step2_kernel<DIM, Real, SPLIT, VISC, R2X, R2Y, PHIA, NA><<<grid, C::NT, C::SMEM_BYTES, s>>>(a);
    return cudaGetLastError();
}

template <int DIM, typename Real, bool SPLIT, bool VISC, int R2X, int R2Y, bool PHIA = false, bool NA = false>
StepKernelInfo step2_info()
{
    using C = Step2Cfg<DIM, Real, SPLIT, VISC, R2X, R2Y, PHIA>;
    StepKernelInfo k;
    k.launch = &launch_step2_impl<DIM, Real, SPLIT, VISC, R2X, R2Y, PHIA, NA>;
    k.tx = C::TX;
    k.ty = C::TY;
    k.threads = C::NT;
    k.smem = C::SMEM_BYTES;
    k.blocks_per_sm = 512 / C::NT;
    k.balanced = true;
    return k;
}

template <typename Real, bool SPLIT, bool VISC, int R2X>
BatchKernelInfo batch2_info()
{
    using C = Step2Cfg<2, Real, SPLIT, VISC, R2X, 1, false, true>;
    BatchKernelInfo k;
    k.func = reinterpret_cast<const void*>(&ark_batch2_kernel<2, Real, SPLIT, VISC, R2X, 1>);
    k.tx = C::TX;
    k.threads = C::NT;
    k.smem = C::SMEM_BYTES;
    return k;
}

}  // namespace ark
