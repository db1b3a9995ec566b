// ark_batch_inst.cuh -- description of one batched step-kernel instance.
#pragma once

#include "ark_aux.cuh"
#include "ark_step.cuh"

namespace ark {

template <typename Real, bool SPLIT, bool VISC, int TX>
BatchKernelInfo batch_info()
{
    using C = StepCfg<2, Real, SPLIT, VISC, TX, 1>;
    BatchKernelInfo k;
    k.func = reinterpret_cast<const void*>(&ark_batch_kernel<2, Real, SPLIT, VISC, TX, 1>);
    k.tx = TX;
    k.threads = TX;
    k.smem = C::SMEM_BYTES;
    return k;
}

}  // namespace ark
