// ark_aux.cuh -- launchers of the non-step kernels and lookup of the step
// kernel instances, used by the host API.
#pragma once

#include <cuda_runtime.h>

#include "ark_common.cuh"

namespace ark {

// CFL wave rate max over all cells of U -> atomicMax into *slot (FP64 bits).
cudaError_t launch_wave_rate(const StepArgs& a, int prec, int visc, const void* U, unsigned long long* slot,
                             cudaStream_t s);

// FP64 full state (device) -> storage state (deviation form for F32_SPLIT), and back.
cudaError_t launch_convert_in(const StepArgs& a, int prec, const double* Uin, void* Uout, cudaStream_t s);
cudaError_t launch_convert_out(const StepArgs& a, int prec, const void* Uin, double* Uout, cudaStream_t s);

// Slab decomposition along x (BC_HALO): the two cell layers next to x side
// `side` (0: low, 1: high) as FP64 full values [NF][nv][ny][2], layer 0 at the
// side; and FP64 ghost layers into a halo buffer of the state's form.
cudaError_t launch_halo_get(const StepArgs& a, int prec, int side, const void* U, double* out, cudaStream_t s);
cudaError_t launch_halo_set(const StepArgs& a, int prec, const double* in, void* halo, cudaStream_t s);

// Horizontal means of rho and p of an FP64 full state, one per row of the last
// axis: per-chunk partial sums into `scratch` (row_means_scratch(a) doubles),
// then each row's chunks summed in order.
size_t row_means_scratch(const StepArgs& a);
cudaError_t launch_row_means(const StepArgs& a, const double* U, double* scratch, double* rho_mean, double* p_mean,
                             cudaStream_t s);

// Diagnostics: per-block FP64 partial sums in a fixed order, then one fixed-order reduction.
enum { DG_MASS = 0, DG_MX, DG_MY, DG_MZ, DG_W, DG_KE, DG_VABS, DG_NSUM };
enum { DG_UMAX = DG_NSUM, DG_RMIN, DG_PMIN, DG_NAN, DG_NTOT };
constexpr int DIAG_BLOCKS = 304;
cudaError_t launch_diagnostics(const StepArgs& a, int prec, const void* U, double* partials, double* out,
                               cudaStream_t s);

// Step kernel instances (ark_step_*.cu).
using StepLauncher = cudaError_t (*)(const StepArgs&, dim3 grid, cudaStream_t);
struct StepKernelInfo {
    StepLauncher launch;
    int tx, ty, threads;
    size_t smem;
    int blocks_per_sm;
    bool balanced = false;   // grid of resident blocks, each an equal share of (tile, plane) units
};
StepKernelInfo step_kernel_2d(int prec, int visc);
StepKernelInfo step_kernel_3d(int prec, int visc);
StepKernelInfo step_kernel_phi(int dim, int prec, int visc);   // caller-supplied potential array
StepKernelInfo step_kernel_noble_abel(int dim, int prec, int visc);   // covolume (Noble-Abel stiffened gas)

// Batched 2D step-kernel instances (ark_batch_2d*.cu): tile widths 64, 128, 256.
struct BatchKernelInfo {
    const void* func;   // ark_batch_kernel instance (argument list: runs, items, nitems, ctr, ctr_cur, ctr_next)
    int tx, threads;
    size_t smem;        // dynamic shared memory per block
};
BatchKernelInfo batch_kernel_2d(int prec, int visc, int width);   // width: 64, 128, 256 threads per row; func == nullptr if not built

}  // namespace ark
