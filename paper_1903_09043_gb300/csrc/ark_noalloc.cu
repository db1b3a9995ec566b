// ark_noalloc.cu -- the CFL time step of a caller's FP64 state, computed
// without allocating any device memory (ark_compute_dt_noalloc in ark.h).
//
// Some callers cannot allocate device memory at the moment they need a time
// step: code running inside a memory pool or arena that owns every byte of the
// device, a host that must not trigger an allocation (which can synchronise
// the device or fail when memory is exhausted), or an embedding runtime that
// forbids library allocations.  This entry point needs no handle: its only
// scratch is a fixed array in the library's own device image.
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/ark.h"
#include "ark_handle.h"
#include "ark_step.cuh"

namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_CELLS_PER_THREAD = 16;
constexpr long long NA_CELLS_PER_BLOCK = (long long)NA_THREADS * NA_CELLS_PER_THREAD;   // 4096 cells
constexpr int NA_MAX_BLOCKS = 16384;                                                      // 128 KiB of scratch
constexpr long long NA_MAX_CELLS = NA_CELLS_PER_BLOCK * NA_MAX_BLOCKS;                   // 67,108,864 cells
constexpr int NA_MAX_DEVICES = 64;

// One wave-rate maximum per block of the first pass (NaN for a block that saw
// a bad cell).  Every device that loads the library holds this array until the
// process exits.  Each call writes the slots it then reads, so nothing needs
// clearing between calls; two calls that overlap on the GPU (different
// streams, no ordering) race on it.
static __device__ __align__(256) double ark_noalloc_scratch[NA_MAX_BLOCKS];

std::mutex g_setup_mutex;
double* g_scratch[NA_MAX_DEVICES] = {};   // device address of the array, per device ordinal

template <int D, bool VISC>
__global__ void __launch_bounds__(NA_THREADS) na_rate_kernel(const __grid_constant__ ark::StepArgs a,
                                                               const double* __restrict__ U, double* partial)
{
    __shared__ double red[NA_THREADS];
    const int nv = a.n[D - 1];
    const ark::PhiRow<double> ph(a);
    const ark::Eos<double> eos{ark::KConst<double>(a)};
    const double invdx[3] = {1.0 / a.dx[0], 1.0 / a.dx[1], 1.0 / a.dx[2]};
    const long long plane = D == 3 ? (long long)a.n[0] * a.n[1] : (long long)a.n[0];
    double m = 0.0;
    int bad = 0;   // a cell with rho <= 0, p + p_inf <= 0 or a NaN rate
    for (int k = 0; k < NA_CELLS_PER_THREAD; ++k) {
        const long long idx = blockIdx.x * NA_CELLS_PER_BLOCK + k * NA_THREADS + threadIdx.x;
        if (idx >= a.ncell) break;
        double b[D + 2];
#pragma unroll
        for (int f = 0; f < D + 2; ++f) b[f] = __ldg(U + f * a.ncell + idx);
        const ark::Row<double> w = ark::row_info<double, false>(a, ph, (int)(idx / plane), nv);
        double pe, rho;
        const double s = ark::wave_rate<D, double, false, VISC>(b, w, eos, invdx, a.mu, a.kappa, pe, rho);
        if (!(rho > 0.0) || !(pe > 0.0) || s != s) bad = 1;
        else if (s > m) m = s;
    }
    red[threadIdx.x] = m;
    // one flag for the block: every slot of the first pass is written on every
    // call, NaN when the block saw a bad cell
    bad = __syncthreads_or(bad);
    for (int s = NA_THREADS / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = bad ? __longlong_as_double(0x7ff8000000000000ll) : red[0];
}

__global__ void __launch_bounds__(NA_THREADS) na_final_kernel(const double* partial, int nblocks, double cfl,
                                                                double* dt_out)
{
    __shared__ double red[NA_THREADS];
    double m = 0.0;
    int bad = 0;
    for (int i = threadIdx.x; i < nblocks; i += NA_THREADS) {
        const double v = partial[i];
        if (v != v) bad = 1;
        else m = fmax(m, v);
    }
    red[threadIdx.x] = m;
    bad = __syncthreads_or(bad);
    for (int s = NA_THREADS / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
        __syncthreads();
    }
    // a bad state yields NaN rather than a finite step from its healthy cells
    if (threadIdx.x == 0) *dt_out = bad ? __longlong_as_double(0x7ff8000000000000ll) : cfl / red[0];
}

// Device address of the scratch array on the current device, looked up once
// per device ordinal and kept for the life of the process.  A cudaDeviceReset
// unloads the module and makes the kept address stale, so the entry point
// must not be used across a reset.
cudaError_t scratch_for_current_device(double** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= NA_MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch[dev]) {
        double* ptr = nullptr;
        e = cudaGetSymbolAddress((void**)&ptr, ark_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch[dev] = ptr;
    }
    *out = g_scratch[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" ark_status ark_compute_dt_noalloc(const ark_params* p, const double* U, double* dt, void* stream)
{
    if (!p || !U || !dt) return ARK_ERR_INVALID_ARG;
    std::string msg;
    const ark_status vs = ark::validate_params(p, msg);   // the rules of ark_create
    if (vs != ARK_OK) return vs;
    if (p->precision != ARK_F64) return ARK_ERR_INVALID_ARG;
    if (p->gravity.phi) return ARK_ERR_UNSUPPORTED;   // the potential array would need a device copy
    if (p->eos.law != ARK_EOS_STIFFENED_GAS) return ARK_ERR_UNSUPPORTED;   // the stiffened-gas rate only
    const int dim = p->grid.dim;
    long long ncell = 1;
    ark::StepArgs a;
    memset(&a, 0, sizeof a);
    a.dim = dim;
    for (int d = 0; d < 3; ++d) {
        if (d < dim) {
            a.n[d] = p->grid.n[d];
            a.dx[d] = (p->grid.hi[d] - p->grid.lo[d]) / p->grid.n[d];
            ncell *= p->grid.n[d];
        } else {
            a.n[d] = 1;
            a.dx[d] = 1.0;
        }
    }
    if (ncell > NA_MAX_CELLS) return ARK_ERR_INVALID_ARG;   // beyond the fixed scratch
    a.gamma = p->eos.gamma;
    a.p_inf = p->eos.p_inf;
    a.g = p->gravity.g;
    a.lo_v = p->grid.lo[dim - 1];
    a.mu = p->mu;
    a.kappa = p->kappa;
    a.cfl = p->cfl;
    a.energy_form = p->energy_form;
    a.K = p->K;
    a.ncell = ncell;
    ark::fill_constants(a);

    // an error already pending from the caller's earlier work is left for the
    // caller and reported here without launching anything
    if (cudaPeekAtLastError() != cudaSuccess) return ARK_ERR_CUDA;
    double* scratch = nullptr;
    if (scratch_for_current_device(&scratch) != cudaSuccess) return ARK_ERR_CUDA;
    const int nblocks = (int)((ncell + NA_CELLS_PER_BLOCK - 1) / NA_CELLS_PER_BLOCK);
    cudaStream_t s = (cudaStream_t)stream;
    const bool visc = p->mu > 0.0 || p->kappa > 0.0;
    if (dim == 2) {
        if (visc) na_rate_kernel<2, true><<<nblocks, NA_THREADS, 0, s>>>(a, U, scratch);
        else na_rate_kernel<2, false><<<nblocks, NA_THREADS, 0, s>>>(a, U, scratch);
    } else {
        if (visc) na_rate_kernel<3, true><<<nblocks, NA_THREADS, 0, s>>>(a, U, scratch);
        else na_rate_kernel<3, false><<<nblocks, NA_THREADS, 0, s>>>(a, U, scratch);
    }
    if (cudaGetLastError() != cudaSuccess) return ARK_ERR_CUDA;
    na_final_kernel<<<1, NA_THREADS, 0, s>>>(scratch, nblocks, p->cfl, dt);
    if (cudaGetLastError() != cudaSuccess) return ARK_ERR_CUDA;
    return ARK_OK;
}
