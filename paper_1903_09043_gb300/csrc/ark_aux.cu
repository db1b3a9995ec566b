// ark_aux.cu -- CFL wave-rate reduction, state conversion, base-state row
// means and conservation diagnostics (GB300, sm_103a).
#include "ark_aux.cuh"
#include "ark_step.cuh"

namespace ark {

namespace {

constexpr int AUX_THREADS = 256;

__device__ __forceinline__ int row_of(const StepArgs& a, long long idx)
{
    const long long plane = a.dim == 3 ? (long long)a.n[0] * a.n[1] : (long long)a.n[0];
    return (int)(idx / plane);
}


// Wave rate of every cell; one atomicMax per block on the FP64 bit pattern
// (positive doubles order like their bit patterns, so the result does not
// depend on the order of the blocks).
template <int D, typename Real, bool SPLIT, bool VISC, bool NA>
__global__ void __launch_bounds__(AUX_THREADS) wave_rate_kernel(const __grid_constant__ StepArgs a, const Real* __restrict__ U,
                                                                  unsigned long long* slot)
{
    __shared__ double red[AUX_THREADS];
    const int nv = a.n[D - 1];
    const PhiRow<Real> ph(a);
    const KConst<Real> kc(a);
    const Eos<Real, NA> eos(kc);
    const Real mu = kc.mu, kappa = kc.kappa;
    const Real invdx[3] = {kc.invdx[0], kc.invdx[1], kc.invdx[2]};
    Real smax = Real(0);
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < a.ncell;
         idx += (long long)gridDim.x * blockDim.x) {
        Real b[D + 2];
#pragma unroll
        for (int k = 0; k < D + 2; ++k) b[k] = __ldg(U + k * a.ncell + idx);
        Row<Real> w = row_info<Real, SPLIT>(a, ph, row_of(a, idx), nv);
        if (a.phiA && !a.energy_form) w.phi = __ldg(static_cast<const Real*>(a.phiA) + idx);   // caller's Phi
        Real p, rho;
        const Real sh = wave_rate<D, Real, SPLIT, VISC>(b, w, eos, invdx, mu, kappa, p, rho);
        if (!(sh <= smax)) smax = (sh == sh) ? sh : smax;
    }
    block_rate_max(double(smax), reinterpret_cast<unsigned long long*>(red), slot);
}

template <int D, typename Real, bool SPLIT>
__global__ void __launch_bounds__(AUX_THREADS) convert_in_kernel(const StepArgs a, const double* __restrict__ Uin,
                                                                   Real* __restrict__ Uout)
{
    const int nv = a.n[D - 1];
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < a.ncell;
         idx += (long long)gridDim.x * blockDim.x) {
        const int r = row_of(a, idx);
        double rho = Uin[idx], W = Uin[(D + 1) * a.ncell + idx];
        if constexpr (SPLIT) {
            rho -= a.base64[0 * (nv + 4) + r + 2];
            W -= a.base64[2 * (nv + 4) + r + 2];
        }
        Uout[idx] = Real(rho);
#pragma unroll
        for (int d = 0; d < D; ++d) Uout[(1 + d) * a.ncell + idx] = Real(Uin[(1 + d) * a.ncell + idx]);
        Uout[(D + 1) * a.ncell + idx] = Real(W);
    }
}

template <int D, typename Real, bool SPLIT>
__global__ void __launch_bounds__(AUX_THREADS) convert_out_kernel(const StepArgs a, const Real* __restrict__ Uin,
                                                                    double* __restrict__ Uout)
{
    const int nv = a.n[D - 1];
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < a.ncell;
         idx += (long long)gridDim.x * blockDim.x) {
        const int r = row_of(a, idx);
        double rho = double(Uin[idx]), W = double(Uin[(D + 1) * a.ncell + idx]);
        if constexpr (SPLIT) {
            rho += a.base64[0 * (nv + 4) + r + 2];
            W += a.base64[2 * (nv + 4) + r + 2];
        }
        Uout[idx] = rho;
#pragma unroll
        for (int d = 0; d < D; ++d) Uout[(1 + d) * a.ncell + idx] = double(Uin[(1 + d) * a.ncell + idx]);
        Uout[(D + 1) * a.ncell + idx] = W;
    }
}

// Halo layers of a slab decomposition along x.  Element e of the FP64 buffer
// [NF][nv][ny][2] is field f, plane k, row j, layer l (l = 0 at the side).
__device__ __forceinline__ void halo_decode(const StepArgs& a, int D, long long e, int& f, int& l, int& j, int& k)
{
    const int nv = a.n[D - 1], ny = D == 3 ? a.n[1] : 1;
    const long long per = (long long)nv * ny * 2;
    f = (int)(e / per);
    const long long r = e - (long long)f * per;
    l = (int)(r & 1);
    const long long jk = r >> 1;
    j = (int)(jk % ny);
    k = (int)(jk / ny);
}

template <int D, typename Real, bool SPLIT>
__global__ void __launch_bounds__(AUX_THREADS) halo_get_kernel(const StepArgs a, int side, const Real* __restrict__ U,
                                                                 double* __restrict__ out)
{
    const int nv = a.n[D - 1], nx = a.n[0], ny = D == 3 ? a.n[1] : 1;
    const long long total = (long long)(D + 2) * nv * ny * 2;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        int f, l, j, k;
        halo_decode(a, D, e, f, l, j, k);
        const int x = side == 0 ? l : nx - 1 - l;
        const long long idx = x + (long long)nx * (j + (long long)ny * k);
        double v = double(U[f * a.ncell + idx]);
        if constexpr (SPLIT) {   // deviations back to full values with the FP64 base row
            if (f == 0) v += a.base64[0 * (nv + 4) + k + 2];
            if (f == D + 1) v += a.base64[2 * (nv + 4) + k + 2];
        }
        out[e] = v;
    }
}

template <int D, typename Real, bool SPLIT>
__global__ void __launch_bounds__(AUX_THREADS) halo_set_kernel(const StepArgs a, const double* __restrict__ in,
                                                                 Real* __restrict__ H)
{
    const int nv = a.n[D - 1], ny = D == 3 ? a.n[1] : 1;
    const long long total = (long long)(D + 2) * nv * ny * 2;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        int f, l, j, k;
        halo_decode(a, D, e, f, l, j, k);
        double v = in[e];
        if constexpr (SPLIT) {   // this subdomain's base row
            if (f == 0) v -= a.base64[0 * (nv + 4) + k + 2];
            if (f == D + 1) v -= a.base64[2 * (nv + 4) + k + 2];
        }
        H[e] = Real(v);
    }
}

// Horizontal means of rho and p, pass 1: block (r, c) sums chunk c of row r
// (ROW_CHUNK cells; fixed-order tree sums) into part[r * chunks + c].  NA:
// the covolume law divides p by 1 - b rho; the stiffened gas (b = 0) skips
// that division, one of the two FP64 divisions per cell of this FP64-bound
// pass.
constexpr long long ROW_CHUNK = 8192;
template <int D, bool NA>
__global__ void __launch_bounds__(AUX_THREADS) row_means_kernel(const StepArgs a, const double* __restrict__ U,
                                                                  double* part_r, double* part_p)
{
    __shared__ double sr[AUX_THREADS], sp[AUX_THREADS];
    const int r = blockIdx.x, c = blockIdx.y, chunks = gridDim.y;   // rows in x: no 65535 limit
    const long long plane = D == 3 ? (long long)a.n[0] * a.n[1] : (long long)a.n[0];
    // a caller's potential (split form: separable, one value per row) from the
    // FP64 row table, else the uniform-gravity potential
    const double phi = a.phiA ? a.base64[3 * (a.n[D - 1] + 4) + r + 2] : -(a.g * (a.lo_v + (r + 0.5) * a.dx[D - 1]));
    const long long i1 = min(plane, (c + 1) * ROW_CHUNK);
    double accr = 0.0, accp = 0.0;
    for (long long i = c * ROW_CHUNK + threadIdx.x; i < i1; i += AUX_THREADS) {
        const long long idx = r * plane + i;
        const double rho = U[idx];
        double m2 = 0.0;
#pragma unroll
        for (int d = 0; d < D; ++d) {
            const double m = U[(1 + d) * a.ncell + idx];
            m2 += m * m;
        }
        const double ke = 0.5 * m2 / rho;
        accr += rho;
        const double re = (a.gamma - 1.0) * (U[(D + 1) * a.ncell + idx] - ke - rho * phi);
        accp += (NA ? re / (1.0 - a.b * rho) : re) - a.dgpinf;
    }
    sr[threadIdx.x] = accr;
    sp[threadIdx.x] = accp;
    __syncthreads();
    for (int s = AUX_THREADS / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            sr[threadIdx.x] += sr[threadIdx.x + s];
            sp[threadIdx.x] += sp[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part_r[(long long)r * chunks + c] = sr[0];
        part_p[(long long)r * chunks + c] = sp[0];
    }
}

// Pass 2: one thread per row sums its chunks in order.
__global__ void row_means_final_kernel(const double* __restrict__ part_r, const double* __restrict__ part_p,
                                       int chunks, int nv, double plane, double* rho_mean, double* p_mean)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nv) return;
    double sr = 0.0, sp = 0.0;
    for (int c = 0; c < chunks; ++c) {
        sr += part_r[(long long)r * chunks + c];
        sp += part_p[(long long)r * chunks + c];
    }
    rho_mean[r] = sr / plane;
    p_mean[r] = sp / plane;
}

template <int D, typename Real, bool SPLIT>
__global__ void __launch_bounds__(AUX_THREADS) diag_kernel(const StepArgs a, const Real* __restrict__ U,
                                                             double* partials)
{
    __shared__ double red[DG_NTOT][AUX_THREADS];
    const int nv = a.n[D - 1];
    double acc[DG_NTOT];
#pragma unroll
    for (int k = 0; k < DG_NSUM; ++k) acc[k] = 0.0;
    acc[DG_UMAX] = 0.0;
    acc[DG_RMIN] = INFINITY;
    acc[DG_PMIN] = INFINITY;
    acc[DG_NAN] = 0.0;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < a.ncell;
         idx += (long long)gridDim.x * blockDim.x) {
        const int r = row_of(a, idx);
        double phi = a.energy_form ? 0.0 : -(a.g * (a.lo_v + (r + 0.5) * a.dx[D - 1]));
        if (a.phiA && !a.energy_form)   // caller's Phi (split form: the FP64 row value)
            phi = SPLIT ? a.base64[3 * (nv + 4) + r + 2] : double(static_cast<const Real*>(a.phiA)[idx]);
        double rho = double(U[idx]), W = double(U[(D + 1) * a.ncell + idx]);
        if constexpr (SPLIT) {
            rho += a.base64[0 * (nv + 4) + r + 2];
            W += a.base64[2 * (nv + 4) + r + 2];
        }
        double m[3] = {0.0, 0.0, 0.0}, ke = 0.0, u2 = 0.0;
#pragma unroll
        for (int d = 0; d < D; ++d) {
            m[d] = double(U[(1 + d) * a.ncell + idx]);
            const double u = m[d] / rho;
            ke += 0.5 * rho * u * u;
            u2 += u * u;
        }
        const double p = (a.gamma - 1.0) * (W - ke - rho * phi) / (1.0 - a.b * rho) - a.dgpinf;   // covolume b
        acc[DG_MASS] += rho;
        acc[DG_MX] += m[0];
        acc[DG_MY] += m[1];
        acc[DG_MZ] += m[2];
        acc[DG_W] += W;
        acc[DG_KE] += ke;
        acc[DG_VABS] += fabs(m[D - 1] / rho);
        acc[DG_UMAX] = fmax(acc[DG_UMAX], sqrt(u2));
        acc[DG_RMIN] = fmin(acc[DG_RMIN], rho);
        acc[DG_PMIN] = fmin(acc[DG_PMIN], p);
        if (!(p == p) || !(rho == rho) || !(W == W)) acc[DG_NAN] += 1.0;
    }
#pragma unroll
    for (int k = 0; k < DG_NTOT; ++k) red[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int s = AUX_THREADS / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
#pragma unroll
            for (int k = 0; k < DG_NSUM; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + s];
            red[DG_UMAX][threadIdx.x] = fmax(red[DG_UMAX][threadIdx.x], red[DG_UMAX][threadIdx.x + s]);
            red[DG_RMIN][threadIdx.x] = fmin(red[DG_RMIN][threadIdx.x], red[DG_RMIN][threadIdx.x + s]);
            red[DG_PMIN][threadIdx.x] = fmin(red[DG_PMIN][threadIdx.x], red[DG_PMIN][threadIdx.x + s]);
            red[DG_NAN][threadIdx.x] += red[DG_NAN][threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x < DG_NTOT) partials[blockIdx.x * DG_NTOT + threadIdx.x] = red[threadIdx.x][0];
}

__global__ void diag_final_kernel(const double* partials, int nblocks, double* out)
{
    // the partials are staged in shared memory by the whole block (coalesced),
    // then one thread per quantity sums them in block index order: a fixed
    // summation order, without a chain of dependent global loads
    extern __shared__ double sp[];
    for (int i = threadIdx.x; i < nblocks * DG_NTOT; i += blockDim.x) sp[i] = partials[i];
    __syncthreads();
    const int k = threadIdx.x;
    if (k >= DG_NTOT) return;
    double v = sp[k];
    for (int b = 1; b < nblocks; ++b) {
        const double x = sp[b * DG_NTOT + k];
        if (k < DG_NSUM || k == DG_NAN) v += x;
        else if (k == DG_UMAX) v = fmax(v, x);
        else v = fmin(v, x);
    }
    out[k] = v;
}

int grid_for(long long n)
{
    long long b = (n + AUX_THREADS - 1) / AUX_THREADS;
    if (b > 152 * 16) b = 152 * 16;
    if (b < 1) b = 1;
    return (int)b;
}

}  // namespace

cudaError_t launch_wave_rate(const StepArgs& a, int prec, int visc, const void* U, unsigned long long* slot,
                             cudaStream_t s)
{
    const int g = grid_for(a.ncell);
    // a covolume takes the Noble-Abel instances; b = 0 is the stiffened gas
#define ARK_WR(D, R, SP, VI)                                                                    \
    do {                                                                                        \
        if (a.b != 0.0) wave_rate_kernel<D, R, SP, VI, true><<<g, AUX_THREADS, 0, s>>>(a, (const R*)U, slot); \
        else wave_rate_kernel<D, R, SP, VI, false><<<g, AUX_THREADS, 0, s>>>(a, (const R*)U, slot);           \
    } while (0)
    if (a.dim == 2) {
        if (prec == P_F64) { if (visc) ARK_WR(2, double, false, true); else ARK_WR(2, double, false, false); }
        else if (prec == P_F32) { if (visc) ARK_WR(2, float, false, true); else ARK_WR(2, float, false, false); }
        else { if (visc) ARK_WR(2, float, true, true); else ARK_WR(2, float, true, false); }
    } else {
        if (prec == P_F64) { if (visc) ARK_WR(3, double, false, true); else ARK_WR(3, double, false, false); }
        else if (prec == P_F32) { if (visc) ARK_WR(3, float, false, true); else ARK_WR(3, float, false, false); }
        else { if (visc) ARK_WR(3, float, true, true); else ARK_WR(3, float, true, false); }
    }
#undef ARK_WR
    return cudaGetLastError();
}

cudaError_t launch_halo_get(const StepArgs& a, int prec, int side, const void* U, double* out, cudaStream_t s)
{
    const long long total = (long long)(a.dim + 2) * a.n[a.dim - 1] * (a.dim == 3 ? a.n[1] : 1) * 2;
    const int g = grid_for(total);
#define ARK_HG(D, R, SP) halo_get_kernel<D, R, SP><<<g, AUX_THREADS, 0, s>>>(a, side, (const R*)U, out)
    if (a.dim == 2) {
        if (prec == P_F64) ARK_HG(2, double, false); else if (prec == P_F32) ARK_HG(2, float, false); else ARK_HG(2, float, true);
    } else {
        if (prec == P_F64) ARK_HG(3, double, false); else if (prec == P_F32) ARK_HG(3, float, false); else ARK_HG(3, float, true);
    }
#undef ARK_HG
    return cudaGetLastError();
}

cudaError_t launch_halo_set(const StepArgs& a, int prec, const double* in, void* halo, cudaStream_t s)
{
    const long long total = (long long)(a.dim + 2) * a.n[a.dim - 1] * (a.dim == 3 ? a.n[1] : 1) * 2;
    const int g = grid_for(total);
#define ARK_HS(D, R, SP) halo_set_kernel<D, R, SP><<<g, AUX_THREADS, 0, s>>>(a, in, (R*)halo)
    if (a.dim == 2) {
        if (prec == P_F64) ARK_HS(2, double, false); else if (prec == P_F32) ARK_HS(2, float, false); else ARK_HS(2, float, true);
    } else {
        if (prec == P_F64) ARK_HS(3, double, false); else if (prec == P_F32) ARK_HS(3, float, false); else ARK_HS(3, float, true);
    }
#undef ARK_HS
    return cudaGetLastError();
}

cudaError_t launch_convert_in(const StepArgs& a, int prec, const double* Uin, void* Uout, cudaStream_t s)
{
    const int g = grid_for(a.ncell);
    if (a.dim == 2) {
        if (prec == P_F64) convert_in_kernel<2, double, false><<<g, AUX_THREADS, 0, s>>>(a, Uin, (double*)Uout);
        else if (prec == P_F32) convert_in_kernel<2, float, false><<<g, AUX_THREADS, 0, s>>>(a, Uin, (float*)Uout);
        else convert_in_kernel<2, float, true><<<g, AUX_THREADS, 0, s>>>(a, Uin, (float*)Uout);
    } else {
        if (prec == P_F64) convert_in_kernel<3, double, false><<<g, AUX_THREADS, 0, s>>>(a, Uin, (double*)Uout);
        else if (prec == P_F32) convert_in_kernel<3, float, false><<<g, AUX_THREADS, 0, s>>>(a, Uin, (float*)Uout);
        else convert_in_kernel<3, float, true><<<g, AUX_THREADS, 0, s>>>(a, Uin, (float*)Uout);
    }
    return cudaGetLastError();
}

cudaError_t launch_convert_out(const StepArgs& a, int prec, const void* Uin, double* Uout, cudaStream_t s)
{
    const int g = grid_for(a.ncell);
    if (a.dim == 2) {
        if (prec == P_F64) convert_out_kernel<2, double, false><<<g, AUX_THREADS, 0, s>>>(a, (const double*)Uin, Uout);
        else if (prec == P_F32) convert_out_kernel<2, float, false><<<g, AUX_THREADS, 0, s>>>(a, (const float*)Uin, Uout);
        else convert_out_kernel<2, float, true><<<g, AUX_THREADS, 0, s>>>(a, (const float*)Uin, Uout);
    } else {
        if (prec == P_F64) convert_out_kernel<3, double, false><<<g, AUX_THREADS, 0, s>>>(a, (const double*)Uin, Uout);
        else if (prec == P_F32) convert_out_kernel<3, float, false><<<g, AUX_THREADS, 0, s>>>(a, (const float*)Uin, Uout);
        else convert_out_kernel<3, float, true><<<g, AUX_THREADS, 0, s>>>(a, (const float*)Uin, Uout);
    }
    return cudaGetLastError();
}

static int row_chunks(const StepArgs& a)
{
    const long long plane = a.dim == 3 ? (long long)a.n[0] * a.n[1] : (long long)a.n[0];
    return (int)((plane + ROW_CHUNK - 1) / ROW_CHUNK);
}

size_t row_means_scratch(const StepArgs& a) { return 2 * (size_t)a.n[a.dim - 1] * (size_t)row_chunks(a); }

cudaError_t launch_row_means(const StepArgs& a, const double* U, double* scratch, double* rho_mean, double* p_mean,
                             cudaStream_t s)
{
    const int nv = a.n[a.dim - 1], chunks = row_chunks(a);
    const long long plane = a.dim == 3 ? (long long)a.n[0] * a.n[1] : (long long)a.n[0];
    double* part_r = scratch;
    double* part_p = scratch + (size_t)nv * chunks;
    const dim3 grid((unsigned)nv, (unsigned)chunks);
    const bool na = a.b != 0.0;
    if (a.dim == 2) {
        if (na) row_means_kernel<2, true><<<grid, AUX_THREADS, 0, s>>>(a, U, part_r, part_p);
        else row_means_kernel<2, false><<<grid, AUX_THREADS, 0, s>>>(a, U, part_r, part_p);
    } else {
        if (na) row_means_kernel<3, true><<<grid, AUX_THREADS, 0, s>>>(a, U, part_r, part_p);
        else row_means_kernel<3, false><<<grid, AUX_THREADS, 0, s>>>(a, U, part_r, part_p);
    }
    row_means_final_kernel<<<(nv + 127) / 128, 128, 0, s>>>(part_r, part_p, chunks, nv, double(plane), rho_mean, p_mean);
    return cudaGetLastError();
}

cudaError_t launch_diagnostics(const StepArgs& a, int prec, const void* U, double* partials, double* out,
                               cudaStream_t s)
{
    const int g = DIAG_BLOCKS;
    if (a.dim == 2) {
        if (prec == P_F64) diag_kernel<2, double, false><<<g, AUX_THREADS, 0, s>>>(a, (const double*)U, partials);
        else if (prec == P_F32) diag_kernel<2, float, false><<<g, AUX_THREADS, 0, s>>>(a, (const float*)U, partials);
        else diag_kernel<2, float, true><<<g, AUX_THREADS, 0, s>>>(a, (const float*)U, partials);
    } else {
        if (prec == P_F64) diag_kernel<3, double, false><<<g, AUX_THREADS, 0, s>>>(a, (const double*)U, partials);
        else if (prec == P_F32) diag_kernel<3, float, false><<<g, AUX_THREADS, 0, s>>>(a, (const float*)U, partials);
        else diag_kernel<3, float, true><<<g, AUX_THREADS, 0, s>>>(a, (const float*)U, partials);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    diag_final_kernel<<<1, 256, (size_t)g * DG_NTOT * sizeof(double), s>>>(partials, g, out);
    return cudaGetLastError();
}

}  // namespace ark
