// ark_api.cu -- host implementation of the C ABI declared in include/ark.h.
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "../../include/ark.h"
#include "ark_aux.cuh"
#include "ark_base.h"
#include "ark_handle.h"

namespace {

ark_status fail(ark_handle* h, ark_status s, const std::string& msg)
{
    if (h) h->err = msg;
    return s;
}

ark_status cuda_fail(ark_handle* h, cudaError_t e, const char* where)
{
    return fail(h, ARK_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define ARK_CUDA(h, call)                                           \
    do {                                                            \
        cudaError_t e_ = (call);                                    \
        if (e_ != cudaSuccess) return cuda_fail((h), e_, #call);    \
    } while (0)

}  // namespace

int ark::nv_of(const ark_handle* h) { return h->p.grid.n[h->dim - 1]; }

ark::StepArgs ark::base_args(const ark_handle* h)
{
    ark::StepArgs a;
    std::memset(&a, 0, sizeof a);
    const ark_params& p = h->p;
    a.dim = h->dim;
    for (int d = 0; d < 3; ++d) {
        a.n[d] = d < h->dim ? p.grid.n[d] : 1;
        a.dx[d] = d < h->dim ? (p.grid.hi[d] - p.grid.lo[d]) / p.grid.n[d] : 1.0;
        a.bc_lo[d] = p.bc.lo[d];
        a.bc_hi[d] = p.bc.hi[d];
        a.Tw_lo[d] = p.bc.T_lo[d];
        a.Tw_hi[d] = p.bc.T_hi[d];
    }
    a.gamma = p.eos.gamma;
    a.p_inf = p.eos.p_inf;
    a.b = p.eos.law == ARK_EOS_NOBLE_ABEL ? p.eos.b : 0.0;
    a.g = p.gravity.g;
    a.lo_v = p.grid.lo[h->dim - 1];
    a.mu = p.mu;
    a.kappa = p.kappa;
    a.K = p.K;
    a.cfl = p.cfl;
    a.low_mach = p.low_mach;
    a.energy_form = p.energy_form;
    a.work_per_block = h->work_per_block;
    a.phiA = h->phiA;
    a.halo[0] = h->halo[0];
    a.halo[1] = h->halo[1];
    a.planes = h->planes;
    a.tiles_x = h->tiles_x;
    a.tiles_y = h->tiles_y;
    a.ncell = h->N;
    a.base = h->base;
    a.base64 = h->base64;
    a.smax = h->smax;
    a.status = h->status;
    a.time = h->time;
    a.dt_last = h->dt_last;
    ark::fill_constants(a);
    return a;
}

namespace {

using ark::base_args;
using ark::nv_of;

}  // namespace

ark_status ark::validate_params(const ark_params* p, std::string& msg)
{
    if (p->grid.dim != 2 && p->grid.dim != 3) { msg = "grid.dim must be 2 or 3"; return ARK_ERR_INVALID_ARG; }
    const int dim = p->grid.dim;
    for (int d = 0; d < dim; ++d) {
        if (p->grid.n[d] < 1) { msg = "grid.n must be >= 1"; return ARK_ERR_INVALID_ARG; }
        if (!std::isfinite(p->grid.lo[d]) || !std::isfinite(p->grid.hi[d])) {
            msg = "grid.lo and grid.hi must be finite"; return ARK_ERR_INVALID_ARG;
        }
        if (!(p->grid.hi[d] > p->grid.lo[d])) { msg = "grid.hi must exceed grid.lo"; return ARK_ERR_INVALID_ARG; }
        for (int s = 0; s < 2; ++s) {
            const int bc = s ? p->bc.hi[d] : p->bc.lo[d];
            if (bc < ARK_BC_PERIODIC || bc > ARK_BC_HALO) { msg = "unknown boundary condition"; return ARK_ERR_INVALID_ARG; }
            if (bc == ARK_BC_HALO && d != 0) {
                msg = "ARK_BC_HALO borders a neighbouring slab along x only"; return ARK_ERR_INVALID_ARG;
            }
            if (bc == ARK_BC_HALO && p->gravity.phi) {
                msg = "ARK_BC_HALO takes uniform gravity only (no potential array)"; return ARK_ERR_UNSUPPORTED;
            }
            if (bc != ARK_BC_PERIODIC && p->grid.n[d] < 2) { msg = "walls and outflow need n >= 2 along their axis"; return ARK_ERR_INVALID_ARG; }
            if (bc == ARK_BC_NOSLIP_FIXED_T && !((s ? p->bc.T_hi[d] : p->bc.T_lo[d]) > 0.0)) { msg = "wall temperature must be > 0"; return ARK_ERR_INVALID_ARG; }
            if (bc == ARK_BC_NOSLIP_FIXED_T && p->precision == ARK_F32_SPLIT && d != dim - 1) {
                msg = "ARK_F32_SPLIT supports fixed-temperature walls only across the gravity axis";
                return ARK_ERR_UNSUPPORTED;
            }
        }
        if ((p->bc.lo[d] == ARK_BC_PERIODIC) != (p->bc.hi[d] == ARK_BC_PERIODIC)) {
            msg = "periodic boundaries come in pairs"; return ARK_ERR_INVALID_ARG;
        }
    }
    if (!std::isfinite(p->gravity.g)) { msg = "gravity.g must be finite"; return ARK_ERR_INVALID_ARG; }
    if (p->bc.lo[dim - 1] == ARK_BC_PERIODIC && p->gravity.g != 0.0) {
        msg = "gravity along a periodic axis"; return ARK_ERR_INVALID_ARG;
    }
    if (p->gravity.phi) {
        if (p->gravity.g != 0.0) { msg = "gravity.g must be 0 when gravity.phi is given"; return ARK_ERR_INVALID_ARG; }
        if (p->precision == ARK_F32_SPLIT) {
            // the split form's base state is one row per level of the gravity axis
            long long plane = 1;
            for (int d = 0; d + 1 < dim; ++d) plane *= p->grid.n[d];
            std::vector<double> rows;
            if (!ark::row_potential(p->gravity.phi, plane, p->grid.n[dim - 1], p->bc.lo[dim - 1], p->bc.hi[dim - 1], rows)) {
                msg = "ARK_F32_SPLIT takes a potential array that depends on the last (gravity) axis only";
                return ARK_ERR_UNSUPPORTED;
            }
        }
    }
    if (!(p->eos.gamma > 1.0) || !std::isfinite(p->eos.gamma)) { msg = "eos.gamma must be finite and > 1"; return ARK_ERR_INVALID_ARG; }
    if (!(p->eos.p_inf >= 0.0) || !std::isfinite(p->eos.p_inf)) {
        msg = "eos.p_inf must be finite and >= 0";
        return ARK_ERR_INVALID_ARG;
    }
    if (p->eos.law != ARK_EOS_STIFFENED_GAS && p->eos.law != ARK_EOS_NOBLE_ABEL) {
        msg = "unknown eos.law"; return ARK_ERR_INVALID_ARG;
    }
    if (!(p->eos.b >= 0.0) || !std::isfinite(p->eos.b)) { msg = "eos.b must be finite and >= 0"; return ARK_ERR_INVALID_ARG; }
    if (p->eos.law == ARK_EOS_STIFFENED_GAS && p->eos.b != 0.0) {
        msg = "eos.b is the covolume of ARK_EOS_NOBLE_ABEL"; return ARK_ERR_INVALID_ARG;
    }
    if (p->eos.b != 0.0 && p->gravity.phi) {
        msg = "a covolume takes uniform gravity only (no potential array)"; return ARK_ERR_UNSUPPORTED;
    }
    if (!(p->K >= 1.0) || !std::isfinite(p->K)) { msg = "K must be finite and >= 1 (sub-characteristic condition)"; return ARK_ERR_INVALID_ARG; }
    if (!(p->cfl > 0.0) || !std::isfinite(p->cfl)) { msg = "cfl must be finite and > 0"; return ARK_ERR_INVALID_ARG; }
    if (!(p->mu >= 0.0) || !(p->kappa >= 0.0) || !std::isfinite(p->mu) || !std::isfinite(p->kappa)) {
        msg = "mu and kappa must be finite and >= 0"; return ARK_ERR_INVALID_ARG;
    }
    if (p->precision < ARK_F64 || p->precision > ARK_F32_SPLIT) { msg = "unknown precision"; return ARK_ERR_INVALID_ARG; }
    if (p->low_mach != 0 && p->low_mach != 1) { msg = "low_mach must be 0 or 1"; return ARK_ERR_INVALID_ARG; }
    if (p->energy_form != 0 && p->energy_form != 1) { msg = "energy_form must be 0 or 1"; return ARK_ERR_INVALID_ARG; }
    if (p->energy_form == 1 && p->precision == ARK_F32_SPLIT) {
        msg = "ARK_F32_SPLIT needs energy_form 0 (its base state carries rho Phi)";
        return ARK_ERR_UNSUPPORTED;
    }
    if (p->precision != ARK_F64) {
        unsigned long long cells = 1;
        for (int d = 0; d < dim; ++d) cells *= (unsigned long long)p->grid.n[d];
        if (cells >= (1ull << 32)) {   // the FP32 kernels index a field with 32-bit offsets
            msg = "the FP32 forms take fewer than 2^32 cells";
            return ARK_ERR_UNSUPPORTED;
        }
    }
    return ARK_OK;
}

namespace {

// The FP64 staging buffer of host states for the FP32 forms, allocated once
// per handle on first use (a per-call allocation of this size returns to the
// OS at the next synchronisation and has to be mapped again every call).
bool ensure_stage(ark_handle* h, size_t bytes)
{
    if (h->stage) return true;
    if (cudaMalloc((void**)&h->stage, bytes) != cudaSuccess) {
        cudaGetLastError();
        h->stage = nullptr;
        return false;
    }
    return true;
}

// Values of one halo buffer: nf fields x nv planes x ny rows x 2 layers.
size_t halo_elems(const ark_handle* h)
{
    return (size_t)h->nf * nv_of(h) * (h->dim == 3 ? h->p.grid.n[1] : 1) * 2;
}

void choose_launch(ark_handle* h, int nsm)
{
    const int dim = h->dim;
    const bool covolume = h->p.eos.law == ARK_EOS_NOBLE_ABEL && h->p.eos.b != 0.0;
    h->kinfo = h->phiA    ? ark::step_kernel_phi(dim, h->prec, h->visc)
               : covolume ? ark::step_kernel_noble_abel(dim, h->prec, h->visc)
               : (dim == 2 ? ark::step_kernel_2d(h->prec, h->visc) : ark::step_kernel_3d(h->prec, h->visc));
    h->tiles_x = (h->p.grid.n[0] + h->kinfo.tx - 1) / h->kinfo.tx;
    h->tiles_y = dim == 3 ? (h->p.grid.n[1] + h->kinfo.ty - 1) / h->kinfo.ty : 1;
    const int tiles = h->tiles_x * h->tiles_y;
    const int nv = nv_of(h);
    if (h->kinfo.balanced) {
        // one wave of resident blocks; block b takes units [b W, (b + 1) W) of the
        // tile-major list of (tile, plane) units, as runs of planes per tile.
        // A grid too small to fill the wave takes runs of at least 4 planes: more
        // blocks and shorter marches (each run adds 4 planes of pipeline warm-up),
        // which is what sets the step time when the GPU is not full.
        const long long total = (long long)tiles * nv;
        const long long resident = (long long)nsm * h->kinfo.blocks_per_sm;
        long long W = (total + resident - 1) / resident;
        if (W < 4) W = 4;
        h->work_per_block = W;
        h->planes = (int)(W < nv ? W : nv);
        h->grid = dim3((unsigned)((total + W - 1) / W), 1, 1);
        return;
    }
    // enough blocks for ~4 waves of resident blocks, each marching >= 8 planes
    const long long want = 4LL * nsm * h->kinfo.blocks_per_sm;
    long long chunks = (want + tiles - 1) / tiles;
    const long long maxc = (nv + 7) / 8;
    if (chunks > maxc) chunks = maxc;
    if (chunks < 1) chunks = 1;
    h->planes = (int)((nv + chunks - 1) / chunks);
    const int nchunk = (nv + h->planes - 1) / h->planes;
    h->grid = dim3(tiles, nchunk, 1);
}

}  // namespace

ark_status ark::ensure_dt(ark_handle* h)
{
    if (h->dt_valid) return ARK_OK;
    unsigned long long* slot = h->smax + (h->step % 3);
    ARK_CUDA(h, cudaMemsetAsync(slot, 0, sizeof(unsigned long long), h->stream));
    ark::StepArgs a = base_args(h);
    ARK_CUDA(h, ark::launch_wave_rate(a, h->prec, h->visc, h->U[h->cur], slot, h->stream));
    h->dt_valid = true;
    return ARK_OK;
}

using ark::ensure_dt;

extern "C" {

const char* ark_status_string(ark_status s)
{
    switch (s) {
    case ARK_OK: return "ok";
    case ARK_ERR_INVALID_ARG: return "invalid argument";
    case ARK_ERR_CUDA: return "CUDA error";
    case ARK_ERR_NONPHYSICAL: return "nonphysical state";
    case ARK_ERR_TIMEOUT: return "timeout";
    case ARK_ERR_UNSUPPORTED: return "unsupported";
    case ARK_ERR_ALLOC: return "allocation failed";
    }
    return "unknown status";
}

const char* ark_last_error(const ark_handle* h) { return h ? h->err.c_str() : "null handle"; }

ark_status ark_create(const ark_params* p, void* cuda_stream, ark_handle** out)
{
    if (!p || !out) return ARK_ERR_INVALID_ARG;
    *out = nullptr;
    std::string msg;
    ark_status st = ark::validate_params(p, msg);
    if (st != ARK_OK) return st;
    ark_handle* h = new (std::nothrow) ark_handle();
    if (!h) return ARK_ERR_ALLOC;
    h->p = *p;
    h->dim = p->grid.dim;
    h->nf = h->dim + 2;
    h->prec = p->precision;
    h->visc = (p->mu > 0.0 || p->kappa > 0.0) ? 1 : 0;
    if (h->dim == 2) h->p.grid.n[2] = 1;
    h->N = (long long)h->p.grid.n[0] * h->p.grid.n[1] * h->p.grid.n[2];
    h->esz = h->prec == ARK_F64 ? 8 : 4;
    h->stream = (cudaStream_t)cuda_stream;

    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) { st = cuda_fail(h, e, "device query"); delete h; return st; }

    const size_t bytes = (size_t)h->nf * h->N * h->esz;
    const int L = nv_of(h) + 4;
    const size_t ctrl_bytes = 64 + 64 + 16 * 8 + (size_t)ark::DIAG_BLOCKS * ark::DG_NTOT * 8;
    if (cudaMalloc(&h->U[0], bytes) != cudaSuccess || cudaMalloc(&h->U[1], bytes) != cudaSuccess ||
        cudaMalloc(&h->ctrl, ctrl_bytes) != cudaSuccess ||
        cudaMallocHost((void**)&h->status_host, 16) != cudaSuccess ||
        (h->prec == ARK_F32_SPLIT && (cudaMalloc(&h->base, (size_t)ark::BSTRIDE * L * sizeof(float)) != cudaSuccess ||
                                      cudaMalloc((void**)&h->base64, 4 * (size_t)L * sizeof(double)) != cudaSuccess))) {
        cudaGetLastError();
        ark_destroy(h);
        return ARK_ERR_ALLOC;
    }
    if (p->gravity.phi) {   // the caller's potential, in the state precision, owned by the handle
        std::vector<float> f32;
        const void* src = p->gravity.phi;
        if (h->esz == 4) {
            f32.resize((size_t)h->N);
            for (long long i = 0; i < h->N; ++i) f32[i] = (float)p->gravity.phi[i];
            src = f32.data();
        }
        if (cudaMalloc(&h->phiA, (size_t)h->N * h->esz) != cudaSuccess) {
            cudaGetLastError();
            ark_destroy(h);
            return ARK_ERR_ALLOC;
        }
        e = cudaMemcpy(h->phiA, src, (size_t)h->N * h->esz, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) { st = cuda_fail(h, e, "potential upload"); ark_destroy(h); return st; }
        if (h->prec == ARK_F32_SPLIT) {   // FP64 potential of each row (checked separable by validate)
            const int nv = nv_of(h);
            ark::row_potential(p->gravity.phi, h->N / nv, nv, p->bc.lo[h->dim - 1], p->bc.hi[h->dim - 1], h->phi_rows);
            e = cudaMemcpy(h->base64 + 3 * (size_t)L, h->phi_rows.data(), (size_t)L * sizeof(double),
                           cudaMemcpyHostToDevice);
            if (e != cudaSuccess) { st = cuda_fail(h, e, "potential rows upload"); ark_destroy(h); return st; }
        }
        h->p.gravity.phi = nullptr;   // the caller's array is not referenced after ark_create
    }
    for (int side = 0; side < 2; ++side) {   // ghost layers of slab boundaries, zero until set
        if ((side ? p->bc.hi[0] : p->bc.lo[0]) != ARK_BC_HALO) continue;
        const size_t hb = halo_elems(h) * h->esz;
        if (cudaMalloc(&h->halo[side], hb) != cudaSuccess) {
            cudaGetLastError();
            ark_destroy(h);
            return ARK_ERR_ALLOC;
        }
        e = cudaMemsetAsync(h->halo[side], 0, hb, h->stream);
        if (e != cudaSuccess) { st = cuda_fail(h, e, "cudaMemsetAsync"); ark_destroy(h); return st; }
    }
    char* c = (char*)h->ctrl;
    h->smax = (unsigned long long*)c;              // 3 slots
    h->status = (unsigned int*)(c + 32);
    h->time = (double*)(c + 64);
    h->dt_last = (double*)(c + 72);
    h->diag_out = (double*)(c + 128);
    h->partials = (double*)(c + 128 + 16 * 8);
    e = cudaMemsetAsync(h->ctrl, 0, ctrl_bytes, h->stream);
    if (e != cudaSuccess) { st = cuda_fail(h, e, "cudaMemsetAsync"); ark_destroy(h); return st; }
    choose_launch(h, nsm);
    *out = h;
    return ARK_OK;
}

ark_status ark_destroy(ark_handle* h)
{
    if (!h) return ARK_ERR_INVALID_ARG;
    if (h->stream || h->U[0]) cudaStreamSynchronize(h->stream);
    cudaFree(h->U[0]);
    cudaFree(h->U[1]);
    cudaFree(h->ctrl);
    cudaFree(h->base);
    cudaFree(h->base64);
    cudaFree(h->stage);
    cudaFree(h->phiA);
    cudaFreeHost(h->status_host);
    cudaFree(h->halo[0]);
    cudaFree(h->halo[1]);
    cudaFree(h->halo_stage);
    delete h;
    return ARK_OK;
}

ark_status ark_set_state(ark_handle* h, const double* U, int on_device)
{
    if (!h || !U) return fail(h, ARK_ERR_INVALID_ARG, "null argument");
    const size_t bytes64 = (size_t)h->nf * h->N * sizeof(double);
    const double* src = U;
    if (!on_device) {
        if (h->prec == ARK_F64) {
            ARK_CUDA(h, cudaMemcpyAsync(h->U[h->cur], U, bytes64, cudaMemcpyHostToDevice, h->stream));
        } else {
            if (!ensure_stage(h, bytes64)) return fail(h, ARK_ERR_ALLOC, "staging buffer");
            ARK_CUDA(h, cudaMemcpyAsync(h->stage, U, bytes64, cudaMemcpyHostToDevice, h->stream));
            src = h->stage;
        }
    } else if (h->prec == ARK_F64) {
        ARK_CUDA(h, cudaMemcpyAsync(h->U[h->cur], U, bytes64, cudaMemcpyDeviceToDevice, h->stream));
    }
    ark::StepArgs a = base_args(h);
    ark_status st = ARK_OK;
    if (h->prec == ARK_F32_SPLIT) {
        const int nv = nv_of(h), L = nv + 4;
        double* means = nullptr;
        cudaError_t e = cudaMallocAsync((void**)&means, (2 * (size_t)nv + ark::row_means_scratch(a)) * sizeof(double),
                                        h->stream);
        if (e == cudaSuccess) e = ark::launch_row_means(a, src, means + 2 * nv, means, means + nv, h->stream);
        std::vector<double> hm(2 * (size_t)nv);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hm.data(), means, hm.size() * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (means) cudaFreeAsync(means, h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "base state");
        std::vector<double> rho(hm.begin(), hm.begin() + nv), pr(hm.begin() + nv, hm.end());
        for (int r = 0; r < nv; ++r)
            if (!(rho[r] > 0.0) || !(pr[r] + h->p.eos.p_inf > 0.0) || !(a.b * rho[r] < 1.0))
                return fail(h, ARK_ERR_NONPHYSICAL, "base state with rho <= 0, p + p_inf <= 0 or b rho >= 1");
        std::vector<double> b64;
        std::vector<float> tab;
        {
            const ark_params& p = h->p;
            const int V = h->dim - 1;
            ark::BaseSpec bs{nv, p.grid.lo[V], (p.grid.hi[V] - p.grid.lo[V]) / nv, p.gravity.g, p.eos.gamma, p.kappa,
                             p.bc.lo[V], p.bc.hi[V], p.bc.T_lo[V], p.bc.T_hi[V], p.eos.p_inf,
                             h->phi_rows.empty() ? nullptr : h->phi_rows.data(), a.b};
            ark::build_base_tables(bs, rho, pr, b64, tab);
        }
        e = cudaMemcpyAsync(h->base64, b64.data(), b64.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h->base, tab.data(), tab.size() * sizeof(float), cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);   // host vectors leave scope
        if (e != cudaSuccess) return cuda_fail(h, e, "base tables");
        (void)L;
    }
    if (h->prec != ARK_F64) {
        cudaError_t e = ark::launch_convert_in(a, h->prec, src, h->U[h->cur], h->stream);
        if (e != cudaSuccess) st = cuda_fail(h, e, "convert_in");
    }
    if (st != ARK_OK) return st;
    ARK_CUDA(h, cudaMemsetAsync(h->ctrl, 0, 128, h->stream));   // smax slots, status, time, dt
    h->step = 0;
    h->dt_valid = false;
    h->state_set = true;
    if (!on_device) ARK_CUDA(h, cudaStreamSynchronize(h->stream));   // caller may reuse U
    return ARK_OK;
}

ark_status ark_get_state(ark_handle* h, double* U, int on_device)
{
    if (!h || !U) return fail(h, ARK_ERR_INVALID_ARG, "null argument");
    if (!h->state_set) return fail(h, ARK_ERR_INVALID_ARG, "state not set");
    const size_t bytes64 = (size_t)h->nf * h->N * sizeof(double);
    if (h->prec == ARK_F64) {
        ARK_CUDA(h, cudaMemcpyAsync(U, h->U[h->cur], bytes64, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                    h->stream));
    } else {
        ark::StepArgs a = base_args(h);
        double* dst = U;
        if (!on_device) {
            if (!ensure_stage(h, bytes64)) return fail(h, ARK_ERR_ALLOC, "staging buffer");
            dst = h->stage;
        }
        cudaError_t e = ark::launch_convert_out(a, h->prec, h->U[h->cur], dst, h->stream);
        if (e == cudaSuccess && !on_device) e = cudaMemcpyAsync(U, h->stage, bytes64, cudaMemcpyDeviceToHost, h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "get_state");
    }
    if (!on_device) ARK_CUDA(h, cudaStreamSynchronize(h->stream));
    return ARK_OK;
}

ark_status ark_compute_dt(ark_handle* h, double* dt_out)
{
    if (!h) return ARK_ERR_INVALID_ARG;
    if (!h->state_set) return fail(h, ARK_ERR_INVALID_ARG, "state not set");
    h->dt_valid = false;
    ark_status st = ensure_dt(h);
    if (st != ARK_OK) return st;
    if (dt_out) {
        unsigned long long bits = 0;
        ARK_CUDA(h, cudaMemcpyAsync(&bits, h->smax + (h->step % 3), sizeof bits, cudaMemcpyDeviceToHost, h->stream));
        ARK_CUDA(h, cudaStreamSynchronize(h->stream));
        double s;
        std::memcpy(&s, &bits, sizeof s);
        *dt_out = h->p.cfl / s;
    }
    return ARK_OK;
}

ark_status ark_step(ark_handle* h, int nsteps, double dt)
{
    if (!h || nsteps < 0) return fail(h, ARK_ERR_INVALID_ARG, "bad arguments");
    if (!h->state_set) return fail(h, ARK_ERR_INVALID_ARG, "state not set");
    if (nsteps == 0) return ARK_OK;
    if (!(dt > 0.0)) {
        ark_status st = ensure_dt(h);
        if (st != ARK_OK) return st;
    }
    ark::StepArgs a = base_args(h);
    a.dt_fixed = dt > 0.0 ? dt : 0.0;
    for (int i = 0; i < nsteps; ++i) {
        const long long n = h->step;
        a.Uin = h->U[h->cur];
        a.Uout = h->U[1 - h->cur];
        a.slot_read = (int)(n % 3);
        a.slot_write = (int)((n + 1) % 3);
        a.slot_reset = (int)((n + 2) % 3);
        cudaError_t e = h->kinfo.launch(a, h->grid, h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "step launch");
        h->cur = 1 - h->cur;
        h->step = n + 1;
    }
    h->dt_valid = true;   // every step leaves the next step's wave rate in its slot
    return ARK_OK;
}

ark_status ark_diagnostics(ark_handle* h, ark_diag* out)
{
    if (!h || !out) return fail(h, ARK_ERR_INVALID_ARG, "null argument");
    if (!h->state_set) return fail(h, ARK_ERR_INVALID_ARG, "state not set");
    ark::StepArgs a = base_args(h);
    ARK_CUDA(h, ark::launch_diagnostics(a, h->prec, h->U[h->cur], h->partials, h->diag_out, h->stream));
    double v[16];
    unsigned char ctrl[128];
    ARK_CUDA(h, cudaMemcpyAsync(v, h->diag_out, sizeof v, cudaMemcpyDeviceToHost, h->stream));
    ARK_CUDA(h, cudaMemcpyAsync(ctrl, h->ctrl, sizeof ctrl, cudaMemcpyDeviceToHost, h->stream));
    ARK_CUDA(h, cudaStreamSynchronize(h->stream));
    double vol = 1.0;
    for (int d = 0; d < h->dim; ++d) vol *= (h->p.grid.hi[d] - h->p.grid.lo[d]) / h->p.grid.n[d];
    std::memset(out, 0, sizeof *out);
    out->mass = v[ark::DG_MASS] * vol;
    out->momentum[0] = v[ark::DG_MX] * vol;
    out->momentum[1] = v[ark::DG_MY] * vol;
    out->momentum[2] = v[ark::DG_MZ] * vol;
    out->energy = v[ark::DG_W] * vol;
    out->kinetic = v[ark::DG_KE] * vol;
    out->max_speed = v[ark::DG_UMAX];
    out->mean_abs_v_last = v[ark::DG_VABS] / (double)h->N;
    out->min_rho = v[ark::DG_RMIN];
    out->min_p = v[ark::DG_PMIN];
    std::memcpy(&out->status, ctrl + 32, sizeof(unsigned));
    std::memcpy(&out->t, ctrl + 64, sizeof(double));
    std::memcpy(&out->dt, ctrl + 72, sizeof(double));
    out->step = h->step;
    if (v[ark::DG_NAN] > 0.0) out->status |= ark::ST_NAN;
    if (out->status) return fail(h, ARK_ERR_NONPHYSICAL, "device reported a nonphysical state");
    return ARK_OK;
}

ark_status ark_time(ark_handle* h, double* t, double* dt)
{
    if (!h) return ARK_ERR_INVALID_ARG;
    double v[2];
    ARK_CUDA(h, cudaMemcpyAsync(v, h->time, sizeof v, cudaMemcpyDeviceToHost, h->stream));
    ARK_CUDA(h, cudaStreamSynchronize(h->stream));
    if (t) *t = v[0];
    if (dt) *dt = v[1];
    return ARK_OK;
}

ark_status ark_sync(ark_handle* h, double timeout_s)
{
    if (!h) return ARK_ERR_INVALID_ARG;
    const auto t0 = std::chrono::steady_clock::now();
    // wait for everything enqueued on h's stream so far, polling an event
    // until the time limit
    auto wait = [&](const char* what) -> ark_status {
        cudaEvent_t ev;
        ARK_CUDA(h, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        cudaError_t e = cudaEventRecord(ev, h->stream);
        if (e != cudaSuccess) { cudaEventDestroy(ev); return cuda_fail(h, e, "cudaEventRecord"); }
        for (;;) {
            e = cudaEventQuery(ev);
            if (e == cudaSuccess) break;
            if (e != cudaErrorNotReady) { cudaEventDestroy(ev); return cuda_fail(h, e, "cudaEventQuery"); }
            const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            if (el > timeout_s) { cudaEventDestroy(ev); return fail(h, ARK_ERR_TIMEOUT, what); }
            std::this_thread::sleep_for(std::chrono::microseconds(50));
        }
        cudaEventDestroy(ev);
        return ARK_OK;
    };
    ark_status st = wait("stream still busy");
    if (st != ARK_OK) return st;
    // the status word is read on h's own stream (whose work is done), so other
    // streams of the device cannot hold the read past the limit
    ARK_CUDA(h, cudaMemcpyAsync(h->status_host, h->status, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream));
    st = wait("status read still pending");
    if (st != ARK_OK) return st;
    if (*h->status_host) return fail(h, ARK_ERR_NONPHYSICAL, "device reported a nonphysical state");
    return ARK_OK;
}

ark_status ark_get_halo(ark_handle* h, int side, double* out, int on_device)
{
    if (!h || !out || (side != 0 && side != 1)) return fail(h, ARK_ERR_INVALID_ARG, "null argument or side not 0/1");
    if (!h->state_set) return fail(h, ARK_ERR_INVALID_ARG, "state not set");
    if (h->p.grid.n[0] < 2) return fail(h, ARK_ERR_INVALID_ARG, "two layers need n[0] >= 2");
    const size_t bytes = halo_elems(h) * sizeof(double);
    double* dst = out;
    if (!on_device) {
        if (!h->halo_stage && cudaMalloc((void**)&h->halo_stage, bytes) != cudaSuccess) {
            cudaGetLastError();
            return fail(h, ARK_ERR_ALLOC, "halo staging buffer");
        }
        dst = h->halo_stage;
    }
    const ark::StepArgs a = base_args(h);
    ARK_CUDA(h, ark::launch_halo_get(a, h->prec, side, h->U[h->cur], dst, h->stream));
    if (!on_device) {
        ARK_CUDA(h, cudaMemcpyAsync(out, dst, bytes, cudaMemcpyDeviceToHost, h->stream));
        ARK_CUDA(h, cudaStreamSynchronize(h->stream));
    }
    return ARK_OK;
}

ark_status ark_set_halo(ark_handle* h, int side, const double* in, int on_device)
{
    if (!h || !in || (side != 0 && side != 1)) return fail(h, ARK_ERR_INVALID_ARG, "null argument or side not 0/1");
    if (!h->halo[side]) return fail(h, ARK_ERR_INVALID_ARG, "that x side is not ARK_BC_HALO");
    if (h->prec == ARK_F32_SPLIT && !h->state_set) return fail(h, ARK_ERR_INVALID_ARG, "the split form needs its state (base rows) first");
    const size_t bytes = halo_elems(h) * sizeof(double);
    const double* src = in;
    if (!on_device) {
        if (!h->halo_stage && cudaMalloc((void**)&h->halo_stage, bytes) != cudaSuccess) {
            cudaGetLastError();
            return fail(h, ARK_ERR_ALLOC, "halo staging buffer");
        }
        ARK_CUDA(h, cudaMemcpyAsync(h->halo_stage, in, bytes, cudaMemcpyHostToDevice, h->stream));
        src = h->halo_stage;
    }
    const ark::StepArgs a = base_args(h);
    ARK_CUDA(h, ark::launch_halo_set(a, h->prec, src, h->halo[side], h->stream));
    if (!on_device) ARK_CUDA(h, cudaStreamSynchronize(h->stream));   // the caller may reuse `in`
    return ARK_OK;
}

ark_status ark_state_device_ptr(ark_handle* h, const void** ptr, size_t* bytes)
{
    if (!h || !ptr || !bytes) return fail(h, ARK_ERR_INVALID_ARG, "null argument");
    *ptr = h->U[h->cur];
    *bytes = (size_t)h->nf * h->N * h->esz;
    return ARK_OK;
}

ark_status ark_launch_shape(const ark_handle* h, int* tx, int* ty, int* planes, int* threads, int* blocks)
{
    if (!h) return ARK_ERR_INVALID_ARG;
    if (tx) *tx = h->kinfo.tx;
    if (ty) *ty = h->kinfo.ty;
    if (planes) *planes = h->planes;
    if (threads) *threads = h->kinfo.threads;
    if (blocks) *blocks = (int)(h->grid.x * h->grid.y);
    return ARK_OK;
}

}  // extern "C"
