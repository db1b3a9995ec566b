// ark_handle.h -- the single-grid handle behind include/ark.h (host code).
#pragma once

#include <string>
#include <vector>

#include "../../include/ark.h"
#include "ark_aux.cuh"

struct ark_handle {
    ark_params p;
    int dim = 2, nf = 4, prec = 0, visc = 0;
    long long N = 0;
    size_t esz = 8;
    cudaStream_t stream = nullptr;
    void* U[2] = {nullptr, nullptr};
    int cur = 0;
    void* base = nullptr;          // Real table [nv + 4][BSTRIDE], row-major
    double* base64 = nullptr;      // FP64 rho0, p0, W0, Phi [4][nv + 4]
    double* stage = nullptr;       // FP64 staging of host states (FP32 forms), nf * N, made on first use
    void* phiA = nullptr;          // caller-supplied potential, N values of the state precision
    std::vector<double> phi_rows;  // F32_SPLIT with a potential array: Phi of rows -2 .. nv + 1
    void* halo[2] = {nullptr, nullptr};   // ghost layers beyond BC_HALO x sides, state precision [nf][nv][ny][2]
    double* halo_stage = nullptr;  // FP64 staging of host halo transfers, nf * nv * ny * 2
    void* ctrl = nullptr;          // smax[3] | status | pad | time | dt_last | diag out[16] | partials
    unsigned long long* smax = nullptr;
    unsigned int* status = nullptr;
    unsigned int* status_host = nullptr;   // pinned host copy of the status word (ark_sync)
    double* time = nullptr;
    double* dt_last = nullptr;
    double* diag_out = nullptr;
    double* partials = nullptr;
    long long step = 0;
    bool dt_valid = false;
    bool state_set = false;
    ark::StepKernelInfo kinfo{};
    dim3 grid;
    int planes = 1, tiles_x = 1, tiles_y = 1;
    long long work_per_block = 0;  // balanced schedule only
    std::string err;
};

namespace ark {
int nv_of(const ark_handle* h);
StepArgs base_args(const ark_handle* h);   // every field but Uin/Uout/dt/slots
ark_status ensure_dt(ark_handle* h);       // wave rate of the current state into slot step % 3
// The parameter rules of ark_create (include/ark.h); msg receives the reason.
ark_status validate_params(const ark_params* p, std::string& msg);
}  // namespace ark
