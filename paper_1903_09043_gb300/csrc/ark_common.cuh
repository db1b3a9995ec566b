// ark_common.cuh -- types shared by the step kernel, the auxiliary kernels and
// the host side of libark (GB300, sm_103a).
#pragma once

#include <cstdint>

namespace ark {

enum BC : int { BC_PERIODIC = 0, BC_REFLECT = 1, BC_NOSLIP_T = 2, BC_OUTFLOW = 3, BC_HALO = 4 };
enum Prec : int { P_F64 = 0, P_F32 = 1, P_F32_SPLIT = 2 };
enum Status : unsigned { ST_NONPHYS = 1u, ST_LTILDE = 2u, ST_NAN = 4u };

// Per-row base-state table (F32_SPLIT only), rows r = -2 .. nv + 1, row-major:
// row r holds its BSTRIDE entries at [(r + 2) * BSTRIDE, (r + 3) * BSTRIDE),
// in the order of BaseField, grouped by four so that a kernel reads a row's
// values with 16-byte loads.  Every entry is formed in FP64 on the host and
// rounded once to the state precision.
enum BaseField : int {
    B_RHO0 = 0,  // rho0_r
    B_P0,        // pe0_r = p0_r + p_inf (effective pressure of the equation of state)
    B_T0,        // T0_r = pe0_r / rho0_r
    B_H0,        // W0_r + p0_r, W0 = (p0 + gamma p_inf)/(gamma-1) + rho0 Phi_r
    B_R0F,       // p0_{r+1} - p0_r - S0_{r+1/2}: base residual of the face above row r
    B_Q0,        // (R0F_r + R0F_{r-1}) / 2: base part of [Pi*] - S_i in the vertical momentum
    B_DPP,       // P0_{r+1/2} - p0_r = (p0_{r+1} - p0_r) / 2
    B_DPM,       // P0_{r-1/2} - p0_r = (p0_{r-1} - p0_r) / 2
    B_DRP,       // rho0_{r+1} - rho0_r
    B_DRM,       // rho0_{r-1} - rho0_r
    B_DWP,       // W0_{r+1} - W0_r
    B_DWM,       // W0_{r-1} - W0_r
    B_DQ0,       // kappa [(T0_{r+1} - T0_r) - (T0_r - T0_{r-1})] / dz^2: base heat divergence
    NBASE
};
constexpr int BSTRIDE = 16;   // entries per row (NBASE rounded up to a multiple of 4)
static_assert(NBASE <= BSTRIDE, "base row too long");
__host__ __device__ constexpr int base_index(int field, int r) { return (r + 2) * BSTRIDE + field; }

// Everything one step launch needs, passed by value.
struct StepArgs {
    int dim;
    int n[3];               // cells per axis (x, y, z); the last active axis is the gravity axis
    double dx[3];           // cell sizes
    double gamma;
    double p_inf;           // stiffened-gas constant (0: ideal gas)
    double b;               // covolume of the Noble-Abel stiffened gas (0: the stiffened gas)
    double g;               // gravity along the last axis: Phi = -g x_last
    double lo_v;            // lower coordinate of the last axis
    double mu, kappa, K, cfl;
    int low_mach;
    int energy_form;        // 0: rho*calE (Sec. 2); 1: rho E with the (uS) source (Appendix B)
    long long work_per_block;   // balanced schedule: (tile, plane) units per block (single-grid kernels)
    int bc_lo[3], bc_hi[3];
    double Tw_lo[3], Tw_hi[3];
    int planes;             // planes of the gravity axis per block
    int tiles_x, tiles_y;   // in-plane tiles
    long long ncell;        // cells per field
    const void* Uin;
    void* Uout;
    const void* base;       // BaseField tables (F32_SPLIT), else nullptr
    const void* phiA;       // caller-supplied potential at the cell centres (Real, one field), or null
    const void* halo[2];    // BC_HALO sides of x (low, high): the neighbouring subdomain's two cell
                            // layers beyond the side, Real [NF][nv][ny][2], layer 1 (adjacent) first
    const double* base64;   // FP64 rho0, p0, W0, Phi per row, rows -2 .. nv + 1 (F32_SPLIT)
    double dt_fixed;        // > 0: fixed step; otherwise cfl / smax[slot_read]
    unsigned long long* smax;  // 3 slots of FP64 bit patterns (max wave rate)
    int slot_read, slot_write, slot_reset;
    unsigned int* status;
    double* time;           // simulated time, advanced by dt each step
    double* dt_last;        // dt of this step
    // constants of the stencil in both precisions, rounded once on the host, so
    // that no kernel converts between precisions (conversions run on GB300's
    // FP64 pipe, 1/64 of its FP32 rate)
    float fK, fhalfInvK, fmu, fkappa, feta, fgamma, fgm1, fpinf, fgpinf, fb, fphi_g, fphi_lo, fphi_dv, finvdx[3];
    float fdphi;            // Phi_{r+1} - Phi_r = -g dz, formed in FP64 (uniform g)
    double dK, dhalfInvK, deta, dgpinf, dinvdx[3];
};

// Set the precomputed constants of a StepArgs whose double fields are filled.
inline void fill_constants(StepArgs& a)
{
    const int V = a.dim - 1;
    a.dK = a.K;
    a.dhalfInvK = 0.5 / a.K;
    a.deta = -2.0 / 3.0 * a.mu;
    a.dgpinf = a.gamma * a.p_inf;
    for (int d = 0; d < 3; ++d) a.dinvdx[d] = 1.0 / a.dx[d];
    a.fK = (float)a.K;
    a.fhalfInvK = (float)a.dhalfInvK;
    a.fmu = (float)a.mu;
    a.fkappa = (float)a.kappa;
    a.feta = (float)a.deta;
    a.fgamma = (float)a.gamma;
    a.fgm1 = (float)(a.gamma - 1.0);
    a.fpinf = (float)a.p_inf;
    a.fgpinf = (float)a.dgpinf;
    a.fb = (float)a.b;
    a.fphi_g = (float)a.g;
    a.fphi_lo = (float)a.lo_v;
    a.fphi_dv = (float)a.dx[V];
    for (int d = 0; d < 3; ++d) a.finvdx[d] = (float)a.dinvdx[d];
    a.fdphi = (float)(-a.g * a.dx[V]);
}

}  // namespace ark
