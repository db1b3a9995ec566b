// ark_base.h -- FP64 base state of the F32_SPLIT form (host code).
#pragma once

#include <cmath>
#include <vector>

#include "ark_common.cuh"

namespace ark {

struct BaseSpec {
    int nv;              // rows along the gravity axis
    double lo_v, dv;     // lower coordinate and cell size of that axis
    double g, gamma, kappa;
    int bc_lo, bc_hi;    // boundary conditions of that axis
    double T_lo, T_hi;   // wall temperatures
    double p_inf;        // stiffened-gas constant (0: ideal gas)
    const double* phi_rows = nullptr;   // potential of rows -2 .. nv + 1 (nv + 4 values), or
                                        // nullptr for uniform gravity, Phi = -g x_last
    double b = 0.0;      // covolume of the Noble-Abel stiffened gas (0: the stiffened gas)
};

// FP64 base state of F32_SPLIT: rows -2 .. nv + 1 from the interior row means,
// ghost rows by the boundary rule of the gravity axis applied to the base,
// then every table entry formed in FP64 and rounded once.  Pressures enter the
// equation of state as pe = p + p_inf: T0 = pe0 / rho0, the wall balance in pe,
// and B_P0 holds pe0.  b64 holds four FP64 rows of nv + 4 values: rho0, p0,
// W0 and the potential Phi of each row.
inline void build_base_tables(const BaseSpec& s, const std::vector<double>& rho_in, const std::vector<double>& p_in,
                              std::vector<double>& b64, std::vector<float>& tab)
{
    const int nv = s.nv, L = nv + 4;
    const double dv = s.dv;
    const double gm1 = s.gamma - 1.0;
    std::vector<double> rho(L), pr(L), T(L), phi(L);
    for (int r = -2; r < nv + 2; ++r) phi[r + 2] = s.phi_rows ? s.phi_rows[r + 2] : -(s.g * (s.lo_v + (r + 0.5) * dv));
    for (int r = 0; r < nv; ++r) {
        rho[r + 2] = rho_in[r];
        pr[r + 2] = p_in[r];
        T[r + 2] = (p_in[r] + s.p_inf) * (1.0 - s.b * rho_in[r]) / rho_in[r];
    }
    for (int side = 0; side < 2; ++side) {
        const int bc = side == 0 ? s.bc_lo : s.bc_hi;
        const double Tw = side == 0 ? s.T_lo : s.T_hi;
        for (int layer = 1; layer <= 2; ++layer) {
            const int g = side == 0 ? -layer : nv - 1 + layer;
            const int m = side == 0 ? layer - 1 : nv - layer;        // mirror row
            const int A = layer == 1 ? m : (side == 0 ? -1 : nv);   // inner neighbour
            if (bc == BC_PERIODIC) {
                const int w = ((g % nv) + nv) % nv;
                rho[g + 2] = rho[w + 2]; pr[g + 2] = pr[w + 2]; T[g + 2] = T[w + 2];
            } else if (bc == BC_OUTFLOW) {
                const int e = side == 0 ? 0 : nv - 1;
                rho[g + 2] = rho[e + 2]; pr[g + 2] = pr[e + 2]; T[g + 2] = T[e + 2];
            } else {
                const double Tg = bc == BC_REFLECT ? T[m + 2] : 2.0 * Tw - T[m + 2];
                const double dphi = phi[g + 2] - phi[A + 2];
                const double K = pr[A + 2] + s.p_inf - 0.5 * rho[A + 2] * dphi;
                double pe;
                if (s.b == 0.0) {
                    pe = K / (1.0 + dphi / (2.0 * Tg));
                } else {   // rho = pe / (T + b pe): the balance is a quadratic in pe (positive root)
                    const double B = Tg - s.b * K + 0.5 * dphi;
                    pe = 2.0 * K * Tg / (B + std::sqrt(B * B + 4.0 * s.b * K * Tg));
                }
                pr[g + 2] = pe - s.p_inf;
                rho[g + 2] = pe / (Tg + s.b * pe);
                T[g + 2] = Tg;
            }
        }
    }
    b64.assign(4 * L, 0.0);
    std::vector<double> W0(L);
    for (int i = 0; i < L; ++i) {
        W0[i] = (pr[i] + s.gamma * s.p_inf) * (1.0 - s.b * rho[i]) / gm1 + rho[i] * phi[i];
        b64[0 * L + i] = rho[i];
        b64[1 * L + i] = pr[i];
        b64[2 * L + i] = W0[i];
        b64[3 * L + i] = phi[i];
    }
    std::vector<double> t((size_t)BSTRIDE * L, 0.0);
    auto at = [&](int f, int i) -> double& { return t[(size_t)i * BSTRIDE + f]; };   // i = r + 2
    for (int i = 0; i < L; ++i) {
        at(B_RHO0, i) = rho[i];
        at(B_P0, i) = pr[i] + s.p_inf;
        at(B_T0, i) = T[i];
        at(B_H0, i) = W0[i] + pr[i];
    }
    for (int i = 0; i + 1 < L; ++i) {
        const double S0 = -0.5 * (rho[i] + rho[i + 1]) * (phi[i + 1] - phi[i]);
        at(B_R0F, i) = (pr[i + 1] - pr[i]) - S0;
        at(B_DPP, i) = 0.5 * (pr[i + 1] - pr[i]);
        at(B_DRP, i) = rho[i + 1] - rho[i];
        at(B_DWP, i) = W0[i + 1] - W0[i];
    }
    for (int i = 1; i < L; ++i) {
        at(B_Q0, i) = 0.5 * (at(B_R0F, i) + at(B_R0F, i - 1));
        at(B_DPM, i) = 0.5 * (pr[i - 1] - pr[i]);
        at(B_DRM, i) = rho[i - 1] - rho[i];
        at(B_DWM, i) = W0[i - 1] - W0[i];
    }
    for (int i = 1; i + 1 < L; ++i)
        at(B_DQ0, i) = s.kappa * ((T[i + 1] - T[i]) - (T[i] - T[i - 1])) / (dv * dv);
    tab.resize(t.size());
    for (size_t i = 0; i < t.size(); ++i) tab[i] = (float)t[i];
}

// Potential of the rows -2 .. nv + 1 of the gravity (last) axis from a caller's
// array that depends on that axis only: interior rows from the array, ghost
// rows by the array's ghost rule along that axis (across a periodic side the
// row on the other side; across a wall or outflow side the linear extension
// (1 + L) Phi_0 - L Phi_1 of the boundary row and its inner neighbour, layer
// L = 1, 2).  Returns false if some cell differs from the first cell of its row.
inline bool row_potential(const double* phi, long long plane, int nv, int bc_lo, int bc_hi, std::vector<double>& rows)
{
    for (int r = 0; r < nv; ++r)
        for (long long i = 1; i < plane; ++i)
            if (!(phi[r * plane + i] == phi[r * plane])) return false;
    rows.assign((size_t)nv + 4, 0.0);
    for (int r = 0; r < nv; ++r) rows[r + 2] = phi[r * plane];
    for (int side = 0; side < 2; ++side)
        for (int layer = 1; layer <= 2; ++layer) {
            const int g = side == 0 ? -layer : nv - 1 + layer;
            const int bc = side == 0 ? bc_lo : bc_hi;
            if (bc == BC_PERIODIC) {
                rows[g + 2] = rows[((g % nv) + nv) % nv + 2];
            } else {
                const int b0 = side == 0 ? 0 : nv - 1, b1 = side == 0 ? 1 : nv - 2;
                rows[g + 2] = (1.0 + layer) * rows[b0 + 2] - layer * rows[(nv > 1 ? b1 : b0) + 2];
            }
        }
    return true;
}

}  // namespace ark
