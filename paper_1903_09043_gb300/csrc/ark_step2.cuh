// ark_step2.cuh -- column-per-thread form of the fused step for the FP32 state
// forms (F32, F32_SPLIT) on GB300 (sm_103a).
//
// Same arithmetic as ark_step.cuh (Sec. 2 of arXiv:1903.09043; see that file),
// organised for a kernel whose cost is instruction issue rather than FP64
// throughput: every thread owns one column (lx, ly) of the tile plus its
// two-cell in-plane halo, R2X x R2Y threads in all, and keeps that column's
// whole vertical pipeline in registers -- primitives of planes f and f-1,
// the faces between them, tilde states of planes f-1 and f-2, the upwind
// flux through the lower face, the dissipative carries.  Shared memory only
// exchanges in-plane neighbours, at constant offsets (t +- 1, t +- R2X), so
// no index arithmetic is left in the plane loop.  One warp spans a row of 32
// columns (3D: 28 output cells plus the halo).
//
// Per front plane f (one __syncthreads after each of A-D):
//   A  own cell of plane f: primitives (registers), in-plane exchange copies;
//   B  own +x / +y faces of plane f, own z face (f-1, f);
//   C  tilde state of plane f-1 (own), dissipative fluxes of plane f-1's
//      own +x / +y faces and of the z face (f-1, f);
//   D  upwind transport fluxes of plane f-2's own +x / +y faces, the z face
//      (f-2, f-1), the in-plane viscous divergence of plane f-1;
//   E  update of plane f-2 (own cell), store, CFL wave rate.
#pragma once

#include "ark_step.cuh"

namespace ark {

template <int DIM, typename Real, bool SPLIT, bool VISC, int R2X_, int R2Y_>
struct Step2Cfg {
    static constexpr int D = DIM, NF = DIM + 2, V = DIM - 1;
    static constexpr int R2X = R2X_, R2Y = R2Y_, NT = R2X * R2Y;
    static constexpr int HY = DIM == 3 ? 2 : 0, H1 = DIM == 3 ? 1 : 0;
    static constexpr int TX = R2X - 4, TY = DIM == 3 ? R2Y - 4 : 1;
    static constexpr int NPX = DIM == 3 ? 6 : 5;                  // in-plane face inputs: u_x[, u_y], dp, z, rz, rc
    static constexpr int NVT = DIM + (VISC ? 1 : 0);              // velocity (+ temperature)
    static constexpr int NV = DIM + 1;                            // dissipative flux components
    static constexpr int NDIR = DIM - 1;                          // in-plane directions
    // shared memory, in units of Real, each array indexed by thread
    static constexpr int O_PX = 0;                                // [2][NPX][NT]
    static constexpr int O_VT = O_PX + 2 * NPX * NT;              // [3][NVT][NT]
    static constexpr int O_F = O_VT + (VISC ? 3 * NVT * NT : 0);   // [2][NDIR][2][NT]  (u*, dPi*)
    static constexpr int O_TL = O_F + 2 * NDIR * 2 * NT;          // [2][NF][NT]
    static constexpr int O_VF = O_TL + 2 * NF * NT;               // [NDIR][NV][NT]
    static constexpr int O_TF = O_VF + (VISC ? NDIR * NV * NT : 0);   // [NDIR][NF][NT]
    static constexpr int N_REAL = O_TF + NDIR * NF * NT;
    static constexpr size_t SMEM_BYTES = ((N_REAL * sizeof(Real) + 15) / 16) * 16 + NT * sizeof(double) + 4 * sizeof(double);
    static_assert(NT % 32 == 0 && NT <= 1024, "block must be whole warps");
};

template <int DIM, typename Real, bool SPLIT, bool VISC, int R2X, int R2Y>
__device__ __forceinline__ void step_block2(const StepArgs& a, const int tile, const int chunk, unsigned char* smem_raw)
{
    using C = Step2Cfg<DIM, Real, SPLIT, VISC, R2X, R2Y>;
    using C1 = StepCfg<DIM, Real, SPLIT, VISC, C::TX, C::TY>;   // for the loader's Stepper type
    constexpr int D = DIM, NF = DIM + 2, V = DIM - 1, NT = C::NT, TX = C::TX, TY = C::TY;
    Real* sm = reinterpret_cast<Real*>(smem_raw);
    double* red = reinterpret_cast<double*>(smem_raw + ((C::N_REAL * sizeof(Real) + 15) / 16) * 16);

    const Stepper<DIM, Real, SPLIT, VISC, C::TX, C::TY> S(a);
    (void)sizeof(C1);
    const int t = threadIdx.x;
    const int lx = t % R2X - 2, ly = t / R2X - C::HY;
    const int x0 = (tile % a.tiles_x) * TX;
    const int y0 = D == 3 ? (tile / a.tiles_x) * TY : 0;
    const int z0 = chunk * a.planes;
    const int z1 = min(z0 + a.planes, S.nv);
    const int nx = S.nx, ny = S.ny, nv = S.nv;
    const long long N = S.N;

    // roles of this column (warp-uniform in y, so whole warps skip what they do not own)
    const bool rowR1 = D == 2 || (ly >= -1 && ly <= TY);
    const bool rowT = D == 2 || (ly >= 0 && ly < TY);
    const bool inR1 = rowR1 && lx >= -1 && lx <= TX;
    const bool inT = rowT && lx >= 0 && lx < TX;
    const bool xfR1 = rowR1 && lx <= TX;                       // own +x face bounds an R1 cell
    const bool yfR1 = D == 3 && ly <= TY && lx >= -1 && lx <= TX; // own +y face bounds an R1 cell
    const bool xfT = rowT && lx >= -1 && lx < TX;              // own +x face bounds an output cell
    const bool yfT = D == 3 && ly >= -1 && ly < TY && lx >= 0 && lx < TX;

    // time step of this step, formed once and shared
    Real* const sdt = reinterpret_cast<Real*>(red + NT);
    if (t == 0) {
        double dt_d = a.dt_fixed;
        if (!(dt_d > 0.0)) dt_d = a.cfl / __longlong_as_double((long long)a.smax[a.slot_read]);
        if (tile == 0 && chunk == 0) {
            a.smax[a.slot_reset] = 0ull;
            *a.time += dt_d;
            *a.dt_last = dt_d;
        }
        sdt[0] = Real(dt_d);
#pragma unroll
        for (int d = 0; d < 3; ++d) sdt[1 + d] = d < D ? Real(dt_d * a.dinvdx[d]) : Real(0);
    }
    __syncthreads();
    const KConst<Real> kc(a);
    const Real dt = sdt[0];
    Real lam[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) lam[d] = sdt[1 + d];
    const Real* __restrict__ Bt = static_cast<const Real*>(a.base);
    const int BL = nv + 4;
    auto base = [&](int field, int r) -> Real { return SPLIT ? __ldg(Bt + field * BL + r + 2) : Real(0); };

    // loader position of this column (clamped into the ghost range)
    const int gx = min(max(x0 + lx, -2), nx + 1);
    const int gy = D == 3 ? min(max(y0 + ly, -2), ny + 1) : 0;
    const bool colin = gx >= 0 && gx < nx && (D == 2 || (gy >= 0 && gy < ny));
    const long long cidx = D == 3 ? gx + (long long)nx * gy : gx;
    const long long plane_cells = D == 3 ? (long long)nx * ny : (long long)nx;
    const bool ocol = inT && (x0 + lx) < nx && (D == 2 || (y0 + ly) < ny);
    const long long oidx = D == 3 ? (x0 + lx) + (long long)nx * (y0 + ly) : (x0 + lx);

    Real raw[NF];
    auto prefetch = [&](int p) {
        if (colin && p >= 0 && p < nv) {
            const long long idx = cidx + plane_cells * p;
#pragma unroll
            for (int k = 0; k < NF; ++k) raw[k] = __ldg(S.U + k * N + idx);
        }
    };
    prefetch(z0 - 2);

    // own-column registers
    struct Prev {                     // plane f-1: conserved values and face inputs
        Real drho, m[D], dW, dp, z, rz, rc;
    } cp;
    Real fxp[2] = {0, 0}, fyp[2] = {0, 0};   // own +x / +y faces of plane f-1 (u*, dPi*)
    Real fx2 = 0, fy2 = 0;            // u* of the own +x / +y faces of plane f-2
    Real zfl[3] = {0, 0, 0};          // face (f-2, f-1): u*, dPi*, dS
    Real tlA[NF + 1];                 // tilde state (+ L) of plane f-2
    Real vt2[C::NVT], vt1[C::NVT];    // velocity (+T) of planes f-2, f-1
    Real zt_lo[NF];
    Real us_lo = 0;
    Real zvA[C::NV], zvB[C::NV], dxy_prev[C::NV];
#pragma unroll
    for (int k = 0; k <= NF; ++k) tlA[k] = 0;
#pragma unroll
    for (int k = 0; k < NF; ++k) zt_lo[k] = 0;
#pragma unroll
    for (int k = 0; k < C::NV; ++k) zvA[k] = zvB[k] = dxy_prev[k] = 0;
#pragma unroll
    for (int k = 0; k < C::NVT; ++k) vt2[k] = vt1[k] = 0;
    Real smax_t = 0;
    unsigned status = 0u;

    constexpr int SX = 1, SY = R2X;

    for (int f = z0 - 2; f <= z1 + 1; ++f) {
        const Real fr = Real(f);
        const int s3 = ((f % 3) + 3) % 3;
        Real* const PXf = sm + C::O_PX + (f & 1) * C::NPX * NT;
        Real* const VT0 = sm + C::O_VT + s3 * C::NVT * NT;                    // plane f
        Real* const VT1 = sm + C::O_VT + ((s3 + 2) % 3) * C::NVT * NT;        // plane f-1
        Real* const VT2 = sm + C::O_VT + ((s3 + 1) % 3) * C::NVT * NT;        // plane f-2
        Real* const Ff = sm + C::O_F + (f & 1) * C::NDIR * 2 * NT;            // in-plane faces of plane f
        Real* const Ff1 = sm + C::O_F + ((f - 1) & 1) * C::NDIR * 2 * NT;     // of plane f-1
        Real* const TL1 = sm + C::O_TL + ((f - 1) & 1) * NF * NT;             // tilde of plane f-1
        Real* const TL2 = sm + C::O_TL + ((f - 2) & 1) * NF * NT;             // tilde of plane f-2
        Real* const VF = sm + C::O_VF;
        Real* const TF = sm + C::O_TF;

        // ---------------- A: own cell of plane f ----------------
        Cell<D, Real> cc;
        {
            const bool fin = f >= 0 && f < nv;
            if (fin && colin) {
                const Row<Real> w = row_info<Real, SPLIT>(a, S.phi, f, nv, fr);
                cc.drho = raw[0];
#pragma unroll
                for (int d = 0; d < D; ++d) cc.m[d] = raw[1 + d];
                cc.dW = raw[D + 1];
                prim<D, Real, SPLIT>(cc, w, S.gm1, S.gamma);
            } else {
                cc = S.fetch(gx, gy, f);
            }
        }
        prefetch(f + 1);
        const Real rcc = cc.rc;
        const Real zc = cc.rho * cc.c, rzc = rcc * cc.rr;
        PXf[0 * NT + t] = cc.u[0];
        if constexpr (D == 3) PXf[1 * NT + t] = cc.u[1];
        PXf[(C::NPX - 4) * NT + t] = cc.dp;
        PXf[(C::NPX - 3) * NT + t] = zc;
        PXf[(C::NPX - 2) * NT + t] = rzc;
        PXf[(C::NPX - 1) * NT + t] = rcc;
        Real vt0[C::NVT];
#pragma unroll
        for (int d = 0; d < D; ++d) vt0[d] = cc.u[d];
        if constexpr (VISC) vt0[D] = cc.dT;
        if constexpr (VISC) {
#pragma unroll
            for (int k = 0; k < C::NVT; ++k) VT0[k * NT + t] = vt0[k];
        }
        __syncthreads();

        // ---------------- B: own +x / +y faces of plane f, own z face (f-1, f) ----------------
        Real fxc[2] = {0, 0}, fyc[2] = {0, 0};
        if (f >= z0 - 1) {
            if (xfR1) {
                const int j = t + SX;
                acoustic_face<Real>(cc.u[0], PXf[j], cc.dp, PXf[(C::NPX - 4) * NT + j], zc, PXf[(C::NPX - 3) * NT + j],
                                    rzc, PXf[(C::NPX - 2) * NT + j], rcc, PXf[(C::NPX - 1) * NT + j], Real(0), Real(0),
                                    kc.K, kc.halfInvK, a.low_mach, fxc[0], fxc[1]);
                Ff[0 * NT + t] = fxc[0];
                Ff[1 * NT + t] = fxc[1];
            }
            if constexpr (D == 3) {
                if (yfR1) {
                    const int j = t + SY;
                    acoustic_face<Real>(cc.u[1], PXf[NT + j], cc.dp, PXf[2 * NT + j], zc, PXf[3 * NT + j], rzc,
                                        PXf[4 * NT + j], rcc, PXf[5 * NT + j], Real(0), Real(0), kc.K, kc.halfInvK,
                                        a.low_mach, fyc[0], fyc[1]);
                    Ff[2 * NT + t] = fyc[0];
                    Ff[3 * NT + t] = fyc[1];
                }
            }
        }
        Real zfu[3] = {0, 0, 0};   // face (f-1, f)
        if (f >= z0 - 1 && inR1) {
            const Real dphi = S.phi.at(fr) - S.phi.at(fr - Real(1));
            zfu[2] = Real(-0.5) * (cp.drho + cc.drho) * dphi;
            acoustic_face<Real>(vt1[V], cc.u[V], cp.dp, cc.dp, cp.z, zc, cp.rz, rzc, cp.rc, rcc, base(B_R0F, f - 1),
                                zfu[2], kc.K, kc.halfInvK, a.low_mach, zfu[0], zfu[1]);
        }
        __syncthreads();

        // ---------------- C: tilde of plane f-1; dissipative fluxes of plane f-1 ----------------
        Real tlB[NF + 1];
#pragma unroll
        for (int k = 0; k <= NF; ++k) tlB[k] = 0;
        if (f >= z0 && inR1) {
            const int q1 = f - 1;
            const Real usx_m = Ff1[t - SX], pix_m = Ff1[NT + t - SX];
            Real ell = lam[0] * (fxp[0] - usx_m);
            Real m_t[D];
            m_t[0] = cp.m[0] - lam[0] * (fxp[1] - pix_m);
            Real W_t = cp.dW - lam[0] * (fxp[1] * fxp[0] - pix_m * usx_m);
            if constexpr (D == 3) {
                const Real usy_m = Ff1[2 * NT + t - SY], piy_m = Ff1[3 * NT + t - SY];
                ell += lam[1] * (fyp[0] - usy_m);
                m_t[1] = cp.m[1] - lam[1] * (fyp[1] - piy_m);
                W_t -= lam[1] * (fyp[1] * fyp[0] - piy_m * usy_m);
            }
            ell += lam[V] * (zfu[0] - zfl[0]);
            m_t[V] = cp.m[V] - lam[V] * (zfu[1] - zfl[1]) + lam[V] * Real(0.5) * (zfu[2] + zfl[2]);
            if constexpr (SPLIT) m_t[V] -= lam[V] * base(B_Q0, q1);
            W_t -= lam[V] * (zfu[1] * zfu[0] - zfl[1] * zfl[0]);
            if constexpr (SPLIT) W_t -= lam[V] * (base(B_DPP, q1) * zfu[0] - base(B_DPM, q1) * zfl[0]) + base(B_H0, q1) * ell;
            if (a.energy_form) W_t += lam[V] * Real(0.5) * (zfu[0] * zfu[2] + zfl[0] * zfl[2]);   // (uS)_i, Appendix B
            const Real L = Real(1) + ell;
            const Real rL = rcp(L);
            tlB[0] = SPLIT ? (cp.drho - base(B_RHO0, q1) * ell) * rL : cp.drho * rL;
#pragma unroll
            for (int d = 0; d < D; ++d) tlB[1 + d] = m_t[d] * rL;
            tlB[D + 1] = W_t * rL;
            tlB[NF] = L;
#pragma unroll
            for (int k = 0; k < NF; ++k) TL1[k * NT + t] = tlB[k];
            const bool valid = (x0 + lx) >= 0 && (x0 + lx) < nx && (D == 2 || ((y0 + ly) >= 0 && (y0 + ly) < ny)) &&
                               q1 >= 0 && q1 < nv;
            if (valid && !(L > Real(0))) status |= ST_LTILDE;
        }
        Real zv_new[C::NV];
#pragma unroll
        for (int k = 0; k < C::NV; ++k) zv_new[k] = 0;
        if constexpr (VISC) {
            const Real mu = kc.mu, kappa = kc.kappa, eta = kc.eta;
            // own +x (and +y) faces of plane f-1's output cells
            if (f >= z0 + 1 && f <= z1) {
                auto face = [&](auto dirc) {
                    constexpr int dir = decltype(dirc)::value;
                    constexpr int sh = dir == 0 ? SX : SY;
                    const int j = t + sh;
                    Real grad[3][3];
#pragma unroll
                    for (int aa = 0; aa < 3; ++aa)
#pragma unroll
                        for (int qq = 0; qq < 3; ++qq) grad[aa][qq] = 0;
#pragma unroll
                    for (int qq = 0; qq < D; ++qq) grad[dir][qq] = (VT1[qq * NT + j] - vt1[qq]) * kc.invdx[dir];
                    if constexpr (D == 3) {
                        constexpr int tt = 1 - dir;
                        constexpr int st = tt == 0 ? SX : SY;
#pragma unroll
                        for (int qq = 0; qq < D; ++qq)
                            grad[tt][qq] = Real(0.25) *
                                           ((VT1[qq * NT + t + st] - VT1[qq * NT + t - st]) +
                                            (VT1[qq * NT + j + st] - VT1[qq * NT + j - st])) *
                                           kc.invdx[tt];
                    }
#pragma unroll
                    for (int qq = 0; qq < D; ++qq)
                        grad[V][qq] = Real(0.25) * ((vt0[qq] - vt2[qq]) + (VT0[qq * NT + j] - VT2[qq * NT + j])) * kc.invdx[V];
                    Real divu = 0;
#pragma unroll
                    for (int aa = 0; aa < D; ++aa) divu += grad[aa][aa];
                    Real work = 0;
#pragma unroll
                    for (int qq = 0; qq < D; ++qq) {
                        Real tau = mu * (grad[dir][qq] + grad[qq][dir]);
                        if (qq == dir) tau += eta * divu;
                        work += tau * Real(0.5) * (vt1[qq] + VT1[qq * NT + j]);
                        VF[(dir * C::NV + qq) * NT + t] = tau;
                    }
                    VF[(dir * C::NV + D) * NT + t] = work + kappa * (VT1[D * NT + j] - vt1[D]) * kc.invdx[dir];
                };
                if (xfT) face(IC<0>{});
                if constexpr (D == 3) {
                    if (yfT) face(IC<1>{});
                }
            }
            // own z face (f-1, f)
            if (f >= z0 && f <= z1 && inT) {
                Real grad[3][3];
#pragma unroll
                for (int aa = 0; aa < 3; ++aa)
#pragma unroll
                    for (int qq = 0; qq < 3; ++qq) grad[aa][qq] = 0;
#pragma unroll
                for (int qq = 0; qq < D; ++qq) grad[V][qq] = (vt0[qq] - vt1[qq]) * kc.invdx[V];
#pragma unroll
                for (int tt = 0; tt < D - 1; ++tt) {
                    const int st = tt == 0 ? SX : SY;
#pragma unroll
                    for (int qq = 0; qq < D; ++qq)
                        grad[tt][qq] = Real(0.25) *
                                       ((VT1[qq * NT + t + st] - VT1[qq * NT + t - st]) +
                                        (VT0[qq * NT + t + st] - VT0[qq * NT + t - st])) *
                                       kc.invdx[tt];
                }
                Real divu = 0;
#pragma unroll
                for (int aa = 0; aa < D; ++aa) divu += grad[aa][aa];
                Real work = 0;
#pragma unroll
                for (int qq = 0; qq < D; ++qq) {
                    Real tau = mu * (grad[V][qq] + grad[qq][V]);
                    if (qq == V) tau += eta * divu;
                    work += tau * Real(0.5) * (vt1[qq] + vt0[qq]);
                    zv_new[qq] = tau;
                }
                zv_new[D] = work + kappa * (vt0[D] - vt1[D]) * kc.invdx[V];
            }
        }
        __syncthreads();

        // ---------------- D: transport fluxes of plane f-2, viscous divergence of plane f-1 ----------------
        Real dxy_new[C::NV];
#pragma unroll
        for (int k = 0; k < C::NV; ++k) dxy_new[k] = 0;
        if constexpr (VISC) {
            if (f >= z0 + 1 && f <= z1 && inT) {
#pragma unroll
                for (int k = 0; k < C::NV; ++k) dxy_new[k] = (VF[k * NT + t] - VF[k * NT + t - SX]) * lam[0];
                if constexpr (D == 3) {
#pragma unroll
                    for (int k = 0; k < C::NV; ++k)
                        dxy_new[k] += (VF[(C::NV + k) * NT + t] - VF[(C::NV + k) * NT + t - SY]) * lam[1];
                }
            }
        }
        Real tfx[NF], tfy[NF];
        if (f >= z0 + 2) {
            if (xfT) {
                const bool upL = fx2 >= Real(0);
#pragma unroll
                for (int k = 0; k < NF; ++k) {
                    tfx[k] = (upL ? tlA[k] : TL2[k * NT + t + SX]) * fx2;
                    TF[k * NT + t] = tfx[k];
                }
            }
            if constexpr (D == 3) {
                if (yfT) {
                    const bool upL = fy2 >= Real(0);
#pragma unroll
                    for (int k = 0; k < NF; ++k) {
                        tfy[k] = (upL ? tlA[k] : TL2[k * NT + t + SY]) * fy2;
                        TF[(NF + k) * NT + t] = tfy[k];
                    }
                }
            }
        }
        Real zt_hi[NF];
        Real us_hi = zfl[0];   // u* of the face (f-2, f-1)
#pragma unroll
        for (int k = 0; k < NF; ++k) zt_hi[k] = 0;
        if (f >= z0 + 1 && inT) {
            const bool upL = us_hi >= Real(0);
#pragma unroll
            for (int k = 0; k < NF; ++k) zt_hi[k] = (upL ? tlA[k] : tlB[k]) * us_hi;
            if constexpr (SPLIT) {
                if (!upL) {
                    zt_hi[0] += base(B_DRP, f - 2) * us_hi;
                    zt_hi[D + 1] += base(B_DWP, f - 2) * us_hi;
                }
            }
        }
        __syncthreads();

        // ---------------- E: update of plane f-2 ----------------
        if (f >= z0 + 2 && inT) {
            const int q = f - 2;
            const Real L = tlA[NF];
            Real nb[NF];
#pragma unroll
            for (int k = 0; k < NF; ++k) {
                Real acc = tlA[k] * L;
                acc -= lam[0] * (tfx[k] - TF[k * NT + t - SX]);
                if constexpr (D == 3) acc -= lam[1] * (tfy[k] - TF[(NF + k) * NT + t - SY]);
                nb[k] = acc;
            }
            Real lowfix[NF];
#pragma unroll
            for (int k = 0; k < NF; ++k) lowfix[k] = zt_lo[k];
            if constexpr (SPLIT) {
                if (us_lo >= Real(0)) {
                    lowfix[0] += base(B_DRM, q) * us_lo;
                    lowfix[D + 1] += base(B_DWM, q) * us_lo;
                } else {
                    lowfix[0] -= base(B_DRP, q - 1) * us_lo;
                    lowfix[D + 1] -= base(B_DWP, q - 1) * us_lo;
                }
            }
#pragma unroll
            for (int k = 0; k < NF; ++k) nb[k] -= lam[V] * (zt_hi[k] - lowfix[k]);
            if constexpr (VISC) {
#pragma unroll
                for (int k = 0; k < C::NV; ++k) nb[1 + k] += dxy_prev[k] + (zvB[k] - zvA[k]) * lam[V];
                if constexpr (SPLIT) nb[D + 1] += dt * base(B_DQ0, q);
            }
            if (ocol) {
                Real* Uo = static_cast<Real*>(a.Uout);
                const long long idx = oidx + plane_cells * q;
#pragma unroll
                for (int k = 0; k < NF; ++k) Uo[k * N + idx] = nb[k];
                const Row<Real> w = row_info<Real, SPLIT>(a, S.phi, q, nv, fr - Real(2));
                Real p, rho;
                const Real sh = wave_rate<D, Real, SPLIT, VISC>(nb, w, S.gm1, S.gamma, kc.invdx, kc.mu, kc.kappa, p, rho);
                if (!(sh <= smax_t)) smax_t = (sh == sh) ? sh : smax_t;
                if (sh != sh || p != p) status |= ST_NAN;
                if (!(rho > Real(0)) || !(p > Real(0))) status |= ST_NONPHYS;
            }
        }

        // ---------------- rotate the column registers ----------------
        if (f >= z0 + 1) {
#pragma unroll
            for (int k = 0; k < NF; ++k) zt_lo[k] = zt_hi[k];
            us_lo = us_hi;
        }
#pragma unroll
        for (int k = 0; k < C::NV; ++k) {
            zvA[k] = zvB[k];
            zvB[k] = zv_new[k];
            dxy_prev[k] = dxy_new[k];
        }
#pragma unroll
        for (int k = 0; k <= NF; ++k) tlA[k] = tlB[k];
        fx2 = fxp[0];
        fy2 = fyp[0];
        fxp[0] = fxc[0];
        fxp[1] = fxc[1];
        fyp[0] = fyc[0];
        fyp[1] = fyc[1];
#pragma unroll
        for (int k = 0; k < 3; ++k) zfl[k] = zfu[k];
#pragma unroll
        for (int k = 0; k < C::NVT; ++k) {
            vt2[k] = vt1[k];
            vt1[k] = vt0[k];
        }
        cp.drho = cc.drho;
#pragma unroll
        for (int d = 0; d < D; ++d) cp.m[d] = cc.m[d];
        cp.dW = cc.dW;
        cp.dp = cc.dp;
        cp.z = zc;
        cp.rz = rzc;
        cp.rc = rcc;
    }

    // block max of the wave rate -> one atomic per block
    red[t] = double(smax_t);
    __syncthreads();
    for (int s = NT / 2; s > 0; s >>= 1) {
        if (t < s) red[t] = fmax(red[t], red[t + s]);
        __syncthreads();
    }
    if (t == 0) atomicMax(a.smax + a.slot_write, (unsigned long long)__double_as_longlong(red[0]));
    if (status) atomicOr(a.status, status);
}

template <int DIM, typename Real, bool SPLIT, bool VISC, int R2X, int R2Y>
__global__ void __launch_bounds__(R2X * R2Y, 512 / (R2X * R2Y)) ark_step2_kernel(const __grid_constant__ StepArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    step_block2<DIM, Real, SPLIT, VISC, R2X, R2Y>(a, blockIdx.x, blockIdx.y, smem_raw);
}

template <int DIM, typename Real, bool SPLIT, bool VISC, int R2X, int R2Y>
__global__ void __launch_bounds__(R2X * R2Y, 512 / (R2X * R2Y))
ark_batch2_kernel(const StepArgs* __restrict__ runs, const BatchItem* __restrict__ items, int nitems, int* ctr,
                  int ctr_cur, int ctr_next)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_item;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = atomicAdd(ctr + ctr_cur, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= nitems) break;
        if (it == 0 && threadIdx.x == 0) ctr[ctr_next] = 0;
        const BatchItem w = items[it];
        step_block2<DIM, Real, SPLIT, VISC, R2X, R2Y>(runs[w.run], w.tile, w.chunk, smem_raw);
    }
}

}  // namespace ark
