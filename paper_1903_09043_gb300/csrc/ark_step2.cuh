// ark_step2.cuh -- column-per-thread form of the fused step for the FP32 state
// forms (F32, F32_SPLIT) on GB300 (sm_103a).
//
// Same arithmetic as ark_step.cuh (Sec. 2 of arXiv:1903.09043; see that file),
// organised for a kernel whose cost is instruction issue rather than FP64
// throughput: every thread owns one column (lx, ly) of the tile plus its
// two-cell in-plane halo, R2X x R2Y threads in all, and keeps that column's
// whole vertical pipeline in registers -- conserved and face values of the
// planes behind the front, tilde states, the upwind flux through the lower
// face, the viscous z flux.  Shared memory exchanges in-plane neighbours
// (every exchange array single-buffered at a fixed offset, so each access is
// the thread's own slot plus a constant) and stages each column's next
// planes (Step2Cfg::RING) where that measured faster than prefetching the next
// plane into registers.
//
// The vertical pipeline is skewed so that one plane needs two barriers.  At
// front plane f:
//   H1  own cell of plane f (primitives; exchange X), z face (f-1, f),
//       tilde state of plane f-1, viscous fluxes of plane f-2's own +x / +y
//       faces (exchange VF) and of the z face (f-2, f-1), upwind transport
//       fluxes of plane f-2's own +x / +y faces (exchange TF) and z face;
//   --- barrier
//   H2  own +x / +y acoustic faces of plane f from X (exchange FF, read in
//       the next H1); exchange of the tilde state of plane f-1 (TL) and of the
//       velocity / temperature data the next plane's viscous fluxes need (VT,
//       DZ, SZ); update of plane f-2 from TF and VF, store, CFL wave rate;
//   --- barrier
// Each exchange array is written in one half and read in the other, so one
// buffer of each suffices.
#pragma once

#include <type_traits>

#include "ark_step.cuh"

namespace ark {

template <int DIM, typename Real, bool SPLIT, bool VISC, int R2X_, int R2Y_, bool PHIA = false, bool ENS = false>
struct Step2Cfg {
    static constexpr int D = DIM, NF = DIM + 2, V = DIM - 1;
    static constexpr int R2X = R2X_, R2Y = R2Y_, NT = R2X * R2Y;
    static constexpr int HY = DIM == 3 ? 2 : 0, H1 = DIM == 3 ? 1 : 0;
    static constexpr int TX = R2X - 4, TY = DIM == 3 ? R2Y - 4 : 1;
    // in-plane face inputs: u_x[, u_y], dp, z, rz, rc (+ rho, Phi with a potential array)
    static constexpr int XI_DP = DIM - 1, XI_Z = XI_DP + 1, XI_RZ = XI_DP + 2, XI_RC = XI_DP + 3;
    static constexpr int XI_RHO = XI_DP + 4, XI_PHI = XI_DP + 5;
    static constexpr int NPX = XI_RC + 1 + (PHIA ? 2 : 0);
    static constexpr int NFF = PHIA ? 3 : 2;                      // per in-plane face: u*, dPi* (+ S)
    static constexpr int NVT = DIM + (VISC ? 1 : 0);              // velocity (+ temperature)
    static constexpr int NV = DIM + 1;                            // dissipative flux components
    static constexpr int NDIR = DIM - 1;                          // in-plane directions
    // shared memory, in units of Real, each array indexed by thread
    static constexpr int O_X = 0;                                 // [NPX]       plane f primitives
    static constexpr int O_FF = O_X + NPX * NT;                   // [NDIR][NFF] u*, dPi* (, S) of own in-plane faces
    static constexpr int O_TL = O_FF + NDIR * NFF * NT;           // [NF]        tilde state
    static constexpr int O_TF = O_TL + NF * NT;                   // [NDIR][NF]  upwind transport fluxes
    static constexpr int O_VT = O_TF + NDIR * NF * NT;            // [NVT]       velocity, T (VISC)
    static constexpr int O_DZ = O_VT + (VISC ? NVT * NT : 0);     // [D]         vertical velocity difference (VISC)
    static constexpr int O_SZ = O_DZ + (VISC ? D * NT : 0);       // [D]         velocity sum of two planes (VISC)
    static constexpr int O_VF = O_SZ + (VISC ? D * NT : 0);       // [NDIR][NV]  dissipative fluxes (VISC)
    static constexpr int N_REAL = O_VF + (VISC ? NDIR * NV * NT : 0);
    static constexpr int BRING = 8;                               // base rows kept in shared memory (split form)
    static constexpr size_t O_BASE = ((N_REAL * sizeof(Real) + 15) / 16) * 16;
    static constexpr size_t O_RED = O_BASE + (SPLIT ? BRING * BSTRIDE * sizeof(float) : 0);
    // Each thread copies its own column three planes ahead into a shared ring
    // of 4 planes (cp.async); in the split form the first BSTRIDE threads copy
    // the base row each plane needs in the same group, so no thread waits on a
    // load before a barrier.  This hides the load latency of a 2D block's short
    // planes (about 1 us each).  The viscous split step of one 2D grid (ENS
    // false: not an ensemble item) keeps the one-plane register prefetch, which
    // its longer planes hide and which measured faster there; in 3D, where a
    // plane takes ten times longer, the ring pays only in the split form (whose
    // base rows it also carries), and plain FP32 keeps the register prefetch.
    static constexpr bool RING = !PHIA && (DIM == 3 ? SPLIT : !(SPLIT && VISC && !ENS));
    static constexpr size_t O_RING = O_RED + NT * sizeof(double) + 4 * sizeof(double);
    static constexpr size_t SMEM_BYTES = O_RING + (RING ? 4 * NF * NT * sizeof(Real) : 0);
    static_assert(NT % 32 == 0 && NT <= 1024, "block must be whole warps");
};

// Four consecutive base-table entries of one row.  The block keeps the rows
// it is using in a shared ring of BRING rows (slot r & (BRING - 1)), filled
// ahead of use (with the state ring's copies, or one plane ahead without the
// ring), so each read is a 16-byte shared broadcast.
struct Base4 {
    float x, y, z, w;
};
template <int BRING>
__device__ __forceinline__ Base4 base4(const float* ring, int group, int r)
{
    const float4 v = *reinterpret_cast<const float4*>(ring + (r & (BRING - 1)) * BSTRIDE + 4 * group);
    return Base4{v.x, v.y, v.z, v.w};
}

// Asynchronous copy of one 4-byte value from global to shared memory, and the
// waits on this thread's own copies (groups complete in the order committed).
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait2() { asm volatile("cp.async.wait_group 2;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Field-parallel arithmetic on pairs of FP32 values (Blackwell's packed FP32x2
// instructions: one issue slot for two lanes' worth of operations).
__device__ __forceinline__ float2 pr(float a, float b) { return make_float2(a, b); }
// c[k] = a[k] * s, k < N
template <int N>
__device__ __forceinline__ void scale_n(float* c, const float* a, float s)
{
    const float2 s2 = pr(s, s);
#pragma unroll
    for (int k = 0; k + 1 < N; k += 2) {
        const float2 r = __fmul2_rn(pr(a[k], a[k + 1]), s2);
        c[k] = r.x;
        c[k + 1] = r.y;
    }
    if constexpr (N % 2) c[N - 1] = a[N - 1] * s;
}
// c[k] = a[k] * s - l0 (b0[k] - m0[k]) [- l1 (b1[k] - m1[k])] - l2 (b2[k] - m2[k]), k < N
template <int N, bool TWO>
__device__ __forceinline__ void flux_update_n(float* c, const float* a, float s, float l0, const float* b0,
                                              const float* m0, float l1, const float* b1, const float* m1, float l2,
                                              const float* b2, const float* m2)
{
    const float2 s2 = pr(s, s), n0 = pr(-l0, -l0), n1 = pr(-l1, -l1), n2 = pr(-l2, -l2), one = pr(-1.f, -1.f);
#pragma unroll
    for (int k = 0; k + 1 < N; k += 2) {
        float2 r = __fmul2_rn(pr(a[k], a[k + 1]), s2);
        r = __ffma2_rn(n0, __ffma2_rn(pr(m0[k], m0[k + 1]), one, pr(b0[k], b0[k + 1])), r);
        if constexpr (TWO) r = __ffma2_rn(n1, __ffma2_rn(pr(m1[k], m1[k + 1]), one, pr(b1[k], b1[k + 1])), r);
        r = __ffma2_rn(n2, __ffma2_rn(pr(m2[k], m2[k + 1]), one, pr(b2[k], b2[k + 1])), r);
        c[k] = r.x;
        c[k + 1] = r.y;
    }
    if constexpr (N % 2) {
        constexpr int k = N - 1;
        float r = a[k] * s - l0 * (b0[k] - m0[k]);
        if constexpr (TWO) r -= l1 * (b1[k] - m1[k]);
        c[k] = r - l2 * (b2[k] - m2[k]);
    }
}

template <int DIM, typename Real, bool SPLIT, bool VISC, int R2X, int R2Y, bool PHIA = false, bool NA = false,
          bool ENS = false>
__device__ __forceinline__ void step_block2(const StepArgs& a, const int tile, const int z0, const int z1, const bool lead,
                                            unsigned char* smem_raw)
{
    using C = Step2Cfg<DIM, Real, SPLIT, VISC, R2X, R2Y, PHIA, ENS>;
    constexpr int D = DIM, NF = DIM + 2, V = DIM - 1, NT = C::NT, TX = C::TX, TY = C::TY;
    static_assert(!SPLIT || sizeof(Real) == 4, "the split form stores FP32 deviations");
    Real* sm = reinterpret_cast<Real*>(smem_raw);
    double* red = reinterpret_cast<double*>(smem_raw + C::O_RED);
    float* const bring = reinterpret_cast<float*>(smem_raw + C::O_BASE);

    const Stepper<DIM, Real, SPLIT, VISC, C::TX, C::TY, PHIA, NA> S(a);
    constexpr int NFF = C::NFF;
    const int t = threadIdx.x;
    const int lx = t % R2X - 2, ly = t / R2X - C::HY;
    const int x0 = (tile % a.tiles_x) * TX;
    const int y0 = D == 3 ? (tile / a.tiles_x) * TY : 0;
    const int nx = S.nx, ny = S.ny, nv = S.nv;
    const long long N = S.N;

    // roles of this column.  A stage runs on every lane of the rows that need
    // it (row roles are warp-uniform: R2X = 32 in 3D, one row in 2D), so no
    // warp diverges on the x halo; the x-halo lanes form values nobody reads,
    // from their own slots and in-bounds neighbour slots of the shared
    // arrays.  Only the lane roles that decide a result -- stores, status
    // words, the wave-rate maximum -- test the column.
    const bool rowR1 = D == 2 || (ly >= -1 && ly <= TY);       // rows of the R1 cells (tilde states)
    const bool rowT = D == 2 || (ly >= 0 && ly < TY);          // rows of the output cells
    const bool rowFy = D == 3 && ly >= -1 && ly < TY;          // own +y face bounds an output cell
    const bool rowFyR1 = D == 3 && ly <= TY;                   // own +y face bounds an R1 cell
    const bool inR1 = rowR1 && lx >= -1 && lx <= TX;

    // time step of this step, formed once and shared
    Real* const sdt = reinterpret_cast<Real*>(red + NT);
    if (t == 0) {
        double dt_d = a.dt_fixed;
        if (!(dt_d > 0.0)) dt_d = a.cfl / __longlong_as_double((long long)a.smax[a.slot_read]);
        if (lead) {   // once per step: clear the slot two steps ahead, advance the clock
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
    const float* __restrict__ Bt = static_cast<const float*>(a.base);
    // the base ring starts with row z0 - 2 (the first front plane); row f + 1 is
    // loaded during plane f by the first BSTRIDE threads
    if constexpr (SPLIT) {
        if (t < BSTRIDE) bring[((z0 - 2) & (C::BRING - 1)) * BSTRIDE + t] = __ldg(Bt + base_index(t, z0 - 2));
        __syncthreads();
    }

    // loader position of this column (clamped into the ghost range); cell
    // offsets within a field are 32-bit (the FP32 forms need ncell < 2^32)
    // position of this column; across a periodic in-plane boundary the halo
    // column is the interior column on the other side (loaded directly, as the
    // ghost rule would give), otherwise clamped into the ghost range
    auto wrap = [](int g, int n) { return g < 0 ? g + n : (g >= n ? g - n : g); };   // |g| stays within 2 of the box
    int gxw = x0 + lx, gyw = D == 3 ? y0 + ly : 0;
    if (a.bc_lo[0] == BC_PERIODIC && nx >= 2) gxw = wrap(gxw, nx);
    if (D == 3 && a.bc_lo[1] == BC_PERIODIC && ny >= 2) gyw = wrap(gyw, ny);
    const int gx = min(max(gxw, -2), nx + 1);
    const int gy = D == 3 ? min(max(gyw, -2), ny + 1) : 0;
    const bool colin = gx >= 0 && gx < nx && (D == 2 || (gy >= 0 && gy < ny));
    const unsigned plane_cells = D == 3 ? (unsigned)nx * (unsigned)ny : (unsigned)nx;
    const unsigned cidx = D == 3 ? (unsigned)gx + (unsigned)nx * (unsigned)gy : (unsigned)gx;
    const bool ocol = rowT && lx >= 0 && lx < TX && (x0 + lx) < nx && (D == 2 || (y0 + ly) < ny);
    const unsigned oidx = D == 3 ? (unsigned)(x0 + lx) + (unsigned)nx * (unsigned)(y0 + ly) : (unsigned)(x0 + lx);
    const Real* __restrict__ Uin = S.U;
    Real* __restrict__ Uo = static_cast<Real*>(a.Uout);

    Real raw[NF];
    Real rawphi = 0;                  // potential of the prefetched cell (PHIA)
    const Real* __restrict__ Pa = static_cast<const Real*>(a.phiA);
    Real* const ringp = reinterpret_cast<Real*>(smem_raw + C::O_RING) + t;   // own slot, [4][NF][NT]
    auto prefetch = [&](int p) {
        if constexpr (C::RING) {   // plane p into ring slot p & 3; one group per plane, even if empty
            if (colin && p >= 0 && p < nv) {
                const unsigned idx = cidx + plane_cells * (unsigned)p;
#pragma unroll
                for (int k = 0; k < NF; ++k) cp_async4(ringp + ((p & 3) * NF + k) * NT, Uin + k * N + idx);
            }
            // base row p + 1, read from plane p + 1 on (the ring's 8 rows hold
            // rows p - 3 .. p + 4 while the copy is in flight)
            if constexpr (SPLIT) {
                if (t < BSTRIDE && p + 1 <= nv + 1)
                    cp_async4(bring + ((p + 1) & (C::BRING - 1)) * BSTRIDE + t, Bt + base_index(t, p + 1));
            }
            cp_async_commit();
        } else {
            if (colin && p >= 0 && p < nv) {
                const unsigned idx = cidx + plane_cells * (unsigned)p;
#pragma unroll
                for (int k = 0; k < NF; ++k) raw[k] = __ldg(Uin + k * N + idx);
                if constexpr (PHIA) rawphi = __ldg(Pa + idx);
            }
        }
    };
    prefetch(z0 - 2);
    if constexpr (C::RING) {
        prefetch(z0 - 1);
        prefetch(z0);
    }

    // exchange arrays: this thread's slot of each
    Real* const X = sm + C::O_X + t;
    Real* const FF = sm + C::O_FF + t;
    Real* const TL = sm + C::O_TL + t;
    Real* const TF = sm + C::O_TF + t;
    Real* const VT = sm + C::O_VT + t;
    Real* const DZ = sm + C::O_DZ + t;
    Real* const SZ = sm + C::O_SZ + t;
    Real* const VF = sm + C::O_VF + t;
    constexpr int SX = 1, SY = R2X;

    // own-column registers
    struct Prev {                     // plane f-1: conserved values and face inputs
        Real drho, m[D], dW, dp, z, rz, rc, phi;
    } cp;
    cp.drho = cp.dW = cp.dp = cp.z = cp.rz = cp.rc = cp.phi = 0;
    Real phi2 = 0;                    // potential of plane f-2 (PHIA)
#pragma unroll
    for (int d = 0; d < D; ++d) cp.m[d] = 0;
    Real fxp[3] = {0, 0, 0}, fyp[3] = {0, 0, 0};   // own +x / +y faces of plane f-1 (u*, dPi*, S)
    Real fx2 = 0, fy2 = 0;            // u* of the own +x / +y faces of plane f-2
    Real zfl[3] = {0, 0, 0};          // face (f-2, f-1): u*, dPi*, dS
    Real tlA[NF + 1];                 // tilde state (+ L) of plane f-2
    Real vt2[C::NVT], vt1[C::NVT];    // velocity (+T) of planes f-2, f-1
    Real zt_lo[NF];                   // upwind transport flux through the face (f-3, f-2)
    Real us_lo = 0;
    Real zvA[C::NV];                  // dissipative flux through the face (f-3, f-2)
#pragma unroll
    for (int k = 0; k <= NF; ++k) tlA[k] = 0;
#pragma unroll
    for (int k = 0; k < NF; ++k) zt_lo[k] = 0;
#pragma unroll
    for (int k = 0; k < C::NV; ++k) zvA[k] = 0;
#pragma unroll
    for (int k = 0; k < C::NVT; ++k) vt2[k] = vt1[k] = 0;
    Real smax_t = 0;
    unsigned status = 0u;

    // One plane of the march.  STEADY: every stage of the pipeline is past its
    // warm-up and f lies inside the box (z0 + 2 <= f <= z1 - 1), so no phase
    // or range test is needed; the warm-up and drain planes take the general
    // form.
    auto plane = [&](const int f, auto steady_c) {
        constexpr bool STEADY = decltype(steady_c)::value;
        const Real fr = Real(f);
        // base rows of the planes this pass touches (split form)
        Base4 bf0{}, b10{}, b11{}, b20{}, b22{}, b23{}, b32{};
        constexpr int BR = C::BRING;
        if constexpr (SPLIT) {
            bf0 = base4<BR>(bring, 0, f);          // row f:   rho0, p0, T0, H0
            if (STEADY || f >= z0) {
                b10 = base4<BR>(bring, 0, f - 1);  // row f-1: rho0, p0, T0, H0
                b11 = base4<BR>(bring, 1, f - 1);  //          R0F, Q0, DPP, DPM
            } else if (f >= z0 - 1) {
                b11 = base4<BR>(bring, 1, f - 1);
            }
            if (STEADY || f >= z0 + 1) {
                b22 = base4<BR>(bring, 2, f - 2);  // row f-2: DRP, DRM, DWP, DWM
                if (STEADY || f >= z0 + 2) {
                    b20 = base4<BR>(bring, 0, f - 2);
                    b23 = base4<BR>(bring, 3, f - 2);  //      DQ0
                    b32 = base4<BR>(bring, 2, f - 3);  // row f-3: DRP, DRM, DWP, DWM
                }
            }
        }

        // ================= H1 =================
        // own cell of plane f
        Cell<D, Real> cc;
        Real ccphi = 0;               // potential of the own cell (PHIA)
        if constexpr (C::RING) {      // plane f, copied three planes ago (planes f+1, f+2 may be in flight)
            cp_async_wait2();
#pragma unroll
            for (int k = 0; k < NF; ++k) raw[k] = ringp[((f & 3) * NF + k) * NT];
        }
        {
            const bool fin = STEADY || (f >= 0 && f < nv);
            if ((STEADY && D == 3) || (fin && colin)) {   // 3D steady planes: all-interior tiles, no ghost call
                Row<Real> w;
                w.rho0 = SPLIT ? bf0.x : Real(0);
                w.p0 = SPLIT ? bf0.y : Real(0);
                w.T0 = SPLIT ? bf0.z : Real(0);
                if constexpr (PHIA) ccphi = rawphi;
                w.phi = a.energy_form ? Real(0) : (PHIA ? ccphi : S.phi.at(fr));
                cc.drho = raw[0];
#pragma unroll
                for (int d = 0; d < D; ++d) cc.m[d] = raw[1 + d];
                cc.dW = raw[D + 1];
                prim<D, Real, SPLIT>(cc, w, S.eos);
            } else {
                cc = S.fetch(gx, gy, f);
                if constexpr (PHIA) ccphi = S.phi_cell(gx, gy, f);
            }
        }
        prefetch(f + (C::RING ? 3 : 1));   // the ring slot of plane f - 1, already read
        const Real rcc = cc.rc;
        const Real zc = cc.rho * cc.c, rzc = rcc * cc.rr;
        X[0 * NT] = cc.u[0];
        if constexpr (D == 3) X[1 * NT] = cc.u[1];
        X[C::XI_DP * NT] = cc.dp;
        X[C::XI_Z * NT] = zc;
        X[C::XI_RZ * NT] = rzc;
        X[C::XI_RC * NT] = rcc;
        if constexpr (PHIA) {
            X[C::XI_RHO * NT] = cc.rho;
            X[C::XI_PHI * NT] = ccphi;
        }
        Real vt0[C::NVT];
#pragma unroll
        for (int d = 0; d < D; ++d) vt0[d] = cc.u[d];
        if constexpr (VISC) vt0[D] = cc.dT;

        // own z face (f-1, f)
        Real zfu[3] = {0, 0, 0};
        if ((STEADY || f >= z0 - 1) && rowR1) {
            // Phi jump across the face: -g dz for uniform g, rounded once from FP64
            zfu[2] = Real(-0.5) * (cp.drho + cc.drho) * (PHIA ? ccphi - cp.phi : Real(a.fdphi));
            acoustic_face<Real>(vt1[V], cc.u[V], cp.dp, cc.dp, cp.z, zc, cp.rz, rzc, cp.rc, rcc,
                                SPLIT ? Real(b11.x) : Real(0), zfu[2], kc.K, kc.halfInvK, a.low_mach, zfu[0], zfu[1]);
        }

        // tilde state of plane f-1
        Real tlB[NF + 1];
#pragma unroll
        for (int k = 0; k <= NF; ++k) tlB[k] = 0;
        if ((STEADY || f >= z0) && rowR1) {
            const int q1 = f - 1;
            const Real usx_m = FF[0 * NT - SX], pix_m = FF[1 * NT - SX];
            Real ell = lam[0] * (fxp[0] - usx_m);
            Real m_t[D];
            m_t[0] = cp.m[0] - lam[0] * (fxp[1] - pix_m);
            Real W_t = cp.dW - lam[0] * (fxp[1] * fxp[0] - pix_m * usx_m);
            if constexpr (PHIA) {   // gravity source of the in-plane faces (the caller's Phi varies in x)
                const Real sx_m = FF[2 * NT - SX];
                m_t[0] += lam[0] * Real(0.5) * (fxp[2] + sx_m);
                if (a.energy_form) W_t += lam[0] * Real(0.5) * (fxp[0] * fxp[2] + usx_m * sx_m);
            }
            if constexpr (D == 3) {
                const Real usy_m = FF[NFF * NT - SY], piy_m = FF[(NFF + 1) * NT - SY];
                ell += lam[1] * (fyp[0] - usy_m);
                m_t[1] = cp.m[1] - lam[1] * (fyp[1] - piy_m);
                W_t -= lam[1] * (fyp[1] * fyp[0] - piy_m * usy_m);
                if constexpr (PHIA) {
                    const Real sy_m = FF[(NFF + 2) * NT - SY];
                    m_t[1] += lam[1] * Real(0.5) * (fyp[2] + sy_m);
                    if (a.energy_form) W_t += lam[1] * Real(0.5) * (fyp[0] * fyp[2] + usy_m * sy_m);
                }
            }
            ell += lam[V] * (zfu[0] - zfl[0]);
            m_t[V] = cp.m[V] - lam[V] * (zfu[1] - zfl[1]) + lam[V] * Real(0.5) * (zfu[2] + zfl[2]);
            if constexpr (SPLIT) m_t[V] -= lam[V] * Real(b11.y);
            W_t -= lam[V] * (zfu[1] * zfu[0] - zfl[1] * zfl[0]);
            if constexpr (SPLIT) W_t -= lam[V] * (Real(b11.z) * zfu[0] - Real(b11.w) * zfl[0]) + Real(b10.w) * ell;
            if (a.energy_form) W_t += lam[V] * Real(0.5) * (zfu[0] * zfu[2] + zfl[0] * zfl[2]);   // (uS)_i, Appendix B
            const Real L = Real(1) + ell;
            const Real rL = rcp(L);
            {
                Real pre[NF];
                pre[0] = SPLIT ? cp.drho - Real(b10.x) * ell : cp.drho;
#pragma unroll
                for (int d = 0; d < D; ++d) pre[1 + d] = m_t[d];
                pre[D + 1] = W_t;
                scale_n<NF>(tlB, pre, rL);
            }
            tlB[NF] = L;
            const bool valid = inR1 && (x0 + lx) >= 0 && (x0 + lx) < nx && (D == 2 || ((y0 + ly) >= 0 && (y0 + ly) < ny)) &&
                               q1 >= 0 && q1 < nv;
            if (valid && !(L > Real(0))) status |= ST_LTILDE;
        }

        // dissipative fluxes of plane f-2's own +x / +y faces and of the z face (f-2, f-1)
        Real zv_new[C::NV];
#pragma unroll
        for (int k = 0; k < C::NV; ++k) zv_new[k] = 0;
        if constexpr (VISC) {
            // tau = mu (grad u + grad u^T) + eta (div u) I and the work and heat
            // fluxes of Sec. 2.2 at one face; only the derivatives tau and
            // div u need are formed.  qt = dx^-1 / 4 scales the averaged
            // tangential differences (an exact power-of-two factor).
            const Real mu = kc.mu, eta = kc.eta, mu2 = Real(2) * kc.mu;
            Real qt[3], kinv[3];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                qt[d] = Real(0.25) * kc.invdx[d];
                kinv[d] = kc.kappa * kc.invdx[d];
            }
            if (STEADY || f >= z0 + 2) {
                auto face = [&](auto dirc) {
                    constexpr int dir = decltype(dirc)::value;
                    constexpr int sh = dir == 0 ? SX : SY;
                    Real vj[C::NVT];
#pragma unroll
                    for (int q = 0; q < C::NVT; ++q) vj[q] = VT[q * NT + sh];
                    Real gn[D];                       // d u_q / d x_dir
#pragma unroll
                    for (int q = 0; q < D; ++q) gn[q] = (vj[q] - vt2[q]) * kc.invdx[dir];
                    Real tau[D];
                    Real divu = gn[dir];
                    if constexpr (D == 3) {
                        constexpr int tt = 1 - dir;
                        constexpr int st = tt == 0 ? SX : SY;
                        auto tder = [&](int q) {
                            return ((VT[q * NT + st] - VT[q * NT - st]) + (VT[q * NT + sh + st] - VT[q * NT + sh - st])) *
                                   qt[tt];
                        };
                        tau[tt] = mu * (gn[tt] + tder(dir));
                        divu += tder(tt);
                    }
                    const Real gv_dir = (DZ[dir * NT] + DZ[dir * NT + sh]) * qt[V];
                    divu += (DZ[V * NT] + DZ[V * NT + sh]) * qt[V];
                    tau[V] = mu * (gn[V] + gv_dir);
                    tau[dir] = mu2 * gn[dir] + eta * divu;
                    Real work = 0;
#pragma unroll
                    for (int q = 0; q < D; ++q) {
                        work += tau[q] * (vt2[q] + vj[q]);
                        VF[(dir * C::NV + q) * NT] = tau[q];
                    }
                    VF[(dir * C::NV + D) * NT] = Real(0.5) * work + (vj[D] - vt2[D]) * kinv[dir];
                };
                if constexpr (D == 3) {
                    // the own +x face (lane .x) and +y face (lane .y) of plane f-2
                    // together, one FP32x2 instruction for both: the same
                    // arithmetic as face() with the roles of x and y swapped.
                    // Rows -1 .. TY-1 need the y face; the x face of row -1 is
                    // formed too and never read.
                    if (rowFy) {
                        const float2 m1 = pr(-1.f, -1.f);
                        auto sub = [&](float2 x, float2 y) { return __ffma2_rn(y, m1, x); };   // x - y
                        auto add = [](float2 x, float2 y) { return __fadd2_rn(x, y); };
                        auto ld = [&](int ix, int iy) { return pr(VT[ix], VT[iy]); };
                        const float2 inv = pr(kc.invdx[0], kc.invdx[1]);
                        const float2 qtt = pr(qt[1], qt[0]);            // tangential scale of each face
                        const float2 qtv = pr(qt[V], qt[V]);
                        const float2 mu_2 = pr(mu, mu), mu2_2 = pr(mu2, mu2), eta_2 = pr(eta, eta);
                        // neighbour values: normal (N), tangential (T), vertical (V) velocity, temperature
                        const float2 jN = ld(0 * NT + SX, 1 * NT + SY), jT = ld(1 * NT + SX, 0 * NT + SY);
                        const float2 jV = ld(2 * NT + SX, 2 * NT + SY), jH = ld(3 * NT + SX, 3 * NT + SY);
                        const float2 oN = pr(vt2[0], vt2[1]), oT = pr(vt2[1], vt2[0]);
                        const float2 oV = pr(vt2[2], vt2[2]), oH = pr(vt2[3], vt2[3]);
                        const float2 gN = __fmul2_rn(sub(jN, oN), inv);
                        const float2 gT = __fmul2_rn(sub(jT, oT), inv);
                        const float2 gV = __fmul2_rn(sub(jV, oV), inv);
                        // averaged tangential differences of the normal (dN) and tangential (dT) components
                        const float2 dN = __fmul2_rn(add(sub(ld(0 * NT + SY, 1 * NT + SX), ld(0 * NT - SY, 1 * NT - SX)),
                                                         sub(ld(0 * NT + SX + SY, 1 * NT + SY + SX),
                                                             ld(0 * NT + SX - SY, 1 * NT + SY - SX))),
                                                     qtt);
                        const float2 dT = __fmul2_rn(add(sub(ld(1 * NT + SY, 0 * NT + SX), ld(1 * NT - SY, 0 * NT - SX)),
                                                         sub(ld(1 * NT + SX + SY, 0 * NT + SY + SX),
                                                             ld(1 * NT + SX - SY, 0 * NT + SY - SX))),
                                                     qtt);
                        const float2 zN = __fmul2_rn(add(pr(DZ[0 * NT], DZ[1 * NT]), pr(DZ[0 * NT + SX], DZ[1 * NT + SY])), qtv);
                        const float2 zV = __fmul2_rn(add(pr(DZ[V * NT], DZ[V * NT]), pr(DZ[V * NT + SX], DZ[V * NT + SY])), qtv);
                        const float2 tauT = __fmul2_rn(mu_2, add(gT, dN));
                        const float2 divu = add(add(gN, dT), zV);
                        const float2 tauV = __fmul2_rn(mu_2, add(gV, zN));
                        const float2 tauN = __ffma2_rn(eta_2, divu, __fmul2_rn(mu2_2, gN));
                        float2 work = __fmul2_rn(tauN, add(oN, jN));
                        work = __ffma2_rn(tauT, add(oT, jT), work);
                        work = __ffma2_rn(tauV, add(oV, jV), work);
                        const float2 heat = __ffma2_rn(sub(jH, oH), pr(kinv[0], kinv[1]), __fmul2_rn(pr(0.5f, 0.5f), work));
                        VF[(0 * C::NV + 0) * NT] = tauN.x;
                        VF[(0 * C::NV + 1) * NT] = tauT.x;
                        VF[(0 * C::NV + 2) * NT] = tauV.x;
                        VF[(0 * C::NV + 3) * NT] = heat.x;
                        VF[(1 * C::NV + 1) * NT] = tauN.y;
                        VF[(1 * C::NV + 0) * NT] = tauT.y;
                        VF[(1 * C::NV + 2) * NT] = tauV.y;
                        VF[(1 * C::NV + 3) * NT] = heat.y;
                    }
                } else {
                    if (rowT) face(IC<0>{});
                }
            }
            if ((STEADY || f >= z0 + 1) && rowT) {
                Real gn[D];                           // d u_q / d z
#pragma unroll
                for (int q = 0; q < D; ++q) gn[q] = (vt1[q] - vt2[q]) * kc.invdx[V];
                Real tau[D];
                Real divu = gn[V];
#pragma unroll
                for (int tt = 0; tt < D - 1; ++tt) {
                    const int st = tt == 0 ? SX : SY;
                    tau[tt] = mu * (gn[tt] + (SZ[V * NT + st] - SZ[V * NT - st]) * qt[tt]);
                    divu += (SZ[tt * NT + st] - SZ[tt * NT - st]) * qt[tt];
                }
                tau[V] = mu2 * gn[V] + eta * divu;
                Real work = 0;
#pragma unroll
                for (int q = 0; q < D; ++q) {
                    work += tau[q] * (vt2[q] + vt1[q]);
                    zv_new[q] = tau[q];
                }
                zv_new[D] = Real(0.5) * work + (vt1[D] - vt2[D]) * kinv[V];
            }
        }

        // upwind transport fluxes of plane f-2's own +x / +y faces
        Real tfx[NF], tfy[NF];
#pragma unroll
        for (int k = 0; k < NF; ++k) tfx[k] = tfy[k] = 0;
        if (STEADY || f >= z0 + 2) {
            if (rowT) {
                const bool upL = fx2 >= Real(0);
                Real up[NF];
#pragma unroll
                for (int k = 0; k < NF; ++k) up[k] = upL ? tlA[k] : TL[k * NT + SX];
                scale_n<NF>(tfx, up, fx2);
#pragma unroll
                for (int k = 0; k < NF; ++k) TF[k * NT] = tfx[k];
            }
            if constexpr (D == 3) {
                if (rowFy) {
                    const bool upL = fy2 >= Real(0);
                    Real up[NF];
#pragma unroll
                    for (int k = 0; k < NF; ++k) up[k] = upL ? tlA[k] : TL[k * NT + SY];
                    scale_n<NF>(tfy, up, fy2);
#pragma unroll
                    for (int k = 0; k < NF; ++k) TF[(NF + k) * NT] = tfy[k];
                }
            }
        }
        // ... and of the z face (f-2, f-1)
        Real zt_hi[NF];
        const Real us_hi = zfl[0];
#pragma unroll
        for (int k = 0; k < NF; ++k) zt_hi[k] = 0;
        if ((STEADY || f >= z0 + 1) && rowT) {
            const bool upL = us_hi >= Real(0);
            Real up[NF];
#pragma unroll
            for (int k = 0; k < NF; ++k) up[k] = upL ? tlA[k] : tlB[k];
            scale_n<NF>(zt_hi, up, us_hi);
            if constexpr (SPLIT) {
                if (!upL) {
                    zt_hi[0] += Real(b22.x) * us_hi;
                    zt_hi[D + 1] += Real(b22.z) * us_hi;
                }
            }
        }
        __syncthreads();

        // ================= H2 =================
        // next base row into the ring (read from the next plane on)
        float bnext = 0.f;
        if constexpr (SPLIT && !C::RING) {
            if (t < BSTRIDE && (STEADY || f + 1 <= nv + 1)) bnext = __ldg(Bt + base_index(t, f + 1));
        }
        // own +x / +y acoustic faces of plane f
        Real fxc[3] = {0, 0, 0}, fyc[3] = {0, 0, 0};
        if constexpr (D == 3 && !PHIA) {
            // 3D: the +x face (lane .x) and the +y face (lane .y) together in
            // FP32x2 instructions, the arithmetic of acoustic_face() per lane.
            // Rows -2 .. TY need the y face; the x face of row -2 is formed too
            // and never read.
            if ((STEADY || (f >= z0 - 1 && f <= z1)) && rowFyR1) {
                const float2 uL = pr(cc.u[0], cc.u[1]), uR = pr(X[0 * NT + SX], X[1 * NT + SY]);
                const float2 dpL = pr(cc.dp, cc.dp), dpR = pr(X[C::XI_DP * NT + SX], X[C::XI_DP * NT + SY]);
                const float zRx = X[C::XI_Z * NT + SX], zRy = X[C::XI_Z * NT + SY];
                const float rzRx = X[C::XI_RZ * NT + SX], rzRy = X[C::XI_RZ * NT + SY];
                const float2 aa = __fmul2_rn(pr(kc.K, kc.K), pr(pmax(zc, zRx), pmax(zc, zRy)));
                const float2 ninv2a = __fmul2_rn(pr(-kc.halfInvK, -kc.halfInvK), pr(pmin(rzc, rzRx), pmin(rzc, rzRy)));
                const float2 half = pr(0.5f, 0.5f), m1 = pr(-1.f, -1.f);
                const float2 jump = __ffma2_rn(dpL, m1, dpR);                                    // dpR - dpL
                const float2 us = __ffma2_rn(jump, ninv2a, __fmul2_rn(half, __fadd2_rn(uL, uR)));
                float2 th = pr(1.f, 1.f);
                if (a.low_mach) {
                    th.x = pmin(vabs(us.x) * pmin(rcc, X[C::XI_RC * NT + SX]), 1.f);
                    th.y = pmin(vabs(us.y) * pmin(rcc, X[C::XI_RC * NT + SY]), 1.f);
                }
                const float2 du = __ffma2_rn(uL, m1, uR);                                        // uR - uL
                const float2 hat = __fmul2_rn(__fmul2_rn(pr(-0.5f, -0.5f), aa), th);
                const float2 dPi = __ffma2_rn(hat, du, __fmul2_rn(half, __fadd2_rn(dpL, dpR)));
                fxc[0] = us.x;
                fxc[1] = dPi.x;
                fyc[0] = us.y;
                fyc[1] = dPi.y;
                FF[0 * NT] = fxc[0];
                FF[1 * NT] = fxc[1];
                FF[NFF * NT] = fyc[0];
                FF[(NFF + 1) * NT] = fyc[1];
            }
        } else if (STEADY || (f >= z0 - 1 && f <= z1)) {
            if (rowR1) {
                // with a Phi array the in-plane faces carry S = -(rho_L + rho_R)(Phi_R - Phi_L) / 2
                if constexpr (PHIA)
                    fxc[2] = Real(-0.5) * (cc.rho + X[C::XI_RHO * NT + SX]) * (X[C::XI_PHI * NT + SX] - ccphi);
                acoustic_face<Real>(cc.u[0], X[SX], cc.dp, X[C::XI_DP * NT + SX], zc, X[C::XI_Z * NT + SX],
                                    rzc, X[C::XI_RZ * NT + SX], rcc, X[C::XI_RC * NT + SX], Real(0), fxc[2],
                                    kc.K, kc.halfInvK, a.low_mach, fxc[0], fxc[1]);
                FF[0 * NT] = fxc[0];
                FF[1 * NT] = fxc[1];
                if constexpr (PHIA) FF[2 * NT] = fxc[2];
            }
            if constexpr (D == 3) {
                if (rowFyR1) {
                    if constexpr (PHIA)
                        fyc[2] = Real(-0.5) * (cc.rho + X[C::XI_RHO * NT + SY]) * (X[C::XI_PHI * NT + SY] - ccphi);
                    acoustic_face<Real>(cc.u[1], X[NT + SY], cc.dp, X[C::XI_DP * NT + SY], zc, X[C::XI_Z * NT + SY], rzc,
                                        X[C::XI_RZ * NT + SY], rcc, X[C::XI_RC * NT + SY], Real(0), fyc[2], kc.K,
                                        kc.halfInvK, a.low_mach, fyc[0], fyc[1]);
                    FF[NFF * NT] = fyc[0];
                    FF[(NFF + 1) * NT] = fyc[1];
                    if constexpr (PHIA) FF[(NFF + 2) * NT] = fyc[2];
                }
            }
        }
        // exchange for the next plane's H1
        if (rowR1) {
#pragma unroll
            for (int k = 0; k < NF; ++k) TL[k * NT] = tlB[k];
            if constexpr (VISC) {
#pragma unroll
                for (int k = 0; k < C::NVT; ++k) VT[k * NT] = vt1[k];
#pragma unroll
                for (int d = 0; d < D; ++d) {
                    DZ[d * NT] = vt0[d] - vt2[d];
                    SZ[d * NT] = vt1[d] + vt0[d];
                }
            }
        }

        // update of plane f-2
        if ((STEADY || f >= z0 + 2) && rowT) {
            const int q = f - 2;
            const Real L = tlA[NF];
            Real nb[NF];
            Real tmx[NF], tmy[NF];
#pragma unroll
            for (int k = 0; k < NF; ++k) {
                tmx[k] = TF[k * NT - SX];
                tmy[k] = D == 3 ? TF[(NF + k) * NT - SY] : Real(0);
            }
            Real lowfix[NF];
#pragma unroll
            for (int k = 0; k < NF; ++k) lowfix[k] = zt_lo[k];
            if constexpr (SPLIT) {
                if (us_lo >= Real(0)) {
                    lowfix[0] += Real(b22.y) * us_lo;
                    lowfix[D + 1] += Real(b22.w) * us_lo;
                } else {
                    lowfix[0] -= Real(b32.x) * us_lo;
                    lowfix[D + 1] -= Real(b32.z) * us_lo;
                }
            }
            flux_update_n<NF, D == 3>(nb, tlA, L, lam[0], tfx, tmx, lam[1], tfy, tmy, lam[V], zt_hi, lowfix);
            if constexpr (VISC) {
#pragma unroll
                for (int k = 0; k < C::NV; ++k) {
                    Real dxy = (VF[k * NT] - VF[k * NT - SX]) * lam[0];
                    if constexpr (D == 3) dxy += (VF[(C::NV + k) * NT] - VF[(C::NV + k) * NT - SY]) * lam[1];
                    nb[1 + k] += dxy + (zv_new[k] - zvA[k]) * lam[V];
                }
                if constexpr (SPLIT) nb[D + 1] += dt * Real(b23.x);
            }
            // the wave rate is formed on every lane of the row; only the
            // output columns store and fold it into the maximum and status
            Row<Real> w;
            w.rho0 = SPLIT ? Real(b20.x) : Real(0);
            w.p0 = SPLIT ? Real(b20.y) : Real(0);
            w.T0 = SPLIT ? Real(b20.z) : Real(0);
            w.phi = a.energy_form ? Real(0) : (PHIA ? phi2 : S.phi.at(fr - Real(2)));
            Real p, rho;
            const Real sh = wave_rate<D, Real, SPLIT, VISC>(nb, w, S.eos, kc.invdx, kc.mu, kc.kappa, p, rho);
            if (ocol) {
                const unsigned idx = oidx + plane_cells * (unsigned)q;
#pragma unroll
                for (int k = 0; k < NF; ++k) Uo[k * N + idx] = nb[k];
            }
            if (ocol && !(sh <= smax_t)) smax_t = (sh == sh) ? sh : smax_t;
            if (ocol && (sh != sh || p != p)) status |= ST_NAN;
            if (ocol && (!(rho > Real(0)) || !(p > Real(0)))) status |= ST_NONPHYS;
        }
        if constexpr (SPLIT && !C::RING) {
            if (t < BSTRIDE && (STEADY || f + 1 <= nv + 1)) bring[((f + 1) & (BR - 1)) * BSTRIDE + t] = bnext;
        }
        __syncthreads();

        // ---------------- rotate the column registers ----------------
        if (STEADY || f >= z0 + 1) {
#pragma unroll
            for (int k = 0; k < NF; ++k) zt_lo[k] = zt_hi[k];
            us_lo = us_hi;
        }
#pragma unroll
        for (int k = 0; k < C::NV; ++k) zvA[k] = zv_new[k];
#pragma unroll
        for (int k = 0; k <= NF; ++k) tlA[k] = tlB[k];
        fx2 = fxp[0];
        fy2 = fyp[0];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            fxp[k] = fxc[k];
            fyp[k] = fyc[k];
        }
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
        if constexpr (PHIA) {
            phi2 = cp.phi;
            cp.phi = ccphi;
        }
    };
    // Steady planes take the specialised body.  In 3D only tiles whose every
    // column loads directly do, and their copy carries no out-of-line ghost
    // call: with the call inside, the copy needs more than the 128 registers
    // a 512-thread block allows and spills.  The 2D copy keeps the ghost path
    // for columns across a wall, which measured faster there.
    bool allin = true;
    if constexpr (DIM == 3) allin = __syncthreads_and(colin);   // every column of the tile loads directly
    for (int f = z0 - 2; f <= z1 + 1; ++f) {
        if (allin && f >= z0 + 2 && f <= z1 - 1) plane(f, std::true_type{});
        else plane(f, std::false_type{});
    }

    // block max of the wave rate -> one atomic per block
    if constexpr (C::RING) cp_async_wait0();   // no copy of this run lands in the next run's ring
    block_rate_max(double(smax_t), reinterpret_cast<unsigned long long*>(red), a.smax + a.slot_write);
    if (status) atomicOr(a.status, status);
}

template <int DIM, typename Real, bool SPLIT, bool VISC, int R2X, int R2Y, bool PHIA = false, bool NA = false>
__global__ void __launch_bounds__(R2X * R2Y, 512 / (R2X * R2Y)) ark_step2_kernel(const __grid_constant__ StepArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // balanced schedule: this block's share of the tile-major (tile, plane) units,
    // marched as one run of planes per tile it touches
    const int nv = a.n[DIM - 1];
    const long long total = (long long)a.tiles_x * a.tiles_y * nv;
    long long u = (long long)blockIdx.x * a.work_per_block;
    const long long end = min(u + a.work_per_block, total);
    bool lead = blockIdx.x == 0;
    while (u < end) {
        const int tile = (int)(u / nv);
        const int z0 = (int)(u - (long long)tile * nv);
        const int z1 = (int)min((long long)nv, z0 + (end - u));
        step_block2<DIM, Real, SPLIT, VISC, R2X, R2Y, PHIA, NA>(a, tile, z0, z1, lead, smem_raw);
        u += z1 - z0;
        lead = false;
        __syncthreads();   // the next run reuses the shared exchange arrays
    }
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
        const StepArgs& r = runs[w.run];
        const int z0 = w.chunk * r.planes;
        step_block2<DIM, Real, SPLIT, VISC, R2X, R2Y, false, false, true>(r, w.tile, z0, min(z0 + r.planes, r.n[DIM - 1]),
                                                      w.tile == 0 && w.chunk == 0, smem_raw);
    }
}

}  // namespace ark
