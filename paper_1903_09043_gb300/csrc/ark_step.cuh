// ark_step.cuh -- the fused explicit step of the all-regime, well-balanced
// acoustic-transport scheme (arXiv:1903.09043, Sec. 2) for GB300 (sm_103a).
//
// One launch = one time step.  Each block owns an in-plane tile of TX x TY
// cells (TY = 1 in 2D) and marches along the gravity axis (y in 2D, z in 3D)
// over `planes` planes.  Per plane f it
//   A  loads U^n of plane f over the tile + 2 ghost cells in-plane (boundary
//      conditions are applied in the loader; no ghost array exists in HBM) and
//      forms the primitives (Sec. 3.2 "conservative to primitive");
//   B  forms the acoustic face values u*, Pi* (theta of Eq. 16) and the
//      gravity source S of plane f-1's in-plane faces and of the faces
//      between planes f-1 and f (Sec. 2.1.2);
//   C  forms L~ and the tilde states of plane f-1 (Sec. 2.1.2) and the
//      first-order viscous / heat fluxes (Sec. 2.2) around plane f-1;
//   D  forms the upwind transport fluxes (Sec. 2.1.3) of plane f-2, updates
//      it, stores U^{n+1} once, and folds its CFL wave rate into a block max.
// Every conserved field is therefore read from HBM once per step (halo reads
// hit L2) and written once.  Planes live in small shared-memory rings; values
// that stay with one output column (z-face fluxes, in-plane viscous sums)
// live in registers.  Multi-dimensional terms are summed unsplit.
//
// Arithmetic forms: F64 (Real = double), F32 (Real = float) and F32_SPLIT
// (Real = float, the state stores deviations from an FP64 base state per row
// of the gravity axis; every base-state term, including the well-balanced
// residual p0_{r+1} - p0_r - S0_{r+1/2}, comes from an FP64 table).
#pragma once

#include <cuda_runtime.h>

#include "ark_common.cuh"

namespace ark {

template <int DIM, typename Real, bool SPLIT, bool VISC, int TX, int TY, bool PHIA = false>
struct StepCfg {
    static constexpr int D = DIM;
    static constexpr int NF = DIM + 2;
    static constexpr bool Y = (DIM == 3);
    static constexpr int HY = Y ? 2 : 0;
    static constexpr int H1 = Y ? 1 : 0;
    static constexpr int NT = TX * TY;
    static constexpr int R2X = TX + 4, R2Y = TY + 2 * HY, NR2 = R2X * R2Y;
    static constexpr int R1X = TX + 2, R1Y = TY + 2 * H1, NR1 = R1X * R1Y;
    // x faces bounding R1 cells: left cell lx in [-2, TX], rows ly in [-H1, TY + H1)
    static constexpr int FXX = TX + 3, NFX = FXX * R1Y;
    // y faces bounding R1 cells (3D): columns lx in [-1, TX], lower cell ly in [-2, TY]
    static constexpr int FYY = TY + 3, NFY = Y ? R1X * FYY : 0;
    // faces of the output cells: x: left lx in [-1, TX - 1]; y: lower ly in [-1, TY - 1]
    static constexpr int NTX = (TX + 1) * TY;
    static constexpr int NTY = Y ? TX * (TY + 1) : 0;
    static constexpr int NVT = D + (VISC ? 1 : 0);   // velocity components (+ temperature)
    static constexpr int NV = D + 1;                 // dissipative flux components (m_d..., W)

    // shared-memory layout, in units of Real
    static constexpr int O_VELT = 0;                                   // [3][NVT][NR2]
    static constexpr int O_FACEF = O_VELT + 3 * NVT * NR2;             // [2][4][NR2] dp, rc, z, rz
    static constexpr int O_UCONS = O_FACEF + 2 * 4 * NR2;              // [2][NF][NR1]
    static constexpr int O_ZF = O_UCONS + 2 * NF * NR1;                // [2][3][NR1] u*, dPi*, dS
    static constexpr int NXYC = PHIA ? 3 : 2;                          // in-plane face values: u*, dPi* (, S)
    static constexpr int O_XYF = O_ZF + 2 * 3 * NR1;                   // [2][NXYC][NFX + NFY]
    static constexpr int O_TL = O_XYF + 2 * NXYC * (NFX + NFY);        // [2][NF + 1][NR1]
    static constexpr int O_TFLUX = O_TL + 2 * (NF + 1) * NR1;          // [NF][NTX + NTY]
    static constexpr int O_VFLUX = O_TFLUX + NF * (NTX + NTY);         // [NV][NTX + NTY]
    static constexpr int O_PH = O_VFLUX + (VISC ? NV * (NTX + NTY) : 0);   // [2][2][NR2] rho, Phi (PHIA)
    static constexpr int N_REAL = O_PH + (PHIA ? 2 * 2 * NR2 : 0);
    static constexpr size_t SMEM_BYTES = ((N_REAL * sizeof(Real) + 15) / 16) * 16 + NT * sizeof(double) + 4 * sizeof(double);

    static constexpr int TXV = TX, TYV = TY;
    __device__ static int i2(int lx, int ly) { return (ly + HY) * R2X + (lx + 2); }
    __device__ static int i1(int lx, int ly) { return (ly + H1) * R1X + (lx + 1); }
    __device__ static int ifx(int lx, int ly) { return (ly + H1) * FXX + (lx + 2); }
    __device__ static int ify(int lx, int ly) { return (ly + 2) * R1X + (lx + 1); }
    __device__ static int itx(int lx, int ly) { return ly * (TX + 1) + (lx + 1); }
    __device__ static int ity(int lx, int ly) { return (ly + 1) * TX + lx; }
};

template <int D, typename Real>
struct Cell {
    Real drho, m[D], dW;            // conserved values (deviation form in F32_SPLIT)
    Real rho, u[D], dp, dT, c;      // full rho, velocity, deviation p and T (full in F64/F32), c
    Real rr;                        // 1 / rho
    Real rc;                        // 1 / c
};

template <typename Real>
struct Row {
    Real rho0, p0, T0, phi;
};

// Reciprocal and square root.
// FP64: Newton-Raphson iteration (the textbook scheme for reciprocals and
// reciprocal square roots, e.g. Markstein, IBM J. Res. Dev. 34 (1990)) from
// the hardware's approximate FP64 seeds (rcp.approx.ftz.f64 and
// rsqrt.approx.ftz.f64, relative error below 2^-22).  Each iteration squares
// the relative error, so two leave it below 2^-88 and the result is within one
// ulp of the correctly rounded value, at a fraction of the FP64-pipe work of
// the IEEE division and square root.  Arguments are positive normal numbers
// (densities, L~, gamma (p + p_inf) / rho); zero, infinite or NaN arguments give NaN,
// which the step's status word reports.
// FP32: the hardware approximations (within 2 ulp), one special-function
// instruction each; the FP32 forms' error budget is several ulp per step.
__device__ __forceinline__ double rcp_seed(double x)
{
#ifdef __CUDA_ARCH__
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    return y;
#else
    return 1.0 / x;   // host-side parsing of device code only
#endif
}
__device__ __forceinline__ double rsqrt_seed(double q)
{
#ifdef __CUDA_ARCH__
    double y;
    asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(q));
    return y;
#else
    return 1.0 / sqrt(q);
#endif
}
__device__ __forceinline__ double rcp(double x)
{
    double y = rcp_seed(x);
    double e = fma(-x, y, 1.0);   // relative error of y
    y = fma(y, e, y);
    e = fma(-x, y, 1.0);
    return fma(y, e, y);
}
__device__ __forceinline__ float rcp(float x) { return __fdividef(1.0f, x); }
// c = sqrt(q) and 1 / c together
__device__ __forceinline__ void sqrt_rsqrt(double q, double& c, double& rc)
{
    double y = rsqrt_seed(q);
    double e = fma(-q * y, y, 1.0);   // 1 - q y^2
    y = fma(0.5 * y, e, y);            // y (1 + e / 2)
    e = fma(-q * y, y, 1.0);
    y = fma(0.5 * y, e, y);
    double s = q * y;                  // sqrt(q), then one correction on the residual q - s^2
    s = fma(fma(-s, s, q), 0.5 * y, s);
    c = s;
    rc = fma(y, fma(-s, y, 1.0), y);   // 1 / c, one reciprocal correction on the rounded c
}
__device__ __forceinline__ void sqrt_rsqrt(float q, float& c, float& rc)
{
    rc = rsqrtf(q);
    c = q * rc;
}

// Math in the state precision, named explicitly so that no float argument is
// ever promoted to a double routine (the FP64 pipe is 1/64 of FP32 on GB300).
__device__ __forceinline__ float vmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double vmax(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float vmin(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double vmin(double a, double b) { return fmin(a, b); }
// Maximum and minimum of non-negative values (rho c, 1/(rho c), 1/c, rates).
// For FP64 they compare the bit patterns as integers, which orders
// non-negative doubles as their values do and keeps the comparison off the
// FP64 pipe; a NaN operand wins the maximum (it is reported by the status word).
__device__ __forceinline__ float pmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ float pmin(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double pmax(double a, double b)
{
    return __longlong_as_double(max(__double_as_longlong(a), __double_as_longlong(b)));
}
__device__ __forceinline__ double pmin(double a, double b)
{
    return __longlong_as_double(min(__double_as_longlong(a), __double_as_longlong(b)));
}
__device__ __forceinline__ float vabs(float a) { return fabsf(a); }
__device__ __forceinline__ double vabs(double a) { return fabs(a); }
__device__ __forceinline__ float vsqrt(float a) { return sqrtf(a); }
__device__ __forceinline__ double vsqrt(double a) { return sqrt(a); }

template <typename Real>
__device__ __forceinline__ Real rsqrt_(Real x);
template <>
__device__ __forceinline__ double rsqrt_<double>(double x) { return rsqrt(x); }
template <>
__device__ __forceinline__ float rsqrt_<float>(float x) { return rsqrtf(x); }

// The stencil constants in the state precision, read from the arguments
// without conversion.
template <typename Real>
struct KConst;
template <>
struct KConst<float> {
    float K, halfInvK, mu, kappa, eta, gamma, gm1, pinf, gpinf, b, invdx[3];
    __device__ explicit KConst(const StepArgs& a)
        : K(a.fK), halfInvK(a.fhalfInvK), mu(a.fmu), kappa(a.fkappa), eta(a.feta), gamma(a.fgamma), gm1(a.fgm1),
          pinf(a.fpinf), gpinf(a.fgpinf), b(a.fb), invdx{a.finvdx[0], a.finvdx[1], a.finvdx[2]} {}
};
template <>
struct KConst<double> {
    double K, halfInvK, mu, kappa, eta, gamma, gm1, pinf, gpinf, b, invdx[3];
    __device__ explicit KConst(const StepArgs& a)
        : K(a.dK), halfInvK(a.dhalfInvK), mu(a.mu), kappa(a.kappa), eta(a.deta), gamma(a.gamma), gm1(a.gamma - 1.0),
          pinf(a.p_inf), gpinf(a.dgpinf), b(a.b), invdx{a.dinvdx[0], a.dinvdx[1], a.dinvdx[2]} {}
};

// Equation of state: the stiffened gas (Harlow and Amsden 1971; temperature
// as in Le Metayer, Massoni and Saurel 2004, with (gamma-1) c_v = 1), which
// the scheme admits as Sec. 4 notes that another equation of state may be
// used; p_inf = 0 is the ideal gas of Sec. 4:
//   p = (gamma-1) rho e - gamma p_inf,  T = (p + p_inf) / rho,
//   c^2 = gamma (p + p_inf) / rho.
// Every formula below reads the pressure either as a difference or as the
// effective pressure pe = p + p_inf.  In F32_SPLIT the base row carries
// pe0 = p0 + p_inf (B_P0), so deviations need no p_inf term at all.
// NA: the Noble-Abel stiffened gas (Le Metayer and Saurel 2016, without the
// reference energy), a second law of the same family: the covolume b leaves
// the fraction fv = 1 - b rho of the volume free,
//   p = (gamma-1) rho e / fv - gamma p_inf,  T = (p + p_inf) fv / rho,
//   c^2 = gamma (p + p_inf) / (rho fv);
// b = 0 is the stiffened gas.  The law is chosen per kernel instance (a
// template flag), so the stiffened-gas instances carry no covolume term.
template <typename Real, bool NA_ = false>
struct Eos {
    static constexpr bool NA = false;
    Real gamma, gm1, pinf, gpinf;   // gpinf = gamma p_inf
    __device__ explicit Eos(const KConst<Real>& k) : gamma(k.gamma), gm1(k.gm1), pinf(k.pinf), gpinf(k.gpinf) {}
};
template <typename Real>
struct Eos<Real, true> {
    static constexpr bool NA = true;
    Real gamma, gm1, pinf, gpinf;   // gpinf = gamma p_inf
    Real b;                         // covolume
    __device__ explicit Eos(const KConst<Real>& k)
        : gamma(k.gamma), gm1(k.gm1), pinf(k.pinf), gpinf(k.gpinf), b(k.b) {}
};

// Phi at the centre of row r of the gravity axis (Phi = -g x_last), in the
// state precision.  The FP64 form evaluates the oracle's expression; kernels
// keep (g, lo, dz) as Real constants so that FP32 forms do no FP64 work per
// plane (GB300's FP64 rate, conversions included, is 1/64 of its FP32 rate).
template <typename Real>
struct PhiRow {
    Real g, lo, dv;
    __device__ explicit PhiRow(const StepArgs& a)
        : g(sizeof(Real) == 8 ? Real(a.g) : Real(a.fphi_g)), lo(sizeof(Real) == 8 ? Real(a.lo_v) : Real(a.fphi_lo)),
          dv(sizeof(Real) == 8 ? Real(a.dx[a.dim - 1]) : Real(a.fphi_dv)) {}
    __device__ Real operator()(int r) const { return at(Real(r)); }
    __device__ Real at(Real r) const { return -(g * (lo + (r + Real(0.5)) * dv)); }
};

template <typename Real, bool SPLIT>
__device__ __forceinline__ Row<Real> row_info(const StepArgs& a, const PhiRow<Real>& ph, int r, int nv,
                                              Real rf = Real(-1e30))
{
    Row<Real> w;
    if constexpr (SPLIT) {
        const Real* B = static_cast<const Real*>(a.base) + base_index(0, r);
        w.rho0 = __ldg(B + B_RHO0);
        w.p0 = __ldg(B + B_P0);
        w.T0 = __ldg(B + B_T0);
    } else {
        w.rho0 = Real(0); w.p0 = Real(0); w.T0 = Real(0);
    }
    w.phi = rf > Real(-1e29) ? ph.at(rf) : ph(r);   // rf: the row as a Real, when the caller has it
    if (a.energy_form) w.phi = Real(0);              // rho E carries no potential energy (Appendix B)
    return w;
}

// Primitive values from conserved values (the equation of state above).
// Split form with a covolume: with re = rho e - rho0 e0 (the stored deviation),
//   dp = ((gamma-1) re + b (p0 + gamma p_inf) drho) / fv,
//   dT = (dp fv - (T0 + b pe0) drho) / rho,
// exact rearrangements of the law about the base row, O(deviation) throughout.
template <int D, typename Real, bool SPLIT, bool NA>
__device__ __forceinline__ void prim(Cell<D, Real>& c, const Row<Real>& w, const Eos<Real, NA>& q)
{
    c.rho = SPLIT ? w.rho0 + c.drho : c.drho;
    const Real rr = rcp(c.rho);
    c.rr = rr;
    Real ke = Real(0);
#pragma unroll
    for (int d = 0; d < D; ++d) {
        c.u[d] = c.m[d] * rr;
        ke += c.m[d] * c.u[d];
    }
    const Real re = c.dW - Real(0.5) * ke - c.drho * w.phi;
    if constexpr (NA) {
        const Real fv = Real(1) - q.b * c.rho;
        const Real rfv = rcp(fv);
        c.dp = SPLIT ? (q.gm1 * re + q.b * (w.p0 + q.gm1 * q.pinf) * c.drho) * rfv : q.gm1 * re * rfv - q.gpinf;
        const Real pe = SPLIT ? w.p0 + c.dp : c.dp + q.pinf;
        c.dT = SPLIT ? (c.dp * fv - (w.T0 + q.b * w.p0) * c.drho) * rr : pe * fv * rr;
        sqrt_rsqrt(q.gamma * pe * rr * rfv, c.c, c.rc);
    } else {
        c.dp = SPLIT ? q.gm1 * re : q.gm1 * re - q.gpinf;
        const Real pe = SPLIT ? w.p0 + c.dp : c.dp + q.pinf;
        c.dT = SPLIT ? (c.dp - w.T0 * c.drho) * rr : pe * rr;
        sqrt_rsqrt(q.gamma * pe * rr, c.c, c.rc);
    }
}

// Conserved values of a ghost built from primitives (rho full, u, dp, dT).
template <int D, typename Real, bool SPLIT, bool NA>
__device__ __forceinline__ void cons_from_prim(Cell<D, Real>& g, const Row<Real>& w, const Eos<Real, NA>& q)
{
    Real ke = Real(0);
#pragma unroll
    for (int d = 0; d < D; ++d) {
        g.m[d] = g.rho * g.u[d];
        ke += g.rho * g.u[d] * g.u[d];
    }
    if constexpr (NA) {
        // rho e = (p + gamma p_inf) fv / (gamma - 1); about the base row,
        // re = (dp fv - b (p0 + gamma p_inf) drho) / (gamma - 1)
        const Real fv = Real(1) - q.b * g.rho;
        const Real re = SPLIT ? (g.dp * fv - q.b * (w.p0 + q.gm1 * q.pinf) * g.drho) / q.gm1
                              : (g.dp + q.gpinf) * fv / q.gm1;
        g.dW = re + Real(0.5) * ke + g.drho * w.phi;
        const Real pe = SPLIT ? w.p0 + g.dp : g.dp + q.pinf;
        g.rr = rcp(g.rho);
        sqrt_rsqrt(q.gamma * pe * g.rr * rcp(fv), g.c, g.rc);
    } else {
        // rho e = (p + gamma p_inf) / (gamma - 1); the deviation form cancels gamma p_inf
        g.dW = (SPLIT ? g.dp : g.dp + q.gpinf) / q.gm1 + Real(0.5) * ke + g.drho * w.phi;
        const Real pe = SPLIT ? w.p0 + g.dp : g.dp + q.pinf;
        g.rr = rcp(g.rho);
        sqrt_rsqrt(q.gamma * pe * g.rr, g.c, g.rc);
    }
}

// Wall ghost (reflective hydrostatic or no-slip fixed-temperature): velocity
// mirrored (normal component, or all components, with sign flip);
// temperature mirrored or reflected about the wall value; pressure from the
// discrete hydrostatic balance of Eq. 18 with the inner neighbour A, in the
// effective pressure pe = p + p_inf (rho = pe / T):
//   pe_g = (pe_A - dPhi rho_A / 2) / (1 + dPhi / (2 T_g)),  rho_g = pe_g / T_g;
// in deviation form, with base ghost row (rho0_g, T0_g) built by the same rule,
//   dp_g = (dp_A - dPhi drho_A / 2 + dPhi rho0_g dT_g / (2 T_g)) / (1 + dPhi / (2 T_g)),
//   drho_g = (dp_g - rho0_g dT_g) / T_g.
//
// NA (covolume b): rho_g = pe_g / (T_g + b pe_g), so the balance is the
// quadratic b pe^2 + (T_g - b K + dPhi/2) pe - K T_g = 0, K = pe_A - rho_A dPhi / 2,
// solved by its positive root 2 K T_g / (B + sqrt(B^2 + 4 b K T_g)), B the
// linear coefficient (no cancellation).  In deviation form, with the base ghost
// row q0 = pe0_g, T0_g (the base quadratic with K0 = q0 + rho0_g dPhi / 2) and
// dK = dp_A - drho_A dPhi / 2, the deviation dp_g solves
//   b dp^2 + beta dp + g1 = 0,  beta = 2 b q0 + T0_g - b K0 + dPhi/2 + dT_g - b dK,
//   g1 = (dT_g - b dK) q0 - K0 dT_g - dK (T0_g + dT_g),
// dp_g = -2 g1 / (beta + sqrt(beta^2 - 4 b g1)), and
//   drho_g = (dp_g T0_g - q0 dT_g) / ((T_g + b pe_g) (T0_g + b q0));
// both reduce term by term to the lines above when b = 0.
template <int D, typename Real, bool SPLIT, bool NA>
__device__ __forceinline__ Cell<D, Real> wall_ghost(const Cell<D, Real>& M, const Cell<D, Real>& A, int bc,
                                                    int axis, Real Tw, const Row<Real>& wg, Real dphi,
                                                    const Eos<Real, NA>& q)
{
    Cell<D, Real> g;
#pragma unroll
    for (int k = 0; k < D; ++k) g.u[k] = (bc == BC_NOSLIP_T || k == axis) ? -M.u[k] : M.u[k];
    Real dTg;
    if (bc == BC_REFLECT) dTg = M.dT;
    else dTg = SPLIT ? -M.dT : Real(2) * Tw - M.dT;
    const Real Tg = SPLIT ? wg.T0 + dTg : dTg;
    if constexpr (NA) {
        if constexpr (SPLIT) {
            const Real q0 = wg.p0, T0 = wg.T0;
            const Real K0 = q0 + Real(0.5) * wg.rho0 * dphi;
            const Real dK = A.dp - Real(0.5) * A.drho * dphi;
            const Real beta = Real(2) * q.b * q0 + T0 - q.b * K0 + Real(0.5) * dphi + dTg - q.b * dK;
            const Real g1 = (dTg - q.b * dK) * q0 - K0 * dTg - dK * (T0 + dTg);
            const Real x = Real(-2) * g1 / (beta + vsqrt(beta * beta - Real(4) * q.b * g1));
            g.dp = x;
            g.drho = (x * T0 - q0 * dTg) / ((Tg + q.b * (q0 + x)) * (T0 + q.b * q0));
        } else {
            const Real K = A.dp + q.pinf - Real(0.5) * A.drho * dphi;
            const Real B = Tg - q.b * K + Real(0.5) * dphi;
            const Real pe = Real(2) * K * Tg / (B + vsqrt(B * B + Real(4) * q.b * K * Tg));
            g.dp = pe - q.pinf;
            g.drho = pe / (Tg + q.b * pe);
        }
    } else {
        Real num = (SPLIT ? A.dp : A.dp + q.pinf) - Real(0.5) * A.drho * dphi;
        if constexpr (SPLIT) num += Real(0.5) * wg.rho0 * dphi * dTg / Tg;
        const Real x = num / (Real(1) + dphi / (Real(2) * Tg));   // dp_g (split) or pe_g
        g.dp = SPLIT ? x : x - q.pinf;
        g.drho = SPLIT ? (x - wg.rho0 * dTg) / Tg : x / Tg;
    }
    g.dT = dTg;
    g.rho = SPLIT ? wg.rho0 + g.drho : g.drho;
    cons_from_prim<D, Real, SPLIT>(g, wg, q);
    return g;
}

// CFL wave rate of one cell (the time step is cfl / max over cells):
//   max( sum_d (|u_d| + c) / dx_d , sum_d 2 max(4 mu / (3 rho), kappa (gamma-1) / rho) / dx_d^2 ).
// b holds the cell's stored values (deviation form in F32_SPLIT); the
// effective pressure pe = p + p_inf and rho are returned for the physical
// checks (both must be positive).
template <int D, typename Real, bool SPLIT, bool VISC, bool NA>
__device__ __forceinline__ Real wave_rate(const Real* b, const Row<Real>& w, const Eos<Real, NA>& q,
                                          const Real* invdx, Real mu, Real kappa, Real& pe, Real& rho)
{
    rho = SPLIT ? w.rho0 + b[0] : b[0];
    const Real rr = rcp(rho);
    Real ke = Real(0), sh = Real(0);
    Real uu[D];
#pragma unroll
    for (int d = 0; d < D; ++d) {
        uu[d] = b[1 + d] * rr;
        ke += b[1 + d] * uu[d];
    }
    const Real re = b[D + 1] - Real(0.5) * ke - b[0] * w.phi;
    Real cs, rcs;
    if constexpr (NA) {   // covolume: the law of prim()
        const Real rfv = rcp(Real(1) - q.b * rho);
        const Real dp = SPLIT ? (q.gm1 * re + q.b * (w.p0 + q.gm1 * q.pinf) * b[0]) * rfv : q.gm1 * re * rfv - q.gpinf;
        pe = SPLIT ? w.p0 + dp : dp + q.pinf;
        sqrt_rsqrt(q.gamma * pe * rr * rfv, cs, rcs);
    } else {
        const Real dp = SPLIT ? q.gm1 * re : q.gm1 * re - q.gpinf;
        pe = SPLIT ? w.p0 + dp : dp + q.pinf;
        sqrt_rsqrt(q.gamma * pe * rr, cs, rcs);
    }
#pragma unroll
    for (int d = 0; d < D; ++d) sh += (vabs(uu[d]) + cs) * invdx[d];
    if constexpr (VISC) {
        const Real nu = Real(4.0 / 3.0) * mu * rr, chi = kappa * q.gm1 * rr;
        const Real dm = pmax(nu, chi);
        Real s2 = Real(0);   // sum_d 2 / dx_d^2 (loop-invariant)
#pragma unroll
        for (int d = 0; d < D; ++d) s2 += Real(2) * invdx[d] * invdx[d];
        sh = pmax(sh, dm * s2);
    }
    return sh;
}

// Potential of a caller-supplied array at any cell within two layers of the
// box (R20): interior cells read the array; a ghost resolves its out-of-range
// axes from the last to the first, as the state's ghost rule does -- across a
// periodic side it takes the cell on the other side, across a wall or outflow
// side the linear extension (1 + L) Phi_0 - L Phi_1 of the boundary cell and
// its inner neighbour along that axis (ghost layer L = 1, 2).
template <int AX, typename Real>
__device__ Real phi_resolve(const StepArgs& a, const Real* __restrict__ P, int i0, int i1, int i2)
{
    if constexpr (AX < 0) {
        return __ldg(P + (i0 + (long long)a.n[0] * (i1 + (long long)a.n[1] * i2)));
    } else {
        int idx[3] = {i0, i1, i2};
        const int n = a.n[AX];
        if (idx[AX] >= 0 && idx[AX] < n) return phi_resolve<AX - 1, Real>(a, P, i0, i1, i2);
        const bool lo = idx[AX] < 0;
        const int bc = lo ? a.bc_lo[AX] : a.bc_hi[AX];
        if (bc == BC_PERIODIC) {
            idx[AX] = ((idx[AX] % n) + n) % n;
            return phi_resolve<AX - 1, Real>(a, P, idx[0], idx[1], idx[2]);
        }
        const int layer = lo ? -idx[AX] : idx[AX] - n + 1;
        int jdx[3] = {i0, i1, i2};
        idx[AX] = lo ? 0 : n - 1;
        jdx[AX] = lo ? 1 : n - 2;
        return Real(1 + layer) * phi_resolve<AX - 1, Real>(a, P, idx[0], idx[1], idx[2]) -
               Real(layer) * phi_resolve<AX - 1, Real>(a, P, jdx[0], jdx[1], jdx[2]);
    }
}

// Loader of any cell within two layers of the tile, boundary rules included.
// PHIA: the potential is the caller's array (phi_resolve) instead of -g x_last,
// so ghosts across in-plane walls see its jumps too.
template <int DIM, typename Real, bool SPLIT, bool VISC, int TX, int TY, bool PHIA = false, bool NA = false>
struct Stepper {
    using C = StepCfg<DIM, Real, SPLIT, VISC, TX, TY>;
    static constexpr int D = DIM;
    static constexpr int NF = DIM + 2;
    static constexpr int V = DIM - 1;   // index of the gravity (marching) axis

    const StepArgs& a;
    const Real* __restrict__ U;
    long long N;
    int nx, ny, nv;
    PhiRow<Real> phi;
    Eos<Real, NA> eos;

    __device__ Stepper(const StepArgs& args) : a(args), phi(args), eos(KConst<Real>(args))
    {
        U = static_cast<const Real*>(a.Uin);
        N = a.ncell;
        nx = a.n[0];
        ny = D == 3 ? a.n[1] : 1;
        nv = a.n[V];
    }

    // Phi at (gx, gy, gv) (ghosts included), in the state precision
    __device__ Real phi_cell(int gx, int gy, int gv) const
    {
        if constexpr (PHIA) {
            const Real* P = static_cast<const Real*>(a.phiA);
            return D == 3 ? phi_resolve<2, Real>(a, P, gx, gy, gv) : phi_resolve<1, Real>(a, P, gx, gv, 0);
        } else {
            return phi(gv);
        }
    }
    // the row values of plane gv with the potential of cell (gx, gy, gv)
    __device__ Row<Real> at(const Row<Real>& w, int gx, int gy, int gv) const
    {
        if constexpr (PHIA) {
            Row<Real> r = w;
            r.phi = a.energy_form ? Real(0) : phi_cell(gx, gy, gv);
            return r;
        } else {
            return w;
        }
    }
    __device__ Cell<D, Real> load_in(int gx, int gy, int gv, const Row<Real>& w) const
    {
        long long idx = D == 3 ? gx + (long long)nx * (gy + (long long)ny * gv) : gx + (long long)nx * gv;
        Cell<D, Real> c;
        c.drho = __ldg(U + idx);
#pragma unroll
        for (int d = 0; d < D; ++d) c.m[d] = __ldg(U + (1 + d) * N + idx);
        c.dW = __ldg(U + (D + 1) * N + idx);
        prim<D, Real, SPLIT>(c, at(w, gx, gy, gv), eos);
        return c;
    }

    // Ghost layer `layer` (1, 2) beyond a BC_HALO side of x at row gy of plane
    // gv: a cell of the neighbouring subdomain (Sec. 3.2: ghost zones hold the
    // neighbours' cells), stored by the caller in the state's form.
    __device__ Cell<D, Real> load_halo(bool lo, int layer, int gy, int gv, const Row<Real>& w) const
    {
        const Real* __restrict__ H = static_cast<const Real*>(a.halo[lo ? 0 : 1]);
        const long long per = (long long)nv * ny * 2;
        const long long idx = ((long long)gv * ny + gy) * 2 + (layer - 1);
        Cell<D, Real> c;
        c.drho = __ldg(H + idx);
#pragma unroll
        for (int d = 0; d < D; ++d) c.m[d] = __ldg(H + (1 + d) * per + idx);
        c.dW = __ldg(H + (D + 1) * per + idx);
        prim<D, Real, SPLIT>(c, w, eos);
        return c;
    }

    // in-plane axis rule (axis 0 = x, axis 1 = y in 3D).  All in-plane
    // ghosts share the row of their plane; for uniform gravity along the last
    // axis dPhi = 0 across in-plane walls, with a Phi array the wall ghost sees
    // the array's jump (ghost minus inner neighbour).
    __device__ Cell<D, Real> fetch_x(int gx, int gy, int gv, const Row<Real>& w) const
    {
        if (gx >= 0 && gx < nx) return load_in(gx, gy, gv, w);
        const bool lo = gx < 0;
        const int bc = lo ? a.bc_lo[0] : a.bc_hi[0];
        if (bc == BC_PERIODIC) return load_in(((gx % nx) + nx) % nx, gy, gv, w);
        if (bc == BC_HALO) return load_halo(lo, lo ? -gx : gx - nx + 1, gy, gv, w);
        if (bc == BC_OUTFLOW) {
            Cell<D, Real> M = load_in(lo ? 0 : nx - 1, gy, gv, w);
            if constexpr (PHIA) cons_from_prim<D, Real, SPLIT>(M, at(w, gx, gy, gv), eos);
            return M;
        }
        const Real Tw = Real(lo ? a.Tw_lo[0] : a.Tw_hi[0]);
        const int x0 = lo ? 0 : nx - 1, x1 = lo ? 1 : nx - 2, g1 = lo ? -1 : nx;
        const Cell<D, Real> M0 = load_in(x0, gy, gv, w);
        const Real d1 = PHIA ? phi_cell(g1, gy, gv) - phi_cell(x0, gy, gv) : Real(0);
        Cell<D, Real> g1c = wall_ghost<D, Real, SPLIT>(M0, M0, bc, 0, Tw, at(w, g1, gy, gv), d1, eos);
        const int layer = lo ? -gx : gx - nx + 1;
        if (layer == 1) return g1c;
        const Cell<D, Real> M1 = load_in(x1, gy, gv, w);
        const Real d2 = PHIA ? phi_cell(gx, gy, gv) - phi_cell(g1, gy, gv) : Real(0);
        return wall_ghost<D, Real, SPLIT>(M1, g1c, bc, 0, Tw, at(w, gx, gy, gv), d2, eos);
    }

    __device__ Cell<D, Real> fetch_h(int gx, int gy, int gv, const Row<Real>& w) const
    {
        if constexpr (D == 3) {
            if (gy < 0 || gy >= ny) {
                const bool lo = gy < 0;
                const int bc = lo ? a.bc_lo[1] : a.bc_hi[1];
                if (bc == BC_PERIODIC) return fetch_x(gx, ((gy % ny) + ny) % ny, gv, w);
                if (bc == BC_OUTFLOW) {
                    Cell<D, Real> M = fetch_x(gx, lo ? 0 : ny - 1, gv, w);
                    if constexpr (PHIA) cons_from_prim<D, Real, SPLIT>(M, at(w, gx, gy, gv), eos);
                    return M;
                }
                const Real Tw = Real(lo ? a.Tw_lo[1] : a.Tw_hi[1]);
                const int y0 = lo ? 0 : ny - 1, y1 = lo ? 1 : ny - 2, g1 = lo ? -1 : ny;
                const Cell<D, Real> M0 = fetch_x(gx, y0, gv, w);
                const Real d1 = PHIA ? phi_cell(gx, g1, gv) - phi_cell(gx, y0, gv) : Real(0);
                Cell<D, Real> g1c = wall_ghost<D, Real, SPLIT>(M0, M0, bc, 1, Tw, at(w, gx, g1, gv), d1, eos);
                const int layer = lo ? -gy : gy - ny + 1;
                if (layer == 1) return g1c;
                const Cell<D, Real> M1 = fetch_x(gx, y1, gv, w);
                const Real d2 = PHIA ? phi_cell(gx, gy, gv) - phi_cell(gx, g1, gv) : Real(0);
                return wall_ghost<D, Real, SPLIT>(M1, g1c, bc, 1, Tw, at(w, gx, gy, gv), d2, eos);
            }
        }
        return fetch_x(gx, gy, gv, w);
    }

    // full rule: the gravity axis is applied last (x, then y, then the last axis).
    // Out of line: only cells of ghost planes and of tiles touching the box edge come here.
    __device__ __noinline__ Cell<D, Real> fetch(int gx, int gy, int gv) const
    {
        if (gv >= 0 && gv < nv) return fetch_h(gx, gy, gv, row_info<Real, SPLIT>(a, phi, gv, nv));
        const bool lo = gv < 0;
        const int bc = lo ? a.bc_lo[V] : a.bc_hi[V];
        if (bc == BC_PERIODIC) {
            const int s = ((gv % nv) + nv) % nv;
            return fetch_h(gx, gy, s, row_info<Real, SPLIT>(a, phi, s, nv));
        }
        const Row<Real> wg = row_info<Real, SPLIT>(a, phi, gv, nv);
        if (bc == BC_OUTFLOW) {
            const int s = lo ? 0 : nv - 1;
            Cell<D, Real> M = fetch_h(gx, gy, s, row_info<Real, SPLIT>(a, phi, s, nv));
            Cell<D, Real> g = M;   // (rho, u, p) copied; base rows of an outflow ghost copy the edge row
            cons_from_prim<D, Real, SPLIT>(g, at(wg, gx, gy, gv), eos);
            return g;
        }
        const Real Tw = Real(lo ? a.Tw_lo[V] : a.Tw_hi[V]);
        const int r0 = lo ? 0 : nv - 1, r1 = lo ? 1 : nv - 2, g1r = lo ? -1 : nv;
        const Row<Real> w0 = row_info<Real, SPLIT>(a, phi, r0, nv);
        const Row<Real> w1g = row_info<Real, SPLIT>(a, phi, g1r, nv);
        const Cell<D, Real> M0 = fetch_h(gx, gy, r0, w0);
        const Real dphi1 = phi_cell(gx, gy, g1r) - phi_cell(gx, gy, r0);
        Cell<D, Real> g1 = wall_ghost<D, Real, SPLIT>(M0, M0, bc, V, Tw, at(w1g, gx, gy, g1r), dphi1, eos);
        if (gv == g1r) return g1;
        const Row<Real> w1 = row_info<Real, SPLIT>(a, phi, r1, nv);
        const Cell<D, Real> M1 = fetch_h(gx, gy, r1, w1);
        const Real dphi2 = phi_cell(gx, gy, gv) - phi_cell(gx, gy, g1r);
        return wall_ghost<D, Real, SPLIT>(M1, g1, bc, V, Tw, at(wg, gx, gy, gv), dphi2, eos);
    }
};

// Acoustic face values of Sec. 2.1.2 with the low-Mach correction (Eq. 16):
//   a = K max(z_L, z_R), z = rho c;  u* = (u_L + u_R)/2 - (p_R - p_L - S)/(2a);
//   theta = min(|u*| / max(c_L, c_R), 1);  Pi* = (p_L + p_R)/2 - a theta (u_R - u_L)/2.
// Deviation form: pjump = (base residual) + dp_R - dp_L - dS, dPi* excludes the
// base face pressure (p0_L + p0_R)/2.  1/(2a) and 1/max(c) use per-cell reciprocals.
template <typename Real>
__device__ __forceinline__ void acoustic_face(Real uL, Real uR, Real dpL, Real dpR, Real zL, Real zR, Real rzL,
                                              Real rzR, Real rcL, Real rcR, Real pjump_base, Real dS, Real K,
                                              Real halfInvK, int low_mach, Real& ustar, Real& dPi)
{
    const Real a = K * pmax(zL, zR);
    const Real inv2a = halfInvK * pmin(rzL, rzR);
    ustar = Real(0.5) * (uL + uR) - (pjump_base + dpR - dpL - dS) * inv2a;
    Real theta = Real(1);
    if (low_mach) theta = pmin(vabs(ustar) * pmin(rcL, rcR), Real(1));
    dPi = Real(0.5) * (dpL + dpR) - Real(0.5) * a * theta * (uR - uL);
}

template <int N>
struct IC {
    static constexpr int value = N;
};

// Block maximum of non-negative CFL rates into *slot: warp-shuffle maxima of
// the FP64 bit patterns (non-negative doubles order like their bit patterns,
// so the result is exact and independent of the order), one shared slot per
// warp, then one atomicMax per block.  Every thread of the block calls it.
__device__ __forceinline__ void block_rate_max(double v, unsigned long long* red, unsigned long long* slot)
{
    unsigned long long b = (unsigned long long)__double_as_longlong(v);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long c = __shfl_xor_sync(0xffffffffu, b, o);
        b = c > b ? c : b;
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) red[w] = b;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long m = red[0];
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) m = red[k] > m ? red[k] : m;
        atomicMax(slot, m);
    }
}

// Store one loaded cell (conserved + primitive values) into the plane rings.
template <class C, int D, typename Real>
__device__ __forceinline__ void store_cell(const Cell<D, Real>& x, Real* vT, Real* ff, Real* uc, int c, int lx, int ly)
{
#pragma unroll
    for (int d = 0; d < D; ++d) vT[d * C::NR2 + c] = x.u[d];
    if constexpr (C::NVT > D) vT[D * C::NR2 + c] = x.dT;
    const Real rc = x.rc;
    ff[0 * C::NR2 + c] = x.dp;
    ff[1 * C::NR2 + c] = rc;
    ff[2 * C::NR2 + c] = x.rho * x.c;
    ff[3 * C::NR2 + c] = rc * x.rr;
    if (lx >= -1 && lx <= C::TXV && ly >= -C::H1 && ly < C::R1Y - C::H1) {
        const int c1 = C::i1(lx, ly);
        uc[c1] = x.drho;
#pragma unroll
        for (int d = 0; d < D; ++d) uc[(1 + d) * C::NR1 + c1] = x.m[d];
        uc[(D + 1) * C::NR1 + c1] = x.dW;
    }
}

// Cells of ghost planes and of tiles that touch the box edge: boundary rules,
// out of line so that the interior path stays in registers.
// PHIA: the cell's density and potential also go to the ring ph (rho, Phi).
template <int DIM, typename Real, bool SPLIT, bool VISC, int TX, int TY, bool PHIA = false, bool NA = false>
__device__ __noinline__ void slow_cell(const Stepper<DIM, Real, SPLIT, VISC, TX, TY, PHIA, NA> S, int gx, int gy, int f,
                                       Real* vT, Real* ff, Real* uc, Real* ph, int c, int lx, int ly)
{
    using C = StepCfg<DIM, Real, SPLIT, VISC, TX, TY, PHIA>;
    const Cell<DIM, Real> x = S.fetch(gx, gy, f);
    store_cell<C, DIM, Real>(x, vT, ff, uc, c, lx, ly);
    if constexpr (PHIA) {
        ph[c] = x.rho;
        ph[C::NR2 + c] = S.phi_cell(gx, gy, f);
    }
}

// One block's share of a step: in-plane tile `tile`, planes [z0, z1) of the
// gravity axis; `lead` marks the one share per step that advances the clock.
// Called by the single-grid kernel (runs of planes of a balanced schedule) and
// by the batched kernel (work items of many runs).
template <int DIM, typename Real, bool SPLIT, bool VISC, int TX, int TY, bool PHIA = false, bool NA = false>
__device__ __forceinline__ void step_block(const StepArgs& a, const int tile, const int z0, const int z1,
                                           const bool lead, unsigned char* smem_raw)
{
    using C = StepCfg<DIM, Real, SPLIT, VISC, TX, TY, PHIA>;
    constexpr int D = DIM, NF = DIM + 2, V = DIM - 1;
    constexpr int NT = C::NT, NR1 = C::NR1, NR2 = C::NR2, NVT = C::NVT;
    constexpr int NSLOT = (NR2 + NT - 1) / NT;
    Real* sm = reinterpret_cast<Real*>(smem_raw);
    double* red = reinterpret_cast<double*>(smem_raw + ((C::N_REAL * sizeof(Real) + 15) / 16) * 16);

    const Stepper<DIM, Real, SPLIT, VISC, TX, TY, PHIA, NA> S(a);
    const int tid = threadIdx.x;
    const int x0 = (tile % a.tiles_x) * TX;
    const int y0 = D == 3 ? (tile / a.tiles_x) * TY : 0;
    const int nx = S.nx, ny = S.ny, nv = S.nv;
    const Real* __restrict__ U = S.U;
    const long long N = S.N;

    // time step of this step (identical in every block), formed once by one
    // thread and shared: nothing FP64 is left for the compiler to recompute
    Real* const sdt = reinterpret_cast<Real*>(red + NT);
    if (tid == 0) {
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
    Real lam[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) lam[d] = sdt[1 + d];
    const Real dt = sdt[0];
    const Real K = kc.K, halfInvK = kc.halfInvK;
    const Real mu = kc.mu, kappa = kc.kappa, eta = kc.eta;
    const Real invdx[3] = {kc.invdx[0], kc.invdx[1], kc.invdx[2]};
    const Real* __restrict__ Bt = static_cast<const Real*>(a.base);
    auto base = [&](int field, int r) -> Real { return SPLIT ? __ldg(Bt + base_index(field, r)) : Real(0); };

    // this thread's output cell
    const int olx = tid % TX, oly = tid / TX;
    const int ogx = x0 + olx, ogy = y0 + oly;
    const bool ocol = ogx < nx && (D == 2 || ogy < ny);

    // this thread's load slots (fixed in-plane positions)
    // (across a periodic in-plane boundary a halo cell is the interior cell on
    // the other side, loaded directly; walls and outflow take the ghost rule)
    int sgx[NSLOT], sgy[NSLOT];
    bool sin[NSLOT];
    long long sidx[NSLOT];
    auto wrap = [](int g, int n) { return g < 0 ? g + n : (g >= n ? g - n : g); };
    const bool perx = a.bc_lo[0] == BC_PERIODIC && nx >= 2, pery = D == 3 && a.bc_lo[1] == BC_PERIODIC && ny >= 2;
#pragma unroll
    for (int s = 0; s < NSLOT; ++s) {
        const int c = tid + s * NT;
        const int lx = c % C::R2X - 2, ly = c / C::R2X - C::HY;
        const int gxw = perx ? wrap(x0 + lx, nx) : x0 + lx, gyw = pery ? wrap(y0 + ly, ny) : y0 + ly;
        sgx[s] = min(max(gxw, -2), nx + 1);
        sgy[s] = D == 3 ? min(max(gyw, -2), ny + 1) : 0;
        sin[s] = c < NR2 && sgx[s] >= 0 && sgx[s] < nx && (D == 2 || (sgy[s] >= 0 && sgy[s] < ny));
        sidx[s] = D == 3 ? sgx[s] + (long long)nx * sgy[s] : sgx[s];
    }
    const long long plane_cells = D == 3 ? (long long)nx * ny : (long long)nx;
    Real raw[NSLOT][NF];
    Real rawphi[NSLOT];        // caller's potential of the prefetched cells (PHIA)
    const Real* __restrict__ Pa = static_cast<const Real*>(a.phiA);
    auto prefetch = [&](int p) {
        if (p < 0 || p >= nv) return;
#pragma unroll
        for (int s = 0; s < NSLOT; ++s) {
            if (sin[s]) {
                const long long idx = sidx[s] + plane_cells * p;
#pragma unroll
                for (int k = 0; k < NF; ++k) raw[s][k] = __ldg(U + k * N + idx);
                if constexpr (PHIA) rawphi[s] = __ldg(Pa + idx);
            }
        }
    };
    prefetch(z0 - 2);

    // register carries along the column
    Real zt_lo[NF];            // transport flux through the lower z face of the output plane
    Real us_lo = Real(0);      // u* there
    Real zvA[C::NV], zvB[C::NV], dxy_prev[C::NV];
#pragma unroll
    for (int q = 0; q < NF; ++q) zt_lo[q] = Real(0);
#pragma unroll
    for (int q = 0; q < C::NV; ++q) { zvA[q] = zvB[q] = dxy_prev[q] = Real(0); }
    Real smax_t = Real(0);
    unsigned status = 0u;

    for (int f = z0 - 2; f <= z1 + 1; ++f) {
        // ring slots of this iteration
        const int s3 = ((f % 3) + 3) % 3;
        Real* const vT_f = sm + C::O_VELT + s3 * NVT * NR2;
        Real* const vT_f1 = sm + C::O_VELT + ((s3 + 2) % 3) * NVT * NR2;
        Real* const vT_f2 = sm + C::O_VELT + ((s3 + 1) % 3) * NVT * NR2;
        Real* const ff_f = sm + C::O_FACEF + (f & 1) * 4 * NR2;
        Real* const ff_f1 = sm + C::O_FACEF + ((f - 1) & 1) * 4 * NR2;
        Real* const uc_f = sm + C::O_UCONS + (f & 1) * NF * NR1;
        Real* const uc_f1 = sm + C::O_UCONS + ((f - 1) & 1) * NF * NR1;
        Real* const zf_up = sm + C::O_ZF + (f & 1) * 3 * NR1;          // face (f-1, f)
        Real* const zf_lo = sm + C::O_ZF + ((f - 1) & 1) * 3 * NR1;    // face (f-2, f-1)
        Real* const xy_f1 = sm + C::O_XYF + ((f - 1) & 1) * C::NXYC * (C::NFX + C::NFY);
        Real* const xy_f2 = sm + C::O_XYF + ((f - 2) & 1) * C::NXYC * (C::NFX + C::NFY);
        Real* const ph_f = sm + C::O_PH + (f & 1) * 2 * NR2;           // rho, Phi of plane f (PHIA)
        Real* const ph_f1 = sm + C::O_PH + ((f - 1) & 1) * 2 * NR2;    // of plane f-1
        Real* const tl_f1 = sm + C::O_TL + ((f - 1) & 1) * (NF + 1) * NR1;
        Real* const tl_f2 = sm + C::O_TL + ((f - 2) & 1) * (NF + 1) * NR1;
        Real* const tfx = sm + C::O_TFLUX;
        Real* const vfx = sm + C::O_VFLUX;
        constexpr int XYS = C::NFX + C::NFY;     // component stride of the in-plane face arrays
        constexpr int TFS = C::NTX + C::NTY;     // component stride of the output-face arrays

        // ---------------- A: plane f (primitives), prefetch of plane f + 1 ----------------
        const Real fr = Real(f);   // plane index as a Real: rows' Phi without further conversions
        const bool fin = f >= 0 && f < nv;
        const Row<Real> wf = row_info<Real, SPLIT>(a, S.phi, fin ? f : 0, nv, fin ? fr : Real(0));
#pragma unroll
        for (int s = 0; s < NSLOT; ++s) {
            const int c = tid + s * NT;
            if (c < NR2) {
                const int lx = c % C::R2X - 2, ly = c / C::R2X - C::HY;
                if (fin && sin[s]) {
                    Cell<D, Real> x;
                    x.drho = raw[s][0];
#pragma unroll
                    for (int d = 0; d < D; ++d) x.m[d] = raw[s][1 + d];
                    x.dW = raw[s][D + 1];
                    Row<Real> w = wf;
                    if constexpr (PHIA) w.phi = a.energy_form ? Real(0) : rawphi[s];
                    prim<D, Real, SPLIT>(x, w, S.eos);
                    store_cell<C, D, Real>(x, vT_f, ff_f, uc_f, c, lx, ly);
                    if constexpr (PHIA) {
                        ph_f[c] = x.rho;
                        ph_f[NR2 + c] = rawphi[s];
                    }
                } else {
                    slow_cell<DIM, Real, SPLIT, VISC, TX, TY, PHIA, NA>(S, sgx[s], sgy[s], f, vT_f, ff_f, uc_f, ph_f, c, lx, ly);
                }
            }
        }
        prefetch(f + 1);
        __syncthreads();

        // ---------------- B: acoustic faces ----------------
        if (f >= z0) {
            // in-plane x faces of plane f-1 bounding R1 cells
            for (int e = tid; e < C::NFX; e += NT) {
                const int lx = e % C::FXX - 2, ly = e / C::FXX - C::H1;
                const int iL = C::i2(lx, ly), iR = iL + 1;
                Real us, dPi, dS = Real(0);
                if constexpr (PHIA) dS = Real(-0.5) * (ph_f1[iL] + ph_f1[iR]) * (ph_f1[NR2 + iR] - ph_f1[NR2 + iL]);
                acoustic_face<Real>(vT_f1[iL], vT_f1[iR], ff_f1[iL], ff_f1[iR], ff_f1[2 * NR2 + iL],
                                    ff_f1[2 * NR2 + iR], ff_f1[3 * NR2 + iL], ff_f1[3 * NR2 + iR], ff_f1[NR2 + iL],
                                    ff_f1[NR2 + iR], Real(0), dS, K, halfInvK, a.low_mach, us, dPi);
                xy_f1[e] = us;
                xy_f1[XYS + e] = dPi;
                if constexpr (PHIA) xy_f1[2 * XYS + e] = dS;
            }
            if constexpr (D == 3) {
                for (int e = tid; e < C::NFY; e += NT) {
                    const int lx = e % C::R1X - 1, ly = e / C::R1X - 2;
                    const int iL = C::i2(lx, ly), iR = iL + C::R2X;
                    Real us, dPi, dS = Real(0);
                    if constexpr (PHIA) dS = Real(-0.5) * (ph_f1[iL] + ph_f1[iR]) * (ph_f1[NR2 + iR] - ph_f1[NR2 + iL]);
                    acoustic_face<Real>(vT_f1[NR2 + iL], vT_f1[NR2 + iR], ff_f1[iL], ff_f1[iR], ff_f1[2 * NR2 + iL],
                                        ff_f1[2 * NR2 + iR], ff_f1[3 * NR2 + iL], ff_f1[3 * NR2 + iR],
                                        ff_f1[NR2 + iL], ff_f1[NR2 + iR], Real(0), dS, K, halfInvK,
                                        a.low_mach, us, dPi);
                    xy_f1[C::NFX + e] = us;
                    xy_f1[XYS + C::NFX + e] = dPi;
                    if constexpr (PHIA) xy_f1[2 * XYS + C::NFX + e] = dS;
                }
            }
        }
        if (f >= z0 - 1) {
            // faces between planes f-1 (low side) and f (high side), over R1 cells
            const Real dphi = S.phi.at(fr) - S.phi.at(fr - Real(1));
            const Real r0f = base(B_R0F, f - 1);
            for (int c = tid; c < NR1; c += NT) {
                const int lx = c % C::R1X - 1, ly = c / C::R1X - C::H1;
                const int i = C::i2(lx, ly);
                const Real dS = Real(-0.5) * (uc_f1[c] + uc_f[c]) * (PHIA ? ph_f[NR2 + i] - ph_f1[NR2 + i] : dphi);
                Real us, dPi;
                acoustic_face<Real>(vT_f1[V * NR2 + i], vT_f[V * NR2 + i], ff_f1[i], ff_f[i], ff_f1[2 * NR2 + i],
                                    ff_f[2 * NR2 + i], ff_f1[3 * NR2 + i], ff_f[3 * NR2 + i], ff_f1[NR2 + i],
                                    ff_f[NR2 + i], r0f, dS, K, halfInvK, a.low_mach, us, dPi);
                zf_up[c] = us;
                zf_up[NR1 + c] = dPi;
                zf_up[2 * NR1 + c] = dS;
            }
        }
        __syncthreads();

        // ---------------- C: tilde states of plane f-1; dissipative fluxes ----------------
        const int q1 = f - 1;
        if (f >= z0) {
            const Real rho0 = base(B_RHO0, q1), H0 = base(B_H0, q1), Q0 = base(B_Q0, q1);
            const Real dPp = base(B_DPP, q1), dPm = base(B_DPM, q1);
            for (int c = tid; c < NR1; c += NT) {
                const int lx = c % C::R1X - 1, ly = c / C::R1X - C::H1;
                const int exp_ = C::ifx(lx, ly), exm = exp_ - 1;
                const Real usx_p = xy_f1[exp_], usx_m = xy_f1[exm];
                const Real pix_p = xy_f1[XYS + exp_], pix_m = xy_f1[XYS + exm];
                const Real usz_p = zf_up[c], usz_m = zf_lo[c];
                const Real piz_p = zf_up[NR1 + c], piz_m = zf_lo[NR1 + c];
                const Real dSz_p = zf_up[2 * NR1 + c], dSz_m = zf_lo[2 * NR1 + c];
                Real ell = lam[0] * (usx_p - usx_m);
                Real m_t[D];
                m_t[0] = uc_f1[NR1 + c] - lam[0] * (pix_p - pix_m);
                Real W_t = uc_f1[(D + 1) * NR1 + c] - lam[0] * (pix_p * usx_p - pix_m * usx_m);
                if constexpr (PHIA) {   // gravity source of the in-plane faces (the caller's Phi varies in x)
                    const Real sx_p = xy_f1[2 * XYS + exp_], sx_m = xy_f1[2 * XYS + exm];
                    m_t[0] += lam[0] * Real(0.5) * (sx_p + sx_m);
                    if (a.energy_form) W_t += lam[0] * Real(0.5) * (usx_p * sx_p + usx_m * sx_m);
                }
                if constexpr (D == 3) {
                    const int eyp = C::NFX + C::ify(lx, ly), eym = eyp - C::R1X;
                    const Real usy_p = xy_f1[eyp], usy_m = xy_f1[eym];
                    const Real piy_p = xy_f1[XYS + eyp], piy_m = xy_f1[XYS + eym];
                    ell += lam[1] * (usy_p - usy_m);
                    m_t[1] = uc_f1[2 * NR1 + c] - lam[1] * (piy_p - piy_m);
                    W_t -= lam[1] * (piy_p * usy_p - piy_m * usy_m);
                    if constexpr (PHIA) {
                        const Real sy_p = xy_f1[2 * XYS + eyp], sy_m = xy_f1[2 * XYS + eym];
                        m_t[1] += lam[1] * Real(0.5) * (sy_p + sy_m);
                        if (a.energy_form) W_t += lam[1] * Real(0.5) * (usy_p * sy_p + usy_m * sy_m);
                    }
                }
                ell += lam[V] * (usz_p - usz_m);
                m_t[V] = uc_f1[(1 + V) * NR1 + c] - lam[V] * (piz_p - piz_m) + lam[V] * Real(0.5) * (dSz_p + dSz_m);
                if constexpr (SPLIT) m_t[V] -= lam[V] * Q0;
                W_t -= lam[V] * (piz_p * usz_p - piz_m * usz_m);
                if constexpr (SPLIT) W_t -= lam[V] * (dPp * usz_p - dPm * usz_m) + H0 * ell;
                if (a.energy_form) W_t += lam[V] * Real(0.5) * (usz_p * dSz_p + usz_m * dSz_m);   // (uS)_i, Appendix B
                const Real L = Real(1) + ell;
                const Real rL = rcp(L);
                tl_f1[c] = SPLIT ? (uc_f1[c] - rho0 * ell) * rL : uc_f1[c] * rL;
#pragma unroll
                for (int d = 0; d < D; ++d) tl_f1[(1 + d) * NR1 + c] = m_t[d] * rL;
                tl_f1[(D + 1) * NR1 + c] = W_t * rL;
                tl_f1[NF * NR1 + c] = L;
                const bool valid = (x0 + lx) >= 0 && (x0 + lx) < nx &&
                                   (D == 2 || ((y0 + ly) >= 0 && (y0 + ly) < ny)) && q1 >= 0 && q1 < nv;
                if (valid && !(L > Real(0))) status |= ST_LTILDE;
            }
        }
        if constexpr (VISC) {
            // dissipative fluxes (Sec. 2.2) from U^n through the in-plane faces of plane
            // f-1's output cells; tangential derivatives averaged over the face's two cells
            if (f >= z0 + 1 && f <= z1) {
                auto face = [&](auto dirc, int lxL, int lyL, int te) {
                    constexpr int dir = decltype(dirc)::value;
                    constexpr int sh = dir == 0 ? 1 : C::R2X;
                    const int iL = C::i2(lxL, lyL), iR = iL + sh;
                    Real grad[3][3];
#pragma unroll
                    for (int aa = 0; aa < 3; ++aa)
#pragma unroll
                        for (int qq = 0; qq < 3; ++qq) grad[aa][qq] = Real(0);
#pragma unroll
                    for (int qq = 0; qq < D; ++qq) grad[dir][qq] = (vT_f1[qq * NR2 + iR] - vT_f1[qq * NR2 + iL]) * invdx[dir];
                    if constexpr (D == 3) {
                        constexpr int t = 1 - dir;
                        constexpr int st = t == 0 ? 1 : C::R2X;
#pragma unroll
                        for (int qq = 0; qq < D; ++qq)
                            grad[t][qq] = Real(0.25) *
                                          ((vT_f1[qq * NR2 + iL + st] - vT_f1[qq * NR2 + iL - st]) +
                                           (vT_f1[qq * NR2 + iR + st] - vT_f1[qq * NR2 + iR - st])) *
                                          invdx[t];
                    }
#pragma unroll
                    for (int qq = 0; qq < D; ++qq)
                        grad[V][qq] = Real(0.25) *
                                      ((vT_f[qq * NR2 + iL] - vT_f2[qq * NR2 + iL]) +
                                       (vT_f[qq * NR2 + iR] - vT_f2[qq * NR2 + iR])) *
                                      invdx[V];
                    Real divu = Real(0);
#pragma unroll
                    for (int aa = 0; aa < D; ++aa) divu += grad[aa][aa];
                    Real work = Real(0);
#pragma unroll
                    for (int qq = 0; qq < D; ++qq) {
                        Real tau = mu * (grad[dir][qq] + grad[qq][dir]);
                        if (qq == dir) tau += eta * divu;
                        work += tau * Real(0.5) * (vT_f1[qq * NR2 + iL] + vT_f1[qq * NR2 + iR]);
                        vfx[qq * TFS + (dir ? C::NTX : 0) + te] = tau;
                    }
                    const Real heat = kappa * (vT_f1[D * NR2 + iR] - vT_f1[D * NR2 + iL]) * invdx[dir];
                    vfx[D * TFS + (dir ? C::NTX : 0) + te] = work + heat;
                };
                for (int e = tid; e < C::NTX + C::NTY; e += NT) {
                    if (e < C::NTX) face(IC<0>{}, e % (TX + 1) - 1, e / (TX + 1), e);
                    else if constexpr (D == 3) {
                        const int e2 = e - C::NTX;
                        face(IC<1>{}, e2 % TX, e2 / TX - 1, e2);
                    }
                }
            }
        }
        // z-face (f-1, f) dissipative flux of this thread's column
        Real zv_new[C::NV];
#pragma unroll
        for (int k = 0; k < C::NV; ++k) zv_new[k] = Real(0);
        if constexpr (VISC) {
            if (f >= z0 && f <= z1) {
                const int iL = C::i2(olx, oly);
                Real grad[3][3];
#pragma unroll
                for (int aa = 0; aa < 3; ++aa)
#pragma unroll
                    for (int qq = 0; qq < 3; ++qq) grad[aa][qq] = Real(0);
#pragma unroll
                for (int qq = 0; qq < D; ++qq) grad[V][qq] = (vT_f[qq * NR2 + iL] - vT_f1[qq * NR2 + iL]) * invdx[V];
#pragma unroll
                for (int t = 0; t < D - 1; ++t) {
                    const int st = t == 0 ? 1 : C::R2X;
#pragma unroll
                    for (int qq = 0; qq < D; ++qq)
                        grad[t][qq] = Real(0.25) *
                                      ((vT_f1[qq * NR2 + iL + st] - vT_f1[qq * NR2 + iL - st]) +
                                       (vT_f[qq * NR2 + iL + st] - vT_f[qq * NR2 + iL - st])) *
                                      invdx[t];
                }
                Real divu = Real(0);
#pragma unroll
                for (int aa = 0; aa < D; ++aa) divu += grad[aa][aa];
                Real work = Real(0);
#pragma unroll
                for (int qq = 0; qq < D; ++qq) {
                    Real tau = mu * (grad[V][qq] + grad[qq][V]);
                    if (qq == V) tau += eta * divu;
                    work += tau * Real(0.5) * (vT_f1[qq * NR2 + iL] + vT_f[qq * NR2 + iL]);
                    zv_new[qq] = tau;
                }
                zv_new[D] = work + kappa * (vT_f[D * NR2 + iL] - vT_f1[D * NR2 + iL]) * invdx[V];
            }
        }
        __syncthreads();

        // ---------------- D: transport fluxes, update of plane f-2 ----------------
        const int q = f - 2;
        Real dxy_new[C::NV];
#pragma unroll
        for (int k = 0; k < C::NV; ++k) dxy_new[k] = Real(0);
        if constexpr (VISC) {
            if (f >= z0 + 1 && f <= z1) {
                // in-plane viscous divergence of plane f-1 for this column
                const int ex = C::itx(olx, oly);
#pragma unroll
                for (int k = 0; k < C::NV; ++k) dxy_new[k] = (vfx[k * TFS + ex] - vfx[k * TFS + ex - 1]) * lam[0];
                if constexpr (D == 3) {
                    const int ey = C::NTX + C::ity(olx, oly);
#pragma unroll
                    for (int k = 0; k < C::NV; ++k) dxy_new[k] += (vfx[k * TFS + ey] - vfx[k * TFS + ey - TX]) * lam[1];
                }
            }
        }
        if (f >= z0 + 2) {
            // upwind transport fluxes through the in-plane faces of the output cells
            for (int e = tid; e < C::NTX + C::NTY; e += NT) {
                int lxL, lyL, fe, upR;
                if (e < C::NTX) {
                    lxL = e % (TX + 1) - 1; lyL = e / (TX + 1);
                    fe = C::ifx(lxL, lyL);
                    upR = 1;
                } else {
                    const int e2 = e - C::NTX;
                    lxL = e2 % TX; lyL = e2 / TX - 1;
                    fe = C::NFX + C::ify(lxL, lyL);
                    upR = C::R1X;
                }
                const Real us = xy_f2[fe];
                const int up = C::i1(lxL, lyL) + (us >= Real(0) ? 0 : upR);
#pragma unroll
                for (int k = 0; k < NF; ++k) tfx[k * TFS + e] = tl_f2[k * NR1 + up] * us;
            }
        }
        Real zt_hi[NF];
        Real us_hi = Real(0);
#pragma unroll
        for (int k = 0; k < NF; ++k) zt_hi[k] = Real(0);
        if (f >= z0 + 1) {
            // transport flux through the face between planes f-2 and f-1 of this column
            const int c1 = C::i1(olx, oly);
            us_hi = zf_lo[c1];
            const Real* src = us_hi >= Real(0) ? tl_f2 : tl_f1;
#pragma unroll
            for (int k = 0; k < NF; ++k) zt_hi[k] = src[k * NR1 + c1] * us_hi;
            if constexpr (SPLIT) {
                // base-state part of the upwind value relative to the row below (plane f-2)
                if (!(us_hi >= Real(0))) {
                    zt_hi[0] += base(B_DRP, f - 2) * us_hi;
                    zt_hi[D + 1] += base(B_DWP, f - 2) * us_hi;
                }
            }
        }
        __syncthreads();
        if (f >= z0 + 2) {
            const int c1 = C::i1(olx, oly);
            const Real L = tl_f2[NF * NR1 + c1];
            const int ex = C::itx(olx, oly);
            const int ey = C::NTX + C::ity(olx, oly);
            Real nb[NF];
#pragma unroll
            for (int k = 0; k < NF; ++k) {
                Real acc = tl_f2[k * NR1 + c1] * L;
                acc -= lam[0] * (tfx[k * TFS + ex] - tfx[k * TFS + ex - 1]);
                if constexpr (D == 3) acc -= lam[1] * (tfx[k * TFS + ey] - tfx[k * TFS + ey - TX]);
                nb[k] = acc;
            }
            // the flux through the upper z face is relative to row q's base; the lower
            // face's flux (computed relative to row q-1) is shifted to row q's base
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
                const long long idx = D == 3 ? ogx + (long long)nx * (ogy + (long long)ny * q) : ogx + (long long)nx * q;
#pragma unroll
                for (int k = 0; k < NF; ++k) Uo[k * N + idx] = nb[k];
                // CFL wave rate of U^{n+1} (next step's dt) and physical checks
                Row<Real> w = row_info<Real, SPLIT>(a, S.phi, q, nv, fr - Real(2));
                if constexpr (PHIA) w.phi = a.energy_form ? Real(0) : __ldg(Pa + idx);
                Real p, rho;
                const Real sh = wave_rate<D, Real, SPLIT, VISC>(nb, w, S.eos, invdx, mu, kappa, p, rho);
                if (!(sh <= smax_t)) smax_t = (sh == sh) ? sh : smax_t;
                if (sh != sh || p != p) status |= ST_NAN;
                if (!(rho > Real(0)) || !(p > Real(0))) status |= ST_NONPHYS;
            }
        }
        // rotate the column carries
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
    }

    // block max of the wave rate -> one atomic per block
    block_rate_max(double(smax_t), reinterpret_cast<unsigned long long*>(red), a.smax + a.slot_write);
    if (status) atomicOr(a.status, status);
}

// One launch = one step of one grid.  Balanced schedule: the grid is one wave
// of resident blocks, and block b marches units [b W, (b + 1) W) of the
// tile-major list of (tile, plane) units, as one run of planes per tile it
// touches (W = work_per_block).
template <int DIM, typename Real, bool SPLIT, bool VISC, int TX, int TY, bool PHIA = false, bool NA = false>
__global__ void __launch_bounds__(TX * TY, sizeof(Real) == 8 ? (DIM == 2 ? 2 : 1) : 2)
ark_step_kernel(const __grid_constant__ StepArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nv = a.n[DIM - 1];
    const long long total = (long long)a.tiles_x * a.tiles_y * nv;
    long long u = (long long)blockIdx.x * a.work_per_block;
    const long long end = min(u + a.work_per_block, total);
    bool lead = blockIdx.x == 0;
    while (u < end) {
        const int tile = (int)(u / nv);
        const int z0 = (int)(u - (long long)tile * nv);
        const int z1 = (int)min((long long)nv, z0 + (end - u));
        step_block<DIM, Real, SPLIT, VISC, TX, TY, PHIA, NA>(a, tile, z0, z1, lead, smem_raw);
        u += z1 - z0;
        lead = false;
        __syncthreads();   // the next run reuses the shared plane rings
    }
}

// Work item of the batched step: one (run, tile, chunk).
struct BatchItem {
    int run, tile, chunk, pad;
};

// One launch = one step of every run of an ensemble.  A fixed grid of blocks
// (resident blocks per SM x SMs) takes work items from an atomic counter
// until none is left; item 0's taker resets the counter of the next step.
// Every run has its own arguments (state pointers, base tables, dt slots).
template <int DIM, typename Real, bool SPLIT, bool VISC, int TX, int TY>
__global__ void __launch_bounds__(TX * TY, sizeof(Real) == 8 ? 1 : 512 / (TX * TY))
ark_batch_kernel(const StepArgs* __restrict__ runs, const BatchItem* __restrict__ items, int nitems, int* ctr,
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
        step_block<DIM, Real, SPLIT, VISC, TX, TY>(r, w.tile, z0, min(z0 + r.planes, r.n[DIM - 1]),
                                                   w.tile == 0 && w.chunk == 0, smem_raw);
    }
}

}  // namespace ark
