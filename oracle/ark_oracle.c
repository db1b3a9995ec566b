/*
 * ark_oracle.c -- plain, slow, FP64 CPU restatement of one explicit time step
 * of the all-regime, well-balanced acoustic-transport scheme of Padioleau et
 * al. (arXiv:1903.09043), used ONLY as test infrastructure: the parity tests,
 * the package smoke check and the CPU-baseline leg of the benchmark call it.
 * The product path never links, loads or calls this file.  It shares no code,
 * header, table or helper with the CUDA library.
 *
 * Structure follows the paper's order (Sec. 2):
 *   1. ghost cells (Sec. 3.2: ghost zones carry the physical boundary
 *      conditions), materialised as arrays;
 *   2. conservative -> primitive variables (Sec. 3.2 kernel list; ideal gas of
 *      Sec. 4: p = (gamma-1) rho e, c^2 = gamma p / rho, p = rho T; with
 *      p_inf > 0 the stiffened gas of R21, which the scheme admits as Sec. 4
 *      notes that another equation of state may be used);
 *   3. acoustic step, Sec. 2.1.2: per-face a, S, u*, theta (Eq. 16,
 *      low_mach_correction), Pi*, then per-cell L~ and tilde states;
 *   4. transport step, Sec. 2.1.3: b^{n+1} = b~ - dt/dx [b~ u*] + b~ dt/dx [u*]
 *      with b~ upwinded on u*;
 *   5. relaxation step, Sec. 2.1.4: Psi^{n+1} = Phi; the conserved energy
 *      rho*calE is unchanged, so nothing is done to the stored state;
 *   (Appendix B, energy_form 1: the energy variable is rho E without rho Phi
 *    and the acoustic step adds dt/dx (uS)_i to it,
 *    (uS)_i = 1/2 (u*_{i+1/2} S_{i+1/2} + u*_{i-1/2} S_{i-1/2});)
 *   6. first-order dissipative fluxes, Sec. 2.2, evaluated from U^n.
 * Multi-dimensional steps sum every direction's face terms into one L~, one
 * tilde state and one update (unsplit).
 *
 * Readings of points the paper leaves open (each is one numbered reading in
 * the design notes; the code states the choice where it is made):
 *   R1 unsplit multi-D; R2 a = K max(rho_L c_L, rho_R c_R); R3 CFL formula;
 *   R4 dissipative fluxes from U^n in the same update; R5 physical heat-flux
 *   sign; R6 viscous stencil; R7 upwind tie u* >= 0 -> left; R10 wall ghosts;
 *   R11 Phi = -g.x at cell centres; R21 stiffened-gas equation of state;
 *   R22 Noble-Abel stiffened gas (covolume b).
 *
 * State layout: nf = dim + 2 fields (rho, m_x, m_y[, m_z], rho*calE), each a
 * block of nx*ny*nz doubles, x fastest.  For dim == 2, nz == 1.
 *
 * Parity pins: every function here is pinned by tests/test_oracle_pins.py
 * (closed forms, invariants, textbook special cases, the paper's table).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "ark_oracle.h"

#ifdef _OPENMP
#include <omp.h>
#endif

void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------------ */
/* one cell: conserved and primitive values at a (possibly ghost) position   */
/* ------------------------------------------------------------------------ */
typedef struct {
    double rho, m[3], W;   /* conserved: rho, rho u, rho*calE               */
    double u[3], p, T, c;  /* primitives                                     */
    double phi;            /* gravitational potential at the cell centre     */
} cell_t;

static int nfields(const orc_problem* P) { return P->dim + 2; }

static long ncells(const orc_problem* P)
{
    return (long)P->n[0] * P->n[1] * (P->dim == 3 ? P->n[2] : 1);
}

/* Phi at the centre of cell index ijk (ghosts included).
 * R11: Phi = -g . x for uniform gravity.
 * R20: a caller-supplied Phi is given at the interior cell centres; a ghost
 * takes, axis by axis as the state does (the last out-of-range axis first, on
 * cells that may be ghosts of earlier axes), the value across a periodic
 * side, or the linear extension of the two nearest interior cells of that
 * axis across a wall or outflow side: Phi_g = (1 + L) Phi_0 - L Phi_1 for
 * ghost layer L = 1, 2 (Phi_0 the boundary cell, Phi_1 its inner neighbour). */
static double phi_at(const orc_problem* P, const int ijk[3])
{
    if (!P->phi) {
        double phi = 0.0;
        for (int d = 0; d < P->dim; ++d) {
            double x = P->lo[d] + (ijk[d] + 0.5) * P->dx[d];
            phi -= P->g[d] * x;
        }
        return phi;
    }
    int d;
    for (d = P->dim - 1; d >= 0; --d)
        if (ijk[d] < 0 || ijk[d] >= P->n[d]) break;
    if (d < 0) {
        long idx = ijk[0] + (long)P->n[0] * (ijk[1] + (long)P->n[1] * (P->dim == 3 ? ijk[2] : 0));
        return P->phi[idx];
    }
    int n = P->n[d];
    int lo_side = ijk[d] < 0;
    int bc = lo_side ? P->bc_lo[d] : P->bc_hi[d];
    int a[3] = {ijk[0], ijk[1], ijk[2]}, b[3] = {ijk[0], ijk[1], ijk[2]};
    if (bc == ORC_BC_PERIODIC) {
        a[d] = ((ijk[d] % n) + n) % n;
        return phi_at(P, a);
    }
    int layer = lo_side ? -ijk[d] : ijk[d] - n + 1;
    a[d] = lo_side ? 0 : n - 1;
    b[d] = lo_side ? 1 : n - 2;
    return (1.0 + layer) * phi_at(P, a) - layer * phi_at(P, b);
}

/* Primitives from conserved values (Sec. 4 ideal gas, R = 1):
 * e = (W - 1/2 rho |u|^2 - rho Phi) / rho, p = (gamma-1) rho e,
 * T = p / rho, c = sqrt(gamma p / rho).
 * R21 stiffened gas (Harlow and Amsden 1971; temperature as in Le Metayer,
 * Massoni and Saurel 2004, with (gamma-1) c_v = 1): p = (gamma-1) rho e -
 * gamma p_inf, T = (p + p_inf) / rho, c = sqrt(gamma (p + p_inf) / rho);
 * p_inf = 0 is the ideal gas.
 * R22 Noble-Abel stiffened gas (Le Metayer and Saurel 2016, without the
 * reference energy): the covolume b leaves the fraction 1 - b rho of the
 * volume free, p = (gamma-1) rho e / (1 - b rho) - gamma p_inf,
 * T = (p + p_inf) (1 - b rho) / rho, c = sqrt(gamma (p + p_inf) / (rho (1 - b rho)));
 * b = 0 is the stiffened gas (the factor 1 - b rho is then exactly 1). */
static void to_primitive(const orc_problem* P, cell_t* c)
{
    double ke = 0.0;
    for (int d = 0; d < 3; ++d) {
        c->u[d] = c->m[d] / c->rho;
        ke += 0.5 * c->rho * c->u[d] * c->u[d];
    }
    double rho_e = c->W - ke - (P->energy_form == 0 ? c->rho * c->phi : 0.0);
    double free_vol = 1.0 - P->b * c->rho;
    c->p = (P->gamma - 1.0) * rho_e / free_vol - P->gamma * P->p_inf;
    c->T = (c->p + P->p_inf) * free_vol / c->rho;
    c->c = sqrt(P->gamma * (c->p + P->p_inf) / (c->rho * free_vol));
}

/* Conserved values from (rho, u, p, phi). */
static void to_conserved(const orc_problem* P, cell_t* c)
{
    double ke = 0.0;
    for (int d = 0; d < 3; ++d) {
        c->m[d] = c->rho * c->u[d];
        ke += 0.5 * c->rho * c->u[d] * c->u[d];
    }
    /* rho e = (p + gamma p_inf) (1 - b rho) / (gamma - 1) (R21, R22) */
    double free_vol = 1.0 - P->b * c->rho;
    c->W = (c->p + P->gamma * P->p_inf) * free_vol / (P->gamma - 1.0) + ke +
           (P->energy_form == 0 ? c->rho * c->phi : 0.0);
    c->T = (c->p + P->p_inf) * free_vol / c->rho;
    c->c = sqrt(P->gamma * (c->p + P->p_inf) / (c->rho * free_vol));
}

static void load_interior(const orc_problem* P, const double* U, const int ijk[3], cell_t* c)
{
    long N = ncells(P);
    long idx = ijk[0] + (long)P->n[0] * (ijk[1] + (long)P->n[1] * (P->dim == 3 ? ijk[2] : 0));
    c->rho = U[idx];
    c->m[0] = c->m[1] = c->m[2] = 0.0;
    for (int d = 0; d < P->dim; ++d) c->m[d] = U[(1 + d) * N + idx];
    c->W = U[(1 + P->dim) * N + idx];
    c->phi = phi_at(P, ijk);
    to_primitive(P, c);
}

/*
 * Value of the state at any index within two layers of the domain.  Ghosts
 * are defined axis by axis in the order x, then y, then z: the rule of the
 * LAST out-of-range axis is applied to cells that may themselves be ghosts
 * of earlier axes, which fixes edge and corner ghosts (what a fill of x
 * ghosts, then y ghosts over the x-extended rows, then z ghosts, produces).
 *
 * R10 wall ghosts: layer 1 mirrors interior cell 0, layer 2 mirrors interior
 * cell 1.  Velocity: reflective wall flips the normal component; no-slip wall
 * flips every component.  Temperature: reflective wall copies the mirror
 * temperature; fixed-temperature wall sets T_g = 2 T_wall - T_mirror.
 * Pressure: the discrete hydrostatic balance of Eq. 18 (well_balanced_formula)
 * between the ghost and its inner neighbour A (interior cell 0 for layer 1,
 * ghost layer 1 for layer 2), with rho_g = (p_g + p_inf) / T_g:
 *   p_g - p_A = -1/2 (rho_A + (p_g + p_inf) / T_g) (Phi_g - Phi_A)
 *   => p_g + p_inf = (p_A + p_inf - 1/2 rho_A dPhi) / (1 + dPhi / (2 T_g)).
 * With a covolume b (R22) the ghost density is (p_g + p_inf) / (T_g + b (p_g + p_inf))
 * and the balance is a quadratic in p_g + p_inf.
 * Outflow: zero-gradient copy of (rho, u, p) of the boundary cell.
 */
static void cell_at(const orc_problem* P, const double* U, const int ijk[3], cell_t* out)
{
    int d;
    for (d = P->dim - 1; d >= 0; --d)
        if (ijk[d] < 0 || ijk[d] >= P->n[d]) break;
    if (d < 0) {
        load_interior(P, U, ijk, out);
        return;
    }
    int n = P->n[d];
    int lo_side = ijk[d] < 0;
    int bc = lo_side ? P->bc_lo[d] : P->bc_hi[d];
    int src[3] = {ijk[0], ijk[1], ijk[2]};

    if (bc == ORC_BC_PERIODIC) {
        src[d] = ((ijk[d] % n) + n) % n;
        cell_at(P, U, src, out);
        return;
    }
    if (bc == ORC_BC_OUTFLOW) {
        src[d] = lo_side ? 0 : n - 1;
        cell_t s;
        cell_at(P, U, src, &s);
        out->rho = s.rho;
        out->u[0] = s.u[0]; out->u[1] = s.u[1]; out->u[2] = s.u[2];
        out->p = s.p;
        out->phi = phi_at(P, ijk);
        to_conserved(P, out);
        return;
    }
    /* walls */
    int layer = lo_side ? -ijk[d] : ijk[d] - n + 1;        /* 1 or 2 */
    src[d] = lo_side ? -ijk[d] - 1 : 2 * n - 1 - ijk[d];   /* mirror */
    cell_t M, A;
    cell_at(P, U, src, &M);
    if (layer == 1) {
        A = M;
    } else {
        int a_idx[3] = {ijk[0], ijk[1], ijk[2]};
        a_idx[d] = lo_side ? -1 : n;
        cell_at(P, U, a_idx, &A);
    }
    double Tg;
    for (int k = 0; k < 3; ++k) out->u[k] = M.u[k];
    if (bc == ORC_BC_REFLECT_HYDRO) {
        out->u[d] = -M.u[d];
        Tg = M.T;
    } else { /* ORC_BC_NOSLIP_FIXED_T */
        for (int k = 0; k < 3; ++k) out->u[k] = -M.u[k];
        double Tw = lo_side ? P->T_lo[d] : P->T_hi[d];
        Tg = 2.0 * Tw - M.T;
    }
    out->phi = phi_at(P, ijk);
    double dphi = out->phi - A.phi;
    double pi_g;
    if (P->b == 0.0) {
        pi_g = (A.p + P->p_inf - 0.5 * A.rho * dphi) / (1.0 + dphi / (2.0 * Tg));
    } else {
        /* R22: rho_g = pi_g / (T_g + b pi_g) turns the balance into
         * b pi^2 + (T_g - b K + dPhi/2) pi - K T_g = 0, K = pi_A - rho_A dPhi / 2;
         * its positive root, in the form without cancellation */
        double K = A.p + P->p_inf - 0.5 * A.rho * dphi;
        double B = Tg - P->b * K + 0.5 * dphi;
        pi_g = 2.0 * K * Tg / (B + sqrt(B * B + 4.0 * P->b * K * Tg));
    }
    out->p = pi_g - P->p_inf;
    out->rho = pi_g / (Tg + P->b * pi_g);
    to_conserved(P, out);
}

void orc_cell_at(const orc_problem* P, const double* U, const int ijk[3], double out[12])
{
    cell_t c;
    cell_at(P, U, ijk, &c);
    out[0] = c.rho; out[1] = c.m[0]; out[2] = c.m[1]; out[3] = c.m[2]; out[4] = c.W;
    out[5] = c.u[0]; out[6] = c.u[1]; out[7] = c.u[2]; out[8] = c.p; out[9] = c.T;
    out[10] = c.c; out[11] = c.phi;
}

/* ------------------------------------------------------------------------ */
/* acoustic face values, Sec. 2.1.2 and Eq. 16                               */
/* ------------------------------------------------------------------------ */
typedef struct { double a, S, ustar, theta, Pistar; } face_t;

/* L is the cell on the low side, R on the high side, d the face normal. */
static void acoustic_face(const orc_problem* P, const cell_t* L, const cell_t* R, int d, face_t* f)
{
    /* R2: sub-characteristic condition a >= max(rho c), a = K max(rho_L c_L, rho_R c_R) */
    double zl = L->rho * L->c, zr = R->rho * R->c;
    f->a = P->K * (zl > zr ? zl : zr);
    /* S_{i+1/2} = -1/2 (rho_i + rho_{i+1}) (Phi_{i+1} - Phi_i) */
    f->S = -0.5 * (L->rho + R->rho) * (R->phi - L->phi);
    /* u* = 1/2 (u_L + u_R) - 1/(2a) (Pi_R - Pi_L - S), Pi^n = p^n */
    f->ustar = 0.5 * (L->u[d] + R->u[d]) - (R->p - L->p - f->S) / (2.0 * f->a);
    /* Eq. 16: theta = min(|u*| / max(c_L, c_R), 1); theta = 1 when disabled */
    if (P->low_mach) {
        double cmax = L->c > R->c ? L->c : R->c;
        double ma = fabs(f->ustar) / cmax;
        f->theta = ma < 1.0 ? ma : 1.0;
    } else {
        f->theta = 1.0;
    }
    /* Pi* = 1/2 (Pi_L + Pi_R) - a theta / 2 (u_R - u_L) */
    f->Pistar = 0.5 * (L->p + R->p) - 0.5 * f->a * f->theta * (R->u[d] - L->u[d]);
}

void orc_face(const orc_problem* P, const double* Lprim, const double* Rprim, int d, double out[5])
{
    /* prim = (rho, u0, u1, u2, p, phi) */
    cell_t L, R;
    memset(&L, 0, sizeof L); memset(&R, 0, sizeof R);
    L.rho = Lprim[0]; L.u[0] = Lprim[1]; L.u[1] = Lprim[2]; L.u[2] = Lprim[3]; L.p = Lprim[4]; L.phi = Lprim[5];
    R.rho = Rprim[0]; R.u[0] = Rprim[1]; R.u[1] = Rprim[2]; R.u[2] = Rprim[3]; R.p = Rprim[4]; R.phi = Rprim[5];
    to_conserved(P, &L);
    to_conserved(P, &R);
    face_t f;
    acoustic_face(P, &L, &R, d, &f);
    out[0] = f.a; out[1] = f.S; out[2] = f.ustar; out[3] = f.theta; out[4] = f.Pistar;
}

/* ------------------------------------------------------------------------ */
/* the step on a window [wlo, whi) of the domain                              */
/* ------------------------------------------------------------------------ */
typedef struct {
    int E[3];      /* extended extents (window + 2 ghosts each side on active axes) */
    long Ntot;
} ext_t;

static long eidx(const ext_t* X, int i, int j, int k)
{
    return i + (long)X->E[0] * (j + (long)X->E[1] * k);
}

int orc_step_window(const orc_problem* P, const double* U, double dt,
                    const int wlo[3], const int whi[3], double* out)
{
    const int dim = P->dim;
    const int nf = nfields(P);
    ext_t X;
    int W[3] = {1, 1, 1};
    for (int d = 0; d < 3; ++d) {
        if (d < dim) {
            W[d] = whi[d] - wlo[d];
            if (W[d] <= 0 || wlo[d] < 0 || whi[d] > P->n[d]) return -1;
            X.E[d] = W[d] + 4;
        } else {
            X.E[d] = 1;
        }
    }
    X.Ntot = (long)X.E[0] * X.E[1] * X.E[2];
    const int H[3] = {2, 2, dim == 3 ? 2 : 0};      /* ghost width per axis */

    cell_t* C = (cell_t*)malloc(sizeof(cell_t) * X.Ntot);
    face_t* F[3] = {0, 0, 0};
    cell_t* Tl = (cell_t*)calloc(X.Ntot, sizeof(cell_t));   /* tilde states (rho, m, W used) */
    double* Lt = (double*)calloc(X.Ntot, sizeof(double));   /* L~ */
    if (!C || !Tl || !Lt) { free(C); free(Tl); free(Lt); return -2; }
    for (int d = 0; d < dim; ++d) {
        F[d] = (face_t*)calloc(X.Ntot, sizeof(face_t));
        if (!F[d]) return -2;
    }
    double lam[3] = {0, 0, 0};
    for (int d = 0; d < dim; ++d) lam[d] = dt / P->dx[d];

    /* 1+2: ghost-extended cells with primitives */
    #pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < X.E[2]; ++k)
        for (int j = 0; j < X.E[1]; ++j)
            for (int i = 0; i < X.E[0]; ++i) {
                int g[3] = {wlo[0] + i - H[0], wlo[1] + j - H[1], (dim == 3 ? wlo[2] : 0) + k - H[2]};
                cell_at(P, U, g, &C[eidx(&X, i, j, k)]);
            }

    /* 3a: acoustic face values.  F[d][e] is the face between ext cell e and e + e_d. */
    for (int d = 0; d < dim; ++d) {
        int sh[3] = {0, 0, 0};
        sh[d] = 1;
        #pragma omp parallel for collapse(2) schedule(static)
        for (int k = 0; k < X.E[2] - sh[2]; ++k)
            for (int j = 0; j < X.E[1] - sh[1]; ++j)
                for (int i = 0; i < X.E[0] - sh[0]; ++i) {
                    long e = eidx(&X, i, j, k);
                    long e1 = eidx(&X, i + sh[0], j + sh[1], k + sh[2]);
                    acoustic_face(P, &C[e], &C[e1], d, &F[d][e]);
                }
    }

    /* 3b: tilde states on window + 1 ghost layer (Sec. 2.1.2, unsplit R1):
     * L~ = 1 + sum_d dt/dx_d [u*]_d
     * L~ rho~   = rho
     * L~ (m_d)~ = m_d - dt/dx_d [Pi*]_d + dt/dx_d S_d,  S_d = 1/2 (S_{+} + S_{-})
     * L~ W~     = W - sum_d dt/dx_d [Pi* u*]_d */
    int tlo[3], thi[3];
    for (int d = 0; d < 3; ++d) { tlo[d] = H[d] ? 1 : 0; thi[d] = H[d] ? X.E[d] - 1 : X.E[d]; }
    #pragma omp parallel for collapse(2) schedule(static)
    for (int k = tlo[2]; k < thi[2]; ++k)
        for (int j = tlo[1]; j < thi[1]; ++j)
            for (int i = tlo[0]; i < thi[0]; ++i) {
                long e = eidx(&X, i, j, k);
                const cell_t* c = &C[e];
                double L = 1.0;
                double mt[3] = {c->m[0], c->m[1], c->m[2]};
                double Wt = c->W;
                for (int d = 0; d < dim; ++d) {
                    int sh[3] = {0, 0, 0};
                    sh[d] = 1;
                    const face_t* fp = &F[d][e];
                    const face_t* fm = &F[d][eidx(&X, i - sh[0], j - sh[1], k - sh[2])];
                    L += lam[d] * (fp->ustar - fm->ustar);
                    mt[d] += -lam[d] * (fp->Pistar - fm->Pistar) + lam[d] * 0.5 * (fp->S + fm->S);
                    Wt -= lam[d] * (fp->Pistar * fp->ustar - fm->Pistar * fm->ustar);
                    /* Appendix B: energy source dt/dx (uS)_i of the acoustic step */
                    if (P->energy_form == 1)
                        Wt += lam[d] * 0.5 * (fp->ustar * fp->S + fm->ustar * fm->S);
                }
                Lt[e] = L;
                Tl[e].rho = c->rho / L;
                for (int q = 0; q < 3; ++q) Tl[e].m[q] = mt[q] / L;
                Tl[e].W = Wt / L;
            }

    /* 4+6: transport step and dissipative fluxes for the window cells. */
    const double eta_over_mu = -2.0 / 3.0;   /* Stokes hypothesis, Eq. 4 */
    #pragma omp parallel for collapse(2) schedule(static)
    for (int k = H[2]; k < X.E[2] - H[2]; ++k)
        for (int j = H[1]; j < X.E[1] - H[1]; ++j)
            for (int i = H[0]; i < X.E[0] - H[0]; ++i) {
                long e = eidx(&X, i, j, k);
                const cell_t* t = &Tl[e];
                double b[5] = {t->rho, t->m[0], t->m[1], t->m[2], t->W};
                double bt[5] = {t->rho, t->m[0], t->m[1], t->m[2], t->W};
                double Lm1 = Lt[e] - 1.0;
                (void)Lm1;
                /* transport: b^{n+1} = b~ - sum_d lam_d [b~_up u*]_d + b~ sum_d lam_d [u*]_d */
                for (int d = 0; d < dim; ++d) {
                    int sh[3] = {0, 0, 0};
                    sh[d] = 1;
                    long em = eidx(&X, i - sh[0], j - sh[1], k - sh[2]);
                    long ep = eidx(&X, i + sh[0], j + sh[1], k + sh[2]);
                    const face_t* fp = &F[d][e];
                    const face_t* fm = &F[d][em];
                    /* R7: upwind on u*, tie u* = 0 takes the left cell */
                    const cell_t* up_p = fp->ustar >= 0.0 ? &Tl[e] : &Tl[ep];
                    const cell_t* up_m = fm->ustar >= 0.0 ? &Tl[em] : &Tl[e];
                    double bp[5] = {up_p->rho, up_p->m[0], up_p->m[1], up_p->m[2], up_p->W};
                    double bm[5] = {up_m->rho, up_m->m[0], up_m->m[1], up_m->m[2], up_m->W};
                    for (int q = 0; q < 5; ++q)
                        b[q] += -lam[d] * (bp[q] * fp->ustar - bm[q] * fm->ustar)
                                + bt[q] * lam[d] * (fp->ustar - fm->ustar);
                }
                /* dissipative fluxes (Sec. 2.2, R4-R6) from U^n */
                if (P->mu != 0.0 || P->kappa != 0.0) {
                    for (int d = 0; d < dim; ++d) {
                        double acc[5] = {0, 0, 0, 0, 0};
                        for (int side = 0; side < 2; ++side) {
                            /* face between cells Lc and Rc, normal d */
                            int li[3] = {i, j, k}, ri[3] = {i, j, k};
                            if (side == 0) { ri[d] += 1; } else { li[d] -= 1; }
                            const cell_t* Lc = &C[eidx(&X, li[0], li[1], li[2])];
                            const cell_t* Rc = &C[eidx(&X, ri[0], ri[1], ri[2])];
                            double grad[3][3];   /* grad[a][q] = d u_q / d x_a at the face */
                            for (int q = 0; q < 3; ++q) for (int a = 0; a < 3; ++a) grad[a][q] = 0.0;
                            for (int q = 0; q < dim; ++q)
                                grad[d][q] = (Rc->u[q] - Lc->u[q]) / P->dx[d];
                            for (int a = 0; a < dim; ++a) {
                                if (a == d) continue;
                                int lp[3] = {li[0], li[1], li[2]}, lmi[3] = {li[0], li[1], li[2]};
                                int rp[3] = {ri[0], ri[1], ri[2]}, rmi[3] = {ri[0], ri[1], ri[2]};
                                lp[a] += 1; lmi[a] -= 1; rp[a] += 1; rmi[a] -= 1;
                                const cell_t* Lp = &C[eidx(&X, lp[0], lp[1], lp[2])];
                                const cell_t* Lmn = &C[eidx(&X, lmi[0], lmi[1], lmi[2])];
                                const cell_t* Rp = &C[eidx(&X, rp[0], rp[1], rp[2])];
                                const cell_t* Rmn = &C[eidx(&X, rmi[0], rmi[1], rmi[2])];
                                for (int q = 0; q < dim; ++q)
                                    grad[a][q] = 0.25 * ((Lp->u[q] - Lmn->u[q]) + (Rp->u[q] - Rmn->u[q])) / P->dx[a];
                            }
                            double divu = 0.0;
                            for (int a = 0; a < dim; ++a) divu += grad[a][a];
                            double work = 0.0;
                            double tau[3] = {0, 0, 0};
                            for (int q = 0; q < dim; ++q) {
                                /* tau_{dq} = mu (d_d u_q + d_q u_d) + eta div u delta_{dq} */
                                tau[q] = P->mu * (grad[d][q] + grad[q][d]);
                                if (q == d) tau[q] += eta_over_mu * P->mu * divu;
                                work += tau[q] * 0.5 * (Lc->u[q] + Rc->u[q]);
                            }
                            /* R5: heat flux enters with the physical (diffusive) sign */
                            double heat = P->kappa * (Rc->T - Lc->T) / P->dx[d];
                            double sgn = side == 0 ? 1.0 : -1.0;
                            for (int q = 0; q < dim; ++q) acc[1 + q] += sgn * tau[q];
                            acc[4] += sgn * (work + heat);
                        }
                        for (int q = 0; q < 5; ++q) b[q] += dt / P->dx[d] * acc[q];
                    }
                }
                /* write out: field order rho, m_0..m_{dim-1}, W */
                long wi = (i - H[0]) + (long)W[0] * ((j - H[1]) + (long)W[1] * (k - H[2]));
                long WN = (long)W[0] * W[1] * W[2];
                out[wi] = b[0];
                for (int q = 0; q < dim; ++q) out[(1 + q) * WN + wi] = b[1 + q];
                out[(1 + dim) * WN + wi] = b[4];
            }

    free(C); free(Tl); free(Lt);
    for (int d = 0; d < dim; ++d) free(F[d]);
    (void)nf;
    return 0;
}

int orc_step(const orc_problem* P, const double* U, double dt, double* Unew)
{
    int wlo[3] = {0, 0, 0}, whi[3] = {P->n[0], P->n[1], P->dim == 3 ? P->n[2] : 1};
    return orc_step_window(P, U, dt, wlo, whi, Unew);
}

/* ------------------------------------------------------------------------ */
/* R3: CFL time step.                                                         */
/*   dt = cfl / max_i max( sum_d (|u_d| + c)/dx_d ,                           */
/*                         sum_d 2 max(4 mu / (3 rho), kappa (gamma-1)/rho)/dx_d^2 ) */
/* ------------------------------------------------------------------------ */
double orc_dt(const orc_problem* P, const double* U)
{
    long N = ncells(P);
    int nz = P->dim == 3 ? P->n[2] : 1;
    double smax = 0.0;
    for (long idx = 0; idx < N; ++idx) {
        int ijk[3] = {(int)(idx % P->n[0]), (int)((idx / P->n[0]) % P->n[1]), (int)(idx / ((long)P->n[0] * P->n[1]))};
        (void)nz;
        cell_t c;
        load_interior(P, U, ijk, &c);
        double s = 0.0, sp = 0.0;
        double nu = 4.0 * P->mu / (3.0 * c.rho);
        double chi = P->kappa * (P->gamma - 1.0) / c.rho;
        double dmax = nu > chi ? nu : chi;
        for (int d = 0; d < P->dim; ++d) {
            s += (fabs(c.u[d]) + c.c) / P->dx[d];
            sp += 2.0 * dmax / (P->dx[d] * P->dx[d]);
        }
        double sc = s > sp ? s : sp;
        if (sc > smax) smax = sc;
    }
    return P->cfl / smax;
}

/* ------------------------------------------------------------------------ */
/* Diagnostics: sums over the interior (times the cell volume) and extrema. */
/* out: [0] mass, [1..3] momentum, [4] total energy (rho calE),              */
/*      [5] kinetic energy, [6] max |u|, [7] mean |u_last|, [8] min rho,     */
/*      [9] min p                                                            */
/* ------------------------------------------------------------------------ */
void orc_diagnostics(const orc_problem* P, const double* U, double out[10])
{
    long N = ncells(P);
    double vol = 1.0;
    for (int d = 0; d < P->dim; ++d) vol *= P->dx[d];
    double s[6] = {0, 0, 0, 0, 0, 0};
    double umax = 0.0, vsum = 0.0, rmin = INFINITY, pmin = INFINITY;
    for (long idx = 0; idx < N; ++idx) {
        int ijk[3] = {(int)(idx % P->n[0]), (int)((idx / P->n[0]) % P->n[1]), (int)(idx / ((long)P->n[0] * P->n[1]))};
        cell_t c;
        load_interior(P, U, ijk, &c);
        s[0] += c.rho;
        for (int d = 0; d < 3; ++d) s[1 + d] += c.m[d];
        s[4] += c.W;
        double u2 = c.u[0] * c.u[0] + c.u[1] * c.u[1] + c.u[2] * c.u[2];
        s[5] += 0.5 * c.rho * u2;
        double um = sqrt(u2);
        if (um > umax) umax = um;
        vsum += fabs(c.u[P->dim - 1]);
        if (c.rho < rmin) rmin = c.rho;
        if (c.p < pmin) pmin = c.p;
    }
    for (int q = 0; q < 6; ++q) out[q] = s[q] * vol;
    out[6] = umax;
    out[7] = vsum / (double)N;
    out[8] = rmin;
    out[9] = pmin;
}

int orc_nfields(const orc_problem* P) { return nfields(P); }
