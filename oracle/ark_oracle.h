/*
 * ark_oracle.h -- interface of the FP64 CPU oracle (test infrastructure only;
 * see ark_oracle.c).  Independent of the CUDA library and of include/ark.h.
 */
#ifndef ARK_ORACLE_H
#define ARK_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_BC_PERIODIC 0
#define ORC_BC_REFLECT_HYDRO 1
#define ORC_BC_NOSLIP_FIXED_T 2
#define ORC_BC_OUTFLOW 3

typedef struct {
    int dim;            /* 2 or 3                                            */
    int n[3];           /* cells per axis; n[2] ignored when dim == 2        */
    double lo[3];       /* lower corner of the box                           */
    double dx[3];       /* cell sizes                                        */
    double gamma;       /* adiabatic index                                   */
    double g[3];        /* uniform gravity, Phi = -g . x                     */
    double mu, kappa;   /* dynamic viscosity, heat conductivity              */
    double K;           /* a = K max(rho c) at each face                      */
    double cfl;
    int low_mach;       /* 1: theta of Eq. 16; 0: theta = 1                  */
    int bc_lo[3], bc_hi[3];
    double T_lo[3], T_hi[3];  /* wall temperatures for ORC_BC_NOSLIP_FIXED_T */
    int energy_form;    /* 0: rho*calE = rho e + rho u^2/2 + rho Phi (Eq. 6, the
                           scheme of Sec. 2); 1: rho E = rho e + rho u^2/2 with
                           the gravity work as a source (Appendix B) */
    const double* phi;  /* NULL: Phi = -g . x.  Else the potential at the cell
                           centres, one value per cell in the layout of a field
                           (R20: ghost values wrap across periodic sides and
                           extend linearly across walls and outflow) */
    double p_inf;       /* stiffened-gas constant of the equation of state,
                           p = (gamma-1) rho e - gamma p_inf, T = (p + p_inf)/rho,
                           c^2 = gamma (p + p_inf)/rho; 0: the ideal gas (R21) */
    double b;           /* covolume of the Noble-Abel stiffened gas (R22):
                           p = (gamma-1) rho e / (1 - b rho) - gamma p_inf,
                           T = (p + p_inf)(1 - b rho)/rho,
                           c^2 = gamma (p + p_inf)/(rho (1 - b rho));
                           0: the stiffened gas above */
} orc_problem;

int orc_nfields(const orc_problem* P);
void orc_set_threads(int n);
int orc_step(const orc_problem* P, const double* U, double dt, double* Unew);
int orc_step_window(const orc_problem* P, const double* U, double dt,
                    const int wlo[3], const int whi[3], double* out);
double orc_dt(const orc_problem* P, const double* U);
void orc_diagnostics(const orc_problem* P, const double* U, double out[10]);
void orc_cell_at(const orc_problem* P, const double* U, const int ijk[3], double out[12]);
void orc_face(const orc_problem* P, const double* Lprim, const double* Rprim, int d, double out[5]);

#ifdef __cplusplus
}
#endif
#endif
