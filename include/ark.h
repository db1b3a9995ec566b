/*
 * ark.h -- C ABI of the GB300 (sm_103a) explicit step of the all-regime,
 * well-balanced acoustic-transport finite-volume scheme for the stratified
 * compressible Navier-Stokes equations (Padioleau, Tremblin, Audit, Kestener,
 * Kokh, arXiv:1903.09043).
 *
 * One call of ark_step advances the cell averages U = (rho, rho u, rho v
 * [, rho w], rho*calE) by one time step of the scheme of Sec. 2:
 *   - acoustic step with the well-balanced gravity source (Sec. 2.1.2):
 *     per face a, S_{i+1/2}, u*, Pi*, with the low-Mach correction theta of
 *     Eq. 16 (Sec. 2.1.5); per cell L~ and the tilde states;
 *   - transport step, upwind on u* (Sec. 2.1.3);
 *   - relaxation step Psi^{n+1} = Phi (Sec. 2.1.4; no change to the state);
 *   - first-order viscous and heat-conduction fluxes (Sec. 2.2);
 *   - the CFL time step of the next step, reduced on the device.
 * rho*calE = rho e + rho |u|^2 / 2 + rho Phi is the total energy including the
 * gravitational energy (Eq. 6, conservation_of_energy).  The equation of
 * state is the stiffened gas p = (gamma - 1) rho e - gamma p_inf,
 * T = (p + p_inf) / rho, c^2 = gamma (p + p_inf) / rho, which with p_inf = 0
 * is the ideal gas of Sec. 4, or the Noble-Abel stiffened gas (a covolume b;
 * see ark_eos); Sec. 4 notes that the scheme takes another equation of
 * state.
 *
 * Conventions for every call:
 *   - Arrays are structure-of-arrays: field f of cell (i, j[, k]) is at
 *     U[f * N + i + nx * (j + ny * k)], N = nx * ny [* nz], x fastest, FP64.
 *     Field order: rho, m_x, m_y, [m_z,] rho*calE (nf = dim + 2 fields).
 *   - All device work is enqueued on the CUDA stream given to ark_create
 *     (NULL = the legacy default stream).  Calls that return host data
 *     synchronise that stream; ark_step does not.
 *   - Every call returns an ark_status; nothing aborts or traps.  The text
 *     of the last error of a handle is returned by ark_last_error.
 *   - Handles are not thread-safe: one host thread at a time per handle.
 */
#ifndef ARK_H
#define ARK_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ARK_OK = 0,
    ARK_ERR_INVALID_ARG = 1,   /* a parameter or pointer is out of its domain       */
    ARK_ERR_CUDA = 2,          /* a CUDA runtime call failed (see ark_last_error)    */
    ARK_ERR_NONPHYSICAL = 3,   /* the device saw rho <= 0, p + p_inf <= 0, L~ <= 0, NaN */
    ARK_ERR_TIMEOUT = 4,       /* a bounded wait on the device ran out               */
    ARK_ERR_UNSUPPORTED = 5,   /* valid input that this build does not implement     */
    ARK_ERR_ALLOC = 6          /* device or host allocation failed                   */
} ark_status;

/* Boundary conditions per face of the box (ghost cells, Sec. 3.2). */
enum {
    ARK_BC_PERIODIC = 0,       /* wrap-around                                        */
    ARK_BC_REFLECT_HYDRO = 1,  /* reflective wall: normal velocity mirrored with sign
                                  flip, temperature mirrored, pressure and density
                                  extrapolated by the discrete hydrostatic balance of
                                  Eq. 18 (Sec. 4.3: "extrapolation of the hydrostatic
                                  balance ... reflexive conditions for the velocity") */
    ARK_BC_NOSLIP_FIXED_T = 2, /* no-slip wall (all velocity components mirrored with
                                  sign flip) at a fixed temperature T_wall: ghost
                                  T = 2 T_wall - T_mirror; p, rho as above (Sec. 4.5) */
    ARK_BC_OUTFLOW = 3,        /* zero-gradient copy of (rho, u, p)                  */
    ARK_BC_HALO = 4            /* x sides only: the side borders another subdomain of
                                  a slab decomposition along x (Sec. 3.2: the domain is
                                  split into subdomains whose ghost zones hold the
                                  neighbours' cells, exchanged every step).  Its two
                                  ghost layers are the values last given to
                                  ark_set_halo (zero before the first); n[0] >= 2.
                                  Uniform gravity only (no potential array); not in
                                  ensembles.                                           */
};

/* Arithmetic of the device state. */
enum {
    ARK_F64 = 0,               /* FP64 state and arithmetic                           */
    ARK_F32 = 1,               /* FP32 state and arithmetic                           */
    ARK_F32_SPLIT = 2          /* FP32 deviations from an FP64 hydrostatic base state
                                  (per row along the gravity axis); the base-state
                                  pressure jump minus the gravity source, and every
                                  base-state quantity, are formed in FP64             */
};

typedef struct {
    int dim;                   /* 2 or 3                                              */
    int n[3];                  /* cells along x, y, z; n[2] is ignored when dim == 2  */
    double lo[3], hi[3];       /* box corners                                         */
} ark_grid;

/* Equation of state (Sec. 4 uses the ideal gas and notes that the scheme
 * admits another law).  With (gamma - 1) c_v = 1:
 *   ARK_EOS_STIFFENED_GAS  p = (gamma-1) rho e - gamma p_inf,  T = (p + p_inf)/rho,
 *                          c^2 = gamma (p + p_inf)/rho; p_inf = 0 is the ideal gas;
 *   ARK_EOS_NOBLE_ABEL     the Noble-Abel stiffened gas, a covolume b leaving the
 *                          fraction 1 - b rho of the volume free:
 *                          p = (gamma-1) rho e / (1 - b rho) - gamma p_inf,
 *                          T = (p + p_inf)(1 - b rho)/rho,
 *                          c^2 = gamma (p + p_inf)/(rho (1 - b rho));
 *                          b = 0 is the stiffened gas.
 * The wall ghosts solve the discrete balance of Eq. 18 with the law's density
 * rho(p, T).  The law is chosen per kernel instance, so the stiffened-gas
 * path carries no covolume arithmetic. */
enum {
    ARK_EOS_STIFFENED_GAS = 0,
    ARK_EOS_NOBLE_ABEL = 1
};

typedef struct {
    double gamma;              /* adiabatic index, > 1                                */
    double p_inf;              /* stiffened-gas constant, finite and >= 0 (0: ideal
                                  gas).  Physical states need rho > 0 and
                                  p + p_inf > 0; p itself may be negative.            */
    int law;                   /* ARK_EOS_STIFFENED_GAS or ARK_EOS_NOBLE_ABEL          */
    double b;                  /* covolume (ARK_EOS_NOBLE_ABEL), finite and >= 0;
                                  physical states also need b rho < 1.  Must be 0
                                  for ARK_EOS_STIFFENED_GAS.  With a covolume,
                                  ARK_F64, ARK_F32 and ARK_F32_SPLIT take uniform
                                  gravity only (no potential array); ensembles and
                                  ark_compute_dt_noalloc take the stiffened gas. */
} ark_eos;

typedef struct {
    double g;                  /* uniform gravity along the LAST axis (y in 2D, z in
                                  3D): Phi = -g * x_last at cell centres; g < 0 pulls
                                  toward the low side.  Phi is time independent.       */
    const double* phi;         /* NULL, or a host array of N values: the potential at
                                  the cell centres (layout of one field), any
                                  direction; then g must be 0.  ark_create copies it.
                                  Ghost values wrap across periodic sides and extend
                                  linearly from the two nearest interior cells across
                                  walls and outflow.  The gravity source S then acts
                                  on every face (Sec. 2.1.2).  ARK_F64 and ARK_F32
                                  take any array; ARK_F32_SPLIT takes an array that
                                  depends on the last (gravity) axis only (one base
                                  row per level, its tables formed in FP64 from the
                                  array's row values) and returns ARK_ERR_UNSUPPORTED
                                  for any other.                                       */
} ark_gravity;

typedef struct {
    int lo[3], hi[3];          /* ARK_BC_* per axis and side                          */
    double T_lo[3], T_hi[3];   /* wall temperatures for ARK_BC_NOSLIP_FIXED_T         */
} ark_bc;

typedef struct {
    ark_grid grid;
    ark_eos eos;
    ark_gravity gravity;
    double mu;                 /* dynamic viscosity; bulk viscosity eta = -2 mu / 3
                                  (Stokes hypothesis, Eq. 4)                          */
    double kappa;              /* heat conductivity, q = -kappa grad T (Eq. 3)        */
    int low_mach;              /* 1: theta of Eq. 16; 0: theta = 1                    */
    double K;                  /* a_{i+1/2} = K max(rho_i c_i, rho_{i+1} c_{i+1}),
                                  K >= 1 (sub-characteristic condition, Sec. 2.1.2)   */
    double cfl;                /* dt = cfl / max_i max(sum_d (|u_d| + c) / dx_d,
                                  sum_d 2 max(4 mu / (3 rho), kappa (gamma - 1) / rho)
                                  / dx_d^2)                                           */
    ark_bc bc;
    int precision;             /* ARK_F64, ARK_F32 or ARK_F32_SPLIT                   */
    int energy_form;           /* 0: the energy field is rho*calE = rho e + rho |u|^2/2
                                  + rho Phi, conserved (Sec. 2); 1: it is rho E = rho e
                                  + rho |u|^2/2 and the acoustic step adds the gravity
                                  work dt/dx (uS)_i (Appendix B, not conservative for
                                  the total energy).  ARK_F32_SPLIT needs 0.           */
} ark_params;

typedef struct {
    double mass;               /* sum rho dV                                          */
    double momentum[3];        /* sum m dV                                            */
    double energy;             /* sum of the energy field dV (rho*calE, or rho E when
                                  energy_form == 1)                                    */
    double kinetic;            /* sum rho |u|^2 / 2 dV                                */
    double max_speed;          /* max |u|                                             */
    double mean_abs_v_last;    /* mean |u_last| (vertical velocity)                   */
    double min_rho, min_p;
    double t;                  /* simulated time                                      */
    long long step;            /* steps taken                                         */
    double dt;                 /* time step of the last step taken                    */
    unsigned int status;       /* device status bits: 1 nonphysical rho/p, 2 L~ <= 0,
                                  4 NaN; cleared by ark_set_state                     */
} ark_diag;

typedef struct ark_handle ark_handle;

/* Create a solver for one grid.  Validates p (dims, sizes >= 1, n >= 2 along
 * wall/outflow axes, finite box corners and gravity, finite gamma > 1,
 * K >= 1, cfl > 0, mu, kappa >= 0, all finite, periodic
 * axes without gravity; ARK_F32_SPLIT: fixed-temperature walls only at the
 * two ends of the gravity axis and energy_form 0; ARK_F32 and ARK_F32_SPLIT:
 * fewer than 2^32 cells, else ARK_ERR_UNSUPPORTED), allocates the device state (two ping-pong copies of nf * N
 * values of the chosen precision) and small scratch on the current device.
 * The state is undefined until ark_set_state.  *out receives the handle,
 * which the caller releases with ark_destroy.
 * Errors: ARK_ERR_INVALID_ARG, ARK_ERR_UNSUPPORTED, ARK_ERR_ALLOC, ARK_ERR_CUDA. */
ark_status ark_create(const ark_params* p, void* cuda_stream, ark_handle** out);

/* Release every device and host resource of h (synchronises its stream). */
ark_status ark_destroy(ark_handle* h);

/* Load the state from U (nf * N FP64 values in the layout above), on the host
 * (on_device = 0) or on the current device (on_device = 1).  For
 * ARK_F32_SPLIT the FP64 base state is the horizontal mean of rho and p of
 * each row along the gravity axis of U.  Resets t, step and status.  The
 * caller keeps ownership of U; the call returns after U may be reused.
 * With a host U and an FP32 form, the first call allocates a device staging
 * buffer of nf * N doubles that h keeps until ark_destroy (ARK_ERR_ALLOC if
 * it cannot); host transfers run fastest from pinned memory. */
ark_status ark_set_state(ark_handle* h, const double* U, int on_device);

/* Store the state into U (same layout, FP64), host or device memory (a host U
 * with an FP32 form uses the staging buffer of ark_set_state). */
ark_status ark_get_state(ark_handle* h, double* U, int on_device);

/* CFL time step of the current state (formula at ark_params.cfl).  Writes it
 * to *dt_out when dt_out != NULL (synchronising), and always leaves it on the
 * device for the next ark_step with dt <= 0. */
ark_status ark_compute_dt(ark_handle* h, double* dt_out);

/* Advance nsteps >= 0 steps.  dt > 0: fixed time step.  dt <= 0: each step
 * uses the CFL time step of its own initial state, reduced on the device by
 * the previous step (the first from ark_compute_dt, run implicitly if
 * needed).  One kernel launch per step; no host synchronisation. */
ark_status ark_step(ark_handle* h, int nsteps, double dt);

/* Conservation sums (FP64 tree sums in fixed order), extrema, t, step, dt and
 * the device status word.  Synchronises.  Returns ARK_ERR_NONPHYSICAL (after
 * filling *out) when the status word is non-zero. */
ark_status ark_diagnostics(ark_handle* h, ark_diag* out);

/* Simulated time and the time step of the last step taken (8 + 8 bytes read
 * back from the device; synchronises the stream).  Either pointer may be NULL. */
ark_status ark_time(ark_handle* h, double* t, double* dt);

/* Wait for the handle's stream with a time limit (seconds); ARK_ERR_TIMEOUT
 * when it is still busy at the limit, ARK_ERR_NONPHYSICAL when the device
 * status word is non-zero, ARK_OK otherwise. */
ark_status ark_sync(ark_handle* h, double timeout_s);

/* Slab decomposition along x (Sec. 3.2, Implementation: regular domain
 * decomposition with ghost zones per direction and side).  A subdomain is an
 * ordinary handle whose inner x sides are ARK_BC_HALO; before each step the
 * caller moves every subdomain's boundary layers to its neighbours' ghost
 * layers and gives all subdomains the same dt (the minimum of their
 * ark_compute_dt, the CFL step of the whole grid).  With FP64 the result
 * equals the undivided grid's.
 * Layout of a halo buffer: nf * nv * ny * 2 FP64 values (ny = 1 in 2D; nv
 * the cells along the last axis), value (f, k, j, l) at
 * [((f * nv + k) * ny + j) * 2 + l]: field f, plane k of the last axis, row j
 * of y (3D), layer l counted from the side (l = 0 the layer at the side).
 *
 * ark_get_halo: the two cell layers of the current state next to x side
 * `side` (0: low, 1: high), full values (the split form adds its FP64 base
 * rows), into `out` (host, or device with on_device = 1; synchronises for a
 * host buffer).  Any x side may be read.  Needs the state set.
 * ark_set_halo: the two ghost layers beyond the ARK_BC_HALO side `side`, in
 * the layout above with l = 0 the ghost layer adjacent to the side: the
 * neighbour's layers as ark_get_halo returns them from its facing side.  The
 * values are converted to the state's form (the split form subtracts its
 * base rows, so it needs its state first, and ark_set_state, which forms new
 * base rows, calls for the halos to be set again) and read by every later
 * ark_step until the next ark_set_halo.  The caller keeps `in`; a host `in` may be
 * reused when the call returns.
 * Errors: ARK_ERR_INVALID_ARG (side not 0/1, that side not ARK_BC_HALO for
 * ark_set_halo, state not set where needed), ARK_ERR_ALLOC (host staging of
 * nf * nv * ny * 2 doubles, made on first use), ARK_ERR_CUDA. */
ark_status ark_get_halo(ark_handle* h, int side, double* out, int on_device);
ark_status ark_set_halo(ark_handle* h, int side, const double* in, int on_device);

/* Device address and byte size of the current state buffer (read only for
 * the caller; valid until the next ark_step or ark_set_state). */
ark_status ark_state_device_ptr(ark_handle* h, const void** ptr, size_t* bytes);

/* Kernel shape chosen for h: in-plane tile (tx, ty), planes per block along
 * the gravity axis, threads per block and blocks per launch. */
ark_status ark_launch_shape(const ark_handle* h, int* tx, int* ty, int* planes, int* threads, int* blocks);

/* CFL time step of an FP64 state that the caller keeps on the device, computed
 * without allocating any device memory and without a handle.  The paper has no
 * counterpart: this exists for callers that cannot allocate device memory
 * when they need a time step (a memory pool or arena that owns the device, a
 * host thread that must not trigger an allocation, which can synchronise the
 * device or fail when memory is full).
 *   p   problem description, checked by the rules of ark_create;
 *       p->precision must be ARK_F64 (the state is FP64)
 *   U   device pointer, nf * N FP64 values in the layout above, read only
 *   dt  device pointer to one double; receives cfl / max wave rate (the
 *       formula at ark_params.cfl), written on `stream`.  If any cell has
 *       rho <= 0, p + p_inf <= 0 or a NaN wave rate, *dt receives NaN
 *       instead, so a bad state never yields a finite step from its healthy
 *       cells.
 * Scratch: a fixed array of 16384 doubles (128 KiB) inside the library's
 * device image, held by every GPU that loads the library until the process
 * exits; it bounds N to 67,108,864 cells (4096 cells per scratch slot).
 * Larger grids are rejected with ARK_ERR_INVALID_ARG before any launch.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current and keeps it for the
 * process; make that first call before any stream capture, and do not use
 * the call across a cudaDeviceReset (the kept address goes stale).  Every
 * call uses the same array and overwrites the slots it reads, so consecutive
 * calls are independent, but calls that overlap on the GPU (unordered
 * streams) race on it.  Calls no allocating routine.  Returns after
 * enqueueing; it does not synchronise.
 * Errors: ARK_ERR_INVALID_ARG (null pointer, parameters outside the rules of
 * ark_create, a precision other than ARK_F64, too many cells),
 * ARK_ERR_UNSUPPORTED (p->gravity.phi set: the potential array would need a
 * device copy), ARK_ERR_CUDA (a launch failed, or an error from the caller's
 * earlier work was already pending: it is reported, not cleared, and nothing
 * is launched). */
ark_status ark_compute_dt_noalloc(const ark_params* p, const double* U, double* dt, void* stream);

/* ---------------------------------------------------------------------------
 * Ensembles: many independent 2D runs advanced together, one kernel launch
 * per step for all of them (not in the paper; an ensemble of its Rayleigh-
 * Benard set-ups of different sizes and Rayleigh numbers).
 * ------------------------------------------------------------------------- */
typedef struct ark_batch ark_batch;

/* Create an ensemble of `count` runs.  params[i] describes run i; every run
 * must be 2D and share the precision (ARK_F64 or ARK_F32_SPLIT) and whether it
 * has dissipation (mu or kappa > 0).  Each run gets its own device state,
 * base state and time-step slots, as with ark_create; work is enqueued on
 * `cuda_stream`.  Errors as ark_create. */
ark_status ark_batch_create(int count, const ark_params* params, void* cuda_stream, ark_batch** out);

/* Load or store run i's state (layout and ownership as ark_set_state /
 * ark_get_state).  All runs must be loaded before the first ark_batch_step;
 * reloading one run after the ensemble has stepped returns ARK_ERR_INVALID_ARG
 * at the next ark_batch_step (runs advance in lockstep). */
ark_status ark_batch_set_state(ark_batch* b, int run, const double* U, int on_device);
ark_status ark_batch_get_state(ark_batch* b, int run, double* U, int on_device);

/* Autotuner: times the batched kernel for every tile width (64, 128, 256
 * cells) and planes per work item (16, 32, 64), `reps` launches each, on the
 * current states without changing them (outputs go to the spare buffers,
 * time and slots to scratch), and keeps the fastest.  Optional outputs. */
ark_status ark_batch_tune(ark_batch* b, int reps, int* tx, int* planes);

/* Advance every run nsteps >= 0 steps, each with its own CFL time step.  One
 * launch per step: a persistent grid (resident blocks x SMs) takes (run, tile,
 * planes) work items from an atomic counter.  Whole 6-step cycles (ping-pong
 * buffers x 3 rotating time-step slots) replay one CUDA graph built on first
 * use.  No host synchronisation. */
ark_status ark_batch_step(ark_batch* b, int nsteps);

/* Diagnostics of run i (as ark_diagnostics). */
ark_status ark_batch_diagnostics(ark_batch* b, int run, ark_diag* out);

/* Chosen tile width, planes per item, number of work items and resident blocks. */
ark_status ark_batch_shape(const ark_batch* b, int* tx, int* planes, int* items, int* blocks);

ark_status ark_batch_destroy(ark_batch* b);
const char* ark_batch_last_error(const ark_batch* b);

const char* ark_last_error(const ark_handle* h);
const char* ark_status_string(ark_status s);

#ifdef __cplusplus
}
#endif
#endif /* ARK_H */
