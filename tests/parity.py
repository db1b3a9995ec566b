"""Error norms and tolerances used by the parity tests.

Relative L-infinity per field with a floor that keeps fields that vanish in
the reference (momenta of a state at rest) meaningful:
  err_f = max |x_f - ref_f| / max(max |ref_f|, s_f),
  s_rho = max rho_ref, s_m = max rho_ref * max c_ref, s_W = max |W_ref|.

Tolerances:
* F64: 1e-12 (the stated FP64 target; the observed one-step difference is a
  few 1e-16, the rounding order of sums and reciprocals differing).
* F32 and F32_SPLIT against the FP64 oracle: a per-step budget of
  8 * 2^-24 ~ 4.8e-7 of the field scale (a handful of float roundings per
  stored value per step), times the number of steps.
"""
import numpy as np

F64_TOL = 1e-12
F32_STEP_TOL = 8 * 2.0 ** -24


def sound_speed(prob, U):
    dim = prob.dim
    rho = U[0]
    ke = 0.5 * sum(U[1 + d] ** 2 for d in range(dim)) / rho
    phi = -prob.g * prob.centers(dim - 1).reshape((-1,) + (1,) * (dim - 1))
    p = (prob.gamma - 1.0) * (U[dim + 1] - ke - rho * phi)
    return np.sqrt(prob.gamma * np.abs(p) / rho)


def field_errors(prob, A, ref):
    dim = prob.dim
    rho_max = np.max(np.abs(ref[0]))
    c_max = np.max(sound_speed(prob, ref))
    errs = []
    for f in range(ref.shape[0]):
        if f == 0:
            floor = rho_max
        elif f <= dim:
            floor = rho_max * c_max
        else:
            floor = np.max(np.abs(ref[f]))
        scale = max(np.max(np.abs(ref[f])), floor)
        errs.append(float(np.max(np.abs(A[f] - ref[f])) / scale))
    return errs


def max_error(prob, A, ref):
    return max(field_errors(prob, A, ref))
