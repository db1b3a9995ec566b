"""Studies of the paper's workloads run through the CUDA library.

    python -m paper_1903_09043_gb300.studies precision   # Gresho 1024^2, Mach sweep, FP32 forms vs FP64
    python -m paper_1903_09043_gb300.studies rb_growth   # 2D Rayleigh-Benard 256x128 onset sweep, 2e4 steps
    python -m paper_1903_09043_gb300.studies rb_onset    # the same, Ra/Ra_c 1.1 .. 30, 8e4 steps, FP64
    python -m paper_1903_09043_gb300.studies rayleigh_taylor  # Sec. 4.4, 200x600 to t = 12.4, theta on/off
    python -m paper_1903_09043_gb300.studies spectrum    # 3D Rayleigh-Benard 512x512x256, FP32 vs FP64 spectrum

Each prints one JSON document.  The FP64 path is the reference of the
precision comparisons: it equals the FP64 CPU oracle within 1e-12 per field
(tests/test_gpu_parity.py), and runs the full sizes in seconds where the
oracle would take hours.
"""
from __future__ import annotations

import argparse
import json
import math

import numpy as np

from . import ark
from . import inputs as I


def _stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


def field_errors(prob, A, ref):
    """Relative L-infinity and L2 per field, with floors (rho scale for rho,
    rho*c scale for momenta, energy scale for rho*calE)."""
    dim = prob.dim
    rho = ref[0]
    ke = 0.5 * sum(ref[1 + d] ** 2 for d in range(dim)) / rho
    phi = -prob.g * prob.centers(dim - 1).reshape((-1,) + (1,) * (dim - 1))
    p = (prob.gamma - 1.0) * (ref[dim + 1] - ke - rho * phi)
    c = np.sqrt(prob.gamma * np.abs(p) / rho)
    floors = [np.max(np.abs(rho))] + [np.max(np.abs(rho)) * np.max(c)] * dim + [np.max(np.abs(ref[dim + 1]))]
    names = ["rho"] + ["m_" + "xyz"[d] for d in range(dim)] + ["rhoE"]
    out = {}
    for f in range(ref.shape[0]):
        sc = max(np.max(np.abs(ref[f])), floors[f])
        d = A[f] - ref[f]
        out[names[f]] = {"linf": float(np.max(np.abs(d)) / sc), "l2": float(np.sqrt(np.mean(d * d)) / sc)}
    return out


def run(prob, U, precision, nsteps, dt=-1.0):
    with ark.Solver(prob, precision, stream=_stream()) as s:
        s.set_state(U)
        s.step(nsteps, dt)
        V = s.get_state()
        d = s.diagnostics(check=False)
    return V, d


def precision(n=1024, machs=(1e-1, 1e-2, 1e-3, 1e-4), t_final=1e-3):
    """Gresho vortex (Sec. 4.2): every form advanced to t_final with one common
    fixed time step (the CFL step of the initial state, rounded to divide t_final)."""
    rows = []
    for mach in machs:
        for low_mach in (1, 0):
            prob, U = I.gresho(n, mach=mach, low_mach=low_mach)
            with ark.Solver(prob, "f64", stream=_stream()) as s:
                s.set_state(U)
                dt0 = s.compute_dt()
            nsteps = int(math.ceil(t_final / dt0))
            dt = t_final / nsteps
            ref, _ = run(prob, U, "f64", nsteps, dt)
            ue, ve = I.gresho_velocity(prob)
            row = {"mach": mach, "low_mach": low_mach, "steps": nsteps, "dt": dt,
                   "l1_velocity_error_vs_exact": {}}
            for prec in ("f64", "f32split", "f32"):
                V = ref if prec == "f64" else run(prob, U, prec, nsteps, dt)[0]
                row["l1_velocity_error_vs_exact"][prec] = float(
                    np.mean(np.abs(V[1] / V[0] - ue) + np.abs(V[2] / V[0] - ve)))
                if prec != "f64":
                    row[prec + "_vs_f64"] = field_errors(prob, V, ref)
                    dv = np.sqrt((V[1] / V[0] - ref[1] / ref[0]) ** 2 + (V[2] / V[0] - ref[2] / ref[0]) ** 2)
                    row[prec + "_velocity_linf_vs_f64"] = float(np.max(dv))
            rows.append(row)
    return {"study": "precision", "workload": f"gresho {n}x{n}", "t_final": t_final, "rows": rows}


def rb_growth(steps=20000, every=500, ratios=(0.9, 1.1, 1.5, 2.0, 3.0, 5.0), roll=True, precisions=("f64", "f32split"),
              low_machs=(1, 0)):
    """2D Rayleigh-Benard 256x128 near onset (Sec. 4.5): growth rate of the mean
    absolute vertical velocity over the last half of the run, from the roll-pair
    perturbation (amplitude 1e-4) or from white noise."""
    rows = []
    for ratio in ratios:
        for low_mach in low_machs:
            for prec in precisions:
                prob, U = I.rayleigh_benard(2, (256, 128), Ra=ratio * I.RA_CRITICAL_RIGID, low_mach=low_mach, roll=roll)
                ts, vs = [], []
                with ark.Solver(prob, prec, stream=_stream()) as s:
                    s.set_state(U)
                    for _ in range(steps // every):
                        s.step(every)
                        d = s.diagnostics(check=False)
                        ts.append(d["t"])
                        vs.append(d["mean_abs_v_last"])
                ts, vs = np.array(ts), np.array(vs)
                half = len(ts) // 2
                rate = float(np.polyfit(ts[half:], np.log(vs[half:]), 1)[0])
                rows.append({"ra_over_ra_c": ratio, "low_mach": low_mach, "precision": prec, "t_final": float(ts[-1]),
                             "growth_rate": rate, "mean_abs_v_final": float(vs[-1])})
    return {"study": "rb_growth", "workload": f"rayleigh_benard 2d 256x128, {steps} steps, "
            + ("roll-pair" if roll else "white-noise") + " perturbation 1e-4", "rows": rows}


def rayleigh_taylor(n=(200, 600), t_final=12.4, chunk=50):
    """Rayleigh-Taylor (Sec. 4.4) on 200 x 600 to t = 12.4 with and without the
    low-Mach correction: growth rate of max |v| over t in [1, 4] (the
    incompressible linear rate of the seeded mode is sqrt(A g k) with Atwood
    number A = 1/3, g = 0.1, k = 4 pi), mixing-zone extent at t_final (rows
    whose mean density lies strictly between 1.05 and 1.95), FP32-split vs FP64."""
    sigma = math.sqrt((1.0 / 3.0) * 0.1 * 4.0 * math.pi)
    rows = []
    for low_mach in (1, 0):
        finals = {}
        for prec in ("f64", "f32split"):
            prob, U = I.rayleigh_taylor(n, low_mach=low_mach)
            ts, vs = [], []
            with ark.Solver(prob, prec, stream=_stream()) as s:
                s.set_state(U)
                while True:
                    d = s.diagnostics(check=False)
                    ts.append(d["t"])
                    vs.append(d["max_speed"])
                    remaining = t_final - d["t"]
                    if remaining <= 1e-12:
                        break
                    dt = s.compute_dt()
                    if remaining > (chunk + 10) * dt:
                        s.step(chunk)                  # CFL steps
                    elif remaining > dt:
                        s.step(1)
                    else:
                        s.step(1, remaining)           # land on t_final
                V = s.get_state()
                steps = s.diagnostics(check=False)["step"]
            ts, vs = np.array(ts), np.array(vs)
            sel = (ts >= 1.0) & (ts <= 4.0)
            rate = float(np.polyfit(ts[sel], np.log(vs[sel]), 1)[0])
            rho_mean = V[0].mean(axis=1)
            mixed = np.nonzero((rho_mean > 1.05) & (rho_mean < 1.95))[0]
            y = prob.centers(1)
            width = float(y[mixed[-1]] - y[mixed[0]]) if mixed.size else 0.0
            finals[prec] = V
            rows.append({"low_mach": low_mach, "precision": prec, "steps": int(steps), "t_final": float(ts[-1]),
                         "growth_rate_t1_4": rate, "growth_rate_over_linear_theory": rate / sigma,
                         "max_speed_final": float(vs[-1]), "mixing_zone_width": width})
        rows[-1]["f32split_density_linf_vs_f64"] = float(np.max(np.abs(finals["f32split"][0] - finals["f64"][0])))
    return {"study": "rayleigh_taylor", "workload": f"rayleigh_taylor {n[0]}x{n[1]} to t = {t_final}",
            "linear_theory_rate": sigma, "rows": rows}


def ke_spectrum(V, prob):
    """Shell-binned kinetic-energy spectrum of the horizontal middle plane."""
    k = prob.n[2] // 2
    rho = V[0, k]
    e = []
    for d in range(3):
        u = V[1 + d, k] / rho
        f = np.fft.fft2(np.sqrt(rho) * u) / u.size
        e.append(np.abs(f) ** 2)
    E = 0.5 * sum(e)
    ny, nx = E.shape
    kx = np.fft.fftfreq(nx) * nx
    ky = np.fft.fftfreq(ny) * ny
    kk = np.sqrt(kx[None, :] ** 2 + ky[:, None] ** 2)
    shells = np.rint(kk).astype(int)
    spec = np.bincount(shells.ravel(), weights=E.ravel())
    return spec[: min(nx, ny) // 2]


def spectrum(steps=200):
    prob, U = I.rayleigh_benard(3, (512, 512, 256), m=0.1, chi=1.1, Ra=1e7, amp=1e-3, seed=4)
    out = {}
    with ark.Solver(prob, "f64", stream=_stream()) as s:
        s.set_state(U)
        dt0 = s.compute_dt()
    dt = 0.9 * dt0   # one fixed step for both forms
    for prec in ("f64", "f32split"):
        V, d = run(prob, U, prec, steps, dt)
        out[prec] = (ke_spectrum(V, prob), d)
    s64, s32 = out["f64"][0], out["f32split"][0]
    rel = np.abs(s32 - s64) / np.maximum(s64, 1e-300)
    return {"study": "spectrum", "workload": "rayleigh_benard 3d 512x512x256", "steps": steps, "dt": dt,
            "shells": len(s64), "max_rel_shell_difference": float(np.max(rel[1:])),
            "median_rel_shell_difference": float(np.median(rel[1:])),
            "total_ke_f64": float(np.sum(s64)), "total_ke_f32split": float(np.sum(s32)),
            "spectrum_f64_first_shells": s64[:12].tolist(), "spectrum_f32split_first_shells": s32[:12].tolist()}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("study", choices=["precision", "rb_growth", "rb_onset", "rayleigh_taylor", "spectrum"])
    ap.add_argument("--n", type=int, default=1024)
    args = ap.parse_args()
    if args.study == "precision":
        res = precision(n=args.n)
    elif args.study == "rb_growth":
        res = rb_growth()
    elif args.study == "rb_onset":
        res = rb_growth(steps=80000, every=2000, ratios=(1.1, 1.5, 2.0, 3.0, 5.0, 10.0, 15.0, 20.0, 25.0, 30.0),
                        precisions=("f64",))
    elif args.study == "rayleigh_taylor":
        res = rayleigh_taylor()
    else:
        res = spectrum()
    print(json.dumps(res))


if __name__ == "__main__":
    main()
