"""Batched ensemble path: one launch per step for many independent 2D runs.

Each run of an ensemble must equal the same run advanced alone (bit for bit:
the per-cell arithmetic is the same kernel body, only the work decomposition
differs), and in FP64 the oracle within the FP64 tolerance."""
import numpy as np
import pytest

import oracle as O
from paper_1903_09043_gb300 import inputs as I
from parity import F64_TOL, max_error

pytestmark = pytest.mark.gpu

O.set_threads(1)


def _stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


def _ensemble(count=6, seed=11):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        nx = [64, 80, 112, 144, 272, 96][i % 6]
        Ra = float(np.exp(rng.uniform(np.log(1e3), np.log(1e6))))
        out.append(I.rayleigh_benard(2, (nx, nx // 2), Ra=Ra, amp=1e-3, rng=rng))
    return out


def _single(prob, U, n, precision):
    from paper_1903_09043_gb300 import ark
    with ark.Solver(prob, precision, stream=_stream()) as s:
        s.set_state(U)
        s.step(n)
        return s.get_state(), s.diagnostics(check=False)


@pytest.mark.parametrize("precision", ["f64", "f32split"])
def test_batch_equals_runs_alone(precision):
    from paper_1903_09043_gb300 import ark
    runs = _ensemble()
    n = 15   # two graph cycles and three single launches
    with ark.Batch([p for p, _ in runs], precision, stream=_stream()) as b:
        for i, (_, U) in enumerate(runs):
            b.set_state(i, U)
        b.step(2)        # direct launches (phases 0, 1)
        b.step(n - 2)    # phases 2..5 direct, then a graph cycle, then one launch
        outs = [b.get_state(i) for i in range(len(runs))]
        diags = [b.diagnostics(i, check=False) for i in range(len(runs))]
    for (prob, U), V, d in zip(runs, outs, diags):
        ref, dref = _single(prob, U, n, precision)
        assert np.array_equal(V, ref)
        assert d["t"] == dref["t"] and d["step"] == n and d["status"] == 0
        if precision == "f64":
            W, t = O.run(prob, U, n)
            assert max_error(prob, V, W) <= F64_TOL
            assert d["t"] == pytest.approx(t, rel=1e-13)


def test_tuning_leaves_states_unchanged_and_picks_a_shape():
    from paper_1903_09043_gb300 import ark
    runs = _ensemble(count=5, seed=3)
    with ark.Batch([p for p, _ in runs], "f32split", stream=_stream()) as b:
        for i, (_, U) in enumerate(runs):
            b.set_state(i, U)
        before = [b.get_state(i) for i in range(len(runs))]
        tx, planes = b.tune(reps=2)
        assert tx in (60, 124, 252, 64, 128, 256) and planes in (16, 32, 64)
        assert b.shape()["tx"] == tx
        for i in range(len(runs)):
            assert np.array_equal(b.get_state(i), before[i])
        b.step(8)
        outs = [b.get_state(i) for i in range(len(runs))]
    for (prob, U), V in zip(runs, outs):
        ref, _ = _single(prob, U, 8, "f32split")
        assert np.array_equal(V, ref)


def test_batch_runs_must_stay_in_lockstep():
    from paper_1903_09043_gb300 import ark
    runs = _ensemble(count=2)
    with ark.Batch([p for p, _ in runs], "f64", stream=_stream()) as b:
        for i, (_, U) in enumerate(runs):
            b.set_state(i, U)
        b.step(3)
        b.set_state(1, runs[1][1])
        with pytest.raises(ark.ArkError) as ei:
            b.step(1)
        assert ei.value.status == ark.ARK_ERR_INVALID_ARG


def test_batch_of_atmospheres_stays_at_rest():
    """Runs keep their own equation of state: the middle one is a stiffened-gas
    column (p_inf = 5) among ideal-gas atmospheres."""
    from paper_1903_09043_gb300 import ark
    runs = [I.atmosphere((n, n // 2 + 3), p_inf=pinf) for n, pinf in ((64, 0.0), (100, 5.0), (130, 0.0))]
    with ark.Batch([p for p, _ in runs], "f32split", stream=_stream()) as b:
        for i, (_, U) in enumerate(runs):
            b.set_state(i, U)
        b.step(300)
        for i in range(len(runs)):
            assert b.diagnostics(i)["max_speed"] < 1e-10


def test_full_ensemble_sampled_against_the_oracle():
    """The benchmark's ensemble (256 runs, 7.09 M cells) in its launch
    configuration (autotuned tiles, graph-replayed steps): every run ends with
    a clean status word, and four sampled runs (the smallest, the largest and
    two drawn ones) equal the oracle within the FP32 budget."""
    from paper_1903_09043_gb300 import ark
    from parity import F32_STEP_TOL, field_errors
    runs = I.ensemble()
    assert len(runs) == 256
    sizes = [p.ncells for p, _ in runs]
    picks = sorted({int(np.argmin(sizes)), int(np.argmax(sizes)), 17, 200})
    n = 8
    with ark.Batch([p for p, _ in runs], "f32split", stream=_stream()) as b:
        for i, (_, U) in enumerate(runs):
            b.set_state(i, U)
        b.tune(reps=2)
        b.step(n)
        outs = {i: b.get_state(i) for i in picks}
        diags = [b.diagnostics(i, check=False) for i in range(len(runs))]
    assert all(d["status"] == 0 and d["step"] == n for d in diags)
    for i in picks:
        prob, U = runs[i]
        ref, _ = O.run(prob, U, n)
        errs = field_errors(prob, outs[i], ref)
        assert max(errs) <= n * F32_STEP_TOL, (i, errs)
