"""The C-ABI library: it loads, exports every entry point include/ark.h
declares, and rejects invalid parameters before touching a device (so these
run without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ark.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ark_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def ark():
    from paper_1903_09043_gb300 import build
    build.build()
    from paper_1903_09043_gb300 import ark as mod
    return mod


def test_library_exports_every_declared_symbol(ark):
    lib = ctypes.CDLL(ark.LIB_PATH)
    names = _declared()
    assert len(names) >= 12
    for name in names:
        assert hasattr(lib, name), name
        assert hasattr(ark, name), f"binding lacks {name}"


def test_status_strings(ark):
    for code in range(7):
        assert ark.ark_status_string(code)
    assert ark.ark_status_string(0) == b"ok"


def _params(ark, **kw):
    from paper_1903_09043_gb300 import inputs as I
    prob, _ = I.rayleigh_benard(2, (16, 8), amp=0.0)
    prob = prob.replace(**{k: v for k, v in kw.items() if k in prob.__dataclass_fields__})
    return ark.params_from_problem(prob, kw.get("precision", ark.ARK_F64))


@pytest.mark.parametrize("mutate,status", [
    (lambda p: setattr(p.grid, "dim", 4), 1),
    (lambda p: setattr(p.eos, "gamma", 1.0), 1),
    (lambda p: setattr(p.eos, "p_inf", -1.0), 1),
    (lambda p: setattr(p.eos, "p_inf", float("inf")), 1),
    (lambda p: setattr(p.eos, "p_inf", float("nan")), 1),
    (lambda p: setattr(p, "K", 0.5), 1),
    (lambda p: setattr(p, "cfl", 0.0), 1),
    (lambda p: setattr(p, "mu", -1.0), 1),
    (lambda p: setattr(p, "low_mach", 3), 1),
    (lambda p: setattr(p, "precision", 7), 1),
    (lambda p: p.bc.lo.__setitem__(0, 9), 1),
    (lambda p: p.bc.lo.__setitem__(0, 1), 1),                       # periodic pair broken
    (lambda p: (p.bc.lo.__setitem__(1, 0), p.bc.hi.__setitem__(1, 0)), 1),   # gravity along periodic axis
    (lambda p: p.grid.n.__setitem__(1, 1), 1),                       # wall axis with one cell
    (lambda p: p.grid.n.__setitem__(0, 0), 1),                       # empty grid
    (lambda p: (setattr(p, "precision", 1), p.grid.n.__setitem__(0, 65536),
                p.grid.n.__setitem__(1, 65536)), 5),                 # 2^32 cells: beyond 32-bit FP32 offsets
    (lambda p: p.bc.T_lo.__setitem__(1, 0.0), 1),                    # non-positive wall temperature
    (lambda p: (setattr(p, "precision", 2), p.bc.lo.__setitem__(0, 2), p.bc.hi.__setitem__(0, 2),
                p.bc.T_lo.__setitem__(0, 1.0), p.bc.T_hi.__setitem__(0, 1.0)), 5),
])
def test_invalid_parameters_rejected_before_device_work(ark, mutate, status):
    p = _params(ark)
    mutate(p)
    h = ark._H()
    st = ark.ark_create(ctypes.byref(p), None, ctypes.byref(h))
    assert st == status
    assert not h.value


def test_null_arguments(ark):
    assert ark.ark_create(None, None, None) == ark.ARK_ERR_INVALID_ARG
    assert ark.ark_destroy(None) == ark.ARK_ERR_INVALID_ARG
    assert ark.ark_step(None, 1, -1.0) == ark.ARK_ERR_INVALID_ARG
    assert ark.ark_last_error(None) == b"null handle"


def test_split_form_needs_a_row_potential(ark):
    """A potential array that varies across the planes (tilted gravity) has
    no one-row-per-level base state: ARK_F32_SPLIT refuses it before any
    device work; the same array is accepted by the validation of the other
    forms, and a potential that varies along the gravity axis only passes."""
    from paper_1903_09043_gb300 import inputs as I
    prob, _ = I.tilted_atmosphere((16, 12))
    p = ark.params_from_problem(prob, ark.ARK_F32_SPLIT)
    h = ark._H()
    assert ark.ark_create(ctypes.byref(p), None, ctypes.byref(h)) == ark.ARK_ERR_UNSUPPORTED
    assert not h.value
    rp, _ = I.row_potential_state(2, (16, 12))
    q = ark.params_from_problem(rp, ark.ARK_F32_SPLIT)
    q.K = 0.5      # then rejected for K, after the potential passed
    assert ark.ark_create(ctypes.byref(q), None, ctypes.byref(h)) == ark.ARK_ERR_INVALID_ARG


@pytest.mark.parametrize("field", ["lo", "hi", "g", "mu", "kappa", "cfl", "K", "gamma"])
def test_non_finite_parameters_rejected(ark, field):
    p = _params(ark)
    inf = float("inf")
    if field in ("lo", "hi"):
        getattr(p.grid, field)[0] = -inf if field == "lo" else inf
    elif field == "g":
        p.gravity.g = float("nan")
    elif field == "gamma":
        p.eos.gamma = inf
    else:
        setattr(p, field, inf if field != "K" else float("nan"))
    h = ark._H()
    assert ark.ark_create(ctypes.byref(p), None, ctypes.byref(h)) == ark.ARK_ERR_INVALID_ARG


def test_equation_of_state_law_validated(ark):
    """The law selector and the covolume are checked before any device work;
    the combinations this build does not implement are refused as such."""
    from paper_1903_09043_gb300 import inputs as I
    h = ark._H()
    for law, b, status in ((2, 0.0, ark.ARK_ERR_INVALID_ARG),                       # unknown law
                           (ark.ARK_EOS_STIFFENED_GAS, 0.2, ark.ARK_ERR_INVALID_ARG),   # covolume without its law
                           (ark.ARK_EOS_NOBLE_ABEL, -0.1, ark.ARK_ERR_INVALID_ARG),
                           (ark.ARK_EOS_NOBLE_ABEL, float("inf"), ark.ARK_ERR_INVALID_ARG)):
        p = _params(ark)
        p.eos.law, p.eos.b = law, b
        assert ark.ark_create(ctypes.byref(p), None, ctypes.byref(h)) == status, (law, b)
    pp, _ = I.periodic_potential_state(2, (8, 8))
    p = ark.params_from_problem(pp.replace(b=0.1), ark.ARK_F64)
    assert p.eos.law == ark.ARK_EOS_NOBLE_ABEL
    assert ark.ark_create(ctypes.byref(p), None, ctypes.byref(h)) == ark.ARK_ERR_UNSUPPORTED
    sp, _ = I.stratified_random(2, (8, 8), b=0.1)
    p = ark.params_from_problem(sp, ark.ARK_F64)
    fake = ctypes.c_void_p(16)
    assert ark.ark_compute_dt_noalloc(ctypes.byref(p), fake, fake, None) == ark.ARK_ERR_UNSUPPORTED


def test_halo_boundary_rules(ark):
    """ARK_BC_HALO (slab boundaries of a decomposition along x) is checked
    before any device work: x sides only, n[0] >= 2, uniform gravity only,
    and not in ensembles."""
    from paper_1903_09043_gb300 import inputs as I
    h = ark._H()
    p = _params(ark)
    p.bc.lo[0] = p.bc.hi[0] = ark.ARK_BC_HALO
    p.grid.n[0] = 1
    assert ark.ark_create(ctypes.byref(p), None, ctypes.byref(h)) == ark.ARK_ERR_INVALID_ARG
    p = _params(ark)
    p.bc.lo[1] = ark.ARK_BC_HALO                       # not along the gravity axis
    assert ark.ark_create(ctypes.byref(p), None, ctypes.byref(h)) == ark.ARK_ERR_INVALID_ARG
    p = _params(ark)
    p.bc.lo[0] = ark.ARK_BC_HALO                       # a halo side facing a periodic one
    assert ark.ark_create(ctypes.byref(p), None, ctypes.byref(h)) == ark.ARK_ERR_INVALID_ARG
    p = _params(ark)
    p.bc.lo[0] = 5                                     # beyond the known rules
    assert ark.ark_create(ctypes.byref(p), None, ctypes.byref(h)) == ark.ARK_ERR_INVALID_ARG
    tp, _ = I.tilted_atmosphere((16, 12))
    q = ark.params_from_problem(tp, ark.ARK_F64)
    q.bc.lo[0] = q.bc.hi[0] = ark.ARK_BC_HALO
    assert ark.ark_create(ctypes.byref(q), None, ctypes.byref(h)) == ark.ARK_ERR_UNSUPPORTED
    assert not h.value
    runs = (ark.ark_params * 2)(_params(ark), _params(ark))
    runs[1].bc.lo[0] = runs[1].bc.hi[0] = ark.ARK_BC_HALO
    b = ctypes.c_void_p()
    assert ark.ark_batch_create(2, runs, None, ctypes.byref(b)) == ark.ARK_ERR_UNSUPPORTED
    assert ark.ark_get_halo(None, 0, None, 0) == ark.ARK_ERR_INVALID_ARG
    assert ark.ark_set_halo(None, 0, None, 0) == ark.ARK_ERR_INVALID_ARG
