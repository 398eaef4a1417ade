"""Host-side checks of the C ABI that need no GPU: the library loads and exports every entry point
that include/cola.h declares, the library's own FP64 time coefficients (§2.2 eqs. cola-kick,
cola-drift; §2.1 growth factors) agree with the oracle's independent ones, and invalid sizes are
rejected on the host before anything touches a device."""

import ctypes
import math
import os
import re

import pytest

from oracle import cosmology as C

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1507_05329_gb300 import build, binding
    build.build()
    return binding.load_library()


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(cola_\w+)\s*\(", text))
    return sorted(names)


def test_library_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 12
    for name in names:
        assert hasattr(lib, name), name
    from paper_1507_05329_gb300 import binding
    assert set(names) == set(binding.SIGNATURES), "binding and header disagree"


def test_schedule_bits_match_the_header():
    """The binding's schedule constants are the header's COLA_SCHED_* macros, bit for bit."""
    from paper_1507_05329_gb300 import binding
    text = open(os.path.join(ROOT, "include", "cola.h")).read()
    macros = dict(re.findall(r"#define COLA_SCHED_(\w+) (\d+)", text))
    assert len(macros) >= 10
    for name, value in macros.items():
        assert getattr(binding, "SCHED_" + name) == int(value), name
    bits = [int(v) for k, v in macros.items() if k != "BUDGET_SHIFT"]
    bits.append(3 << int(macros["BUDGET_SHIFT"]))
    for i, a in enumerate(bits):   # no two knobs share a bit
        for b in bits[i + 1:]:
            assert a & b == 0, (a, b)


def test_strerror(lib):
    assert lib.cola_strerror(0) == b"ok"
    assert b"overflow" in lib.cola_strerror(4)


PARAMS = [
    dict(),
    dict(ic_mode=1),
    dict(drift_ansatz=1),
    dict(omega_m=0.31, nlpt=-1.0, nstep=20),
]


@pytest.mark.parametrize("kw", PARAMS)
def test_step_scalars_match_oracle(lib, kw):
    from paper_1507_05329_gb300 import Params, step_scalars
    p = Params(**kw)
    op = C.Params(**{("np_side" if k == "np_side" else k): v for k, v in kw.items()})
    keys = ["a", "a_lo", "a_hi", "force_scale", "c1", "c2", "kick", "drift", "dd1", "dd2"]
    for i in range(1, p.nstep + 1):
        got = step_scalars(p, i)
        ref = C.step_scalars(op, i)
        for k, key in enumerate(keys):
            assert got[k] == pytest.approx(ref[key], rel=1e-11, abs=1e-14), (i, key)
        assert got[10] == pytest.approx(C.d1(ref["a"], op.omega_m), rel=1e-11)
        assert got[11] == pytest.approx(C.d2(ref["a"], op.omega_m), rel=1e-11)
    ic = step_scalars(p, 0)
    a1 = 1.0 / p.nstep
    assert ic[10] == pytest.approx(C.d1(a1, op.omega_m), rel=1e-11)
    f1, f2 = C.lpt_velocity_factors(1.0, op.omega_m)
    assert ic[8] == pytest.approx(f1, rel=1e-10) and ic[9] == pytest.approx(f2, rel=1e-10)


@pytest.mark.parametrize("bad", [
    dict(nmesh=7), dict(np_side=3), dict(nmesh=14), dict(np_side=48, nmesh=50), dict(nstep=0),
    dict(omega_m=-0.1), dict(box=0.0), dict(nlpt=0.0), dict(ic_mode=2), dict(nmesh=8192),
])
def test_create_rejects_invalid_parameters_on_host(lib, bad):
    from paper_1507_05329_gb300 import Params, binding
    p = Params(**bad)
    out = ctypes.c_void_p()
    cp = p.to_c()
    assert lib.cola_create(ctypes.byref(cp), None, ctypes.byref(out)) == 1
    assert not out.value
    scal = (ctypes.c_double * 12)()
    assert lib.cola_step_scalars(ctypes.byref(cp), 1, scal, 12) == 1
    assert binding.STATUS[1].startswith("invalid")


def test_step_scalars_rejects_bad_index(lib):
    from paper_1507_05329_gb300 import Params
    cp = Params().to_c()
    out = (ctypes.c_double * 12)()
    assert lib.cola_step_scalars(ctypes.byref(cp), 11, out, 12) == 1
    assert lib.cola_step_scalars(ctypes.byref(cp), 1, out, 11) == 1


@pytest.mark.parametrize("kw", [dict(), dict(omega_m=0.3, h=0.67, n_s=1.0, sigma8=0.9)])
def test_library_linear_power_matches_golden_bbks_and_oracle_amplitude(lib, kw):
    """The library's own P(k) (host_cosmo.cpp, written independently of the oracle): its transfer
    function equals the published BBKS coefficients (tests/golden/bbks_transfer.txt) and its
    amplitude the oracle's sigma8 normalisation, whose integral is pinned by closed forms."""
    from paper_1507_05329_gb300 import Params, binding
    from tests.test_oracle_cosmology import bbks_from_golden
    import numpy as np
    p = Params(**kw)
    op = C.Params(**kw)
    k = np.logspace(-4, 1.5, 47)
    pw, tr = binding.linear_power(p, k)
    q = k / (op.omega_m * op.h)
    np.testing.assert_allclose(tr, bbks_from_golden(q), rtol=1e-13)
    np.testing.assert_allclose(pw, C.linear_power(k, op), rtol=1e-9)
    # sigma(8 Mpc/h) of the library's amplitude times the pinned shape, by the oracle's quadrature
    amp = pw[20] / (k[20] ** op.n_s * tr[20] ** 2)
    assert math.sqrt(C.sigma2_quad(amp, op)) == pytest.approx(op.sigma8, rel=1e-8)


def test_linear_power_rejects_bad_input(lib):
    from paper_1507_05329_gb300 import Params
    import numpy as np
    cp = Params().to_c()
    k = (ctypes.c_double * 2)(0.1, -1.0)
    out = (ctypes.c_double * 2)()
    assert lib.cola_linear_power(ctypes.byref(cp), k, 2, out, None) == 1
    assert lib.cola_linear_power(ctypes.byref(cp), k, 1, out, None) == 0
    bad = Params(np_side=7).to_c()
    assert lib.cola_linear_power(ctypes.byref(bad), k, 1, out, None) == 1
