"""C ABI checks that need no GPU: the library builds, loads, exports every
entry point declared in include/gsis.h, and rejects bad arguments before
touching the device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    with open(os.path.join(ROOT, "include", "gsis.h")) as fh:
        text = fh.read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[\w\s\*]*?\b(gsis_\w+)\s*\(", text, re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2501_02245_gb300 import build
    build.build()
    from paper_2501_02245_gb300 import gsis
    return gsis.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("gsis_init", "gsis_set_mesh", "gsis_set_velocity_grid", "gsis_iterate", "gsis_moments",
              "gsis_free", "gsis_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for n in declared_functions():
        assert hasattr(lib, n), n


def test_binding_names_match_header():
    from paper_2501_02245_gb300 import gsis
    assert set(gsis.EXPORTED) == set(declared_functions())


def test_init_rejects_bad_parameters(lib):
    from paper_2501_02245_gb300.gsis import Params, GSIS_ERR_ARG
    ctx = ctypes.c_void_p()
    good = dict(Kn=0.1, omega=0.81, adaptive=0, Kn_ref=0.0, adapt_every=5, wall_layers=2, vdf_dtype=0,
                macro_steps=10, cfl=5.0, k_sub=2, dt=0.0, tol=1e-6, presolve_max_blocks=0, spin_limit=0)
    for key, bad in (("Kn", -1.0), ("Kn", 0.0), ("cfl", 0.0), ("macro_steps", -3), ("vdf_dtype", 7), ("dt", -1.0),
                     ("k_sub", -1)):
        p = dict(good); p[key] = bad
        st = lib.gsis_init(ctypes.byref(Params(**p)), None, None, ctypes.byref(ctx))
        assert st == GSIS_ERR_ARG, (key, bad, st)
    assert lib.gsis_init(None, None, None, ctypes.byref(ctx)) == GSIS_ERR_ARG


def test_init_refuses_internal_degrees_of_freedom(lib):
    """d_r < 0 is invalid; d_r > 0 (the two-VDF model) is valid but not built."""
    from paper_2501_02245_gb300.gsis import Params, GSIS_ERR_ARG, GSIS_ERR_UNSUPPORTED
    ctx = ctypes.c_void_p()
    base = dict(Kn=0.1, omega=0.74, adaptive=0, Kn_ref=0.0, adapt_every=5, wall_layers=2, vdf_dtype=0,
                macro_steps=10, cfl=5.0, k_sub=2, dt=0.0, tol=1e-6, presolve_max_blocks=0, spin_limit=0)
    for d_r, want in ((-1, GSIS_ERR_ARG), (2, GSIS_ERR_UNSUPPORTED)):
        p = Params(**base, d_r=d_r, Z_r=2.667, A=(ctypes.c_double * 4)(0.786, -0.201, -0.059, 0.842))
        assert lib.gsis_init(ctypes.byref(p), None, None, ctypes.byref(ctx)) == want


def test_init_refuses_knudsen_numbers_outside_the_quotient_range(lib):
    """The kinetic update's quotient needs 1/tau = rho T^(1-omega)/mu(T0) inside
    the FP32 exponent range: Kn outside [1e-15, 1e15] is refused before any
    device call; the ends of the range are accepted by the parameter checks."""
    from paper_2501_02245_gb300.gsis import Params, GSIS_ERR_UNSUPPORTED
    ctx = ctypes.c_void_p()
    base = dict(omega=0.74, adaptive=0, Kn_ref=0.0, adapt_every=5, wall_layers=2, vdf_dtype=0,
                macro_steps=10, cfl=5.0, k_sub=2, dt=0.0, tol=1e-6, presolve_max_blocks=0, spin_limit=0)
    for Kn in (1e-16, 2e15, 1e300):
        p = Params(**base, Kn=Kn)
        assert lib.gsis_init(ctypes.byref(p), None, None, ctypes.byref(ctx)) == GSIS_ERR_UNSUPPORTED
    for Kn in (1e-15, 1e15):
        p = Params(**base, Kn=Kn)
        assert lib.gsis_init(ctypes.byref(p), None, None, ctypes.byref(ctx)) != GSIS_ERR_UNSUPPORTED


def test_null_safety(lib):
    lib.gsis_free(None)
    assert lib.gsis_last_error(None) == b"NULL context"
    assert lib.gsis_iterate(None, 1, None) == 1
    A = (ctypes.c_double * 4)(0.786, -0.201, -0.059, 0.842)
    assert lib.gsis_two_vdf_reference(None, None, 1, 2, 2.667, A, None) == 1
    assert lib.gsis_two_vdf_moments(None, None, 1, 2, None) == 1
