"""Reduced-precision VDF storage (FP32 / BF16 / FP16 with FP32 sweep arithmetic;
FP64 moments across rows, conservation correction and synthetic solve) against
the FP64 oracle on the same inputs.

Bounds (relative to the field's maximum, every iteration), two units of the
storage format's rounding of one stored value:
  FP32 storage: 2e-5 on rho, u, T (unit roundoff 2^-24 ~ 6e-8 per value; the
                bound leaves room for growth through the iteration);
  FP16 storage: 1e-3 on rho and T (2 x 2^-11 = 9.8e-4);
  BF16 storage: 4e-3 on rho and T (2 x 2^-9 = 3.9e-3).  These small test
                grids (about 1,000 velocities) average few rounding errors per
                moment; the full workloads are measured in bench.py.
The heat flux into the wall (cylinder) is the small difference of the
incident and re-emitted energy fluxes, so its error relative to its largest
magnitude is several times that of the moments: bounded by 16 storage
rounding units (FP32 16 x 2^-24 = 9.5e-7, BF16 16 x 2^-9 = 3.1e-2, FP16
16 x 2^-12 = 3.9e-3; measured 2.9e-7, 6.8e-3 and 7.7e-4).
"""
import numpy as np
import pytest

from workloads import shock_1d_case, cylinder_case
from helpers import run_oracle, run_gpu, rel_err

pytestmark = pytest.mark.gpu

BOUNDS = {"f32": 2e-5, "bf16": 3.9e-3, "f16": 9.8e-4}
WALL_Q_BOUNDS = {"f32": 9.5e-7, "bf16": 3.1e-2, "f16": 3.9e-3}


def _check(case, n_iter, dtype):
    o, ho = run_oracle(case, n_iter)
    s, hg, _ = run_gpu(case, n_iter, vdf_dtype=dtype)
    qo = o.wall_heat_flux()
    if np.any(qo != 0.0):
        eq = rel_err(s.moments(["wall_q"])["wall_q"], qo)
        print("%s wall heat flux relative error %.3e" % (dtype, eq))
        assert eq < WALL_Q_BOUNDS[dtype], "%s: wall heat flux relative error %.3e" % (dtype, eq)
    worst = 0.0
    for a, b in zip(hg, ho):
        e = max(rel_err(a[:, 0], b[:, 0]), rel_err(a[:, 4], b[:, 4]))
        if dtype == "f32":
            e = max(e, rel_err(a[:, 1:4], b[:, 1:4]))
        worst = max(worst, e)
    s.close()
    assert worst < BOUNDS[dtype], "%s: worst relative error %.3e" % (dtype, worst)
    return worst


@pytest.mark.parametrize("dtype", ["f32", "bf16", "f16"])
def test_shock_reduced_precision(dtype):
    case = shock_1d_case(n_cells=30, half_width=7.5, nv=(20, 10, 9), vmax=8.0, macro_steps=30)
    _check(case, 5, dtype)


@pytest.mark.parametrize("dtype", ["f32", "bf16", "f16"])
def test_cylinder_reduced_precision(dtype):
    case = cylinder_case(Ma=2.0, Kn=0.1, n_r=6, n_theta=8, nv=(14, 12, 6), adaptive=False, macro_steps=10,
                         cfl=5.0, k_sub=2, vbox=((-10, 10), (-9, 9), (-8, 8)))
    case.dt = 0.5
    _check(case, 3, dtype)
