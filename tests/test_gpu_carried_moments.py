"""The velocity moments of f^{n+1} that a GSIS iteration carries to the next
one (the heat flux of the Shakhov reference distribution and the
diffuse-wall sums) are formed without a pass over the velocities: the
moments of f^{n+1/2} moved to the new macroscopic velocity plus the factored
moments of the two corrected Maxwellians of Eq. updatef, and the wall sums of
f^{n+1/2} plus those of the correction.  They must equal a direct reduction
over the corrected VDF: to rounding in FP64; in FP32 storage, to the storage
rounding of the corrected values and the FP32 row sums of the reduction."""
import numpy as np
import pytest

from workloads import cylinder_case
from helpers import moment_scales

pytestmark = pytest.mark.gpu


def _case():
    case = cylinder_case(Ma=2.0, Kn=0.1, n_r=10, n_theta=16, nv=(14, 12, 6), adaptive=False, macro_steps=10,
                         cfl=5.0, k_sub=2, vbox=((-10, 10), (-9, 9), (-8, 8)), presolve_max_blocks=2)
    case.dt = 0.5
    return case


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-11), ("f32", 1e-5)])
def test_carried_moments_match_a_direct_reduction(dtype, tol):
    from paper_2501_02245_gb300 import Solver
    s = Solver.from_case(_case(), vdf_dtype=dtype)
    rep = s.iterate(2)
    n = rep["n_dvm"]
    carried = s.vdf_moments(n, direct=False)
    direct = s.vdf_moments(n, direct=True)
    s.close()
    assert np.isfinite(carried).all() and np.isfinite(direct).all()
    assert np.abs(direct[:, 13:]).max() > 0, "the case has diffuse-wall cells"
    err = (np.abs(carried - direct) / moment_scales(direct)).max(axis=0)
    assert err.max() < tol, "per-component error %s" % np.array2string(err, precision=2)


def test_moment_hook_rejects_misuse():
    from paper_2501_02245_gb300 import Solver, GsisError
    s = Solver.from_case(_case(), vdf_dtype="f64")
    with pytest.raises(GsisError):       # no iteration yet
        s.vdf_moments(1, direct=True)
    rep = s.iterate(1)
    with pytest.raises(GsisError):       # destination too small
        s.vdf_moments(rep["n_dvm"] - 1, direct=False)
    s.close()
