"""GPU parity of the reduced velocity distributions (xi_z integrated out: G =
int f dxi_z and H = int xi_z^2 f dxi_z on a (xi_x, xi_y) grid, the paper's 2D
memory saver) against the reduced oracle, element by element every
iteration, and the argument checks of the reduced grid."""
import numpy as np
import pytest

from workloads import cylinder_case, sphere_case
from helpers import RTOL_W, rel_err, w_rel_err, run_oracle, run_gpu, vdf_by_cell, moment_scales, compare_derived

pytestmark = pytest.mark.gpu


def _compare(case, n_iter, flags=None, vdf_dtype="f64", w_tol=RTOL_W, f_tol=1e-10, hot_tol=1e-9, q_tol=1e-9):
    o, ho = run_oracle(case, n_iter, flags=flags)
    s, hg, reps = run_gpu(case, n_iter, vdf_dtype=vdf_dtype, flags=flags)
    assert np.array_equal(s.dvm_flags(), o.dvm)
    assert reps[-1]["n_v"] == o.vg.nv == 2 * case.vgrid.n[0] * case.vgrid.n[1]
    for it, (a, b) in enumerate(zip(hg, ho)):
        e = w_rel_err(a, b)
        assert e < w_tol, "iteration %d: W relative error %.3e" % (it, e)
        assert np.all(a[:, 3] == 0.0)   # u_z stays exactly zero
    ho_ = np.concatenate([o.hot_sigma[:, [0, 1, 2, 0, 0, 1], [0, 1, 2, 1, 2, 2]], o.hot_q], axis=1)
    assert rel_err(s.hot(), ho_, max(np.max(np.abs(ho_)), 1e-12)) < hot_tol
    nd = int(o.dvm.sum())
    fg = vdf_by_cell(s, nd, o.N, o.vg.nv)
    assert rel_err(fg[o.dvm], o.f[o.dvm]) < f_tol
    qo = o.wall_heat_flux()
    qg = s.moments(["wall_q"])["wall_q"]
    assert rel_err(qg, qo) < q_tol, "wall heat flux relative error %.3e" % rel_err(qg, qo)
    compare_derived(s, o, max(hot_tol, q_tol))   # wall pressure and shear, constitutive stress and heat flux
    return o, s


def test_reduced_cylinder_all_kinetic():
    """Reduced distributions on a 14 x 12 (xi_x, xi_y) grid (336 stored values
    per cell: G then H), O-grid with wall, wrap and far field, NS presolve."""
    case = cylinder_case(Ma=2.0, Kn=0.1, n_r=6, n_theta=8, nv=(14, 12, 0), adaptive=False, macro_steps=10,
                         cfl=5.0, k_sub=2, vbox=((-10, 10), (-9, 9), (0, 1)), relax=1.0, reduced=True)
    case.dt = 0.5
    o, s = _compare(case, 3)
    s.close()


def test_reduced_cylinder_adaptive_forced_region():
    """Adaptive start (reduced Grad-13 seeds of the entering cells, reduced
    Grad-13 interface distributions of the NS neighbours)."""
    case = cylinder_case(Ma=2.0, Kn=0.02, n_r=8, n_theta=10, nv=(16, 14, 0), adaptive=True, Kn_ref=0.02,
                         macro_steps=20, cfl=5.0, k_sub=2, presolve_max_blocks=3, vbox=((-10, 10), (-9, 9), (0, 1)),
                         reduced=True)
    case.tol = 0.0
    case.adapt_every = 1000
    o = run_oracle(case, 0)[0]
    flags = o.dvm.copy()
    assert 0 < flags.sum() < flags.size
    o, s = _compare(case, 3, flags=flags)
    s.close()


def test_reduced_cylinder_full_velocity_grid():
    """The benchmark's reduced velocity grid, 48 x 48 nodes on the paper's
    [-14, 14] x [-12, 12] box (4,608 stored values per cell), on a 32 x 32
    O-grid at Ma = 5, Kn = 0.01 (adaptive)."""
    case = cylinder_case(n_r=32, n_theta=32, nv=(48, 48, 0), presolve_max_blocks=3, macro_steps=20, relax=1.0,
                         reduced=True)
    case.tol = 0.0
    case.adapt_every = 1000
    o = run_oracle(case, 0)[0]
    o, s = _compare(case, 2, flags=o.dvm.copy())
    s.close()


@pytest.mark.parametrize("dtype,tol", [("f32", 2e-5)])
def test_reduced_fp32_storage(dtype, tol):
    """FP32 storage and arithmetic of the kinetic step on the reduced grid,
    FP64 moments and synthetic solve: within the FP32 rounding of the FP64
    oracle."""
    case = cylinder_case(Ma=2.0, Kn=0.1, n_r=6, n_theta=8, nv=(14, 12, 0), adaptive=False, macro_steps=10,
                         cfl=5.0, k_sub=2, vbox=((-10, 10), (-9, 9), (0, 1)), relax=1.0, reduced=True)
    case.dt = 0.5
    o, ho = run_oracle(case, 3)
    s, hg, reps = run_gpu(case, 3, vdf_dtype=dtype)
    for a, b in zip(hg, ho):
        assert w_rel_err(a, b) < tol
    s.close()


def test_reduced_carried_moments_equal_a_direct_reduction():
    """The moments an iteration carries forward (taken without a pass over
    the velocities after Eq. updatef) equal a direct reduction of the reduced
    VDF, including the xi_z^2 parts from the H plane."""
    case = cylinder_case(Ma=2.0, Kn=0.1, n_r=6, n_theta=8, nv=(14, 12, 0), adaptive=False, macro_steps=10,
                         cfl=5.0, k_sub=2, vbox=((-10, 10), (-9, 9), (0, 1)), relax=1.0, reduced=True)
    case.dt = 0.5
    s, hg, reps = run_gpu(case, 2)
    nd = reps[-1]["n_dvm"]
    carried = s.vdf_moments(nd, direct=False)
    direct = s.vdf_moments(nd, direct=True)
    err = (np.abs(carried - direct) / moment_scales(direct)).max(axis=0)
    assert err.max() < 1e-11, "per-component error %s" % np.array2string(err, precision=2)
    assert np.abs(direct[:, 13:]).max() > 0            # the case has diffuse-wall cells
    assert np.max(np.abs(direct[:, 6])) > 0.1          # the zz moment comes from H
    assert np.all(direct[:, [3, 8, 9, 12]] == 0.0)     # c_z, c_x c_z, c_y c_z, c_z c^2 vanish
    s.close()


def test_reduced_grid_rejects_3d_flows():
    """A reduced grid on a 3D mesh (faces with z components), or with u_z != 0
    in the state: GSIS_ERR_ARG at the first gsis_iterate."""
    from paper_2501_02245_gb300 import Solver, gsis
    from workloads.cases import VGrid
    case = sphere_case(Ma=2.0, Kn=0.1, n_r=3, n_pol=4, n_az=4, nv=(10, 8, 8), adaptive=False, macro_steps=5,
                       presolve_max_blocks=0)
    case.vgrid = VGrid((10, 8, 2), (-10.0, -9.0, 0.0), (10.0, 9.0, 1.0), reduced=True)
    s = Solver.from_case(case)
    with pytest.raises(gsis.GsisError) as ei:
        s.iterate(0)
    assert ei.value.status == gsis.GSIS_ERR_ARG
    s.close()
    case = cylinder_case(Ma=2.0, Kn=0.1, n_r=4, n_theta=6, nv=(10, 8, 0), adaptive=False, vbox=((-10, 10), (-9, 9), (0, 1)),
                         presolve_max_blocks=0, reduced=True)
    case.W0[5, 3] = 0.1
    s = Solver.from_case(case)
    with pytest.raises(gsis.GsisError) as ei:
        s.iterate(0)
    assert ei.value.status == gsis.GSIS_ERR_ARG
    s.close()
