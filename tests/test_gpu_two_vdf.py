"""GPU parity of the two-VDF reference pair (gsis_two_vdf_reference) and of
the two-VDF moments (gsis_two_vdf_moments) with the pinned oracle
(oracle.rykov.RykovGrid.reference, .moments), element by element on a full
3D velocity grid.  The reference pair: the paper's nitrogen gas, a made-up A matrix (so that
no mixing coefficient can be swapped unnoticed), and the monatomic case,
where the pair must reduce to the oracle's conservation-corrected Shakhov
form and g1 = 0.  The refusals of the entry point are host-side checks made
before any launch."""
import ctypes

import numpy as np
import pytest

from workloads import shock_1d_case, cylinder_case
from oracle import model as M
from oracle.rykov import RykovGrid, NITROGEN, MONATOMIC_A

pytestmark = pytest.mark.gpu

# rho, u (3), T_t, T_r, q_t (3), q_r (3): out of equilibrium, with heat fluxes
STATES = np.array([
    [1.0, 0.0, 0.0, 0.0, 1.0, 1.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0],
    [1.3, 0.4, -0.25, 0.1, 1.6, 1.2, 0.07, -0.04, 0.02, -0.03, 0.05, 0.01],
    [0.7, -0.8, 0.3, -0.2, 0.9, 1.4, -0.05, 0.03, -0.01, 0.04, -0.02, 0.03],
    [2.2, 1.1, 0.0, 0.0, 2.1, 1.7, 0.2, 0.0, 0.0, 0.1, 0.0, 0.0],
    [0.45, 0.2, 0.6, -0.3, 1.25, 0.8, 0.01, 0.02, -0.03, -0.02, 0.01, 0.0],
])
GASES = {
    "nitrogen": (NITROGEN["d_r"], NITROGEN["Z_r"], NITROGEN["A"]),
    "made_up": (3, 4.2, (0.7, 0.15, -0.12, 0.9)),
    "monatomic": (0, 2.667, MONATOMIC_A),
}


def _solver():
    from paper_2501_02245_gb300 import Solver
    case = shock_1d_case(n_cells=8, half_width=4.0, nv=(16, 12, 10), vmax=8.0, macro_steps=5)
    return case, Solver.from_case(case)


@pytest.mark.parametrize("gas", list(GASES))
def test_two_vdf_reference_pair_matches_the_oracle(gas):
    d_r, Zr, A = GASES[gas]
    case, s = _solver()
    S = STATES.copy()
    if gas == "monatomic":
        S[:, 9:12] = 0.0          # no internal heat flux without internal modes
    g = s.two_vdf_reference(S, d_r, Zr, A)
    vg = RykovGrid(M.VelocityGrid(case.vgrid.n, case.vgrid.lo, case.vgrid.hi), d_r)
    assert g.shape == (len(S), 2, vg.n0)
    for k, st in enumerate(S):
        ref = vg.reference(st[0], st[1:4], st[4], st[5], st[6:9], st[9:12], Zr, A)
        r0, r1 = vg.split(ref)
        scale = np.max(np.abs(ref))
        assert np.max(np.abs(g[k, 0] - r0)) < 1e-11 * scale, (gas, k)
        assert np.max(np.abs(g[k, 1] - r1)) < 1e-11 * scale, (gas, k)
        if gas == "monatomic":
            sh = vg.base.corrected_shakhov(st[0], st[1:4], st[4], st[6:9])
            assert np.max(np.abs(g[k, 0] - sh)) < 1e-11 * scale
            assert np.max(np.abs(g[k, 1])) == 0.0
        else:
            assert np.max(np.abs(r1)) > 0.1 * np.max(np.abs(r0))   # the f1 half is not trivial
    s.close()


def test_two_vdf_reference_refusals():
    """Bad arguments, states and grids are refused before any launch and the
    context stays usable; n = 0 does nothing."""
    import torch
    from paper_2501_02245_gb300 import gsis, Solver
    case, s = _solver()
    lib = s.lib
    A = (ctypes.c_double * 4)(*NITROGEN["A"])
    out = torch.zeros((2, 2, s.nv), dtype=torch.float64, device="cuda")
    good = torch.from_numpy(STATES[:2].copy()).to("cuda")
    bad = STATES[:2].copy()
    bad[1, 4] = -1.0
    badd = torch.from_numpy(bad).to("cuda")
    torch.cuda.synchronize()
    vp = ctypes.c_void_p
    call = lambda S, n, d_r, Zr: lib.gsis_two_vdf_reference(s.ctx, vp(S.data_ptr()), n, d_r, Zr, A,
                                                            vp(out.data_ptr()))
    assert call(badd, 2, 2, 2.667) == gsis.GSIS_ERR_ARG
    assert call(good, 2, -1, 2.667) == gsis.GSIS_ERR_ARG
    assert call(good, 2, 2, 0.5) == gsis.GSIS_ERR_ARG
    assert call(good, 70000, 2, 2.667) == gsis.GSIS_ERR_ARG
    assert call(good, 0, 2, 2.667) == gsis.GSIS_OK
    assert torch.count_nonzero(out).item() == 0
    assert call(good, 2, 2, 2.667) == gsis.GSIS_OK
    assert torch.count_nonzero(out).item() > 0
    s.close()
    red = cylinder_case(Ma=2.0, Kn=0.1, n_r=4, n_theta=6, nv=(10, 10, 2), vbox=((-8, 8), (-7, 7), (0, 1)),
                        adaptive=False, macro_steps=5, presolve_max_blocks=0, reduced=True)
    r = Solver.from_case(red)
    assert lib.gsis_two_vdf_reference(r.ctx, vp(good.data_ptr()), 2, 2, 2.667, A,
                                      vp(out.data_ptr())) == gsis.GSIS_ERR_UNSUPPORTED
    r.close()


@pytest.mark.parametrize("d_r", [2, 0])
def test_two_vdf_moments_match_the_oracle(d_r):
    """gsis_two_vdf_moments against the oracle's Eq. getmoment
    (RykovGrid.moments) on pairs far from equilibrium: the Grad-13 pair of a
    stressed, heat-conducting state plus a second population, so that every
    moment (stress, both heat fluxes, T_t != T_r) is nonzero."""
    case, s = _solver()
    vg = RykovGrid(M.VelocityGrid(case.vgrid.n, case.vgrid.lo, case.vgrid.hi), d_r)
    sig = np.array([[0.05, -0.02, 0.01], [-0.02, -0.03, 0.0], [0.01, 0.0, -0.02]])
    F = []
    for st in STATES[1:]:
        f = (vg.grad13(st[0], st[1:4], st[4], st[5], sig, st[6:9], st[9:12])
             + vg.equilibrium(0.3, np.array([-0.5, 0.2, 0.1]), 1.9, 0.7))
        F.append(np.stack(vg.split(f)))
    F = np.array(F)
    m = s.two_vdf_moments(F, d_r)
    assert m.shape == (len(F), 18)
    for k in range(len(F)):
        rho, u, Tt, Tr, sg, qt, qr = vg.moments(vg.join(F[k, 0], F[k, 1]))
        ref = np.concatenate([[rho], u, [Tt, Tr], [sg[0, 0], sg[1, 1], sg[2, 2], sg[0, 1], sg[0, 2], sg[1, 2]],
                              qt, qr])
        assert np.max(np.abs(m[k] - ref)) < 1e-11 * max(1.0, np.max(np.abs(ref))), k
        assert min(np.linalg.norm(ref[6:12]), np.linalg.norm(ref[12:15]), np.linalg.norm(ref[15:18])) > 1e-3
        assert d_r == 0 or abs(Tt - Tr) > 1e-2
    s.close()
