"""Pins of the two-VDF oracle of a gas with internal degrees of freedom
(oracle.rykov; CPU only).

What fixes each function, other than its own formula:
* d_r = 0: the whole GSIS iteration must be the pinned Shakhov oracle's;
* the collision term conserves mass, momentum and total energy, and moves
  internal energy by (rho d_r / 2)(T - T_r)/Z_r per collision time (the
  source of Eq. macroscopic_equation_2), T the equilibrium temperature;
* the A matrix is the matrix of the heat-flux relaxation rates (Sec. 2);
* the Grad-13 distributions of Eq. G13_VDF carry the state they are built
  from;
* the synthetic equations: the energy-exchange source, the conductivities of
  the paper's nitrogen Eucken factors, and a steady viscous shock between
  the Rankine-Hugoniot states of gamma = 7/5;
* Eq. updatef leaves every kinetic cell with the conserved moments of the new
  macroscopic state, a uniform equilibrium stream is a fixed point, and a
  nitrogen shock relaxes its internal temperature behind the translational
  one;
* on a 2D flow the reduced-grid iteration is the xi_z integral of the 3D one.
"""
import os

import numpy as np
import pytest

from workloads import shock_1d_case, cylinder_case
from workloads.cases import Case, VGrid, rankine_hugoniot
from workloads.meshes import cartesian_1d, cartesian_2d, BC_FARFIELD, BC_PERIODIC, BC_NONE
from oracle import model as M
from oracle.reduced import ReducedGrid
from oracle.mesh import Topology
from oracle.macro import MacroGeometry
from oracle.gsis import OracleSolver
from oracle.rykov import (RykovGrid, RykovSolver, GasParams, NITROGEN, MONATOMIC_A, conserved6, primitive6,
                          residual6, macro_solve6, heat_flux_relaxation, equilibrium_temperature)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
N2 = (NITROGEN["d_r"], NITROGEN["Z_r"], NITROGEN["A"])


def _grid3(n=(14, 12, 12), box=8.0):
    return RykovGrid(M.VelocityGrid(n, (-box,) * 3, (box,) * 3), NITROGEN["d_r"])


def _grid_red(n=(16, 14)):
    return RykovGrid(ReducedGrid(n, (-8.0, -7.5), (8.5, 7.5)), NITROGEN["d_r"])


STATE = dict(rho=1.3, u=np.array([0.4, -0.25, 0.0]), Tt=1.6, Tr=1.2)
SIGMA = np.array([[0.05, -0.02, 0.0], [-0.02, -0.03, 0.0], [0.0, 0.0, -0.02]])
QT = np.array([0.07, -0.04, 0.0])
QR = np.array([-0.03, 0.05, 0.0])


def _nonequilibrium(vg):
    """A distribution pair far from the reference: the Grad-13 pair of a
    stressed, heat-conducting state plus a second, hotter population."""
    s = STATE
    f = vg.grad13(s["rho"], s["u"], s["Tt"], s["Tr"], SIGMA, QT, QR)
    extra = vg.equilibrium(0.4, np.array([-0.6, 0.3, 0.0]), 2.2, 0.8)
    return f + extra


# ----------------------------------------------------------------------------- d_r = 0
def test_monatomic_case_is_the_shakhov_oracle():
    """With d_r = 0 and A_tt = 2/3 (Pr = 2/3) there is no internal mode
    (f1 = 0, e_r = 0, T = T_t, q0 = q_t): the two-VDF iteration must be the
    pinned Shakhov iteration, on a shock with a 3D velocity grid and on an
    adaptive cylinder with reduced distributions whose region is re-identified
    mid-run."""
    shock = shock_1d_case(Ma=2.0, n_cells=16, half_width=8.0, nv=(12, 8, 8), macro_steps=10, k_sub=2)
    cyl = cylinder_case(Ma=2.0, Kn=0.1, n_r=6, n_theta=8, nv=(10, 10, 2), vbox=((-8, 8), (-7, 7), (0, 1)),
                        adaptive=True, Kn_ref=0.05, macro_steps=10, presolve_max_blocks=2, relax=1.0, reduced=True)
    cyl.adapt_every = 2
    for case in (shock, cyl):
        o = OracleSolver(case).run(3)
        r = RykovSolver(case, 0, NITROGEN["Z_r"], MONATOMIC_A).run(3)
        assert np.array_equal(r.dvm, o.dvm)
        assert np.max(np.abs(r.W[:, :5] - o.W)) < 1e-12 * np.max(np.abs(o.W))
        assert np.array_equal(r.W[:, 5], r.W[:, 4])
        assert np.max(np.abs(r.f[:, :o.vg.nv] - o.f)) < 1e-12 * np.max(np.abs(o.f))
        assert np.all(r.f[:, o.vg.nv:] == 0.0)
        assert np.allclose(r.eps_history, o.eps_history, rtol=1e-10, atol=0.0)


# ----------------------------------------------------------------------------- collision term
def test_equilibrium_temperature_and_conserved_variables():
    """T = (3 T_t + d_r T_r)/(3 + d_r): T_t = 2, T_r = 1, d_r = 2 give 8/5; the
    conserved variables round-trip and rho e counts both energies."""
    assert equilibrium_temperature(2.0, 1.0, 2) == 1.6
    W = np.array([1.3, 0.4, -0.25, 0.1, 1.6, 1.2])
    U = conserved6(W, 2)
    assert np.isclose(U[4], 1.3 * (1.5 * 1.6 + 0.5 * (0.16 + 0.0625 + 0.01) + 1.2), rtol=1e-15)
    assert np.isclose(U[5], 1.3 * 1.2, rtol=1e-15)
    assert np.allclose(primitive6(U, 2), W, rtol=1e-14)


@pytest.mark.parametrize("grid", ["3d", "reduced"])
def test_collision_term_conserves_and_exchanges_internal_energy(grid):
    """sum_v w psi (g - f) over both VDFs: zero for mass, momentum and total
    energy (to rounding, on the discrete grid), and (rho d_r/2)(T - T_r)/Z_r
    for the internal energy (Eq. macroscopic_equation_2's source times tau)."""
    vg = _grid3() if grid == "3d" else _grid_red()
    f = _nonequilibrium(vg)
    rho, u, Tt, Tr, sig, qt, qr = vg.moments(f)
    assert Tt != Tr and np.linalg.norm(qt) > 1e-3 and np.linalg.norm(qr) > 1e-3
    g = vg.reference(rho, u, Tt, Tr, qt, qr, NITROGEN["Z_r"], NITROGEN["A"])
    dU = vg.conserved(g) - vg.conserved(f)
    scale = np.max(np.abs(vg.conserved(f)))
    assert np.max(np.abs(dU[:5])) < 1e-13 * scale
    T = (3.0 * Tt + 2.0 * Tr) / 5.0
    assert abs(dU[5] - rho * (T - Tr) / NITROGEN["Z_r"]) < 1e-13 * scale


@pytest.mark.parametrize("grid", ["3d", "reduced"])
def test_equilibrium_pair_is_the_collision_fixed_point(grid):
    """With T_t = T_r and no heat flux the reference pair is the equilibrium
    pair itself: f0 = M~(T), f1 = (d_r/2) T M~(T)."""
    vg = _grid3() if grid == "3d" else _grid_red()
    z = np.zeros(3)
    feq = vg.equilibrium(1.3, STATE["u"], 1.4, 1.4)
    g = vg.reference(1.3, STATE["u"], 1.4, 1.4, z, z, NITROGEN["Z_r"], NITROGEN["A"])
    assert np.max(np.abs(g - feq)) < 1e-14 * np.max(feq)
    f0, f1 = vg.split(feq)
    assert np.allclose(f1, 1.4 * f0[vg.idx1], rtol=1e-15)


def test_heat_fluxes_relax_at_the_rates_of_the_A_matrix():
    """The A matrix is the matrix of heat-flux relaxation rates (Sec. 2): in
    one collision time the reference pair moves (q_t, q_r) by
    -(A_tt q_t + A_tr q_r, A_rt q_t + A_rr q_r).  On a fine grid (quadrature
    error far below the rates) for the nitrogen A and for a second, made-up
    matrix (so that no entry can be swapped with another unnoticed)."""
    vg = RykovGrid(M.VelocityGrid((48, 48, 48), (-11.0,) * 3, (11.0,) * 3), 2)
    s = STATE
    f = vg.grad13(s["rho"], s["u"], s["Tt"], s["Tr"], SIGMA, QT, QR)
    rho, u, Tt, Tr, sig, qt, qr = vg.moments(f)
    assert np.allclose(qt, QT, atol=1e-10) and np.allclose(qr, QR, atol=1e-10)
    for A in (NITROGEN["A"], (0.7, 0.15, -0.12, 0.9)):
        g = vg.reference(rho, u, Tt, Tr, qt, qr, NITROGEN["Z_r"], A)
        g0, g1 = vg.split(g)
        dqt = vg.base.heat_flux_about(g0, u) - qt
        dqr = vg.w * (vg.c1(u).T @ g1) - qr
        et, er = heat_flux_relaxation(qt, qr, A)
        assert np.max(np.abs(dqt - et)) < 1e-9 and np.max(np.abs(dqr - er)) < 1e-9
        assert np.max(np.abs(et)) > 0.02


@pytest.mark.parametrize("grid", ["3d", "reduced"])
def test_grad13_pair_carries_its_state(grid):
    """Eq. G13_VDF: the pair built from (rho, u, T_t, T_r, sigma, q_t, q_r) has
    those moments -- mass, momentum, both temperatures exactly (the
    conservation readings), stress and heat fluxes to quadrature accuracy."""
    if grid == "3d":
        vg = RykovGrid(M.VelocityGrid((36, 36, 36), (-9.0,) * 3, (9.0,) * 3), 2)
    else:
        vg = RykovGrid(ReducedGrid((40, 40), (-9.0, -9.0), (9.0, 9.0)), 2)
    s = STATE
    f = vg.grad13(s["rho"], s["u"], s["Tt"], s["Tr"], SIGMA, QT, QR)
    rho, u, Tt, Tr, sig, qt, qr = vg.moments(f)
    assert abs(rho - s["rho"]) < 1e-14 and np.allclose(u, s["u"], atol=1e-14)
    assert abs(Tt - s["Tt"]) < 1e-13 and abs(Tr - s["Tr"]) < 1e-13
    assert np.allclose(sig, SIGMA, atol=1e-10) and np.allclose(qt, QT, atol=1e-10)
    assert np.allclose(qr, QR, atol=1e-10)


# ----------------------------------------------------------------------------- synthetic equations
def _geo(mesh):
    topo = Topology(mesh)
    return topo, MacroGeometry(topo)


def _zero_hot(n):
    return (np.zeros((n, 3, 3)), np.zeros((n, 3)), np.zeros((n, 3)))


def test_exchange_source_of_a_uniform_gas():
    """A uniform nitrogen gas at rest with T_t = 1.5, T_r = 1 on a periodic
    mesh: every face flux cancels, the internal-energy residual is the source
    of Eq. macroscopic_equation_2, V d_r rho (T - T_r)/(2 Z_r tau) with
    tau = mu(T_t)/(rho T_t) and T = 1.3, and the other residuals vanish
    (total energy is exchanged, not created).  That the exchange drives both
    temperatures to the equilibrium of the total energy is pinned by the
    nitrogen shock below."""
    d_r, Zr, A = N2
    mu0, omega = 0.05, NITROGEN["omega"]
    mesh = cartesian_2d(4, 3, 0.0, 1.0, 0.0, 0.75, dim=2, bc_types=[BC_PERIODIC] * 4 + [BC_NONE] * 2,
                        bc_states=[[1.0, 0.0, 0.0, 0.0, 1.0]] * 6)
    topo, geo = _geo(mesh)
    gas = GasParams(d_r, Zr, A, mu0, omega)
    W = np.tile([1.2, 0.0, 0.0, 0.0, 1.5, 1.0], (topo.ncell, 1))
    U = conserved6(W, d_r)
    R = residual6(geo, mesh.bc_state, U, _zero_hot(topo.ncell), gas)[0]
    tau = mu0 * 1.5 ** omega / (1.2 * 1.5)
    S = 1.2 * (1.3 - 1.0) / (Zr * tau)           # d_r rho / 2 = rho for d_r = 2
    assert np.allclose(R[:, 5] / topo.vol, S, rtol=1e-13)
    assert np.max(np.abs(R[:, :5])) < 1e-13 * np.max(np.abs(R[:, 5]))


def test_heat_conduction_uses_the_papers_eucken_factors():
    """T_t = T_r = 1 + b y^2 with the gas at rest and a temperature-independent
    viscosity: the conduction terms are d/dy(kappa dT/dy) = 2 b kappa with
    kappa_t = f_t (3/2) mu and kappa_r = f_r (d_r/2) mu, f_t and f_r the
    Eucken factors that are pinned to the values the paper prints for
    nitrogen; the total energy carries both, the internal energy kappa_r
    alone.  (The viscous part is isolated as R(2 mu) - R(mu): the splitting
    does not depend on mu and the exchange source vanishes at T_t = T_r.)"""
    d_r, Zr, A = N2
    b, mu0 = 0.2, 0.04
    mesh = cartesian_2d(6, 8, 0.0, 1.0, 0.0, 1.0, dim=2, bc_types=[BC_FARFIELD] * 4 + [BC_NONE] * 2,
                        bc_states=[[1.0, 0.0, 0.0, 0.0, 1.0]] * 6)
    topo, geo = _geo(mesh)
    x = mesh.flat(mesh.centers)
    W = np.zeros((topo.ncell, 6)); W[:, 0] = 1.0
    W[:, 4] = W[:, 5] = 1.0 + b * x[:, 1] ** 2
    U = conserved6(W, d_r)
    hot = _zero_hot(topo.ncell)
    R1 = residual6(geo, mesh.bc_state, U, hot, GasParams(d_r, Zr, A, mu0, 0.0))[0]
    R2 = residual6(geo, mesh.bc_state, U, hot, GasParams(d_r, Zr, A, 2.0 * mu0, 0.0))[0]
    Rv = R2 - R1
    ijk = np.array([topo.ijk(c) for c in range(topo.ncell)])
    sel = (ijk[:, 0] >= 2) & (ijk[:, 0] <= 3) & (ijk[:, 1] >= 2) & (ijk[:, 1] <= 5)
    ft, fr = M.eucken_factors(A, d_r)
    kt, kr = ft * 1.5 * mu0, fr * 0.5 * d_r * mu0
    assert np.allclose(Rv[sel, 5] / topo.vol[sel], 2 * b * kr, rtol=1e-11)
    assert np.allclose(Rv[sel, 4] / topo.vol[sel], 2 * b * (kt + kr), rtol=1e-11)
    assert np.max(np.abs(Rv[sel, :4])) < 1e-13


def _n2_shock_case(Ma=2.0, n=80, hw=20.0, nv=(8, 4, 4), vmax=7.0, iterations=10, macro_steps=50):
    """Normal shock in nitrogen: Rankine-Hugoniot end states of gamma = 7/5
    (the equilibrium gas with d_r = 2), tanh start, upstream mean free path
    = length unit."""
    g = 1.4
    r2, u2, T2 = rankine_hugoniot(Ma, g)
    u1 = Ma * np.sqrt(g)
    W1 = np.array([1.0, u1, 0.0, 0.0, 1.0])
    W2 = np.array([r2, u2, 0.0, 0.0, T2])
    mesh = cartesian_1d(n, -hw, hw, W1, W2)
    x = mesh.flat(mesh.centers)[:, 0]
    s = 0.5 * (1.0 + np.tanh(x / 2.0))
    W0 = W1[None] + (W2 - W1)[None] * s[:, None]
    vg = VGrid(tuple(nv), (-vmax + 0.5 * u1, -vmax, -vmax), (vmax + 0.5 * u1, vmax, vmax))
    return Case("n2_shock", mesh, vg, W0, Kn=1.0, omega=NITROGEN["omega"], iterations=iterations,
                macro_steps=macro_steps, cfl=50.0, k_sub=4, dt=1.0), (W1, W2)


def test_navier_stokes_nitrogen_shock_between_rankine_hugoniot_states():
    """The six-variable synthetic equations with HoT = 0 are a two-temperature
    Navier-Stokes solver: from the tanh start between the Rankine-Hugoniot
    states of a Ma = 2 shock with gamma = 7/5 (rho2 = 8/3, T2 = 27/16, which
    holds only if the internal energy is carried and exchanged) the
    iteration reaches a steady shock: zero residual, both end cells at the
    Rankine-Hugoniot states with T_r = T_t, the fluxes rho u,
    rho u^2 + P_xx and (rho e + P_xx) u + q_t + q_r constant through it, and
    the internal temperature lagging behind the translational one inside."""
    case, (W1, W2) = _n2_shock_case(n=120, hw=30.0)   # wide enough for the T_r relaxation tail
    s = RykovSolver(case, *N2)
    d_r = N2[0]
    assert abs(W2[0] - 8.0 / 3.0) < 1e-14 and abs(W2[4] - 27.0 / 16.0) < 1e-14
    U = conserved6(s.W, d_r)
    hot = _zero_hot(s.N)
    for _ in range(18):
        U = macro_solve6(s.geo, s.bc_state, U, hot, s.gas, 20.0, 4, 100)
    R = residual6(s.geo, s.bc_state, U, hot, s.gas)[0]
    assert np.max(np.abs(R)) < 1e-9 * 2.0 * np.sqrt(1.4) ** 3 * 4
    W = primitive6(U, d_r)
    assert np.allclose(W[0], [*W1, 1.0], rtol=1e-6, atol=1e-9)
    assert np.allclose(W[-1], [*W2, W2[4]], rtol=1e-6, atol=1e-9)
    sig, qt, qr = s.nsf_field(W)
    rho, u, Tt, Tr = W[:, 0], W[:, 1], W[:, 4], W[:, 5]
    Pxx = rho * Tt + sig[:, 0, 0]
    e = 1.5 * Tt + 0.5 * u * u + Tr
    fl = np.stack([rho * u, rho * u * u + Pxx, (rho * e + Pxx) * u + qt[:, 0] + qr[:, 0]], 1)[1:-1]
    assert np.max(np.abs(fl / fl[0] - 1.0)) < 0.02
    assert np.max(Tt - Tr) > 0.05 and np.min(Tt - Tr) > -1e-6


# ----------------------------------------------------------------------------- GSIS iteration
def test_uniform_equilibrium_stream_is_a_gsis_fixed_point():
    """A uniform nitrogen stream in equilibrium (T_r = T_t) between two
    far-field ends of that same state stays put through the whole iteration:
    reference pair, sweep, six-variable solve and Eq. updatef."""
    W1 = np.array([1.0, 1.5, 0.0, 0.0, 1.0])
    case, _ = _n2_shock_case(n=10, hw=3.0, nv=(32, 20, 20), vmax=12.0, macro_steps=20)
    case.mesh = cartesian_1d(10, -3.0, 3.0, W1, W1)
    case.W0 = np.tile(W1, (10, 1))
    s = RykovSolver(case, *N2).run(3)
    assert np.max(np.abs(s.W - np.tile([*W1, 1.0], (10, 1)))) < 1e-12
    assert max(s.eps_history) < 1e-12


def test_updatef_gives_both_vdfs_the_new_state():
    """Eq. updatef with the equilibrium pair f_eq(W) = (M~, (d_r/2) T_r M~):
    after every GSIS iteration each kinetic cell's discrete mass, momentum,
    total and internal energy equal the new macroscopic state (the internal
    energy through f1 alone), on the 3D grid and on the reduced grid of an
    adaptive cylinder."""
    shock, _ = _n2_shock_case(n=24, hw=10.0, nv=(12, 8, 8), macro_steps=10)
    cyl = cylinder_case(Ma=2.0, Kn=0.1, n_r=6, n_theta=8, nv=(10, 10, 2), vbox=((-8, 8), (-7, 7), (0, 1)),
                        adaptive=True, Kn_ref=0.05, macro_steps=10, presolve_max_blocks=2, relax=1.0, reduced=True)
    cyl.omega = NITROGEN["omega"]
    for case in (shock, cyl):
        o = RykovSolver(case, *N2)
        o.initialise()
        for _ in range(2):
            o.step()
            assert np.max(np.abs(o.W - o.W_half)) > 1e-6
            for c in np.nonzero(o.dvm)[0]:
                Uf = o.vg.conserved(o.f[c])
                Uw = conserved6(o.W[c], N2[0])
                assert np.max(np.abs(Uf - Uw)) < 1e-12 * np.max(np.abs(Uw))


def test_nitrogen_shock_relaxes_its_internal_temperature_behind_the_translational_one():
    """Kinetic nitrogen shock (Ma = 2, 10 GSIS iterations from the tanh start):
    the residual falls every iteration; the internal temperature lags the
    translational one inside the shock (T_t - T_r up to a few tenths, the
    energy exchange taking Z_r collision times) and the two agree, near the
    Rankine-Hugoniot end states, to the transient of an unconverged run."""
    case, (W1, W2) = _n2_shock_case(n=40, hw=15.0, nv=(16, 10, 10), iterations=10, macro_steps=20)
    s = RykovSolver(case, *N2).run()
    e = s.eps_history
    assert all(e[i + 1] < e[i] for i in range(len(e) - 1)) and e[-1] < 0.5 * e[0]
    Tt, Tr = s.W[:, 4], s.W[:, 5]
    assert 0.1 < np.max(Tt - Tr) < 0.6 and np.min(Tt - Tr) > -5e-3
    assert abs(Tt[0] - 1.0) < 2e-3 and abs(Tr[0] - 1.0) < 2e-3
    assert abs(Tt[-1] - W2[4]) < 2e-2 and abs(Tr[-1] - W2[4]) < 2e-2


def test_reduced_two_vdf_iteration_is_the_xi_z_integral_of_the_3d_one(monkeypatch):
    """On a 2D flow with first-order face values the kinetic step is linear in
    (f0, f1), so the reduced iteration (f0 as its G and H planes, f1 as its
    xi_z integral) is the xi_z integral of the 3D one: after two nitrogen
    GSIS iterations of an all-kinetic cylinder the six-variable states agree
    to the xi_z quadrature error, and so do the reduced f1 and the integral
    of the 3D f1."""
    from oracle import kinetic as K
    monkeypatch.setattr(K, "slope", lambda *a: 0.0)
    nz = 24
    base = dict(Ma=2.0, Kn=0.1, n_r=6, n_theta=8, adaptive=False, macro_steps=10, cfl=5.0, k_sub=2, relax=1.0,
                presolve_max_blocks=3)
    c3 = cylinder_case(nv=(14, 12, nz), vbox=((-10, 10), (-9, 9), (-12, 12)), **base)
    cr = cylinder_case(nv=(14, 12, nz), vbox=((-10, 10), (-9, 9), (-12, 12)), **base)
    cr.vgrid = VGrid((14, 12, 2), (-10.0, -9.0, 0.0), (10.0, 9.0, 1.0), reduced=True)
    for c in (c3, cr):
        c.dt = 0.5
        c.omega = NITROGEN["omega"]
    o3 = RykovSolver(c3, *N2).run(2)
    orr = RykovSolver(cr, *N2).run(2)
    assert np.max(np.abs(orr.W - o3.W)) < 1e-8 * np.max(np.abs(o3.W))
    assert np.max(np.abs(o3.W[:, 4] - o3.W[:, 5])) > 1e-3        # the internal mode is out of equilibrium
    dz = 24.0 / nz
    n2 = 14 * 12
    for cell in (0, 7, 30):
        f1 = o3.vg.split(o3.f[cell])[1].reshape(nz, n2)
        ref = dz * f1.sum(axis=0)
        red = orr.vg.split(orr.f[cell])[1]
        assert np.max(np.abs(red - ref)) < 1e-8 * np.max(np.abs(ref))


# ----------------------------------------------------------------------------- unstructured meshes, hybrid grids
def test_collision_term_conserves_on_a_hybrid_grid():
    """The conservation readings hold with per-node weights too: on a stretched
    hybrid velocity grid the two-VDF collision term conserves mass, momentum
    and total energy to rounding and moves internal energy at the exchange
    rate, exactly as on the uniform grid."""
    from oracle.hybrid import HybridGrid, stretched_edges
    vg = RykovGrid(HybridGrid(*[stretched_edges(-9.0, 9.0, n, c, 1.1) for n, c in ((18, 0.4), (16, -0.2),
                                                                                     (14, 0.0))]), 2)
    f = _nonequilibrium(vg)
    rho, u, Tt, Tr, sig, qt, qr = vg.moments(f)
    g = vg.reference(rho, u, Tt, Tr, qt, qr, NITROGEN["Z_r"], NITROGEN["A"])
    dU = vg.conserved(g) - vg.conserved(f)
    scale = np.max(np.abs(vg.conserved(f)))
    assert np.max(np.abs(dU[:5])) < 1e-13 * scale
    T = (3.0 * Tt + 2.0 * Tr) / 5.0
    assert abs(dU[5] - rho * (T - Tr) / NITROGEN["Z_r"]) < 1e-13 * scale and abs(Tt - Tr) > 0.05


def test_monatomic_case_on_triangles_with_a_hybrid_grid_is_the_unstructured_oracle():
    """d_r = 0 on a triangulated, heated channel with a hybrid velocity grid
    and one wall layer: the two-VDF iteration is the (pinned) unstructured
    Shakhov iteration."""
    from oracle.hybrid import HybridGrid, stretched_edges
    from oracle.unstructured import UnstructuredSolver
    from test_oracle_unstructured import _channel
    hg = HybridGrid(*[stretched_edges(-8.0, 9.0, n, c, 1.1) for n, c in ((14, 0.6), (12, 0.0), (8, 0.0))])
    case = _channel(True, triangles=True, vgrid=hg)
    case.adaptive, case.Kn_ref, case.wall_layers, case.adapt_every = True, 1e9, 1, 1000
    o = UnstructuredSolver(case).run(3)
    r = RykovSolver(case, 0, NITROGEN["Z_r"], MONATOMIC_A).run(3)
    assert np.array_equal(r.dvm, o.dvm) and 0 < o.dvm.sum() < o.N
    assert np.max(np.abs(r.W[:, :5] - o.W)) < 1e-12 * np.max(np.abs(o.W))
    assert np.max(np.abs(r.f[:, :o.vg.nv] - o.f)) < 1e-12 * np.max(np.abs(o.f))


def test_nitrogen_on_tetrahedra_with_a_hybrid_grid():
    """Nitrogen in the heated box split into tetrahedra, hybrid velocity grid:
    after every GSIS iteration each kinetic cell carries the six new conserved
    moments (Eq. updatef), the internal mode is out of equilibrium at the
    heated walls, and the residual falls."""
    from oracle.hybrid import HybridGrid, stretched_edges
    from test_oracle_unstructured import _box_case
    hg = HybridGrid(*[stretched_edges(-7.0, 8.0, n, c, 1.1) for n, c in ((10, 0.6), (10, 0.0), (8, 0.1))])
    case = _box_case(True, tets=True, vgrid=hg)
    case.omega = NITROGEN["omega"]
    s = RykovSolver(case, *N2)
    s.initialise()
    for _ in range(3):
        s.step()
        for c in np.nonzero(s.dvm)[0]:
            Uf = s.vg.conserved(s.f[c])
            Uw = conserved6(s.W[c], N2[0])
            assert np.max(np.abs(Uf - Uw)) < 1e-12 * np.max(np.abs(Uw))
    assert np.max(np.abs(s.W[:, 4] - s.W[:, 5])) > 1e-3
    assert s.eps_history[-1] < s.eps_history[0]
