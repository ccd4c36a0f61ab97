"""Pins of the oracle functions that the GSIS iteration rests on (CPU only).

Each test checks the oracle against a closed form, an invariant, or a limit
that the mathematics fixes: the Navier-Stokes-Fourier face fluxes of the
synthetic solve (Eq. NSF_constitutive inside Eq. macro) on quadratic fields
where the discrete flux difference is exact, the wall flux on linear fields,
the wall correction at equilibrium, both remaining branches of Eq. Kn_Gll,
the continuum limit of the high-order terms (Eq. full_constitutive: HoT =
O(Kn^2)), the steady viscous shock of the synthetic equations (constant
fluxes, Rankine-Hugoniot end states), and the conservation property of
Eq. updatef.
"""
import numpy as np
import pytest

from workloads import shock_1d_case, cylinder_case
from workloads.cases import Case, VGrid, rankine_hugoniot
from workloads.meshes import cartesian_2d, cylinder_ogrid, BC_FARFIELD, BC_WALL, BC_PERIODIC, BC_NONE
from oracle import model as M
from oracle import kinetic as K
from oracle.mesh import Topology
from oracle.macro import MacroGeometry, residual, cell_gradients, wall_nsf_flux, macro_solve
from oracle.gsis import OracleSolver, prim_to_U, U_to_prim

FF, WL, PER, NO = BC_FARFIELD, BC_WALL, BC_PERIODIC, BC_NONE


# ----------------------------------------------------------------------------- viscous face flux
def _cart(ni, nj, x0, x1, y0, y1, types):
    states = [[1.0, 0.0, 0.0, 0.0, 1.0]] * 6
    return cartesian_2d(ni, nj, x0, x1, y0, y1, dim=2, bc_types=types, bc_states=states)


def _viscous_residual(mesh, W, mu0, omega):
    """Viscous part of the synthetic-equation residual: R(mu0) - R(0).  The
    inviscid splitting does not depend on the viscosity, so the difference
    is the NSF (and work) flux balance alone."""
    topo = Topology(mesh)
    geo = MacroGeometry(topo)
    U = prim_to_U(W)
    z = np.zeros((topo.ncell, 3, 3)); zq = np.zeros((topo.ncell, 3))
    R1 = residual(geo, mesh.bc_state, U, z, zq, mu0, omega)[0]
    R0 = residual(geo, mesh.bc_state, U, z, zq, 0.0, omega)[0]
    return topo, R1 - R0


def _interior(topo, margin=2):
    """Cells at least `margin` cells away from every non-periodic boundary:
    their least-squares gradients and those of their face neighbours use cell
    values only (no boundary state)."""
    ijk = np.array([topo.ijk(c) for c in range(topo.ncell)])
    ok = np.ones(topo.ncell, dtype=bool)
    for d in range(topo.dim):
        ok &= (ijk[:, d] >= margin) & (ijk[:, d] <= topo.n[d] - 1 - margin)
    return ok


def test_shear_stress_of_a_parabolic_profile():
    """u_x = a y^2 (uniform rho, T): the momentum equation's viscous term is
    d/dy(mu du_x/dy) = 2 a mu per unit volume.  On a uniform Cartesian mesh
    the face gradient along y is the exact difference quotient of the
    quadratic, so the discrete viscous residual equals 2 a mu V exactly; the
    energy residual is the difference of sigma_xy u_x through the top and
    bottom faces, with sigma_xy = -mu 2 a y_f and u_x the mean of the two
    cells (the work term of the face flux)."""
    a, mu0 = 0.3, 0.05
    mesh = _cart(6, 8, 0.0, 1.0, 0.5, 1.5, [FF, FF, FF, FF, NO, NO])
    x = mesh.flat(mesh.centers)
    W = np.zeros((mesh.ncell, 5)); W[:, 0] = 1.0; W[:, 4] = 1.0
    W[:, 1] = a * x[:, 1] ** 2
    topo, Rv = _viscous_residual(mesh, W, mu0, 0.81)
    sel = _interior(topo)
    V = topo.vol[sel]
    assert np.allclose(Rv[sel, 1] / V, 2 * a * mu0, rtol=1e-11)
    assert np.max(np.abs(Rv[sel, 0])) < 1e-15
    assert np.max(np.abs(Rv[sel, 2:4])) < 1e-12 * a * mu0
    dy = 1.0 / 8
    y = x[sel, 1]
    yt, yb = y + dy / 2, y - dy / 2
    uft = a * (y ** 2 + (y + dy) ** 2) / 2
    ufb = a * (y ** 2 + (y - dy) ** 2) / 2
    S = 1.0 / 6
    RE = mu0 * 2 * a * S * (yt * uft - yb * ufb)
    assert np.allclose(Rv[sel, 4], RE, rtol=1e-11)


def test_shear_stress_uses_the_transposed_gradient():
    """u_y = b x^2: the same shear with the roles of x and y exchanged; the
    stress sigma_xy = -mu (du_x/dy + du_y/dx) carries it through du_y/dx,
    so the y-momentum viscous residual is 2 b mu V."""
    b, mu0 = -0.4, 0.02
    mesh = _cart(8, 6, 0.5, 1.5, 0.0, 1.0, [FF, FF, FF, FF, NO, NO])
    x = mesh.flat(mesh.centers)
    W = np.zeros((mesh.ncell, 5)); W[:, 0] = 1.0; W[:, 4] = 1.0
    W[:, 2] = b * x[:, 0] ** 2
    topo, Rv = _viscous_residual(mesh, W, mu0, 0.81)
    sel = _interior(topo)
    assert np.allclose(Rv[sel, 2] / topo.vol[sel], 2 * b * mu0, rtol=1e-11)
    assert np.max(np.abs(Rv[sel, 1])) < 1e-12 * abs(b) * mu0


def test_normal_stress_of_a_compression():
    """u_x = a x^2: sigma_xx = -mu (2 du/dx - 2/3 div u) = -4/3 mu du/dx, so
    the viscous momentum residual is 4/3 mu 2 a V (the bulk term of
    Eq. NSF_constitutive), and the 2/3 div u part of sigma_yy cancels
    between the top and bottom faces."""
    a, mu0 = 0.25, 0.03
    mesh = _cart(8, 6, 0.5, 1.5, 0.0, 1.0, [FF, FF, FF, FF, NO, NO])
    x = mesh.flat(mesh.centers)
    W = np.zeros((mesh.ncell, 5)); W[:, 0] = 1.0; W[:, 4] = 1.0
    W[:, 1] = a * x[:, 0] ** 2
    topo, Rv = _viscous_residual(mesh, W, mu0, 0.81)
    sel = _interior(topo)
    assert np.allclose(Rv[sel, 1] / topo.vol[sel], 4.0 / 3.0 * mu0 * 2 * a, rtol=1e-11)
    assert np.max(np.abs(Rv[sel, 2])) < 1e-12 * a * mu0


def test_heat_conduction_of_a_parabolic_temperature():
    """T = 1 + b y^2 with the gas at rest and a temperature-independent
    viscosity (omega = 0): the energy equation's conduction term is
    d/dy(kappa dT/dy) = kappa 2 b with kappa = 15/4 mu (Pr = 2/3 for the
    monatomic gas), exact for the difference quotient of a quadratic."""
    b, mu0 = 0.2, 0.04
    mesh = _cart(6, 8, 0.0, 1.0, 0.0, 1.0, [FF, FF, FF, FF, NO, NO])
    x = mesh.flat(mesh.centers)
    W = np.zeros((mesh.ncell, 5)); W[:, 0] = 1.0
    W[:, 4] = 1.0 + b * x[:, 1] ** 2
    topo, Rv = _viscous_residual(mesh, W, mu0, 0.0)
    sel = _interior(topo)
    assert np.allclose(Rv[sel, 4] / topo.vol[sel], 3.75 * mu0 * 2 * b, rtol=1e-11)
    assert np.max(np.abs(Rv[sel, :4])) < 1e-14


def test_viscous_residual_on_the_ogrid():
    """On the body-fitted O-grid (non-uniform, non-orthogonal faces): a
    linear velocity field has a constant NSF stress, so the viscous momentum
    residual of every interior cell vanishes (its faces close); and for
    u_x = a y^2 the viscous residual per volume converges to 2 a mu under
    refinement."""
    a, mu0 = 0.3, 0.05
    errs = []
    for nr, nt in ((8, 32), (16, 64)):
        m = cylinder_ogrid(nr, nt, 1.0, 2.0, 1.0 / nr, 2.0, [1.0, 0.0, 0.0, 0.0, 1.0])
        m.bc_type[0] = FF
        m.bc_state[0] = [1.0, 0.0, 0.0, 0.0, 1.0]
        x = m.flat(m.centers)
        W = np.zeros((m.ncell, 5)); W[:, 0] = 1.0; W[:, 4] = 1.0
        W[:, 1] = 0.3 * x[:, 0] - 0.2 * x[:, 1]
        W[:, 2] = 0.1 * x[:, 0] + 0.4 * x[:, 1]
        topo, Rl = _viscous_residual(m, W, mu0, 0.81)
        sel = _interior(topo)
        assert np.max(np.abs(Rl[sel, 1:4])) < 1e-11 * mu0 * np.max(topo.vol)
        W[:, 1] = a * x[:, 1] ** 2
        W[:, 2] = 0.0
        topo, Rv = _viscous_residual(m, W, mu0, 0.81)
        errs.append(np.max(np.abs(Rv[sel, 1] / topo.vol[sel] / (2 * a * mu0) - 1)))
    assert errs[1] < 0.5 * errs[0] and errs[1] < 0.01


# ----------------------------------------------------------------------------- wall flux
def test_wall_nsf_flux_of_linear_profiles():
    """Gas between a wall at y = 0 (temperature T_w, at rest) and the far
    field, with u_x = a y and T = T_w + b y: both profiles are linear and
    meet the wall values, so the wall gradients are exact and the NSF wall
    flux through the outward area S = -|S| e_y is mass 0, momentum
    (mu(T_w) a |S|, -p_c |S|, 0) and energy q.S = kappa(T_w) b |S|."""
    a, b, Tw, mu0, om = 0.5, 0.3, 1.5, 0.05, 0.81
    states = [[0] * 5, [0] * 5, [0, 0, 0, 0, Tw], [1.0, 0.0, 0.0, 0.0, 1.0], [0] * 5, [0] * 5]
    mesh = cartesian_2d(4, 6, 0.0, 1.0, 0.0, 1.0, dim=2, bc_types=[PER, PER, WL, FF, NO, NO], bc_states=states)
    topo = Topology(mesh)
    geo = MacroGeometry(topo)
    x = topo.centers
    rho = np.full(topo.ncell, 1.2)
    u = np.zeros((topo.ncell, 3)); u[:, 0] = a * x[:, 1]
    T = Tw + b * x[:, 1]
    gu, gT = cell_gradients(geo, mesh.bc_state, rho, u, T)
    F = wall_nsf_flux(geo, mesh.bc_state, rho, u, T, gu, gT, mu0, om)
    idx = np.nonzero(geo.bT == WL)[0]
    assert len(idx) == 4
    c = geo.bC[idx]
    S = geo.bSabs[idx]
    mu_w = mu0 * Tw ** om
    assert np.max(np.abs(F[:, 0])) == 0.0
    assert np.allclose(F[:, 1], mu_w * a * S, rtol=1e-12)
    assert np.allclose(F[:, 2], -rho[c] * T[c] * S, rtol=1e-12)
    assert np.max(np.abs(F[:, 3])) < 1e-15
    assert np.allclose(F[:, 4], 3.75 * mu_w * b * S, rtol=1e-12)


def test_wall_correction_vanishes_at_wall_equilibrium():
    """A kinetic wall cell holding the Maxwellian of a gas at rest at the
    wall temperature: the diffuse wall re-emits the same half-range, the
    kinetic wall flux is the pressure alone, and the NSF wall flux of the
    uniform state is that same pressure, so the frozen wall correction of the
    synthetic solve is zero (up to the velocity quadrature of the pressure)."""
    case = cylinder_case(Ma=2.0, Kn=0.1, n_r=4, n_theta=6, nv=(24, 24, 24), adaptive=False,
                         vbox=((-9, 9), (-9, 9), (-9, 9)), presolve_max_blocks=0)
    o = OracleSolver(case)
    o.initialise()
    Tw = case.mesh.bc_state[0][4]
    rho = 1.3
    o.W[:] = [rho, 0.0, 0.0, 0.0, Tw]
    for c in range(o.N):
        o.f[c] = M.corrected_maxwellian(rho, np.zeros(3), Tw, o.vg)
    inp = o.kinetic_inputs()
    corr = o.wall_correction(o.W, inp.mw)
    idx = np.nonzero(o.geo.bT == WL)[0]
    scale = rho * Tw * np.max(o.geo.bSabs[idx])
    assert corr.shape == (len(idx), 5) and len(idx) == case.mesh.nj
    # (the half-range sums of an oblique face on a 24^3 grid are exact to ~1e-8; a wrong sign or
    # factor in either flux would leave an O(1) correction)
    assert np.max(np.abs(corr)) < 1e-7 * scale
    # a gas at a different temperature: the wall exchanges heat, the correction does not vanish
    for c in range(o.N):
        o.f[c] = M.corrected_maxwellian(rho, np.zeros(3), 1.2 * Tw, o.vg)
    o.W[:, 4] = 1.2 * Tw
    corr = o.wall_correction(o.W, inp.mw)
    assert np.max(np.abs(corr[:, 4])) > 1e-3 * scale


# ----------------------------------------------------------------------------- Eq. Kn_Gll
def _kn_case(W_of_x, half=3.0, n=12):
    case = shock_1d_case(n_cells=n, half_width=half, nv=(8, 4, 4))
    x = case.mesh.flat(case.mesh.centers)[:, 0]
    case.mesh.bc_state[0] = W_of_x(np.array([-half]))[0]
    case.mesh.bc_state[1] = W_of_x(np.array([half]))[0]
    case.W0 = W_of_x(x)
    return case, x


def test_kn_gll_speed_branch():
    """|grad U|/U with U = |u| for a linear stream u_x = U0 + c x (uniform rho,
    T): lambda c / U where the stream is supersonic, and lambda c / a (the
    local sound speed a = sqrt(gamma T) replacing U) where U < a, the
    stagnation reading of the garbled branch."""
    c = 0.1
    for U0 in (3.0, 0.3):
        case, x = _kn_case(lambda x: np.stack([np.ones_like(x), U0 + c * x, 0 * x, 0 * x, np.ones_like(x)], 1))
        s = OracleSolver(case)
        kn = s.kn_gll_field(case.W0)
        lam = M.mu0_from_kn(case.Kn) * np.sqrt(np.pi / 2)          # rho = T = 1
        U = U0 + c * x
        expect = lam * c / np.maximum(U, np.sqrt(5.0 / 3.0))
        assert np.allclose(kn, expect, rtol=1e-12)
        assert (U0 > 1.3) == bool(np.all(U > np.sqrt(5.0 / 3.0)))


def test_kn_gll_temperature_branch():
    """|grad T|/T for T = 1 + 0.05 x with the gas at rest and uniform rho:
    lambda(T) 0.05 / T with the local mean free path
    lambda = mu(T)/p sqrt(pi T/2) and mu = mu0 T^omega."""
    case, x = _kn_case(lambda x: np.stack([np.ones_like(x), 0 * x, 0 * x, 0 * x, 1.0 + 0.05 * x], 1))
    s = OracleSolver(case)
    kn = s.kn_gll_field(case.W0)
    T = 1.0 + 0.05 * x
    lam = M.mu0_from_kn(case.Kn) * T ** case.omega / T * np.sqrt(np.pi * T / 2)
    assert np.allclose(kn, lam * 0.05 / T, rtol=1e-12)


def test_kn_gll_takes_the_largest_ratio():
    """With density, speed and temperature gradients together the criterion
    is the largest of the three ratios, not their sum."""
    case, x = _kn_case(lambda x: np.stack([1.0 + 0.02 * x, 2.0 + 0.3 * x, 0 * x, 0 * x, 1.0 + 0.01 * x], 1),
                       half=2.0)
    s = OracleSolver(case)
    kn = s.kn_gll_field(case.W0)
    rho, U, T = 1.0 + 0.02 * x, 2.0 + 0.3 * x, 1.0 + 0.01 * x
    lam = M.mu0_from_kn(case.Kn) * T ** case.omega / (rho * T) * np.sqrt(np.pi * T / 2)
    r = np.maximum(np.maximum(0.02 / rho, 0.3 / np.maximum(U, np.sqrt(5 / 3 * T))), 0.01 / T)
    assert np.allclose(kn, lam * r, rtol=1e-12)
    assert np.all(r == 0.3 / np.maximum(U, np.sqrt(5 / 3 * T)))


# ----------------------------------------------------------------------------- continuum limit
def _frozen_state_hot(Kn, n=64, amp=0.1):
    """Kinetic steady state for a frozen smooth macroscopic state on a
    periodic 1D domain of unit length: a gas at rest at uniform pressure with
    T = 1 + amp sin(2 pi x), rho = 1/T.  The kinetic step is repeated (the
    reference distribution taking the heat flux of the current f each time,
    as in the GSIS iteration) until f stops changing.  Returns the maximum
    kinetic normal stress (its NSF value is zero: u = 0), the maximum heat
    flux HoT (kinetic minus Fourier) and the maximum Fourier heat flux, over
    the cells away from the periodic wrap (the Cartesian wrap is not closed
    geometrically, so the least-squares gradients of the two end cells are
    not those of the profile)."""
    mesh = cartesian_2d(n, 1, 0.0, 1.0, 0.0, 1.0, dim=1, bc_types=[PER, PER, NO, NO, NO, NO],
                        bc_states=[[0.0] * 5] * 6)
    x = mesh.flat(mesh.centers)[:, 0]
    T = 1.0 + amp * np.sin(2 * np.pi * x)
    W = np.stack([1.0 / T, 0 * x, 0 * x, 0 * x, T], 1)
    case = Case("periodic", mesh, VGrid((40, 12, 12), (-7.0, -6.0, -6.0), (7.0, 6.0, 6.0)), W, Kn=Kn,
                presolve_max_blocks=0)
    s = OracleSolver(case)
    s.initialise()
    prev = s.f.copy()
    for _ in range(80):
        K.sweep(s.topo, s.vg, s.f, s.dvm, s.kinetic_inputs())
        if np.max(np.abs(s.f - prev)) < 1e-11 * np.max(np.abs(s.f)):
            break
        prev = s.f.copy()
    else:
        raise AssertionError("kinetic steady state not reached")
    sig_n, q_n = s.nsf_field(W)
    sxx = np.array([M.moments(s.f[c], s.vg)[3][0, 0] for c in range(s.N)])
    qk = np.array([M.heat_flux_about(s.f[c], W[c, 1:4], s.vg)[0] for c in range(s.N)])
    keep = slice(3, n - 3)
    return (np.max(np.abs(sxx[keep])), np.max(np.abs((qk - q_n[:, 0])[keep])),
            np.max(np.abs(q_n[keep, 0])))


def test_high_order_terms_vanish_like_kn_squared():
    """Continuum limit of Eq. full_constitutive: the kinetic stress and heat
    flux agree with Eq. NSF_constitutive to first order in Kn (Chapman-Enskog:
    the Shakhov model with Pr = 2/3 and kappa = 15/4 mu), so the high-order
    terms fall like Kn^2 while the Fourier flux itself falls like Kn.
    Halving Kn must divide the HoT by clearly more than 2 (a first-order
    error, e.g. a wrong conductivity or Prandtl number, gives 2)."""
    s1, h1, q1 = _frozen_state_hot(0.01)
    s2, h2, q2 = _frozen_state_hot(0.005)
    assert abs(q1 / q2 - 2.0) < 0.01                  # Fourier flux ~ Kn
    assert s1 / s2 > 3.0 and h1 / h2 > 3.0           # HoT ~ Kn^2
    assert h2 < 0.02 * q2 and s2 < 0.02 * q2


# ----------------------------------------------------------------------------- steady viscous shock
def test_navier_stokes_shock_is_steady_between_rankine_hugoniot_states():
    """The synthetic equations with HoT = 0 are a Navier-Stokes solver: from
    the tanh start between the Rankine-Hugoniot states of a Ma = 2 shock
    (gamma = 5/3: rho2/rho1 = 2.2857, T2/T1 = 2.0781) the pseudo-time
    iteration reaches a steady viscous shock whose residual vanishes (every
    face carries the same mass, momentum and energy flux: rho u,
    rho u^2 + P_xx, (rho E + P_xx) u + q_x), whose end cells hold the two
    Rankine-Hugoniot states, and whose cell-centred fluxes are constant to
    the discretisation error."""
    case = shock_1d_case(n_cells=80, half_width=20.0, nv=(8, 4, 4))
    s = OracleSolver(case)
    N = s.N
    z = np.zeros((N, 3, 3)); zq = np.zeros((N, 3))
    U = prim_to_U(case.W0)
    for _ in range(15):
        U = macro_solve(s.geo, s.bc_state, U, z, zq, s.mu0, s.omega, 20.0, 4, 100)
    R = residual(s.geo, s.bc_state, U, z, zq, s.mu0, s.omega)[0]
    Fscale = 2.0 * np.sqrt(5 / 3) ** 3 * 4          # rho u^3 of the upstream state, order of magnitude
    assert np.max(np.abs(R)) < 1e-9 * Fscale
    W = U_to_prim(U)
    r2, u2, T2 = rankine_hugoniot(2.0)
    assert abs(r2 - 2.2857142857142856) < 1e-15 and abs(T2 - 2.078125) < 1e-15
    assert np.allclose(W[0], [1.0, 2.0 * np.sqrt(5 / 3), 0, 0, 1.0], rtol=1e-6, atol=1e-9)
    assert np.allclose(W[-1], [r2, u2, 0, 0, T2], rtol=1e-6, atol=1e-9)
    sig, q = s.nsf_field(W)
    rho, u, T = W[:, 0], W[:, 1], W[:, 4]
    Pxx = rho * T + sig[:, 0, 0]
    E = 1.5 * T + 0.5 * u * u
    fl = np.stack([rho * u, rho * u * u + Pxx, (rho * E + Pxx) * u + q[:, 0]], 1)[1:-1]
    assert np.max(np.abs(fl / fl[0] - 1.0)) < 0.02
    # the shock is there: the density rises from rho1 to rho2 across it
    assert W[N // 2 - 10, 0] < 1.3 and W[N // 2 + 10, 0] > 2.2


# ----------------------------------------------------------------------------- Eq. updatef
@pytest.mark.parametrize("relax", [1.0, 0.7])
def test_updatef_gives_the_new_conserved_moments(relax):
    """Eq. updatef, f^{n+1} = f^{n+1/2} + M~(W^{n+1}) - M~(W^{n+1/2}): the
    moments of f^{n+1/2} are W^{n+1/2} and those of M~ are exact, so after
    every GSIS iteration the discrete mass, momentum and energy of each
    kinetic cell equal the new macroscopic state W^{n+1} (with or without
    the under-relaxation of the synthetic correction)."""
    case = cylinder_case(Ma=2.0, Kn=0.1, n_r=6, n_theta=8, nv=(14, 12, 6), adaptive=False, macro_steps=10,
                         vbox=((-10, 10), (-9, 9), (-8, 8)), presolve_max_blocks=3, relax=relax)
    case.dt = 0.5
    o = OracleSolver(case)
    o.initialise()
    for _ in range(2):
        o.step()
        assert np.max(np.abs(o.W - o.W_half)) > 1e-6      # the synthetic solve moved the state
        for c in range(o.N):
            Uf = M.conserved(o.f[c], o.vg)
            Uw = M.conserved_from_primitive(o.W[c, 0], o.W[c, 1:4], o.W[c, 4])
            assert np.max(np.abs(Uf - Uw)) < 1e-12 * np.max(np.abs(Uw))
