"""Pins of the oracle's discretisation and GSIS driver (CPU only)."""
import numpy as np
import pytest

from workloads import shock_1d_case, cylinder_case, cartesian_1d, cylinder_ogrid, sphere_ogrid
from workloads.meshes import BC_FARFIELD, BC_WALL, BC_PERIODIC, BC_NONE
from oracle import model as M
from oracle import kinetic as K
from oracle.mesh import Topology
from oracle.macro import MacroGeometry, kfvs, _half_range, euler_flux_dot, residual, lsq_grad
from oracle.gsis import OracleSolver, residual_eps, prim_to_U


# ----------------------------------------------------------------------------- geometry
@pytest.mark.parametrize("mesh", [
    cartesian_1d(7, -1.0, 2.0, [1, 1, 0, 0, 1], [1, 1, 0, 0, 1]),
    cylinder_ogrid(6, 8, 0.5, 5.0, 0.05, 2.0, [1, 1, 0, 0, 1]),
    sphere_ogrid(4, 6, 8, 0.5, 5.0, 0.1, 2.0, [1, 1, 0, 0, 1]),
])
def test_cells_are_closed(mesh):
    """Outward area vectors of every cell sum to zero (geometric conservation)."""
    topo = Topology(mesh)
    for c in range(topo.ncell):
        s = sum(sd.S_out for sd in topo.sides[c])
        scale = max(np.linalg.norm(sd.S_out) for sd in topo.sides[c])
        assert np.linalg.norm(s) < 1e-13 * scale
        assert topo.vol[c] > 0


def test_cylinder_volume_is_polygon_area():
    """Cells are straight-sided quadrilaterals of unit depth: the total volume
    is the annulus between two regular n-gons, n/2 (r_o^2 - r_i^2) sin(2 pi/n)."""
    n = 16
    mesh = cylinder_ogrid(10, n, 0.5, 5.0, 0.02, 2.0, [1, 1, 0, 0, 1])
    exact = 0.5 * n * (5.0 ** 2 - 0.5 ** 2) * np.sin(2 * np.pi / n)
    assert abs(mesh.volumes.sum() / exact - 1.0) < 1e-13


@pytest.mark.parametrize("mesh", [
    cylinder_ogrid(6, 8, 0.5, 5.0, 0.05, 2.0, [1, 1, 0, 0, 1]),
    sphere_ogrid(4, 6, 8, 0.5, 5.0, 0.1, 2.0, [1, 1, 0, 0, 1]),
])
def test_lsq_gradient_exact_for_linear_fields(mesh):
    topo = Topology(mesh)
    geo = MacroGeometry(topo)
    a = np.array([0.3, -1.2, 0.7])[:mesh.dim]
    lin = lambda x: 2.0 + x[..., :mesh.dim] @ a
    phi = lin(topo.centers)
    bv = np.zeros((topo.ncell, 6))
    for c in range(topo.ncell):
        for si, sd in enumerate(topo.sides[c]):
            bv[c, si] = lin(sd.xf)
    g = lsq_grad(geo, phi, bv)
    assert np.max(np.abs(g[:, :mesh.dim] - a[None, :])) < 1e-11


# ----------------------------------------------------------------------------- macro fluxes
def test_kfvs_consistency_and_supersonic_limit():
    """Kinetic flux-vector splitting: a uniform state gives the Euler flux
    exactly (the two half-range fluxes add up to the full-range moments); a
    state moving along n at 9 thermal speeds sends no molecules back (the
    backward half-range weight erfc(9/sqrt 2)/2 ~ 1e-19), so the flux is the
    left state's Euler flux whatever the right state is."""
    rng = np.random.default_rng(1)
    F = 20
    r = rng.uniform(0.5, 2, F); u = rng.uniform(-1, 1, (F, 3)); p = rng.uniform(0.5, 2, F)
    n = rng.normal(size=(F, 3)); n /= np.linalg.norm(n, axis=1)[:, None]
    U = np.concatenate([r[:, None], r[:, None] * u, (1.5 * p + 0.5 * r * np.sum(u * u, 1))[:, None]], 1)
    assert np.allclose(kfvs(r, u, p, r, u, p, n), euler_flux_dot(U, n), rtol=1e-13, atol=1e-13)
    T = p / r
    u2 = (9.0 * np.sqrt(T))[:, None] * n
    U2 = np.concatenate([r[:, None], r[:, None] * u2, (1.5 * p + 0.5 * r * np.sum(u2 * u2, 1))[:, None]], 1)
    rR, uR2 = r * 2, (9.0 * np.sqrt(3 * p / (r * 2)))[:, None] * n   # right state also at 9 thermal speeds along +n
    assert np.allclose(kfvs(r, u2, p, rR, uR2, 3 * p, n), euler_flux_dot(U2, n), rtol=1e-13, atol=1e-14)


def test_kfvs_effusion_closed_form_and_quadrature():
    """Gas at rest: the one-way flux through a face is the effusion flux
    rho sqrt(T / (2 pi)) of mass and rho T sqrt(2 T / pi) of energy (kinetic
    theory), and the normal momentum flux is p / 2.  A moving state: the
    closed-form half-range moments equal a brute-force sum over a fine
    uniform velocity grid of the Maxwellian's molecules with xi.n > 0."""
    r, T = np.array([1.7]), np.array([2.3])
    n = np.array([[0.0, 0.0, 1.0]])
    F = _half_range(r, np.zeros((1, 3)), T, n, 1.0)[0]
    assert abs(F[0] / (r[0] * np.sqrt(T[0] / (2 * np.pi))) - 1) < 1e-14
    assert abs(F[3] / (0.5 * r[0] * T[0]) - 1) < 1e-14
    assert abs(F[4] / (r[0] * T[0] * np.sqrt(2 * T[0] / np.pi)) - 1) < 1e-14
    u = np.array([[0.7, -0.4, 0.3]]); nn = np.array([[0.6, 0.0, 0.8]]); T = np.array([1.4])
    vg = M.VelocityGrid((96, 96, 96), (-9, -9, -9), (9, 9, 9))
    f = M.maxwellian(1.0, u[0], T[0], vg.xi)
    xn = vg.xi @ nn[0]
    g = vg.w * np.where(xn > 0, xn * f, 0.0)
    brute = np.array([g.sum(), g @ vg.xi[:, 0], g @ vg.xi[:, 1], g @ vg.xi[:, 2],
                      0.5 * g @ np.sum(vg.xi ** 2, 1)])
    F = _half_range(np.array([1.0]), u, T, nn, 1.0)[0]
    assert np.max(np.abs(F - brute)) < 2e-3 * np.max(np.abs(F))   # midpoint rule across the xi.n = 0 kink


def test_macro_residual_vanishes_for_uniform_stream_on_ogrid():
    W = [1.0, 2.0, 0.5, 0.0, 1.0]
    mesh = cylinder_ogrid(5, 8, 0.5, 5.0, 0.1, 2.0, W)
    mesh.bc_type[0] = BC_FARFIELD
    mesh.bc_state[0] = W
    topo = Topology(mesh)
    geo = MacroGeometry(topo)
    Wc = np.tile(W, (topo.ncell, 1))
    R, _, _ = residual(geo, mesh.bc_state, prim_to_U(Wc), np.zeros((topo.ncell, 3, 3)),
                       np.zeros((topo.ncell, 3)), 0.01, 0.81)
    assert np.max(np.abs(R)) < 1e-13


# ----------------------------------------------------------------------------- kinetic step
def _tiny_1d(n=6, Kn=1.0, nv=(10, 4, 4), delta=1.0):
    c = shock_1d_case(Ma=2.0, n_cells=n, half_width=n / 4.0, nv=nv, delta=delta)
    c.Kn = Kn
    return c


def test_first_order_sweep_equals_dense_implicit_solve(monkeypatch):
    """With slopes switched off the scheme is the first-order implicit upwind
    system (1/tau + sum_out xi.S/V) f_c - sum_in |xi.S|/V f_nb = g/tau + inflow;
    in 1D one symmetric Gauss-Seidel pass solves it exactly.  Compare with a
    dense Gaussian elimination per velocity."""
    case = _tiny_1d()
    s = OracleSolver(case); s.initialise()
    inp = s.kinetic_inputs()
    monkeypatch.setattr(K, "slope", lambda *a: 0.0)
    f = s.f.copy()
    K.sweep(s.topo, s.vg, f, s.dvm, inp)
    N, vg, topo = s.N, s.vg, s.topo
    for v in range(vg.nv):
        A = np.zeros((N, N)); b = np.zeros(N)
        for c in range(N):
            A[c, c] += 1.0 / inp.tau[c]
            b[c] += inp.gt[c][v] / inp.tau[c]
            for sd in topo.sides[c]:
                if sd.nbr < 0 and sd.bc == BC_NONE:
                    continue
                xn = vg.xi[v] @ sd.S_out / topo.vol[c]
                if xn > 0:
                    A[c, c] += xn
                elif sd.nbr >= 0:
                    A[c, sd.nbr] += xn
                else:
                    b[c] -= xn * inp.ff[sd.bc_side][v]
        ref = np.linalg.solve(A, b)
        assert np.max(np.abs(f[:, v] - ref)) <= 1e-13 * max(1e-300, np.max(np.abs(ref)))


def test_second_order_sweeps_converge_to_discrete_steady_state():
    """Repeated kinetic steps (frozen g~, tau) converge to the solution of the
    second-order steady scheme: for every cell and velocity
    (1/V) sum_F xi.S_F f_F = (g~ - f)/tau with f_F the upwind MUSCL-minmod
    face value (written out here independently of the oracle)."""
    case = _tiny_1d(n=8, Kn=0.3)
    s = OracleSolver(case); s.initialise()
    inp = s.kinetic_inputs()
    for _ in range(60):
        K.sweep(s.topo, s.vg, s.f, s.dvm, inp)
    f, vg, topo = s.f, s.vg, s.topo
    N = s.N

    def mm(a, b):
        return np.where(a * b > 0, np.sign(a) * np.minimum(np.abs(a), np.abs(b)), 0.0)

    slopes = np.zeros_like(f)
    for c in range(1, N - 1):
        slopes[c] = mm(f[c] - f[c - 1], f[c + 1] - f[c])
    xi = vg.xi[:, 0]
    ff_lo, ff_hi = inp.ff[0], inp.ff[1]
    res = 0.0
    for c in range(N):
        dx = topo.vol[c]
        # face c+1/2 and c-1/2 values
        right = np.where(xi > 0, f[c] + 0.5 * slopes[c], (f[c + 1] - 0.5 * slopes[c + 1]) if c + 1 < N else ff_hi)
        left = np.where(xi > 0, (f[c - 1] + 0.5 * slopes[c - 1]) if c > 0 else ff_lo, f[c] - 0.5 * slopes[c])
        r = xi * (right - left) / dx - (inp.gt[c] - f[c]) / inp.tau[c]
        res = max(res, np.max(np.abs(r)) / np.max(np.abs(inp.gt[c] / inp.tau[c])))
    assert res < 1e-11


def test_free_molecular_closed_form():
    """tau -> infinity (Kn = 1e4): the steady 1D solution between two
    far-field Maxwellians is M1 for xi_x > 0 and M2 for xi_x < 0 everywhere."""
    case = _tiny_1d(n=6, Kn=1e4)
    s = OracleSolver(case); s.initialise()
    inp = s.kinetic_inputs()
    for _ in range(8):
        K.sweep(s.topo, s.vg, s.f, s.dvm, inp)
    xi = s.vg.xi[:, 0]
    expect = np.where(xi > 0, inp.ff[0], inp.ff[1])
    assert np.max(np.abs(s.f - expect[None, :])) < 1e-3 * np.max(expect)   # O(1/Kn) collision term
    # density of the half-range mix, summed independently half by half
    w = s.vg.w
    rho_closed = w * (np.sum(inp.ff[0][xi > 0]) + np.sum(inp.ff[1][xi < 0]))
    assert abs(M.moments(s.f[3], s.vg)[0] / rho_closed - 1) < 1e-3


def test_wall_density_gives_zero_mass_flux():
    vg = M.VelocityGrid((12, 10, 6), (-6, -6, -6), (6, 6, 6))
    f = M.maxwellian(1.3, [0.4, -0.2, 0], 1.5, vg.xi)
    S = np.array([-0.3, -0.9, 0.0])
    Mw = M.maxwellian(1.0, np.zeros(3), 2.0, vg.xi)
    rw = K.wall_density(f, S, Mw, vg)
    xn = vg.xi @ S
    face = np.where(xn > 0, f, rw * Mw)
    assert abs(np.sum(xn * face)) < 1e-14 * np.sum(np.abs(xn * face))


# ----------------------------------------------------------------------------- whole iteration
def test_uniform_stream_is_gsis_fixed_point_1d():
    W1 = np.array([1.0, 1.5, 0.0, 0.0, 1.0])
    case = shock_1d_case(n_cells=10, half_width=3.0, nv=(32, 20, 20), vmax=12.0, macro_steps=20)
    case.mesh = cartesian_1d(10, -3, 3, W1, W1)
    case.W0 = np.tile(W1, (10, 1))
    s = OracleSolver(case).run(3)
    assert np.max(np.abs(s.W - case.W0)) < 1e-12
    assert max(s.eps_history) < 1e-12


def test_uniform_stream_is_gsis_fixed_point_ogrid():
    """A uniform stream through an O-grid annulus with far-field boundaries on
    both radial sides (2D faces, periodic wrap, MUSCL, HLLC, viscous terms)."""
    W = np.array([1.0, 1.2, -0.4, 0.0, 1.0])
    case = cylinder_case(n_r=4, n_theta=6, nv=(24, 24, 6), Kn=0.5, adaptive=False, macro_steps=10,
                         vbox=((-9, 9), (-9, 9), (-6, 6)))
    case.mesh.bc_type[0] = BC_FARFIELD
    case.mesh.bc_state[0] = W
    case.mesh.bc_state[1] = W
    case.W0 = np.tile(W, (case.mesh.ncell, 1))
    s = OracleSolver(case).run(2)
    assert np.max(np.abs(s.W - case.W0)) < 1e-11


def test_residual_eps_definition():
    """Convergence criterion of Sec. 4 on a hand-computed two-cell example."""
    Wp = np.array([[1.0, 1.0, 0.0, 0.0, 2.0], [2.0, 0.0, 1.0, 0.0, 1.0]])
    Wn = Wp.copy(); Wn[0, 0] = 1.1; Wn[1, 4] = 1.3
    vol = np.array([1.0, 3.0])
    e_rho = np.sqrt(0.01 * 1.0 / (1.0 * 1 + 4.0 * 3))
    e_T = np.sqrt(0.09 * 3.0 / (4.0 * 1 + 1.0 * 3))
    assert abs(residual_eps(Wn, Wp, vol) - max(e_rho, e_T)) < 1e-15


def test_kn_gll_linear_density():
    """Eq. Kn_Gll for rho = 1 + 0.01 x, uniform u and T: interior cells give
    lambda |d rho/dx| / rho with lambda = mu(T)/p sqrt(pi T/2)."""
    W1 = [1.0, 1.0, 0, 0, 1.0]
    case = shock_1d_case(n_cells=12, half_width=3.0, nv=(8, 4, 4))
    x = case.mesh.flat(case.mesh.centers)[:, 0]
    case.mesh.bc_state[0] = [1 + 0.01 * -3.0, 1.0, 0, 0, 1.0]
    case.mesh.bc_state[1] = [1 + 0.01 * 3.0, 1.0, 0, 0, 1.0]
    case.W0 = np.stack([1 + 0.01 * x, np.ones_like(x), 0 * x, 0 * x, np.ones_like(x)], 1)
    s = OracleSolver(case)
    kn = s.kn_gll_field(case.W0)
    mu0 = M.mu0_from_kn(case.Kn)
    lam = mu0 / (1 + 0.01 * x) * np.sqrt(np.pi / 2)
    assert np.allclose(kn, lam * 0.01 / (1 + 0.01 * x), rtol=1e-12)


def test_no_dvm_cells_is_pure_navier_stokes():
    """Kn_ref above every Kn_Gll: no DVM cell, HoT = 0, so each GSIS iteration
    is exactly one block of NS pseudo-steps (continuum limit of the coupling)."""
    from oracle.macro import macro_solve
    from oracle.gsis import U_to_prim
    case = shock_1d_case(n_cells=16, half_width=4.0, nv=(8, 4, 4), macro_steps=15)
    case.adaptive = True; case.Kn_ref = 1e30; case.presolve_max_blocks = 0
    s = OracleSolver(case).run(2)
    assert not s.dvm.any()
    s2 = OracleSolver(case)
    z = np.zeros((s2.N, 3, 3)); zq = np.zeros((s2.N, 3))
    U = prim_to_U(case.W0)
    for _ in range(2):
        U = macro_solve(s2.geo, s2.bc_state, U, z, zq, s2.mu0, s2.omega, case.cfl, case.k_sub, case.macro_steps,
                        case.dt, U.copy())
    assert np.max(np.abs(U_to_prim(U) - s.W)) < 1e-14


def test_wall_kinetic_flux_of_gas_at_rest():
    """A Maxwellian at rest at the wall temperature meets a diffuse wall: the
    re-emitted half-range equals the incoming one, so the face distribution is
    that Maxwellian; the wall flux is the pressure rho T_w S, no mass, no energy."""
    vg = M.VelocityGrid((32, 32, 32), (-8, -8, -8), (8, 8, 8))
    rho, Tw = 1.7, 1.3
    f = M.maxwellian(rho, [0.0, 0.0, 0.0], Tw, vg.xi)
    Mw = M.maxwellian(1.0, [0.0, 0.0, 0.0], Tw, vg.xi)
    S = np.array([-0.6, -0.8, 0.0]) * 0.05
    F = K.wall_kinetic_flux(f, S, Mw, vg)
    assert abs(F[0]) < 1e-14
    assert np.allclose(F[1:4], rho * Tw * S, rtol=1e-10, atol=1e-14)
    assert abs(F[4]) < 1e-13


def test_wall_heat_flux_free_molecular_closed_form():
    """A DVM wall cell holding the Maxwellian of a gas at rest at T_g next to a
    diffuse wall at T_w: the emitted half carries rho_w M(0, T_w) with
    rho_w sqrt(T_w) = rho sqrt(T_g) (zero net mass flux), so the energy flux
    into the wall is the effusion difference rho sqrt(2/pi) sqrt(T_g) (T_g - T_w)
    per unit area (kinetic theory of free-molecular heat transfer)."""
    case = cylinder_case(Ma=2.0, Kn=0.1, n_r=4, n_theta=6, nv=(40, 40, 40), adaptive=False,
                         vbox=((-9, 9), (-9, 9), (-9, 9)), presolve_max_blocks=0)
    o = OracleSolver(case)
    o.initialise()
    Tg, rho = 1.3, 0.8
    for c in range(o.N):
        o.f[c] = M.maxwellian(rho, np.zeros(3), Tg, o.vg.xi)
    q = o.wall_heat_flux()
    Tw = case.mesh.bc_state[0][4]
    exact = rho * np.sqrt(2 / np.pi) * np.sqrt(Tg) * (Tg - Tw)
    walls = np.nonzero(q)[0]
    assert len(walls) == 6                       # the first radial layer
    # velocity quadrature across the xi.n = 0 kink: 0.05 % for faces aligned with the grid, 0.7 % oblique
    assert np.max(np.abs(q[walls] / exact - 1)) < 1e-2


def test_wall_loads_free_molecular_closed_forms():
    """A DVM wall cell holding the Maxwellian of a gas drifting at speed U
    along its wall face, next to a diffuse wall at T_w (kinetic theory of
    free-molecular surface loads): the incoming half carries, per unit area,
    the mass flux rho sqrt(T/2pi), the normal momentum rho T/2 and the
    tangential momentum rho U sqrt(T/2pi); the emitted half rho_w M(0, T_w)
    (rho_w sqrt(T_w) = rho sqrt(T)) adds the normal momentum
    rho sqrt(T T_w)/2 and no tangential momentum.  So the wall pressure is
    rho (T + sqrt(T T_w))/2, the shear rho U sqrt(T/2pi) along the drift,
    and the heat flux into the wall rho sqrt(T/2pi) (2 (T - T_w) + U^2/2)."""
    case = cylinder_case(Ma=2.0, Kn=0.1, n_r=4, n_theta=6, nv=(40, 40, 40), adaptive=False,
                         vbox=((-9, 9), (-9, 9), (-9, 9)), presolve_max_blocks=0)
    o = OracleSolver(case)
    o.initialise()
    Tg, rho, U = 1.3, 0.8, 0.6
    geo = o.geo
    Tw = case.mesh.bc_state[0][4]
    walls = np.nonzero(geo.bT == BC_WALL)[0]
    assert len(walls) == 6
    tang = {}
    for f_i in walls:
        c = geo.bC[f_i]
        n = geo.bn[f_i]
        t = np.array([-n[1], n[0], 0.0])          # along the wall face, in the flow plane
        tang[c] = (n, t)
        o.f[c] = M.maxwellian(rho, U * t, Tg, o.vg.xi)
    L = o.wall_loads()
    a = rho * np.sqrt(Tg / (2 * np.pi))
    for c, (n, t) in tang.items():
        q, p, tau = L[c, 0], L[c, 1], L[c, 2:5]
        # velocity quadrature across the xi.n = 0 kink (oblique faces): 1 %
        assert abs(p / (0.5 * rho * (Tg + np.sqrt(Tg * Tw))) - 1) < 1e-2
        assert np.linalg.norm(tau - a * U * t) < 1e-2 * a * U
        assert abs(np.dot(tau, n)) < 1e-12                 # shear is tangential by construction
        assert abs(q / (a * (2 * (Tg - Tw) + 0.5 * U * U)) - 1) < 1e-2
    others = np.setdiff1d(np.arange(o.N), list(tang))
    assert np.all(L[others] == 0.0)


def test_wall_loads_of_ns_cells_at_rest_at_wall_temperature():
    """An NS wall cell of a uniform gas at rest at T_w: the NSF wall flux has
    no viscous stress and no heat flux, so the wall pressure is rho T_w and
    the shear and heat flux vanish."""
    case = cylinder_case(Ma=2.0, Kn=0.1, n_r=4, n_theta=6, nv=(8, 8, 4), adaptive=False,
                         presolve_max_blocks=0)
    o = OracleSolver(case)
    o.initialise()
    Tw = case.mesh.bc_state[0][4]
    o.W[:] = [0.7, 0.0, 0.0, 0.0, Tw]
    o.dvm[:] = False
    L = o.wall_loads()
    walls = np.unique(o.geo.bC[o.geo.bT == BC_WALL])
    assert np.allclose(L[walls, 1], 0.7 * Tw, rtol=1e-13)
    assert np.max(np.abs(L[walls][:, [0, 2, 3, 4]])) < 1e-13


def test_constitutive_fields_are_the_kinetic_moments_at_the_half_step():
    """Eq. full_constitutive: sigma_NSF(W) + HoT is the kinetic stress and
    heat flux of f^{n+1/2} in DVM cells when evaluated at W = W^{n+1/2} (the
    NSF parts cancel), and the NSF values in NS cells."""
    case = cylinder_case(Ma=2.0, Kn=0.1, n_r=5, n_theta=8, nv=(10, 10, 6), adaptive=True, Kn_ref=0.05,
                         vbox=((-8, 8), (-8, 8), (-8, 8)), presolve_max_blocks=2)
    case.macro_steps = 10
    o = OracleSolver(case)
    o.initialise()
    o.step()
    assert 0 < o.dvm.sum() < o.N
    o.W = o.W_half.copy()
    sig, q = o.constitutive()
    sig_n, q_n = o.nsf_field(o.W_half)
    # the kinetic moments of f^{n+1/2}: f^{n+1} minus the correction of Eq. updatef
    W_new = o.W_history[-1]
    for c in np.nonzero(o.dvm)[0]:
        fh = o.f[c] - (o.vg.corrected_maxwellian(W_new[c, 0], W_new[c, 1:4], W_new[c, 4]) -
                       o.vg.corrected_maxwellian(o.W_half[c, 0], o.W_half[c, 1:4], o.W_half[c, 4]))
        _, _, _, sk, qk = o.vg.moments(fh)
        assert np.max(np.abs(sig[c] - sk)) < 1e-11 * max(1.0, np.max(np.abs(sk)))
        assert np.max(np.abs(q[c] - qk)) < 1e-11 * max(1.0, np.max(np.abs(qk)))
    ns = ~o.dvm
    assert np.array_equal(sig[ns], sig_n[ns]) and np.array_equal(q[ns], q_n[ns])
