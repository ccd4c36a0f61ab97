"""Pins of the reduced (xi_z-integrated) distributions of oracle.reduced (CPU
only).  Each reduced function is checked against the xi_z integral of the
pinned 3D function of oracle.model, done by brute force on a fine xi_z grid
(the midpoint rule on a Gaussian converges spectrally), and the reduced GSIS
iteration against the 3D one on the same 2D flow."""
import numpy as np
import pytest

from workloads import cylinder_case
from workloads.cases import VGrid
from oracle import model as M
from oracle.reduced import ReducedGrid
from oracle.gsis import OracleSolver

NX, NY = (14, 12)
BOX = ((-7.0, 8.0), (-6.5, 7.0))


def grids(nz=400, zmax=14.0):
    """The reduced grid and a 3D grid with the same (xi_x, xi_y) nodes and a
    fine xi_z axis; integrate(f3) gives (G, H) of a 3D distribution."""
    rg = ReducedGrid((NX, NY), (BOX[0][0], BOX[1][0]), (BOX[0][1], BOX[1][1]))
    g3 = M.VelocityGrid((NX, NY, nz), (BOX[0][0], BOX[1][0], -zmax), (BOX[0][1], BOX[1][1], zmax))
    dz = 2.0 * zmax / nz

    def integrate(f3):
        f = f3.reshape(nz, NY * NX)
        z = g3.axes[2][:, None]
        return np.concatenate([dz * f.sum(axis=0), dz * (z * z * f).sum(axis=0)])
    return rg, g3, integrate


STATE = dict(rho=1.3, u=np.array([0.4, -0.25, 0.0]), T=1.6)
SIGMA = np.array([[0.05, -0.02, 0.0], [-0.02, -0.03, 0.0], [0.0, 0.0, -0.02]])
Q = np.array([0.07, -0.04, 0.0])


def test_grid_layout_and_weights():
    rg = ReducedGrid((4, 3), (-1.0, -3.0), (1.0, 3.0))
    assert rg.nv == 24 and rg.n2 == 12
    assert np.isclose(rg.w, 0.5 * 2.0)
    v = 1 + 4 * 2          # node (ix=1, iy=2) of the G plane, x fastest
    assert np.allclose(rg.xi[v], [-0.25, 2.0, 0.0]) and rg.plane[v] == 0
    assert np.allclose(rg.xi[12 + v], rg.xi[v]) and rg.plane[12 + v] == 1
    assert np.all(rg.psi[12:, :4] == 0.0) and np.all(rg.psi[12:, 4] == 0.5)


@pytest.mark.parametrize("which", ["maxwellian", "shakhov", "grad13"])
def test_reduced_distributions_are_xi_z_integrals(which):
    """G = int f dxi_z and H = int xi_z^2 f dxi_z of the 3D Maxwellian,
    Shakhov reference and Grad-13 distribution of oracle.model."""
    rg, g3, integrate = grids()
    s = STATE
    if which == "maxwellian":
        f3, red = M.maxwellian(s["rho"], s["u"], s["T"], g3.xi), rg.maxwellian(s["rho"], s["u"], s["T"])
    elif which == "shakhov":
        f3 = M.reference_g0t(s["rho"], s["u"], s["T"], Q, g3.xi)
        red = rg.shakhov(s["rho"], s["u"], s["T"], Q)
    else:
        f3 = M.grad13(s["rho"], s["u"], s["T"], SIGMA, Q, g3.xi)
        red = rg.grad13(s["rho"], s["u"], s["T"], SIGMA, Q)
    ref = integrate(f3)
    assert np.max(np.abs(red - ref)) < 1e-12 * np.max(np.abs(ref))


def test_reduced_moments_equal_3d_moments():
    """Density, velocity, temperature, stress (with sigma_zz from H) and heat
    flux (with the xi_z^2 part from H) of the reduced form of a Grad-13
    distribution equal the 3D moments of that distribution."""
    rg, g3, integrate = grids()
    s = STATE
    f3 = M.grad13(s["rho"], s["u"], s["T"], SIGMA, Q, g3.xi)
    r3 = M.moments(f3, g3)
    rr = rg.moments(integrate(f3))
    for a, b in zip(rr, r3):
        assert np.max(np.abs(np.asarray(a) - np.asarray(b))) < 1e-11 * max(1.0, np.max(np.abs(b)))
    assert np.allclose(rg.conserved(integrate(f3)), M.conserved(f3, g3), rtol=1e-12, atol=1e-14)
    assert np.allclose(rg.heat_flux_about(integrate(f3), [0.1, 0.2, 0.0]),
                       M.heat_flux_about(f3, [0.1, 0.2, 0.0], g3), rtol=1e-11, atol=1e-14)


def test_reduced_conservation_correction():
    """The corrected reduced Maxwellian and Shakhov reference carry exactly
    the conserved moments of their state (mass, x/y momentum, energy with the
    xi_z^2 part from H), and the correction is the xi_z integral of the 3D
    correction: on a 3D grid with the same (xi_x, xi_y) nodes and a fine
    xi_z axis the 3D corrected distribution integrates to the reduced one."""
    rg, g3, integrate = grids()
    s = STATE
    U = M.conserved_from_primitive(s["rho"], s["u"], s["T"])
    for red, f3 in ((rg.corrected_maxwellian(s["rho"], s["u"], s["T"]),
                     M.corrected_maxwellian(s["rho"], s["u"], s["T"], g3)),
                    (rg.corrected_shakhov(s["rho"], s["u"], s["T"], Q),
                     M.corrected_shakhov(s["rho"], s["u"], s["T"], Q, g3))):
        assert np.allclose(rg.conserved(red), U, rtol=1e-13, atol=1e-14)
        ref = integrate(f3)
        assert np.max(np.abs(red - ref)) < 1e-10 * np.max(np.abs(ref))
    # the correction is not trivial on this coarse (xi_x, xi_y) grid
    raw = rg.maxwellian(s["rho"], s["u"], s["T"])
    assert np.max(np.abs(rg.conserved(raw) - U)) > 1e-6


def test_reduced_gsis_matches_3d_gsis_on_a_2d_flow(monkeypatch):
    """The cylinder (all kinetic, started from the NS presolve) with the
    reduced distributions and with a 3D velocity grid whose xi_z axis (24
    nodes on [-12, 12]) resolves the Gaussians: with the first-order face
    values the kinetic step is linear in f, so the reduced iteration is the
    xi_z integral of the 3D one, and the macroscopic states after two GSIS
    iterations agree to the xi_z quadrature error, as does the reduced VDF
    with the xi_z integral of the 3D VDF.  (The limited second-order slopes
    are nonlinear in f: the reduced scheme limits the stored G and H, which
    is a discretisation of its own, not the xi_z integral of limiting f.)"""
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
    o3 = OracleSolver(c3).run(2)
    orr = OracleSolver(cr).run(2)
    assert np.max(np.abs(orr.W - o3.W)) < 1e-8 * np.max(np.abs(o3.W))
    dz = 24.0 / nz
    z = o3.vg.axes[2]
    n2 = 14 * 12
    for cell in (0, 7, 30):
        f = o3.f[cell].reshape(nz, n2)
        ref = np.concatenate([dz * f.sum(axis=0), dz * ((z * z)[:, None] * f).sum(axis=0)])
        assert np.max(np.abs(orr.f[cell] - ref)) < 1e-8 * np.max(np.abs(ref))
