"""Workload descriptors: mesh + velocity grid + initial macroscopic state + run
parameters, for the shock, cylinder, sphere and shock-batch workloads.

Non-dimensional units throughout: free-stream (upstream) density, temperature
and gas constant are 1, so sqrt(R T_inf) = 1 and the most-probable speed is
sqrt(2).  The length unit is the cylinder/sphere diameter, or the upstream mean
free path for the 1D shock.  Only geometry and initial fields live here; the
solver parameters (Kn, viscosity index, ...) are plain numbers handed to both
the oracle and the CUDA path.
"""
from dataclasses import dataclass, field
import numpy as np

from .meshes import Mesh, cartesian_1d, cylinder_ogrid, sphere_ogrid

GAMMA = 5.0 / 3.0      # monatomic gas
OMEGA = 0.81           # viscosity index of the monatomic workloads


@dataclass
class VGrid:
    """Uniform midpoint velocity grid: n[d] nodes on [lo[d], hi[d]] per axis.
    reduced: the xi_z axis is integrated out (2D flows): two reduced
    distributions on the n[0] x n[1] grid, n[2] / lo[2] / hi[2] unused."""
    n: tuple
    lo: tuple
    hi: tuple
    reduced: bool = False

    @property
    def nv(self):
        if self.reduced:
            return int(2 * self.n[0] * self.n[1])
        return int(self.n[0] * self.n[1] * self.n[2])


@dataclass
class Case:
    name: str
    mesh: Mesh
    vgrid: VGrid
    W0: np.ndarray              # [ncell, 5] initial (rho, ux, uy, uz, T), flat cell order
    Kn: float
    omega: float = OMEGA
    adaptive: bool = False
    Kn_ref: float = 0.0
    adapt_every: int = 5
    wall_layers: int = 2
    macro_steps: int = 400
    cfl: float = 5.0
    k_sub: int = 2
    iterations: int = 60
    tol: float = 1e-6
    presolve_max_blocks: int = 0   # NS presolve: blocks of macro_steps pseudo-steps
    dt: float = 0.0                # time step of Eq. macro; 0 means the steady form (dt -> inf)
    relax: float = 1.0             # weight of the synthetic correction of W (1 = plain scheme)
    extra: dict = field(default_factory=dict)


def rankine_hugoniot(Ma, gamma=GAMMA):
    """Downstream (rho, u, T) of a normal shock for upstream rho=T=1, u=Ma*sqrt(gamma)."""
    M2 = Ma * Ma
    r = (gamma + 1.0) * M2 / ((gamma - 1.0) * M2 + 2.0)
    p = (2.0 * gamma * M2 - (gamma - 1.0)) / (gamma + 1.0)
    u1 = Ma * np.sqrt(gamma)
    return r, u1 / r, p / r


def shock_1d_case(Ma=2.0, n_cells=200, half_width=25.0, nv=(48, 24, 24), vmax=6.0 * np.sqrt(2.0),
                  delta=2.0, iterations=60, macro_steps=50, cfl=100.0, k_sub=4, dt=1.0):
    """Normal shock structure: upstream mean free path = length unit (Kn = 1).

    Initial state: tanh blend of the Rankine-Hugoniot end states with width
    delta; both ends are far-field boundaries with those end states.  The
    synthetic solve keeps a finite time step dt: a standing shock between two
    fixed end states can translate freely, and the time term holds the mass in
    the domain fixed up to the boundary fluxes.  50 pseudo-steps with 4
    relaxation sweeps per GSIS iteration: the residual history is the same as
    with 200 steps and 8 sweeps.
    """
    r2, u2, T2 = rankine_hugoniot(Ma)
    u1 = Ma * np.sqrt(GAMMA)
    W1 = np.array([1.0, u1, 0.0, 0.0, 1.0])
    W2 = np.array([r2, u2, 0.0, 0.0, T2])
    mesh = cartesian_1d(n_cells, -half_width, half_width, W1, W2)
    x = mesh.flat(mesh.centers)[:, 0]
    s = 0.5 * (1.0 + np.tanh(x / delta))
    W0 = W1[None, :] + (W2 - W1)[None, :] * s[:, None]
    vg = VGrid(tuple(nv), (-vmax,) * 3, (vmax,) * 3)
    return Case(f"shock1d_Ma{Ma:g}_{n_cells}", mesh, vg, np.ascontiguousarray(W0), Kn=1.0,
                iterations=iterations, macro_steps=macro_steps, cfl=cfl, k_sub=k_sub, dt=dt,
                extra={"W1": W1, "W2": W2, "Ma": Ma})


def cylinder_case(Ma=5.0, Kn=0.01, n_r=128, n_theta=128, nv=(48, 48, 24),
                  vbox=((-14.0, 14.0), (-12.0, 12.0), (-12.0, 12.0)), wall_T=2.0,
                  adaptive=True, Kn_ref=0.01, r_out=5.0, first_cell_mfp=0.1,
                  macro_steps=100, cfl=5.0, k_sub=2, iterations=60, presolve_max_blocks=200, relax=0.7,
                  reduced=False):
    """Hypersonic flow past a cylinder of unit diameter on a body-fitted O-grid.

    First radial cell = first_cell_mfp free-stream mean free paths (= Kn * D).
    The initial field is the uniform free stream; runs start with a
    Navier-Stokes presolve.  The synthetic correction is under-relaxed (relax)
    against the entropy mode of the stagnation region.  100 pseudo-steps of
    the synthetic solve per GSIS iteration: the residual history of the
    cylinder is the same with 50 to 400.  reduced: xi_z integrated out (two
    reduced distributions on the nv[0] x nv[1] grid of the first two axes of
    vbox; nv[2] and vbox[2] unused).
    """
    u = Ma * np.sqrt(GAMMA)
    Winf = np.array([1.0, u, 0.0, 0.0, 1.0])
    mesh = cylinder_ogrid(n_r, n_theta, 0.5, r_out, first_cell_mfp * Kn, wall_T, Winf)
    W0 = np.tile(Winf, (mesh.ncell, 1))
    if reduced:
        vg = VGrid((nv[0], nv[1], 2), (vbox[0][0], vbox[1][0], 0.0), (vbox[0][1], vbox[1][1], 1.0), reduced=True)
    else:
        vg = VGrid(tuple(nv), tuple(b[0] for b in vbox), tuple(b[1] for b in vbox))
    return Case(f"cylinder_Ma{Ma:g}_Kn{Kn:g}_{n_r}x{n_theta}", mesh, vg, W0, Kn=Kn,
                adaptive=adaptive, Kn_ref=Kn_ref, macro_steps=macro_steps, cfl=cfl, k_sub=k_sub,
                iterations=iterations, presolve_max_blocks=presolve_max_blocks, relax=relax,
                extra={"Winf": Winf, "Ma": Ma, "wall_T": wall_T})


def sphere_case(Ma=5.0, Kn=0.005, n_r=96, n_pol=64, n_az=64, nv=(48, 48, 48),
                vbox=((-14.0, 14.0), (-12.0, 12.0), (-12.0, 12.0)), wall_T=2.0,
                adaptive=True, Kn_ref=0.01, r_out=5.0, first_cell_mfp=0.1,
                macro_steps=100, cfl=5.0, k_sub=2, iterations=60, presolve_max_blocks=20, relax=0.7):
    """Hypersonic flow past a sphere of unit diameter on a spherical O-grid
    (under-relaxed synthetic correction, as for the cylinder).  The NS
    presolve is cut at 20 blocks (2,000 pseudo-steps): on the full 96x64x64
    mesh a wake mode grows in the steady NS iteration after ~35 blocks
    (Re ~ 1,600 at Kn = 0.005), while the shock layer is in place after 20."""
    u = Ma * np.sqrt(GAMMA)
    Winf = np.array([1.0, u, 0.0, 0.0, 1.0])
    mesh = sphere_ogrid(n_r, n_pol, n_az, 0.5, r_out, first_cell_mfp * Kn, wall_T, Winf)
    W0 = np.tile(Winf, (mesh.ncell, 1))
    vg = VGrid(tuple(nv), tuple(b[0] for b in vbox), tuple(b[1] for b in vbox))
    return Case(f"sphere_Ma{Ma:g}_Kn{Kn:g}_{n_r}x{n_pol}x{n_az}", mesh, vg, W0, Kn=Kn,
                adaptive=adaptive, Kn_ref=Kn_ref, macro_steps=macro_steps, cfl=cfl, k_sub=k_sub,
                iterations=iterations, presolve_max_blocks=presolve_max_blocks, relax=relax,
                extra={"Winf": Winf, "Ma": Ma, "wall_T": wall_T})


def batch_vgrid_n(Ma):
    """Velocity nodes per axis for a shock of Mach Ma: 24 at Ma=1.5 growing to
    64 at Ma=8, rounded to a multiple of 8."""
    n = 8 * int(round((24.0 + 40.0 * (Ma - 1.5) / 6.5) / 8.0))
    return int(min(64, max(24, n)))


def batch_vgrid_half_width(Ma):
    """Half-width of the velocity box for a shock of Mach Ma, in units of
    sqrt(R T1): covers the upstream speed plus 4 thermal widths of either end,
    scaled so that Ma=2 gives 6 most-probable speeds."""
    r2, u2, T2 = rankine_hugoniot(Ma)
    u1 = Ma * np.sqrt(GAMMA)
    L = max(u1 + 4.0, 4.0 * np.sqrt(T2))
    r2b, u2b, T2b = rankine_hugoniot(2.0)
    L2 = max(2.0 * np.sqrt(GAMMA) + 4.0, 4.0 * np.sqrt(T2b))
    return L * (6.0 * np.sqrt(2.0)) / L2


def shock_batch_cases(n=64, seed=2501, ma_range=(1.5, 8.0), cells_range=(100, 800), iterations=60,
                      macro_steps=50):
    """Seeded batch of independent 1D shocks with uneven meshes and velocity grids."""
    rng = np.random.default_rng(seed)
    cases = []
    for b in range(n):
        Ma = float(rng.uniform(*ma_range))
        nc = int(rng.integers(cells_range[0], cells_range[1] + 1))
        nvx = batch_vgrid_n(Ma)
        L = batch_vgrid_half_width(Ma)
        c = shock_1d_case(Ma=Ma, n_cells=nc, half_width=nc / 8.0, nv=(nvx, nvx, nvx), vmax=L,
                          iterations=iterations, macro_steps=macro_steps)
        c.name = f"batch{b:02d}_Ma{Ma:.3f}_{nc}"
        c.extra["vdf_dtype"] = "f32" if b % 2 == 0 else "bf16"
        cases.append(c)
    return cases
