"""Kinetic (discrete-velocity) step of Sec. 3.1 in plain FP64 numpy (oracle;
test infrastructure only).

The paper writes the step as an implicit finite-volume update,
(f^{n+1/2} - f^n)/dt + (1/V_i) sum_j xi_n f_ij^{n+1/2} S_ij = (g^n - f^{n+1/2})/tau^n,
with second-order face values and the details left to its references.  The
reading taken (stated once, used everywhere):

* steady form, dt -> infinity;
* face value f_ij: upwind cell value plus half its limited index-space slope,
  slope = minmod(f_c - f_{c-d}, f_{c+d} - f_c) when both neighbours along d
  are DVM cells, 0 otherwise (first order next to boundaries and NS cells);
* the outgoing part of the upwind cell value is implicit, every other term
  (own slope, neighbour face values) takes the latest value available;
* one symmetric Gauss-Seidel pass: backward over hyperplanes h = i + j + k
  (towards the low-index side, where the body walls of the O-grids lie),
  then forward.  Molecules travelling towards a wall are swept first, the
  wall density is then taken from their outgoing flux, and the re-emitted
  molecules are swept out in the same kinetic step.  Cells of one hyperplane
  never appear in each other's stencil, so the order inside a hyperplane does
  not matter.

Boundary and interface face values for incoming velocities (xi . n < 0):
far field -> conservation-corrected Maxwellian M~ of the boundary state (so a
uniform stream is an exact fixed point); diffuse wall -> rho_w M(0, T_w) with
rho_w from zero net mass flux through the face, using the outgoing half of the
cell's latest f (its value before its own update in the current pass, like
every other explicit term); NS neighbour -> Grad-13 VDF of Eq. G13_VDF from the
neighbour's W and NSF stress/heat flux, conservation-corrected to its W.
"""
import numpy as np

from .mesh import BC_NONE, BC_FARFIELD, BC_WALL


def minmod(a, b):
    return np.where((a > 0) & (b > 0), np.minimum(a, b),
                    np.where((a < 0) & (b < 0), np.maximum(a, b), 0.0))


class KineticInputs:
    """Per-step inputs frozen at the start of the kinetic step."""

    def __init__(self, gt, tau, ghost, ff_maxwellian, wall_maxwellian):
        self.gt = gt                    # {cell: g~ vector} for DVM cells
        self.tau = tau                  # {cell: tau}
        self.ghost = ghost              # {cell: Grad-13 VDF} for NS cells next to DVM cells
        self.ff = ff_maxwellian         # {bc_side: Maxwellian of the far-field state}
        self.mw = wall_maxwellian       # {bc_side: M(0, T_w) with unit density}


def wall_density(f_cell, S_out, Mw, vg):
    """Diffuse-wall density: the emitted half-range rho_w M_w carries the mass
    that the outgoing half of f brings to the face (zero net mass flux).  On
    the reduced grid only the G plane carries mass."""
    xn = vg.xi @ S_out
    out = xn > 0
    if vg.reduced:
        m = vg.psi[:, 0]
        return np.sum(np.where(out, xn * f_cell * m, 0.0)) / np.sum(np.where(~out, -xn * Mw * m, 0.0))
    num = np.sum(np.where(out, xn * f_cell, 0.0))
    den = np.sum(np.where(~out, -xn * Mw, 0.0))
    return num / den


def wall_kinetic_flux(f_cell, S_out, Mw, vg):
    """Flux of (mass, momentum, energy) through a diffuse-wall face carried by
    the face distribution: the cell's f for outgoing velocities (xi . S > 0)
    and rho_w M_w, with rho_w from zero net mass flux of that same f, for the
    incoming ones: sum_v w (xi . S) (1, xi, |xi|^2/2) f_face."""
    xi = vg.xi
    xn = xi @ S_out
    rho_w = wall_density(f_cell, S_out, Mw, vg)
    face = np.where(xn > 0, f_cell, rho_w * Mw)
    g = vg.w * xn * face
    if vg.reduced:   # per-plane weights of mass, momentum and energy
        return g @ vg.psi
    return np.array([np.sum(g), g @ xi[:, 0], g @ xi[:, 1], g @ xi[:, 2],
                     np.sum(g * 0.5 * np.sum(xi * xi, axis=1))])


def slope(topo, f, dvm, c, d):
    cm = topo.step(c, d, -1)
    cp = topo.step(c, d, +1)
    if cm < 0 or cp < 0 or not dvm[cm] or not dvm[cp]:
        return 0.0
    return minmod(f[c] - f[cm], f[cp] - f[c])


def update_cell(topo, vg, f, dvm, inp, c):
    """Solve the implicit first-order part for cell c at every velocity."""
    xi = vg.xi
    V = topo.vol[c]
    tau = inp.tau[c]
    den = np.full(vg.nv, 1.0 / tau)
    num = inp.gt[c] / tau
    for sd in topo.sides[c]:
        if sd.nbr < 0 and sd.bc == BC_NONE:
            continue
        xn = (xi @ sd.S_out) / V
        out = xn > 0
        sc = slope(topo, f, dvm, c, sd.d)
        den = den + np.where(out, xn, 0.0)
        num = num - np.where(out, xn * (sd.s * 0.5) * sc, 0.0)
        if sd.nbr >= 0:
            if dvm[sd.nbr]:
                fin = f[sd.nbr] - (sd.s * 0.5) * slope(topo, f, dvm, sd.nbr, sd.d)
            else:
                fin = inp.ghost[sd.nbr]
        elif sd.bc == BC_FARFIELD:
            fin = inp.ff[sd.bc_side]
        elif sd.bc == BC_WALL:
            fin = wall_density(f[c], sd.S_out, inp.mw[sd.bc_side], vg) * inp.mw[sd.bc_side]
        else:
            raise ValueError("unknown boundary")
        num = num - np.where(out, 0.0, xn * fin)
    f[c] = num / den


def sweep(topo, vg, f, dvm, inp):
    """One backward and one forward Gauss-Seidel pass over the DVM cells in
    hyperplane order; f is updated in place (rows of NS cells are untouched)."""
    cells = [c for c in range(topo.ncell) if dvm[c]]
    cells.sort(key=lambda c: (topo.hyperplane(c), c))
    for c in reversed(cells):
        update_cell(topo, vg, f, dvm, inp, c)
    for c in cells:
        update_cell(topo, vg, f, dvm, inp, c)
    return f

