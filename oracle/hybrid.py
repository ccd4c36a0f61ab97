"""Non-uniform (hybrid) velocity grid for the oracle (test infrastructure only).

The paper's three-dimensional runs (Secs. 4.3, 4.4) discretise velocity space
with cells of varying size instead of the uniform grid of Sec. 4.2; it does
not print their construction.  The reading taken here: a tensor product of
three non-uniform 1D partitions of [lo, hi], each velocity cell represented
by its midpoint with the cell's volume as quadrature weight,

    xi_v = (x_i, y_j, z_k),   w_v = dx_i dy_j dz_k,

the natural generalisation of the uniform midpoint rule of oracle.model
(which it reproduces when every partition is uniform).  Refining near the
bulk velocity and coarsening in the tails is what makes such grids cheaper
than a uniform one for hypersonic flows.

The class offers the same methods as oracle.model.VelocityGrid (the GSIS
driver of oracle.gsis calls only these), written with per-node weights.
For the routines of oracle.kinetic it presents itself like the reduced grid:
`reduced` is set, the scalar weight `w` is 1 and the weights sit in the
rows of `psi` (mass, momentum, energy per node), which is how those routines
weigh wall fluxes and the diffuse-wall density.
"""
import numpy as np

from . import model as M


def partition(edges):
    """Midpoints and widths of the 1D cells between consecutive edges."""
    e = np.asarray(edges, dtype=np.float64)
    assert e.ndim == 1 and len(e) >= 2 and np.all(np.diff(e) > 0)
    return 0.5 * (e[1:] + e[:-1]), np.diff(e)


def stretched_edges(lo, hi, n, centre, ratio):
    """n cells on [lo, hi] whose widths grow geometrically by `ratio` per cell
    away from `centre` (ratio = 1: uniform); the edges include lo, centre and
    hi when centre lies inside."""
    if ratio == 1.0:
        return np.linspace(lo, hi, n + 1)
    nl = max(1, int(round(n * (centre - lo) / (hi - lo))))
    nr = max(1, n - nl)

    def side(length, m):
        w = ratio ** np.arange(m)
        return np.concatenate([[0.0], np.cumsum(w)]) * (length / np.sum(w))
    left = centre - side(centre - lo, nl)[::-1]
    right = centre + side(hi - centre, nr)
    return np.concatenate([left, right[1:]])


class HybridGrid:
    """Tensor product of three non-uniform midpoint partitions given by their
    cell edges; node v = ix + nx (iy + ny iz) (x fastest)."""

    reduced = True   # oracle.kinetic: weights in psi, scalar w = 1

    def __init__(self, edges_x, edges_y, edges_z):
        self.axes, self.widths = [], []
        for e in (edges_x, edges_y, edges_z):
            c, h = partition(e)
            self.axes.append(c)
            self.widths.append(h)
        self.n = tuple(len(a) for a in self.axes)
        Z, Y, X = np.meshgrid(self.axes[2], self.axes[1], self.axes[0], indexing="ij")
        self.xi = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
        WZ, WY, WX = np.meshgrid(self.widths[2], self.widths[1], self.widths[0], indexing="ij")
        self.wv = (WX * WY * WZ).ravel()
        self.nv = self.xi.shape[0]
        self.w = 1.0
        x2 = np.sum(self.xi * self.xi, axis=1)
        self.psi = self.wv[:, None] * np.stack([np.ones(self.nv), self.xi[:, 0], self.xi[:, 1], self.xi[:, 2],
                                                0.5 * x2], axis=1)

    # ---------------------------------------------------------------- distributions (oracle.model)
    def maxwellian(self, rho, u, T):
        return M.maxwellian(rho, u, T, self.xi)

    def shakhov(self, rho, u, T, q):
        return M.reference_g0t(rho, u, T, q, self.xi)

    def grad13(self, rho, u, T, sigma, q):
        return M.grad13(rho, u, T, sigma, q, self.xi)

    # ---------------------------------------------------------------- moments (Eq. getmoment)
    def conserved(self, f):
        """(rho, rho u, rho E) = sum_v w_v (1, xi, |xi|^2/2) f_v."""
        return self.psi.T @ f

    def moments(self, f):
        rho, u, T = M.primitive_from_conserved(self.conserved(f))
        c = self.xi - u[None, :]
        c2 = np.sum(c * c, axis=1)
        wf = self.wv * f
        P = np.einsum("vi,vj,v->ij", c, c, wf)
        sigma = P - np.trace(P) / 3.0 * np.eye(3)
        q = 0.5 * (c.T @ (c2 * wf))
        return rho, u, T, sigma, q

    def heat_flux_about(self, f, u):
        c = self.xi - np.asarray(u)[None, :]
        return 0.5 * (c.T @ (np.sum(c * c, axis=1) * self.wv * f))

    # ---------------------------------------------------------------- conservation correction
    def conservation_correct(self, base, Mx, U):
        """The Lagrange-multiplier correction of oracle.model.conservation_correct
        with per-node weights: base + M (a0 + a.xi + a4 |xi|^2), a from
        sum_v w_v psi_v phi_v^T M_v a = U - sum_v w_v psi_v base_v."""
        x2 = np.sum(self.xi * self.xi, axis=1)
        phi = np.stack([np.ones(self.nv), self.xi[:, 0], self.xi[:, 1], self.xi[:, 2], x2], axis=1)
        A = np.einsum("va,vb,v->ab", self.psi, phi, Mx)
        a = np.linalg.solve(A, np.asarray(U) - self.psi.T @ base)
        return base + Mx * (phi @ a)

    def corrected_maxwellian(self, rho, u, T):
        Mx = self.maxwellian(rho, u, T)
        return self.conservation_correct(Mx, Mx, M.conserved_from_primitive(rho, u, T))

    def corrected_shakhov(self, rho, u, T, q):
        return self.conservation_correct(self.shakhov(rho, u, T, q), self.maxwellian(rho, u, T),
                                         M.conserved_from_primitive(rho, u, T))
