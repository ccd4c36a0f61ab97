"""Reduced velocity distributions for 2D flows (oracle; test infrastructure only).

In a flow with no dependence on z and u_z = 0 (the cylinder), the kinetic
equation can be integrated over xi_z: the paper's 2D runs store two reduced
functions on a (xi_x, xi_y) grid instead of f on a 3D grid (Sec. 3.3, and the
70 x 60 velocity grid of Sec. 4.2):

    G(xi_x, xi_y) = int f dxi_z,        H(xi_x, xi_y) = int xi_z^2 f dxi_z.

Both obey the same transport (xi_z never enters a face flux of a 2D mesh), and
every quantity the method needs follows from them: mass, x/y momentum and
xi_z-free moments from G; the xi_z^2 parts of energy, P_zz and the heat flux
from H.  Reference distributions are the xi_z integrals of the 3D ones of
oracle.model, written out here by hand with the Gaussian moments
int xi_z^{2k} exp(-xi_z^2/(2T)) dxi_z / sqrt(2 pi T) = 1, T, 3T^2 for k = 0, 1, 2
(and zero for odd powers):

    M2 = rho/(2 pi T) exp(-c^2/(2T)),   c = (xi_x - u_x, xi_y - u_y)
    Maxwellian:  G = M2,  H = T M2
    Shakhov (alpha = 2/(15 T p), q.c = q_x c_x + q_y c_y):
        G = M2 [1 + alpha q.c (c^2/(2T) - 2)]
        H = T M2 [1 + alpha q.c (c^2/(2T) - 1)]
    Grad-13 (s = sigma_xx c_x^2 + 2 sigma_xy c_x c_y + sigma_yy c_y^2):
        G = M2 [1 + (s + T sigma_zz)/(2 rho T^2) + q.c/(rho T^2) ((c^2 + T)/(5T) - 1)]
        H = T M2 [1 + (s + 3T sigma_zz)/(2 rho T^2) + q.c/(rho T^2) ((c^2 + 3T)/(5T) - 1)]

A reduced VDF is one array over the nodes of both planes: the G values of the
n_x n_y grid nodes, then the H values (plane index = node // (n_x n_y)).  The
quadrature weight is dxi_x dxi_y.
"""
import numpy as np


class ReducedGrid:
    """Uniform midpoint (xi_x, xi_y) grid carrying the two reduced planes.

    xi: [nv, 3] node velocities for the transport (xi_z = 0 on both planes);
    plane: [nv] 0 for G, 1 for H; psi: [nv, 5] weights of the conserved
    quantities (mass, x/y/z momentum, energy) per node, so that
    sum_v w psi_v f_v = (rho, rho u, rho E)."""

    reduced = True

    def __init__(self, n, lo, hi):
        self.n = (int(n[0]), int(n[1]), 2)
        self.lo = (float(lo[0]), float(lo[1]))
        self.hi = (float(hi[0]), float(hi[1]))
        self.axes = []
        for d in range(2):
            h = (self.hi[d] - self.lo[d]) / self.n[d]
            self.axes.append(self.lo[d] + (np.arange(self.n[d]) + 0.5) * h)
        self.w = float(np.prod([(self.hi[d] - self.lo[d]) / self.n[d] for d in range(2)]))
        Y, X = np.meshgrid(self.axes[1], self.axes[0], indexing="ij")
        x2 = np.stack([X.ravel(), Y.ravel()], axis=1)            # [n2, 2], x fastest
        self.n2 = x2.shape[0]
        self.nv = 2 * self.n2
        self.plane = np.repeat([0, 1], self.n2)
        self.xi = np.zeros((self.nv, 3))
        self.xi[:, :2] = np.concatenate([x2, x2])
        g = (self.plane == 0).astype(np.float64)
        h = 1.0 - g
        e2 = 0.5 * np.sum(self.xi[:, :2] ** 2, axis=1)
        self.psi = np.stack([g, g * self.xi[:, 0], g * self.xi[:, 1], np.zeros(self.nv), g * e2 + 0.5 * h], axis=1)

    # ---------------------------------------------------------------- distributions
    def _planes(self, rho, u, T):
        c = self.xi[:, :2] - np.asarray(u)[None, :2]
        c2 = np.sum(c * c, axis=1)
        M2 = rho / (2.0 * np.pi * T) * np.exp(-c2 / (2.0 * T))
        scale = np.where(self.plane == 0, 1.0, T)
        return c, c2, M2, scale

    def maxwellian(self, rho, u, T):
        _, _, M2, scale = self._planes(rho, u, T)
        return scale * M2

    def shakhov(self, rho, u, T, q):
        c, c2, M2, scale = self._planes(rho, u, T)
        alpha = 2.0 / (15.0 * T * rho * T)
        qc = c @ np.asarray(q)[:2]
        k = np.where(self.plane == 0, -2.0, -1.0)
        return scale * M2 * (1.0 + alpha * qc * (c2 / (2.0 * T) + k))

    def grad13(self, rho, u, T, sigma, q):
        c, c2, M2, scale = self._planes(rho, u, T)
        S = np.asarray(sigma)
        s = S[0, 0] * c[:, 0] ** 2 + 2.0 * S[0, 1] * c[:, 0] * c[:, 1] + S[1, 1] * c[:, 1] ** 2
        zz = np.where(self.plane == 0, T, 3.0 * T)          # xi_z^2 -> T on G, 3T on H
        qc = c @ np.asarray(q)[:2]
        rT2 = rho * T * T
        return scale * M2 * (1.0 + (s + zz * S[2, 2]) / (2.0 * rT2) + qc / rT2 * ((c2 + zz) / (5.0 * T) - 1.0))

    # ---------------------------------------------------------------- moments
    def conserved(self, f):
        """(rho, rho u, rho E) = sum_v w psi_v f_v."""
        return self.w * (self.psi.T @ f)

    def heat_flux_about(self, f, u):
        """q = 1/2 int c (c^2 + xi_z^2) f: 1/2 sum w c (c^2 G + H) (q_z = 0)."""
        c = self.xi[:, :2] - np.asarray(u)[None, :2]
        c2 = np.sum(c * c, axis=1)
        wgt = np.where(self.plane == 0, c2, 1.0)
        q = 0.5 * self.w * (c.T @ (wgt * f))
        return np.array([q[0], q[1], 0.0])

    def moments(self, f):
        """rho, u, T, traceless stress, heat flux (about the distribution's own
        velocity): P_ij from G for i, j in {x, y}, P_zz = sum w H."""
        U = self.conserved(f)
        rho = U[0]
        u = np.array([U[1] / rho, U[2] / rho, 0.0])
        c = self.xi[:, :2] - u[None, :2]
        g = self.plane == 0
        P = np.zeros((3, 3))
        P[:2, :2] = self.w * np.einsum("vi,vj,v->ij", c[g], c[g], f[g])
        P[2, 2] = self.w * np.sum(f[~g])
        T = np.trace(P) / (3.0 * rho)
        sigma = P - np.trace(P) / 3.0 * np.eye(3)
        return rho, u, T, sigma, self.heat_flux_about(f, u)

    # ---------------------------------------------------------------- conservation correction
    def conservation_correct(self, base, M, U):
        """The xi_z integral of the 3D correction of oracle.model
        (base + M (a0 + a.xi + a4 |xi|^2); a_z = 0 in a flow symmetric in
        xi_z): base + a0 M + a_x xi_x M + a_y xi_y M + a4 (xi_x^2 + xi_y^2 + k T) M,
        with k = 1 on G and 3 on H (the reduced M carries T on H, so
        M k T is the xi_z^2 part), and (a0, a_x, a_y, a4) from the 4 x 4
        system that makes mass, x/y momentum and energy exact.  T is the
        Maxwellian's own temperature, read from its planes."""
        g = self.plane == 0
        T = np.sum(M[~g]) / np.sum(M[g])
        k = np.where(g, 1.0, 3.0)
        x2 = np.sum(self.xi[:, :2] ** 2, axis=1)
        phi = np.stack([M, self.xi[:, 0] * M, self.xi[:, 1] * M, (x2 + k * T) * M], axis=1)
        psi = self.psi[:, [0, 1, 2, 4]]
        A = self.w * (psi.T @ phi)
        rhs = np.asarray(U)[[0, 1, 2, 4]] - self.w * (psi.T @ base)
        a = np.linalg.solve(A, rhs)
        return base + phi @ a

    def corrected_maxwellian(self, rho, u, T):
        M = self.maxwellian(rho, u, T)
        return self.conservation_correct(M, M, _cons(rho, u, T))

    def corrected_shakhov(self, rho, u, T, q):
        return self.conservation_correct(self.shakhov(rho, u, T, q), self.maxwellian(rho, u, T), _cons(rho, u, T))


def _cons(rho, u, T):
    u = np.asarray(u)
    return np.array([rho, rho * u[0], rho * u[1], rho * u[2], rho * (1.5 * T + 0.5 * np.dot(u, u))])
