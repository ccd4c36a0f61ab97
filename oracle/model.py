"""Gas model of Sec. 2 in plain FP64 numpy (oracle; test infrastructure only).

Units: R = 1, so p = rho*T and sqrt(R T) = sqrt(T).  Monatomic reduction
(d_r = 0, A_tt = 2/3): the rotational VDF f1 vanishes, g_0r = g_0t and the
relaxation model becomes the Shakhov model with Pr = 2/3.  The general
two-temperature relations that the reduction rests on are kept here too
(conductivities from the A matrix, the q0/q1 mixing) so that tests can check
the reduction itself.
"""
import numpy as np

GAMMA = 5.0 / 3.0


# --------------------------------------------------------------------------- velocity grid
class VelocityGrid:
    """Uniform midpoint quadrature on a truncated box (Sec. 4.2: the velocity
    space is 'uniformly discretized').  Node k of axis d sits at
    lo + (k + 1/2) (hi - lo)/n; every node carries the weight prod_d (hi-lo)/n.
    Flat index v = ix + nx*(iy + ny*iz)."""

    def __init__(self, n, lo, hi):
        self.n = tuple(int(a) for a in n)
        self.lo = tuple(float(a) for a in lo)
        self.hi = tuple(float(a) for a in hi)
        self.axes = []
        for d in range(3):
            h = (self.hi[d] - self.lo[d]) / self.n[d]
            self.axes.append(self.lo[d] + (np.arange(self.n[d]) + 0.5) * h)
        self.w = float(np.prod([(self.hi[d] - self.lo[d]) / self.n[d] for d in range(3)]))
        Z, Y, X = np.meshgrid(self.axes[2], self.axes[1], self.axes[0], indexing="ij")
        self.xi = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)   # [Nv, 3]
        self.nv = self.xi.shape[0]

    # The distributions and moments on this grid, as methods so that the GSIS
    # driver works unchanged on the reduced (xi_z-integrated) grid of
    # oracle.reduced, which has the same methods.
    reduced = False

    def maxwellian(self, rho, u, T):
        return maxwellian(rho, u, T, self.xi)

    def shakhov(self, rho, u, T, q):
        return reference_g0t(rho, u, T, q, self.xi)

    def grad13(self, rho, u, T, sigma, q):
        return grad13(rho, u, T, sigma, q, self.xi)

    def conserved(self, f):
        return conserved(f, self)

    def moments(self, f):
        return moments(f, self)

    def heat_flux_about(self, f, u):
        return heat_flux_about(f, u, self)

    def conservation_correct(self, base, M, U):
        return conservation_correct(base, M, U, self)

    def corrected_maxwellian(self, rho, u, T):
        return corrected_maxwellian(rho, u, T, self)

    def corrected_shakhov(self, rho, u, T, q):
        return corrected_shakhov(rho, u, T, q, self)


# --------------------------------------------------------------------------- transport coefficients
def mu0_from_kn(Kn, L=1.0, p0=1.0, T0=1.0):
    """Invert the Knudsen-number definition of Sec. 2,
    Kn = mu(T0)/(p0 L) * sqrt(pi R T0 / 2), for mu(T0)."""
    return Kn * p0 * L / np.sqrt(np.pi * T0 / 2.0)


def viscosity(T, mu0, omega, T0=1.0):
    """Power-law viscosity mu(T) = mu(T0) (T/T0)^omega (Sec. 2)."""
    return mu0 * (T / T0) ** omega


def conductivities(mu, A, d_r, R=1.0):
    """Eq. mu_kappa: [kappa_t, kappa_r] = (mu R / 2) A^{-1} [5, d_r]."""
    Am = np.array([[A[0], A[1]], [A[2], A[3]]], dtype=np.float64)
    k = 0.5 * mu * R * np.linalg.solve(Am, np.array([5.0, float(d_r)]))
    return k[0], k[1]


def eucken_factors(A, d_r):
    """Eucken factors f_t = kappa_t/(mu c_vt), f_r = kappa_r/(mu c_vr) with
    c_vt = 3R/2 and c_vr = d_r R/2 (the figures quoted for nitrogen in Sec. 4)."""
    kt, kr = conductivities(1.0, A, d_r)
    return kt / 1.5, kr / (0.5 * d_r)


def kappa_monatomic(mu):
    """d_r = 0 reduction of Eq. mu_kappa with A_tt = 2/3: kappa = 15/4 mu (Pr = 2/3)."""
    return 3.75 * mu


def heat_flux_mixing(qt, qr, A, Zr):
    """q0, q1 as the linear combinations of q_t and q_r given in Sec. 2."""
    q0 = ((2.0 - 3.0 * A[0]) * Zr + 1.0) * qt - 3.0 * A[1] * Zr * qr
    q1 = -A[2] * Zr * qt + (-A[3] * Zr + 1.0) * qr
    return q0, q1


# --------------------------------------------------------------------------- distributions
def maxwellian(rho, u, T, xi):
    """rho (2 pi T)^{-3/2} exp(-|xi-u|^2/(2T)), evaluated per node."""
    c = xi - np.asarray(u)[None, :]
    return rho * (2.0 * np.pi * T) ** -1.5 * np.exp(-np.sum(c * c, axis=1) / (2.0 * T))


def reference_g0t(rho, u, T, q, xi):
    """Reference distribution g_0t of Sec. 2 (R = 1, p_t = rho T_t):
    M * [1 + 2 q.c/(15 T p) (c^2/(2T) - 5/2)]."""
    c = xi - np.asarray(u)[None, :]
    c2 = np.sum(c * c, axis=1)
    qc = c @ np.asarray(q)
    p = rho * T
    return maxwellian(rho, u, T, xi) * (1.0 + 2.0 * qc / (15.0 * T * p) * (c2 / (2.0 * T) - 2.5))


def reference_g0r(rho, u, T, q0, xi):
    """g_0r of Sec. 2: same form as g_0t at the equilibrium temperature T with q0."""
    return reference_g0t(rho, u, T, q0, xi)


def grad13(rho, u, T, sigma, q, xi):
    """Eq. G13_VDF for f_0 (R = 1): f_eq [1 + sigma:cc/(2 rho T^2)
    + q.c/(rho T^2) (c^2/(5T) - 1)]."""
    c = xi - np.asarray(u)[None, :]
    c2 = np.sum(c * c, axis=1)
    scc = np.einsum("vi,ij,vj->v", c, np.asarray(sigma), c)
    qc = c @ np.asarray(q)
    return maxwellian(rho, u, T, xi) * (1.0 + scc / (2.0 * rho * T * T)
                                        + qc / (rho * T * T) * (c2 / (5.0 * T) - 1.0))


# --------------------------------------------------------------------------- moments
def conserved(f, vg):
    """(rho, rho u, rho E) = sum_v w (1, xi, |xi|^2/2) f  (Eq. getmoment)."""
    xi, w = vg.xi, vg.w
    rho = w * np.sum(f)
    mom = w * (xi.T @ f)
    E = w * np.sum(0.5 * np.sum(xi * xi, axis=1) * f)
    return np.array([rho, mom[0], mom[1], mom[2], E])


def primitive_from_conserved(U):
    """rho, u, T from (rho, rho u, rho E) with E = 3/2 T + u^2/2 (d_r = 0)."""
    rho = U[0]
    u = U[1:4] / rho
    T = (2.0 * U[4] / rho - np.dot(u, u)) / 3.0
    return rho, u, T


def conserved_from_primitive(rho, u, T):
    u = np.asarray(u)
    return np.array([rho, rho * u[0], rho * u[1], rho * u[2], rho * (1.5 * T + 0.5 * np.dot(u, u))])


def moments(f, vg):
    """Eq. getmoment for f_0: rho, u, T_t, traceless stress sigma, heat flux q
    (central moments about the distribution's own bulk velocity)."""
    xi, w = vg.xi, vg.w
    rho, u, T = primitive_from_conserved(conserved(f, vg))
    c = xi - u[None, :]
    c2 = np.sum(c * c, axis=1)
    P = w * np.einsum("vi,vj,v->ij", c, c, f)
    sigma = P - np.trace(P) / 3.0 * np.eye(3)
    q = 0.5 * w * (c.T @ (c2 * f))
    return rho, u, T, sigma, q


def heat_flux_about(f, u, vg):
    """q = 1/2 sum_v w c c^2 f with c = xi - u for a given bulk velocity u."""
    c = vg.xi - np.asarray(u)[None, :]
    c2 = np.sum(c * c, axis=1)
    return 0.5 * vg.w * (c.T @ (c2 * f))


# --------------------------------------------------------------------------- conservation correction
def conservation_correct(base, M, U, vg):
    """Discrete conservation correction (the paper states conservation of the
    collision term but not how a discrete velocity grid keeps it; the reading
    taken is the Lagrange-multiplier correction of Gamba & Tharkabhushanam,
    J. Comput. Phys. 228 (2009), written with Maxwellian weighting):

        result = base + M * (a0 + a1 xi_x + a2 xi_y + a3 xi_z + a4 |xi|^2)

    with a the solution of  sum_v w psi_v phi_v^T M_v a = U - sum_v w psi_v base_v,
    psi = (1, xi, |xi|^2/2), phi = (1, xi, |xi|^2).  Afterwards
    sum_v w psi_v result_v = U up to rounding."""
    xi, w = vg.xi, vg.w
    x2 = np.sum(xi * xi, axis=1)
    psi = np.stack([np.ones(vg.nv), xi[:, 0], xi[:, 1], xi[:, 2], 0.5 * x2], axis=1)
    phi = np.stack([np.ones(vg.nv), xi[:, 0], xi[:, 1], xi[:, 2], x2], axis=1)
    A = w * np.einsum("va,vb,v->ab", psi, phi, M)
    rhs = np.asarray(U) - w * (psi.T @ base)
    a = np.linalg.solve(A, rhs)
    return base + M * (phi @ a)


def corrected_maxwellian(rho, u, T, vg):
    """M~(W): the Maxwellian of (rho, u, T) corrected so that its discrete
    conserved moments equal (rho, rho u, rho E) exactly (the f_eq of Eq. updatef)."""
    M = maxwellian(rho, u, T, vg.xi)
    return conservation_correct(M, M, conserved_from_primitive(rho, u, T), vg)


def corrected_shakhov(rho, u, T, q, vg):
    """g~ : reference distribution g = g_0t (Eq. general_model with d_r = 0,
    so g = (1 - 1/Z_r) g_t + g_r / Z_r reduces to g_0t) with the discrete
    conservation correction towards the cell's (rho, rho u, rho E)."""
    M = maxwellian(rho, u, T, vg.xi)
    g = reference_g0t(rho, u, T, q, vg.xi)
    return conservation_correct(g, M, conserved_from_primitive(rho, u, T), vg)


def nsf_stress_heatflux(mu, grad_u, grad_T):
    """Eq. NSF_constitutive (d_r = 0): sigma = -mu (grad u + grad u^T - 2/3 div u I),
    q = -kappa grad T with kappa = 15/4 mu.  grad_u[i, j] = d u_j / d x_i."""
    G = np.asarray(grad_u)
    div = np.trace(G)
    sigma = -mu * (G + G.T - 2.0 / 3.0 * div * np.eye(3))
    q = -kappa_monatomic(mu) * np.asarray(grad_T)
    return sigma, q
