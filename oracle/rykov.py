"""Two-VDF model of a molecular gas with d_r internal degrees of freedom
(Sec. 2: Eqs. getmoment, general_model, the reference distributions g_0t,
g_0r, g_1t, g_1r, the q0/q1 mixing, mu_kappa, macroscopic_equation_2) and its
GSIS iteration (Sec. 3.1, 3.2, 3.4), in plain FP64 numpy (oracle; test
infrastructure only).

The Shakhov oracle (oracle.model, oracle.kinetic, oracle.macro, oracle.gsis)
is the d_r = 0 case of this module; this module reuses its transport sweep,
least-squares gradients and half-range (KFVS) moments unchanged and adds what
the internal mode brings:

* a second distribution f1 on the same velocity nodes (on the reduced grid of
  oracle.reduced only its xi_z integral, one plane, is needed: the internal
  energy and the in-plane internal heat flux are its only moments);
* the reference distribution of each VDF, g = (1 - 1/Z_r) g_t + g_r / Z_r,
  from the translational state (T_t, q_t, q_r) and the equilibrium one
  (T, q0, q1);
* the synthetic equations with six conserved variables (rho, rho u, rho e,
  rho e_r), the internal heat flux and the energy-exchange source of
  Eq. macroscopic_equation_2.

Units: R = 1.  Primitive state per cell: (rho, u_x, u_y, u_z, T_t, T_r);
conserved: (rho, rho u, rho e, rho e_r) with e = (3 T_t + |u|^2)/2 + e_r and
e_r = d_r T_r / 2.  With d_r = 0 there is no internal mode: T_r is defined as
T_t, f1 and e_r vanish, and every function here reduces to the Shakhov one.

Readings taken where the paper is silent (each is used once, here):

* discrete conservation: g_0t and g_0r are conservation-corrected Shakhov
  forms (oracle.model.conservation_correct) towards (rho, rho u, and the
  translational energy at T_t, respectively at T); the Maxwellian factor of
  the q_r and q1 terms of g_1t, g_1r is the corrected Maxwellian of that
  temperature, so that the q terms carry neither mass nor internal energy on
  the grid and the collision term conserves mass, momentum and total energy
  to rounding;
* f_eq of Eq. updatef for the two VDFs: the equilibrium of Eq. G13_VDF,
  f0 = M~(rho, u, T_t) and f1 = (d_r/2) T_r M~(rho, u, T_t);
* synthetic solve: the KFVS splitting of oracle.macro for the translational
  part; the internal energy is carried by the mass flux of each half-range
  ((d_r/2) T_r of the side it comes from); the energy-exchange source is
  taken point-implicitly in the pseudo-time step (its derivative with respect
  to rho e_r, -1/(Z_r tau), enters the diagonal of the internal-energy row);
  the spectral radius keeps the frozen translational sound speed
  sqrt(5 T_t / 3);
* Kn_Gll: lambda from T_t and the temperature ratio |grad T|/T taken with the
  equilibrium temperature T;
* residual epsilon: T_t and T_r are two quantities of the maximum.
"""
import numpy as np

from . import model as M
from .reduced import ReducedGrid
from .mesh import Topology, BC_FARFIELD, BC_WALL
from .kinetic import KineticInputs, sweep, wall_kinetic_flux
from .macro import MacroGeometry, lsq_grad, minmod, _half_range
from .hybrid import HybridGrid
from .unstructured import PolygonMesh, PolyhedralMesh, topology_of, UnstructuredGeometry, wall_layer_flags

NITROGEN = {"d_r": 2, "Z_r": 2.667, "omega": 0.74, "A": (0.786, -0.201, -0.059, 0.842)}
MONATOMIC_A = (2.0 / 3.0, 0.0, 0.0, 1.0)


def equilibrium_temperature(Tt, Tr, d_r):
    """T = (3 T_t + d_r T_r)/(3 + d_r) (Sec. 2)."""
    return (3.0 * Tt + d_r * Tr) / (3.0 + d_r)


def conserved6(W, d_r):
    """Primitive [.., 6] -> conserved (rho, rho u, rho e, rho e_r)."""
    W = np.asarray(W, dtype=np.float64)
    rho, u, Tt, Tr = W[..., 0], W[..., 1:4], W[..., 4], W[..., 5]
    er = 0.5 * d_r * Tr
    U = np.empty_like(W)
    U[..., 0] = rho
    U[..., 1:4] = rho[..., None] * u
    U[..., 4] = rho * (1.5 * Tt + 0.5 * np.sum(u * u, axis=-1) + er)
    U[..., 5] = rho * er
    return U


def primitive6(U, d_r):
    """Conserved [.., 6] -> primitive (rho, u, T_t, T_r); T_r = T_t when d_r = 0."""
    U = np.asarray(U, dtype=np.float64)
    rho = U[..., 0]
    u = U[..., 1:4] / rho[..., None]
    Tt = (2.0 * (U[..., 4] - U[..., 5]) / rho - np.sum(u * u, axis=-1)) / 3.0
    Tr = 2.0 * U[..., 5] / (d_r * rho) if d_r > 0 else Tt
    W = np.empty_like(U)
    W[..., 0] = rho
    W[..., 1:4] = u
    W[..., 4] = Tt
    W[..., 5] = Tr
    return W


class RykovGrid:
    """Velocity nodes of the two VDFs: the n0 nodes of a base grid (the 3D grid
    of oracle.model or the reduced grid of oracle.reduced) carry f0, then n1
    nodes carry f1 (all base nodes on a 3D grid; the G plane on the reduced
    grid, where f1 stands for its xi_z integral).  One vector of length
    n0 + n1 per cell, so that the transport sweep of oracle.kinetic runs on it
    unchanged.

    psi [nv, 6]: weights of (mass, x/y/z momentum, total energy, internal
    energy) per node, sum_v w psi_v f_v = (rho, rho u, rho e, rho e_r).
    The mass column is zero on the f1 nodes, so the diffuse-wall density of
    oracle.kinetic comes from f0 alone."""

    reduced = True   # oracle.kinetic takes the mass weight from psi

    def __init__(self, base, d_r):
        self.base = base
        self.d_r = int(d_r)
        self.w = base.w
        self.n0 = base.nv
        self.idx1 = np.nonzero(base.plane == 0)[0] if isinstance(base, ReducedGrid) else np.arange(base.nv)
        # quadrature weight of each f1 node relative to w (per node on a hybrid grid, whose w is 1)
        self.w1 = base.wv[self.idx1] if isinstance(base, HybridGrid) else 1.0
        self.n1 = len(self.idx1)
        self.nv = self.n0 + self.n1
        self.xi = np.concatenate([base.xi, base.xi[self.idx1]])
        if base.reduced:
            psi0 = base.psi
        else:
            x = base.xi
            psi0 = np.stack([np.ones(base.nv), x[:, 0], x[:, 1], x[:, 2], 0.5 * np.sum(x * x, axis=1)], axis=1)
        self.psi = np.zeros((self.nv, 6))
        self.psi[:self.n0, :5] = psi0
        self.psi[self.n0:, 4] = self.w1
        self.psi[self.n0:, 5] = self.w1

    def split(self, f):
        return f[:self.n0], f[self.n0:]

    def join(self, f0, f1):
        return np.concatenate([f0, f1])

    def c1(self, u):
        """Thermal velocities of the f1 nodes."""
        return self.base.xi[self.idx1] - np.asarray(u)[None, :]

    def conserved(self, f):
        return self.w * (self.psi.T @ f)

    # ---------------------------------------------------------------- moments (Eq. getmoment)
    def moments(self, f):
        """rho, u, T_t, T_r, traceless stress, q_t, q_r of (f0, f1): the f0 moments
        of the base grid, d_r/2 rho T_r = sum w f1 and q_r = sum w c f1 about the
        bulk velocity of f0."""
        f0, f1 = self.split(f)
        rho, u, Tt, sigma, qt = self.base.moments(f0)
        if self.d_r > 0:
            Tr = 2.0 * self.w * np.sum(self.w1 * f1) / (self.d_r * rho)
        else:
            Tr = Tt
        qr = self.w * (self.c1(u).T @ (self.w1 * f1))
        return rho, u, Tt, Tr, sigma, qt, qr

    # ---------------------------------------------------------------- distributions
    def _f1_part(self, scale, f0_shape, Mc, q, rho, u, T):
        """f1 values of scale * (f0-shaped distribution) + M (q.c)/(rho T), the
        common form of g_1t, g_1r and the f1 of Eq. G13_VDF (R = 1)."""
        qc = self.c1(u) @ np.asarray(q)
        return scale * f0_shape[self.idx1] + Mc[self.idx1] * qc / (rho * T)

    def reference(self, rho, u, Tt, Tr, qt, qr, Zr, A):
        """g = (1 - 1/Z_r) g_t + g_r / Z_r for both VDFs (Eq. general_model
        rearranged: (g_t - f)/tau + (g_r - g_t)/(Z_r tau) = (g - f)/tau), from
        the reference distributions of Sec. 2 with the conservation readings of
        the module docstring."""
        d_r = self.d_r
        T = equilibrium_temperature(Tt, Tr, d_r)
        q0, q1 = M.heat_flux_mixing(np.asarray(qt), np.asarray(qr), A, Zr)
        g0t = self.base.corrected_shakhov(rho, u, Tt, qt)
        g0r = self.base.corrected_shakhov(rho, u, T, q0)
        Mt = self.base.corrected_maxwellian(rho, u, Tt)
        Mr = self.base.corrected_maxwellian(rho, u, T)
        g1t = self._f1_part(0.5 * d_r * Tr, g0t, Mt, qr, rho, u, Tt)
        g1r = self._f1_part(0.5 * d_r * T, g0r, Mr, q1, rho, u, T)
        a = 1.0 - 1.0 / Zr
        b = 1.0 / Zr
        return self.join(a * g0t + b * g0r, a * g1t + b * g1r)

    def equilibrium(self, rho, u, Tt, Tr):
        """f_eq of Eq. updatef: f0 = M~(rho, u, T_t), f1 = (d_r/2) T_r M~."""
        Mt = self.base.corrected_maxwellian(rho, u, Tt)
        return self.join(Mt, 0.5 * self.d_r * Tr * Mt[self.idx1])

    def grad13(self, rho, u, Tt, Tr, sigma, qt, qr):
        """Eq. G13_VDF for both VDFs, f0 conservation-corrected to
        (rho, rho u, translational energy) and f1 built on it."""
        g = self.base.grad13(rho, u, Tt, sigma, qt)
        Mt = self.base.maxwellian(rho, u, Tt)
        f0 = self.base.conservation_correct(g, Mt, M.conserved_from_primitive(rho, u, Tt))
        Mc = self.base.corrected_maxwellian(rho, u, Tt)
        return self.join(f0, self._f1_part(0.5 * self.d_r * Tr, f0, Mc, qr, rho, u, Tt))

    def boundary_maxwellian(self, rho, u, T):
        """Far-field distribution: both VDFs in equilibrium at T (T_r = T_t = T)."""
        return self.equilibrium(rho, u, T, T)

    def wall_maxwellian(self, Tw):
        """Unit-density emission shape of a diffuse wall at T_w: f0 = M(0, T_w),
        f1 = (d_r/2) T_w M(0, T_w) (internal mode accommodated too)."""
        Mw = self.base.maxwellian(1.0, np.zeros(3), Tw)
        return self.join(Mw, 0.5 * self.d_r * Tw * Mw[self.idx1])


def heat_flux_relaxation(qt, qr, A):
    """Relaxation rates of the heat fluxes that the A matrix prescribes (Sec. 2):
    tau dq_t/dt = -(A_tt q_t + A_tr q_r), tau dq_r/dt = -(A_rt q_t + A_rr q_r)."""
    qt = np.asarray(qt); qr = np.asarray(qr)
    return -(A[0] * qt + A[1] * qr), -(A[2] * qt + A[3] * qr)


# --------------------------------------------------------------------------- synthetic equations
def conductivity_factors(A, d_r):
    """kappa_t / mu and kappa_r / mu of Eq. mu_kappa (R = 1)."""
    Am = np.array([[A[0], A[1]], [A[2], A[3]]], dtype=np.float64)
    k = 0.5 * np.linalg.solve(Am, np.array([5.0, float(d_r)]))
    return k[0], k[1]


def boundary_values6(geo, bc_state, rho, u, Tt, Tr):
    """Boundary values per (cell, side) for the least-squares gradients: far
    field -> the boundary state (in equilibrium, T_r = T_t = T_inf); wall ->
    u = 0, T_t = T_r = T_w, rho = cell value; other sides -> cell values."""
    N = geo.N
    out = {k: np.zeros((N, 6)) for k in ("rho", "ux", "uy", "uz", "Tt", "Tr", "U")}
    for si in range(6):
        bc = geo.side_bc[:, si]
        ff = bc == BC_FARFIELD
        wl = bc == BC_WALL
        st = bc_state[np.maximum(geo.side_bside[:, si], 0)]
        out["rho"][:, si] = np.where(ff, st[:, 0], rho)
        for a, key in enumerate(("ux", "uy", "uz")):
            out[key][:, si] = np.where(ff, st[:, 1 + a], 0.0)
        out["Tt"][:, si] = np.where(ff | wl, st[:, 4], Tt)
        out["Tr"][:, si] = np.where(ff | wl, st[:, 4], Tr)
        out["U"][:, si] = np.where(ff, np.linalg.norm(st[:, 1:4], axis=1), 0.0)
    return out


def gradients6(geo, bc_state, W):
    """Least-squares gradients of u (gu[c, i, j] = d u_j / d x_i), T_t and T_r."""
    rho, u, Tt, Tr = W[:, 0], W[:, 1:4], W[:, 4], W[:, 5]
    bv = boundary_values6(geo, bc_state, rho, u, Tt, Tr)
    gu = np.stack([lsq_grad(geo, u[:, a], bv[k]) for a, k in enumerate(("ux", "uy", "uz"))], axis=2)
    return gu, lsq_grad(geo, Tt, bv["Tt"]), lsq_grad(geo, Tr, bv["Tr"])


def nsf6(mu, gu, gTt, gTr, A, d_r):
    """Eq. NSF_constitutive with the conductivities of Eq. mu_kappa:
    sigma = -mu (grad u + grad u^T - 2/3 div u I), q_t = -kappa_t grad T_t,
    q_r = -kappa_r grad T_r."""
    kt, kr = conductivity_factors(A, d_r)
    div = np.trace(gu, axis1=1, axis2=2)
    sym = gu + np.transpose(gu, (0, 2, 1))
    sigma = -mu[:, None, None] * (sym - 2.0 / 3.0 * div[:, None, None] * np.eye(3)[None])
    return sigma, -(kt * mu)[:, None] * gTt, -(kr * mu)[:, None] * gTr


def kfvs6(rL, uL, pL, TrL, rR, uR, pR, TrR, n, d_r):
    """KFVS of oracle.macro for (mass, momentum, translational energy) plus the
    internal energy each half-range carries with its mass flux, (d_r/2) T_r of
    the side it comes from; the total energy flux is the sum of both energies.
    Per unit area through unit normal n; returns [F, 6]."""
    FL = _half_range(rL, uL, pL / rL, n, 1.0)
    FR = _half_range(rR, uR, pR / rR, n, -1.0)
    erL = 0.5 * d_r * TrL * FL[:, 0]
    erR = 0.5 * d_r * TrR * FR[:, 0]
    F = np.zeros((len(rL), 6))
    F[:, :5] = FL + FR
    F[:, 4] += erL + erR
    F[:, 5] = erL + erR
    return F


def euler_flux_dot6(U, S, d_r):
    """Euler flux of conserved states U[F, 6] dotted with S[F, 3]: p_t = rho T_t
    in the momentum and total energy fluxes, rho e_r convected."""
    W = primitive6(U, d_r)
    rho, u = W[:, 0], W[:, 1:4]
    p = rho * W[:, 4]
    uS = np.sum(u * S, axis=1)
    F = np.zeros_like(U)
    F[:, 0] = rho * uS
    F[:, 1:4] = U[:, 1:4] * uS[:, None] + p[:, None] * S
    F[:, 4] = (U[:, 4] + p) * uS
    F[:, 5] = U[:, 5] * uS
    return F


def exchange_source(W, mu0, omega, d_r, Zr):
    """Energy-exchange source of Eq. macroscopic_equation_2, d_r rho (T - T_r)
    / (2 Z_r tau) with tau = mu(T_t)/p_t, and its derivative with respect to
    rho e_r at fixed rho e, -1/(Z_r tau)."""
    rho, Tt, Tr = W[:, 0], W[:, 4], W[:, 5]
    tau = M.viscosity(Tt, mu0, omega) / (rho * Tt)
    T = equilibrium_temperature(Tt, Tr, d_r)
    return 0.5 * d_r * rho * (T - Tr) / (Zr * tau), -1.0 / (Zr * tau)


def wall_nsf_flux6(geo, bc_state, W, gu, gTt, gTr, mu0, omega, A, d_r):
    """NSF flux through every wall face: no mass flux, cell pressure p_t,
    stress at u = 0 and heat fluxes at T_t = T_r = T_w from the cell gradients
    corrected along the cell-to-face line; [wall faces, 6]."""
    idx = np.nonzero(geo.bT == BC_WALL)[0]
    c = geo.bC[idx]
    Sb = geo.bS[idx]
    Tw = bc_state[geo.bSide[idx], 4]
    e_b = geo.be[idx]
    db = geo.bdist[idx]

    def wall_grad(gc, phic, phiw):
        return gc + ((phiw - phic) / db - np.sum(gc * e_b, axis=1))[:, None] * e_b

    u = W[:, 1:4]
    guw = np.stack([wall_grad(gu[c, :, j], u[c, j], 0.0) for j in range(3)], axis=2)
    sig, qt, qr = nsf6(M.viscosity(Tw, mu0, omega), guw, wall_grad(gTt[c], W[c, 4], Tw),
                       wall_grad(gTr[c], W[c, 5], Tw), A, d_r)
    F = np.zeros((len(idx), 6))
    F[:, 1:4] = (W[c, 0] * W[c, 4])[:, None] * Sb + np.einsum("fij,fj->fi", sig, Sb)
    F[:, 4] = np.sum((qt + qr) * Sb, axis=1)
    F[:, 5] = np.sum(qr * Sb, axis=1)
    return F


class GasParams:
    """Gas of Sec. 2: d_r, Z_r, A = (A_tt, A_tr, A_rt, A_rr), mu(T0) and omega."""

    def __init__(self, d_r, Zr, A, mu0, omega):
        self.d_r = int(d_r)
        self.Zr = float(Zr)
        self.A = tuple(float(a) for a in A)
        self.mu0 = float(mu0)
        self.omega = float(omega)


def residual6(geo, bc_state, U, hot, gas, bface_corr=None):
    """R_c = -sum over faces of the outward flux + V_c Q_c (Eq. macro with the
    equations of Eq. macroscopic_equation_2), for the six conserved variables.
    hot = (sigma [N,3,3], q_t [N,3], q_r [N,3]) high-order terms (zero in NS
    cells).  Face fluxes as in oracle.macro.residual: KFVS on index-space MUSCL
    states of (rho, u, p_t, T_r), NSF from face gradients corrected along the
    line of centres at the mean cell velocity and temperatures, plus the mean
    HoT of the two cells; far field = KFVS against the boundary state plus the
    cell's HoT; wall = wall_nsf_flux6 (+ bface_corr at the walls of DVM
    cells).  Returns R[N, 6], lambda|S| per interior face, its sum per cell
    and d Q_e_r / d(rho e_r) per cell (for the point-implicit diagonal)."""
    d_r, mu0, omega, A = gas.d_r, gas.mu0, gas.omega, gas.A
    hs, hqt, hqr = hot
    N = geo.N
    W = primitive6(U, d_r)
    rho, u, Tt, Tr = W[:, 0], W[:, 1:4], W[:, 4], W[:, 5]
    p = rho * Tt
    a = np.sqrt(M.GAMMA * Tt)
    mu_c = M.viscosity(Tt, mu0, omega)
    gu, gTt, gTr = gradients6(geo, bc_state, W)
    R = np.zeros((N, 6))
    lam_sum = np.zeros(N)

    prim = np.concatenate([rho[:, None], u, p[:, None], Tr[:, None]], axis=1)
    slopes = np.zeros((N, 3, 6))
    for d in range(3):
        lo, hi = geo.nb[:, d, 0], geo.nb[:, d, 1]
        ok = (lo >= 0) & (hi >= 0)
        slopes[:, d, :] = np.where(ok[:, None], minmod(prim - prim[np.maximum(lo, 0)],
                                                       prim[np.maximum(hi, 0)] - prim), 0.0)

    L, Rr, d = geo.L, geo.R, geo.dirs
    qL = prim[L] + 0.5 * slopes[L, d, :]
    qR = prim[Rr] - 0.5 * slopes[Rr, d, :]
    Fi = kfvs6(qL[:, 0], qL[:, 1:4], qL[:, 4], qL[:, 5], qR[:, 0], qR[:, 1:4], qR[:, 4], qR[:, 5],
               geo.n, d_r) * geo.Sabs[:, None]
    uf = 0.5 * (u[L] + u[Rr])
    muf = M.viscosity(0.5 * (Tt[L] + Tt[Rr]), mu0, omega)

    def face_grad(gc, phiL, phiR):
        gav = 0.5 * (gc[L] + gc[Rr])
        return gav + ((phiR - phiL) / geo.dist - np.sum(gav * geo.e, axis=1))[:, None] * geo.e

    guf = np.stack([face_grad(gu[:, :, j], u[L, j], u[Rr, j]) for j in range(3)], axis=2)
    sig_f, qt_f, qr_f = nsf6(muf, guf, face_grad(gTt, Tt[L], Tt[Rr]), face_grad(gTr, Tr[L], Tr[Rr]), A, d_r)
    Sig = sig_f + 0.5 * (hs[L] + hs[Rr])
    Qt = qt_f + 0.5 * (hqt[L] + hqt[Rr])
    Qr = qr_f + 0.5 * (hqr[L] + hqr[Rr])
    SigS = np.einsum("fij,fj->fi", Sig, geo.S)
    QrS = np.sum(Qr * geo.S, axis=1)
    Fv = np.zeros((len(L), 6))
    Fv[:, 1:4] = SigS
    Fv[:, 4] = np.sum(SigS * uf, axis=1) + np.sum(Qt * geo.S, axis=1) + QrS
    Fv[:, 5] = QrS
    F = Fi + Fv
    np.add.at(R, L, -F)
    np.add.at(R, Rr, F)
    lam = (np.abs(np.sum(uf * geo.n, axis=1)) + 0.5 * (a[L] + a[Rr])
           + 5.0 * muf / (0.5 * (rho[L] + rho[Rr]) * geo.dist))
    lamS = lam * geo.Sabs
    np.add.at(lam_sum, L, lamS)
    np.add.at(lam_sum, Rr, lamS)

    C = geo.bC
    ff = geo.bT == BC_FARFIELD
    wl = geo.bT == BC_WALL
    st = bc_state[geo.bSide]
    Fb = np.zeros((len(C), 6))
    if np.any(ff):
        idx = np.nonzero(ff)[0]
        c = C[idx]
        sr = st[idx]
        Fb[idx] = kfvs6(rho[c], u[c], p[c], Tr[c], sr[:, 0], sr[:, 1:4], sr[:, 0] * sr[:, 4], sr[:, 4],
                        geo.bn[idx], d_r) * geo.bSabs[idx, None]
        Sb = geo.bS[idx]
        SigS = np.einsum("fij,fj->fi", hs[c], Sb)
        QrS = np.sum(hqr[c] * Sb, axis=1)
        Fb[idx, 1:4] += SigS
        Fb[idx, 4] += np.sum(SigS * 0.5 * (u[c] + sr[:, 1:4]), axis=1) + np.sum(hqt[c] * Sb, axis=1) + QrS
        Fb[idx, 5] += QrS
    if np.any(wl):
        Fb[np.nonzero(wl)[0]] = wall_nsf_flux6(geo, bc_state, W, gu, gTt, gTr, mu0, omega, A, d_r)
    if bface_corr is not None:
        Fb = Fb + bface_corr
    np.add.at(R, C, -Fb)
    use = ff | wl
    lam_b = np.abs(np.sum(u[C] * geo.bn, axis=1)) + a[C] + 5.0 * mu_c[C] / (rho[C] * 2.0 * geo.bdist)
    np.add.at(lam_sum, C[use], (lam_b * geo.bSabs)[use])

    dQ = np.zeros(N)
    if d_r > 0:
        Q, dQ = exchange_source(W, mu0, omega, d_r, gas.Zr)
        R[:, 5] += geo.topo.vol * Q
    return R, lamS, lam_sum, dQ


def relax_step6(geo, bc_state, U, hot, gas, cfl, k_sub, dt=0.0, Un=None, bface_corr=None):
    """One DP-LUR pseudo-time step of oracle.macro.relax_step for six variables;
    the internal-energy row's diagonal gains -V dQ/d(rho e_r) = V/(Z_r tau)."""
    R, lamS, lam_sum, dQ = residual6(geo, bc_state, U, hot, gas, bface_corr)
    vol = geo.topo.vol
    D = np.repeat(((1.0 / cfl + 0.5) * lam_sum)[:, None], 6, axis=1)
    if dt > 0.0:
        R = R - (vol / dt)[:, None] * (U - Un)
        D = D + (vol / dt)[:, None]
    D[:, 5] -= vol * dQ
    dU = R / D
    L, Rr = geo.L, geo.R
    for _ in range(k_sub):
        off = np.zeros_like(U)
        dFR = euler_flux_dot6(U[Rr] + dU[Rr], geo.S, gas.d_r) - euler_flux_dot6(U[Rr], geo.S, gas.d_r)
        dFL = euler_flux_dot6(U[L] + dU[L], -geo.S, gas.d_r) - euler_flux_dot6(U[L], -geo.S, gas.d_r)
        np.add.at(off, L, 0.5 * (dFR - lamS[:, None] * dU[Rr]))
        np.add.at(off, Rr, 0.5 * (dFL - lamS[:, None] * dU[L]))
        dU = (R - off) / D
    return U + dU


def macro_solve6(geo, bc_state, U0, hot, gas, cfl, k_sub, steps, dt=0.0, Un=None, bface_corr=None):
    """steps pseudo-time steps of the six-variable synthetic equations from U0
    (dt = 0: steady form; dt > 0: the time term of Eq. macro about Un)."""
    U = U0.copy()
    for _ in range(steps):
        U = relax_step6(geo, bc_state, U, hot, gas, cfl, k_sub, dt, Un, bface_corr)
    return U


# --------------------------------------------------------------------------- GSIS iteration
def residual_eps6(Wn, Wp, vol):
    """Convergence criterion of Sec. 4 over rho, u (one vector quantity), T_t
    and T_r; a quantity whose denominator is exactly zero is left out."""
    out = [0.0]
    for sl in (slice(0, 1), slice(1, 4), slice(4, 5), slice(5, 6)):
        num = np.sum(np.sum((Wn[:, sl] - Wp[:, sl]) ** 2, axis=1) * vol)
        den = np.sum(np.sum(Wp[:, sl] ** 2, axis=1) * vol)
        if den > 0.0:
            out.append(np.sqrt(num / den))
    return max(out)


class RykovSolver:
    """Adaptive GSIS (the steps of oracle.gsis.OracleSolver) for the two-VDF gas.
    case: a workload descriptor (mesh -- structured, or a polygon or polyhedral
    mesh of oracle.unstructured --, velocity grid -- uniform, reduced or a
    HybridGrid --, initial W0 with 5 columns (T_r = T_t) or 6, Kn, run
    parameters); gas: d_r, Z_r, A (mu0 and omega come from the case)."""

    def __init__(self, case, d_r, Zr, A, flags_override=None):
        self.case = case
        self.unstructured = isinstance(case.mesh, (PolygonMesh, PolyhedralMesh))
        if self.unstructured:
            self.topo = topology_of(case.mesh)
            self.geo = UnstructuredGeometry(self.topo)
        else:
            self.topo = Topology(case.mesh)
            self.geo = MacroGeometry(self.topo)
        if isinstance(case.vgrid, HybridGrid):
            base = case.vgrid
        elif getattr(case.vgrid, "reduced", False):
            base = ReducedGrid(case.vgrid.n, case.vgrid.lo, case.vgrid.hi)
        else:
            base = M.VelocityGrid(case.vgrid.n, case.vgrid.lo, case.vgrid.hi)
        self.vg = RykovGrid(base, d_r)
        self.gas = GasParams(d_r, Zr, A, M.mu0_from_kn(case.Kn), case.omega)
        self.bc_state = np.array(case.mesh.bc_state, dtype=np.float64)
        W0 = np.array(case.W0, dtype=np.float64)
        if W0.shape[1] == 5:
            W0 = np.concatenate([W0, W0[:, 4:5]], axis=1)
        self.W = W0
        self.N = self.topo.ncell
        self.f = np.zeros((self.N, self.vg.nv))
        self.dvm = np.zeros(self.N, dtype=bool)
        self.flags_override = flags_override
        self.eps_history = []
        self.kn_gll = np.zeros(self.N)
        self.hot = self.zero_hot()
        self.iteration = 0
        self.presolve_blocks = 0

    def zero_hot(self):
        return (np.zeros((self.N, 3, 3)), np.zeros((self.N, 3)), np.zeros((self.N, 3)))

    # ----------------------------------------------------------------- helpers
    def nsf_field(self, W):
        gu, gTt, gTr = gradients6(self.geo, self.bc_state, W)
        mu = M.viscosity(W[:, 4], self.gas.mu0, self.gas.omega)
        return nsf6(mu, gu, gTt, gTr, self.gas.A, self.gas.d_r)

    def kn_gll_field(self, W):
        """Eq. Kn_Gll with lambda = mu(T_t)/p_t sqrt(pi T_t / 2), |grad U| divided
        by max(U, a) (a = sqrt(5 T_t / 3)) and T the equilibrium temperature."""
        rho, u, Tt, Tr = W[:, 0], W[:, 1:4], W[:, 4], W[:, 5]
        d_r = self.gas.d_r
        T = equilibrium_temperature(Tt, Tr, d_r)
        U = np.linalg.norm(u, axis=1)
        bv = boundary_values6(self.geo, self.bc_state, rho, u, Tt, Tr)
        bT = equilibrium_temperature(bv["Tt"], bv["Tr"], d_r)
        g_rho = lsq_grad(self.geo, rho, bv["rho"])
        g_U = lsq_grad(self.geo, U, bv["U"])
        g_T = lsq_grad(self.geo, T, bT)
        a = np.sqrt(M.GAMMA * Tt)
        lam = M.viscosity(Tt, self.gas.mu0, self.gas.omega) / (rho * Tt) * np.sqrt(np.pi * Tt / 2.0)
        r = np.maximum(np.maximum(np.linalg.norm(g_rho, axis=1) / rho,
                                  np.linalg.norm(g_U, axis=1) / np.maximum(U, a)),
                       np.linalg.norm(g_T, axis=1) / T)
        return lam * r

    def region(self, W):
        """DVM-region rule of Sec. 3.2 plus wall_layers cell layers at walls."""
        if self.flags_override is not None:
            return np.array(self.flags_override, dtype=bool)
        self.kn_gll = self.kn_gll_field(W)
        flag = self.kn_gll >= self.case.Kn_ref
        mesh = self.case.mesh
        if self.unstructured:
            return flag | wall_layer_flags(self.topo, self.case.wall_layers)
        if self.case.wall_layers > 0:
            for d in range(3):
                for hi in (0, 1):
                    if mesh.bc_type[2 * d + hi] != BC_WALL:
                        continue
                    for c in range(self.N):
                        m = self.topo.ijk(c)[d]
                        if (m if hi == 0 else self.topo.n[d] - 1 - m) < self.case.wall_layers:
                            flag[c] = True
        return flag

    def seed_vdf(self, cells, W):
        """Eq. G13_VDF for both VDFs from W and its NSF stress / heat fluxes."""
        sig, qt, qr = self.nsf_field(W)
        for c in cells:
            self.f[c] = self.vg.grad13(W[c, 0], W[c, 1:4], W[c, 4], W[c, 5], sig[c], qt[c], qr[c])

    def set_region(self, new_flags, W):
        entering = [c for c in range(self.N) if new_flags[c] and not self.dvm[c]]
        for c in range(self.N):
            if self.dvm[c] and not new_flags[c]:
                self.f[c] = 0.0
        self.dvm = np.array(new_flags, dtype=bool)
        if entering:
            self.seed_vdf(entering, W)

    # ----------------------------------------------------------------- phases
    def presolve(self):
        """Sec. 3.4 Step 1: the synthetic equations with HoT = 0."""
        d_r = self.gas.d_r
        U = conserved6(self.W, d_r)
        for b in range(self.case.presolve_max_blocks):
            Wp = primitive6(U, d_r)
            U = macro_solve6(self.geo, self.bc_state, U, self.zero_hot(), self.gas, self.case.cfl,
                             self.case.k_sub, self.case.macro_steps)
            self.presolve_blocks = b + 1
            if residual_eps6(primitive6(U, d_r), Wp, self.topo.vol) < self.case.tol:
                break
        self.W = primitive6(U, d_r)

    def initialise(self):
        if self.case.presolve_max_blocks > 0:
            self.presolve()
        if self.case.adaptive:
            self.set_region(self.region(self.W), self.W)
        else:
            self.dvm[:] = True
            for c in range(self.N):
                self.f[c] = self.vg.equilibrium(self.W[c, 0], self.W[c, 1:4], self.W[c, 4], self.W[c, 5])

    def kinetic_inputs(self):
        """Reference distributions, tau = mu(T_t)/p_t, Grad-13 ghosts and
        boundary distributions from W^n (q_t, q_r of f^n about u^n)."""
        W, vg, gas = self.W, self.vg, self.gas
        gt, tau, ghost, ff, mw = {}, {}, {}, {}, {}
        for c in range(self.N):
            if not self.dvm[c]:
                continue
            rho, u, Tt, Tr = W[c, 0], W[c, 1:4], W[c, 4], W[c, 5]
            f0, f1 = vg.split(self.f[c])
            qt = vg.base.heat_flux_about(f0, u)
            qr = vg.w * (vg.c1(u).T @ (vg.w1 * f1))
            gt[c] = vg.reference(rho, u, Tt, Tr, qt, qr, gas.Zr, gas.A)
            tau[c] = M.viscosity(Tt, gas.mu0, gas.omega) / (rho * Tt)
        need = set()
        for c in range(self.N):
            if self.dvm[c]:
                for sd in self.topo.sides[c]:
                    if sd.nbr >= 0 and not self.dvm[sd.nbr]:
                        need.add(sd.nbr)
        if need:
            sig, qtn, qrn = self.nsf_field(W)
            for c in need:
                ghost[c] = vg.grad13(W[c, 0], W[c, 1:4], W[c, 4], W[c, 5], sig[c], qtn[c], qrn[c])
        for s in range(6):
            st = self.bc_state[s]
            if self.case.mesh.bc_type[s] == BC_FARFIELD:
                ff[s] = vg.boundary_maxwellian(st[0], st[1:4], st[4])
            elif self.case.mesh.bc_type[s] == BC_WALL:
                mw[s] = vg.wall_maxwellian(st[4])
        return KineticInputs(gt, tau, ghost, ff, mw)

    def wall_correction(self, W_half, mw):
        """Per wall face: kinetic wall flux of f^{n+1/2} (six components) minus
        the NSF wall flux at W^{n+1/2} for a DVM cell, zero for an NS cell."""
        geo = self.geo
        idx = np.nonzero(geo.bT == BC_WALL)[0]
        corr = np.zeros((len(idx), 6))
        if len(idx) == 0:
            return corr
        gu, gTt, gTr = gradients6(geo, self.bc_state, W_half)
        F_nsf = wall_nsf_flux6(geo, self.bc_state, W_half, gu, gTt, gTr, self.gas.mu0, self.gas.omega,
                               self.gas.A, self.gas.d_r)
        for r, f_i in enumerate(idx):
            c = geo.bC[f_i]
            if self.dvm[c]:
                corr[r] = wall_kinetic_flux(self.f[c], geo.bS[f_i], mw[geo.bSide[f_i]], self.vg) - F_nsf[r]
        return corr

    def step(self):
        """One GSIS iteration (the six steps of oracle.gsis.OracleSolver.step);
        returns epsilon."""
        case, vg, gas = self.case, self.vg, self.gas
        d_r = gas.d_r
        if case.adaptive and self.iteration == case.adapt_every and self.flags_override is None:
            self.set_region(self.region(self.W), self.W)
        inp = self.kinetic_inputs()
        sweep(self.topo, vg, self.f, self.dvm, inp)
        W_half = self.W.copy()
        sig_k = np.zeros((self.N, 3, 3)); qt_k = np.zeros((self.N, 3)); qr_k = np.zeros((self.N, 3))
        for c in range(self.N):
            if self.dvm[c]:
                rho, u, Tt, Tr, sig, qt, qr = vg.moments(self.f[c])
                W_half[c] = [rho, u[0], u[1], u[2], Tt, Tr]
                sig_k[c] = sig; qt_k[c] = qt; qr_k[c] = qr
        sig_n, qt_n, qr_n = self.nsf_field(W_half)
        dv = self.dvm
        self.hot = (np.where(dv[:, None, None], sig_k - sig_n, 0.0), np.where(dv[:, None], qt_k - qt_n, 0.0),
                    np.where(dv[:, None], qr_k - qr_n, 0.0))
        self.W_half = W_half
        bcorr = np.zeros((len(self.geo.bC), 6))
        bcorr[self.geo.bT == BC_WALL] = self.wall_correction(W_half, inp.mw)
        U = macro_solve6(self.geo, self.bc_state, conserved6(W_half, d_r), self.hot, gas, case.cfl, case.k_sub,
                         case.macro_steps, case.dt, conserved6(self.W, d_r), bcorr)
        W_new = primitive6(U, d_r)
        if case.relax != 1.0:
            W_new = W_half + case.relax * (W_new - W_half)
        for c in range(self.N):
            if self.dvm[c]:
                a = vg.equilibrium(W_new[c, 0], W_new[c, 1:4], W_new[c, 4], W_new[c, 5])
                b = vg.equilibrium(W_half[c, 0], W_half[c, 1:4], W_half[c, 4], W_half[c, 5])
                self.f[c] = self.f[c] + a - b
        eps = residual_eps6(W_new, self.W, self.topo.vol)
        self.W = W_new
        self.eps_history.append(eps)
        self.iteration += 1
        return eps

    def run(self, iterations=None):
        self.initialise()
        for _ in range(self.case.iterations if iterations is None else iterations):
            self.step()
        return self
