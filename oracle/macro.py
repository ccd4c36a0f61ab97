"""Macroscopic synthetic solve of Sec. 3.1 (Eq. macro with the constitutive
relations of Eq. full_constitutive) in plain FP64 numpy (oracle; test
infrastructure only).

The paper defers the fluxes F and sources Q of Eq. macro to an appendix of
another paper.  The reading taken, for the monatomic gas (no source):

* conserved U = (rho, rho u, rho E), E = 3/2 T + |u|^2/2, p = rho T;
* inviscid face flux: kinetic flux-vector splitting (the flux of the left
  face state's Maxwellian molecules moving along +n plus the right one's
  moving along -n, in closed form) on MUSCL states of (rho, u, p)
  reconstructed in index space with minmod (first order at boundaries).
  This is the Euler flux the discrete-velocity upwind scheme itself carries
  for Maxwellian states, so the synthetic equations and the kinetic step
  dissipate alike; with a contact-preserving Riemann solver (HLLC) an
  entropy mode at the stagnation line, which the kinetic step damps and the
  synthetic solve does not, grew from one GSIS iteration to the next;
* viscous face flux: NSF stress and heat flux (Eq. NSF_constitutive) from
  the mean of the two cells' least-squares gradients, corrected along the
  line of centres, at the mean cell velocity and temperature; plus the mean
  of the two cells' high-order terms (HoT, zero in NS cells);
* boundaries: far field = the same splitting against the boundary state
  (the kinetic step's incoming far-field Maxwellian) plus the cell's HoT (no
  NSF part: the far field is taken as gradient-free);
  wall of an NS cell (and in the NS presolve) = cell pressure, no mass flux,
  NSF at u = 0, T = T_w from a one-sided gradient; wall of a DVM cell = the
  kinetic wall flux of f^{n+1/2} plus the change of that NSF wall flux since
  W^{n+1/2}, so that at convergence the synthetic equations see exactly the
  wall flux of the kinetic solution (slip and temperature jump included);
* pseudo-time relaxation: data-parallel line-free relaxation (DP-LUR of
  Wright, Candler & Bose, AIAA J. 36 (1998)) with a scalar diagonal
  (1/CFL + 1/2) sum_F lambda_F |S_F|, lambda_F = |u.n| + a + 5 mu/(rho d),
  and k_sub Jacobi sweeps over the off-diagonal Rusanov-split Euler fluxes.
"""
import numpy as np
from scipy.special import erf

from .mesh import BC_NONE, BC_FARFIELD, BC_WALL
from .model import GAMMA, viscosity, kappa_monatomic


class MacroGeometry:
    """Face lists and least-squares weights derived from a Topology."""

    def __init__(self, topo):
        self.topo = topo
        N = topo.ncell
        self.N = N
        self.L, self.R, self.S = topo.interior_faces()
        self.dirs = np.array([0] * 0)
        # per-interior-face direction (for MUSCL)
        dirs = []
        for c in range(N):
            for sd in topo.sides[c]:
                if sd.s > 0 and sd.nbr >= 0:
                    dirs.append(sd.d)
        self.dirs = np.array(dirs, dtype=np.int64)
        self.Sabs = np.linalg.norm(self.S, axis=1)
        self.n = self.S / self.Sabs[:, None]
        e = topo.centers[self.R] - topo.centers[self.L]
        self.dist = np.linalg.norm(e, axis=1)
        self.e = e / self.dist[:, None]
        (self.bC, self.bS, self.bX, self.bSide, self.bT) = topo.boundary_faces()
        self.bSabs = np.linalg.norm(self.bS, axis=1)
        self.bn = self.bS / np.where(self.bSabs > 0, self.bSabs, 1.0)[:, None]
        eb = self.bX - topo.centers[self.bC]
        self.bdist = np.linalg.norm(eb, axis=1)
        self.be = eb / self.bdist[:, None]
        # neighbour table for index-space MUSCL: nb[c, d, 0/1] (-1 if none)
        self.nb = -np.ones((N, 3, 2), dtype=np.int64)
        for c in range(N):
            for sd in topo.sides[c]:
                self.nb[c, sd.d, 0 if sd.s < 0 else 1] = sd.nbr
        # least-squares weights: grad = sum_sides w[c, side] (phi_side - phi_c)
        self.lsq_w = np.zeros((N, 6, 3))
        self.side_nbr = -np.ones((N, 6), dtype=np.int64)
        self.side_bc = -np.ones((N, 6), dtype=np.int64)
        self.side_bside = -np.ones((N, 6), dtype=np.int64)
        dim = topo.dim
        for c in range(N):
            rows, used = [], []
            for si, sd in enumerate(topo.sides[c]):
                self.side_nbr[c, si] = sd.nbr
                self.side_bc[c, si] = sd.bc
                self.side_bside[c, si] = sd.bc_side
                if sd.nbr >= 0:
                    rows.append(topo.centers[sd.nbr] - topo.centers[c]); used.append(si)
                elif sd.bc in (BC_FARFIELD, BC_WALL):
                    rows.append(sd.xf - topo.centers[c]); used.append(si)
            A = np.array(rows)[:, :dim]
            P = np.linalg.solve(A.T @ A, A.T)          # dim x nrows
            for r, si in enumerate(used):
                self.lsq_w[c, si, :dim] = P[:, r]


def lsq_grad(geo, phi, bvals):
    """Least-squares gradient of cell field phi [N] with boundary values
    bvals[N, 6] (used on FARFIELD/WALL sides)."""
    g = np.zeros((geo.N, 3))
    for si in range(6):
        nbr = geo.side_nbr[:, si]
        val = np.where(nbr >= 0, phi[np.maximum(nbr, 0)], bvals[:, si])
        use = (nbr >= 0) | (geo.side_bc[:, si] == BC_FARFIELD) | (geo.side_bc[:, si] == BC_WALL)
        g += geo.lsq_w[:, si, :] * np.where(use, val - phi, 0.0)[:, None]
    return g


def primitives(U):
    rho = U[:, 0]
    u = U[:, 1:4] / rho[:, None]
    T = (2.0 * U[:, 4] / rho - np.sum(u * u, axis=1)) / 3.0
    return rho, u, T


def boundary_values(geo, bc_state, rho, u, T):
    """Boundary values per (cell, side) for rho, u (3), T, |u| used by the
    least-squares gradients: far field -> boundary state, wall -> u = 0,
    T = T_w, rho = cell value."""
    N = geo.N
    out = {k: np.zeros((N, 6)) for k in ("rho", "ux", "uy", "uz", "T", "U")}
    for si in range(6):
        bside = geo.side_bside[:, si]
        bc = geo.side_bc[:, si]
        ff = bc == BC_FARFIELD
        wl = bc == BC_WALL
        st = bc_state[np.maximum(bside, 0)]
        out["rho"][:, si] = np.where(ff, st[:, 0], rho)
        for a, key in enumerate(("ux", "uy", "uz")):
            out[key][:, si] = np.where(ff, st[:, 1 + a], 0.0)
        out["T"][:, si] = np.where(ff, st[:, 4], np.where(wl, st[:, 4], T))
        out["U"][:, si] = np.where(ff, np.linalg.norm(st[:, 1:4], axis=1), 0.0)
    return out


def cell_gradients(geo, bc_state, rho, u, T):
    bv = boundary_values(geo, bc_state, rho, u, T)
    gu = np.stack([lsq_grad(geo, u[:, a], bv[k]) for a, k in enumerate(("ux", "uy", "uz"))], axis=2)
    gT = lsq_grad(geo, T, bv["T"])
    return gu, gT          # gu[c, i, j] = d u_j / d x_i


def nsf(mu, gu, gT):
    """Eq. NSF_constitutive (vectorised): sigma[c], q[c]."""
    div = np.trace(gu, axis1=1, axis2=2)
    sym = gu + np.transpose(gu, (0, 2, 1))
    sigma = -mu[:, None, None] * (sym - 2.0 / 3.0 * div[:, None, None] * np.eye(3)[None])
    q = -kappa_monatomic(mu)[:, None] * gT
    return sigma, q


def minmod(a, b):
    return np.where((a > 0) & (b > 0), np.minimum(a, b),
                    np.where((a < 0) & (b < 0), np.maximum(a, b), 0.0))


def _half_range(r, u, T, n, sign):
    """Flux of mass, momentum and energy carried by the molecules of the
    Maxwellian (r, u, T) that cross a face of unit normal n in the direction
    sign * n: the half-range moments of the normal Gaussian N(u.n, T),
    M0 = int_+ xi_n g, M1 = int_+ xi_n^2 g, M2 = int_+ xi_n^3 g, with the
    tangential thermal motion averaged in closed form."""
    un = np.sum(u * n, axis=1)
    st = np.sqrt(T)
    P = 0.5 * (1.0 + sign * erf(un / (np.sqrt(2.0) * st)))
    D = sign * st * np.exp(-0.5 * un * un / T) / np.sqrt(2.0 * np.pi)
    M0 = un * P + D
    M1 = (un * un + T) * P + un * D
    M2 = (un ** 3 + 3.0 * un * T) * P + (un * un + 2.0 * T) * D
    ut = u - un[:, None] * n
    mom = r[:, None] * (M1[:, None] * n + ut * M0[:, None])
    en = 0.5 * r * (M2 + (np.sum(ut * ut, axis=1) + 2.0 * T) * M0)
    return np.concatenate([(r * M0)[:, None], mom, en[:, None]], axis=1)


def kfvs(rL, uL, pL, rR, uR, pR, n):
    """Kinetic flux-vector splitting: the flux of the left Maxwellian's
    molecules moving along +n plus that of the right Maxwellian's molecules
    moving along -n (the Euler flux the discrete-velocity upwind scheme carries
    for Maxwellian states), per unit area through unit normal n."""
    return _half_range(rL, uL, pL / rL, n, 1.0) + _half_range(rR, uR, pR / rR, n, -1.0)


def euler_flux_dot(U, S):
    """Analytic Euler flux of conserved states U[F,5] dotted with vectors S[F,3]."""
    rho = U[:, 0]
    u = U[:, 1:4] / rho[:, None]
    p = (GAMMA - 1.0) * (U[:, 4] - 0.5 * rho * np.sum(u * u, axis=1))
    uS = np.sum(u * S, axis=1)
    return np.concatenate([(rho * uS)[:, None], U[:, 1:4] * uS[:, None] + p[:, None] * S,
                           ((U[:, 4] + p) * uS)[:, None]], axis=1)


def wall_nsf_flux(geo, bc_state, rho, u, T, gu, gT, mu0, omega):
    """NSF flux through every wall face (in the order of the wall faces in
    geo): no mass flux, cell pressure, NSF stress and heat flux at u = 0,
    T = T_w from the cell gradient corrected along the cell-to-face line."""
    wl = geo.bT == BC_WALL
    idx = np.nonzero(wl)[0]
    c = geo.bC[idx]
    Sb = geo.bS[idx]
    Tw = bc_state[geo.bSide[idx], 4]
    e_b = geo.be[idx]
    db = geo.bdist[idx]

    def wall_grad(gc, phic, phiw):
        corr = (phiw - phic) / db - np.sum(gc * e_b, axis=1)
        return gc + corr[:, None] * e_b

    guw = np.stack([wall_grad(gu[c, :, j], u[c, j], 0.0) for j in range(3)], axis=2)
    gTw = wall_grad(gT[c], T[c], Tw)
    sig_w, q_w = nsf(viscosity(Tw, mu0, omega), guw, gTw)
    SigS = np.einsum("fij,fj->fi", sig_w, Sb)
    F = np.zeros((len(idx), 5))
    F[:, 1:4] = (rho[c] * T[c])[:, None] * Sb + SigS
    F[:, 4] = np.sum(q_w * Sb, axis=1)
    return F


def residual(geo, bc_state, U, hot_sigma, hot_q, mu0, omega, bface_corr=None):
    """R_c = -sum over faces of the outward flux (Eq. macro, steady part);
    returns R[N, 5] and the face spectral radii needed by the relaxation.
    bface_corr [boundary faces, 5] is a frozen correction added to the
    boundary face fluxes (used at the walls of DVM cells)."""
    N = geo.N
    rho, u, T = primitives(U)
    p = rho * T
    a = np.sqrt(GAMMA * p / rho)
    mu_c = viscosity(T, mu0, omega)
    gu, gT = cell_gradients(geo, bc_state, rho, u, T)
    R = np.zeros((N, 5))
    lam_sum = np.zeros(N)

    # ---- MUSCL slopes in index space on (rho, u, p)
    prim = np.concatenate([rho[:, None], u, p[:, None]], axis=1)     # [N, 5]
    slopes = np.zeros((N, 3, 5))
    for d in range(3):
        lo = geo.nb[:, d, 0]
        hi = geo.nb[:, d, 1]
        ok = (lo >= 0) & (hi >= 0)
        dm = prim - prim[np.maximum(lo, 0)]
        dp = prim[np.maximum(hi, 0)] - prim
        slopes[:, d, :] = np.where(ok[:, None], minmod(dm, dp), 0.0)

    # ---- interior faces
    L, Rr, d = geo.L, geo.R, geo.dirs
    qL = prim[L] + 0.5 * slopes[L, d, :]
    qR = prim[Rr] - 0.5 * slopes[Rr, d, :]
    Fi = kfvs(qL[:, 0], qL[:, 1:4], qL[:, 4], qR[:, 0], qR[:, 1:4], qR[:, 4], geo.n) * geo.Sabs[:, None]
    uf = 0.5 * (u[L] + u[Rr])
    Tf = 0.5 * (T[L] + T[Rr])
    muf = viscosity(Tf, mu0, omega)
    e = geo.e
    dist = geo.dist

    def face_grad(gc, phiL, phiR):
        gav = 0.5 * (gc[L] + gc[Rr])
        corr = (phiR - phiL) / dist - np.sum(gav * e, axis=1)
        return gav + corr[:, None] * e

    guf = np.stack([face_grad(gu[:, :, j], u[L, j], u[Rr, j]) for j in range(3)], axis=2)
    gTf = face_grad(gT, T[L], T[Rr])
    sig_f, q_f = nsf(muf, guf, gTf)
    Sig = sig_f + 0.5 * (hot_sigma[L] + hot_sigma[Rr])
    Q = q_f + 0.5 * (hot_q[L] + hot_q[Rr])
    SigS = np.einsum("fij,fj->fi", Sig, geo.S)
    Fv = np.concatenate([np.zeros((len(L), 1)), SigS,
                         (np.sum(SigS * uf, axis=1) + np.sum(Q * geo.S, axis=1))[:, None]], axis=1)
    F = Fi + Fv
    np.add.at(R, L, -F)
    np.add.at(R, Rr, F)
    lam = (np.abs(np.sum(0.5 * (u[L] + u[Rr]) * geo.n, axis=1)) + 0.5 * (a[L] + a[Rr])
           + 5.0 * muf / (0.5 * (rho[L] + rho[Rr]) * dist))
    lamS = lam * geo.Sabs
    np.add.at(lam_sum, L, lamS)
    np.add.at(lam_sum, Rr, lamS)

    # ---- boundary faces
    C = geo.bC
    ff = geo.bT == BC_FARFIELD
    wl = geo.bT == BC_WALL
    st = bc_state[geo.bSide]
    Fb = np.zeros((len(C), 5))
    if np.any(ff):
        idx = np.nonzero(ff)[0]
        c = C[idx]
        sr = st[idx]
        Fb[idx] = kfvs(rho[c], u[c], p[c], sr[:, 0], sr[:, 1:4], sr[:, 0] * sr[:, 4],
                       geo.bn[idx]) * geo.bSabs[idx, None]
        # the cell's high-order terms cross the far-field face unchanged (no NSF part)
        Sb = geo.bS[idx]
        SigS = np.einsum("fij,fj->fi", hot_sigma[c], Sb)
        ufb = 0.5 * (u[c] + sr[:, 1:4])
        Fb[idx, 1:4] += SigS
        Fb[idx, 4] += np.sum(SigS * ufb, axis=1) + np.sum(hot_q[c] * Sb, axis=1)
    if np.any(wl):
        idx = np.nonzero(wl)[0]
        Fb[idx] = wall_nsf_flux(geo, bc_state, rho, u, T, gu, gT, mu0, omega)
    if bface_corr is not None:
        Fb = Fb + bface_corr
    np.add.at(R, C, -Fb)
    use = ff | wl
    lam_b = (np.abs(np.sum(u[C] * geo.bn, axis=1)) + a[C] + 5.0 * mu_c[C] / (rho[C] * 2.0 * geo.bdist))
    np.add.at(lam_sum, C[use], (lam_b * geo.bSabs)[use])
    return R, lamS, lam_sum


def relax_step(geo, bc_state, U, hot_sigma, hot_q, mu0, omega, cfl, k_sub, dt=0.0, Un=None, bface_corr=None):
    """One DP-LUR pseudo-time step; returns the new U.  With dt > 0 the
    residual carries the physical-time term of Eq. macro, -V (U - U^n)/dt,
    and the diagonal gains V/dt (dual time stepping)."""
    R, lamS, lam_sum = residual(geo, bc_state, U, hot_sigma, hot_q, mu0, omega, bface_corr)
    D = (1.0 / cfl + 0.5) * lam_sum
    if dt > 0.0:
        vol = geo.topo.vol
        R = R - (vol / dt)[:, None] * (U - Un)
        D = D + vol / dt
    dU = R / D[:, None]
    L, Rr = geo.L, geo.R
    for _ in range(k_sub):
        off = np.zeros_like(U)
        # neighbour R seen from L (S points L->R) and neighbour L seen from R (-S)
        dFR = euler_flux_dot(U[Rr] + dU[Rr], geo.S) - euler_flux_dot(U[Rr], geo.S)
        dFL = euler_flux_dot(U[L] + dU[L], -geo.S) - euler_flux_dot(U[L], -geo.S)
        np.add.at(off, L, 0.5 * (dFR - lamS[:, None] * dU[Rr]))
        np.add.at(off, Rr, 0.5 * (dFL - lamS[:, None] * dU[L]))
        dU = (R - off) / D[:, None]
    return U + dU


def macro_solve(geo, bc_state, U0, hot_sigma, hot_q, mu0, omega, cfl, k_sub, steps, dt=0.0, Un=None,
                bface_corr=None):
    """steps DP-LUR pseudo-time steps of the synthetic equations (Eq. macro)
    from U0.  dt = 0 is the steady form (dt -> infinity); dt > 0 keeps the
    time term (U - Un)/dt of Eq. macro with Un the previous GSIS state.
    bface_corr [boundary faces, 5] is a frozen correction of the boundary
    face fluxes: at the wall of a DVM cell, the kinetic wall flux of f^{n+1/2}
    minus the NSF wall flux at W^{n+1/2}; zero elsewhere."""
    U = U0.copy()
    for _ in range(steps):
        U = relax_step(geo, bc_state, U, hot_sigma, hot_q, mu0, omega, cfl, k_sub, dt, Un, bface_corr)
    return U
