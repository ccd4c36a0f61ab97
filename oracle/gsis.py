"""The adaptive GSIS iteration (Secs. 3.1, 3.2, 3.4 and the convergence
criterion of Sec. 4) in plain FP64 numpy (oracle; test infrastructure only).

One GSIS iteration n -> n+1:
 1. reference state: for each DVM cell, g~ from W^n and the heat flux of f^n,
    tau = mu(T)/p (Sec. 2); Grad-13 ghosts (Eq. G13_VDF) for NS cells next to
    DVM cells from W^n and NSF stress/heat flux; diffuse-wall densities;
 2. kinetic step (oracle.kinetic.sweep) -> f^{n+1/2};
 3. moments of f^{n+1/2} (Eq. getmoment) -> W^{n+1/2}; HoT = kinetic stress /
    heat flux minus NSF at W^{n+1/2} (Eq. full_constitutive), zero in NS cells;
 4. synthetic solve (Eq. macro) over ALL cells from W^{n+1/2} -> W^{n+1};
 5. Eq. updatef in DVM cells: f^{n+1} = f^{n+1/2} + M~(W^{n+1}) - M~(W^{n+1/2});
 6. residual epsilon between W^{n+1} and W^n (convergence criterion, Sec. 4).
Adaptive runs (Sec. 3.4): Step 1 NS presolve, Step 2 region from Eq. Kn_Gll,
Step 3 one re-identification after `adapt_every` GSIS iterations.
"""
import numpy as np

from . import model as M
from .reduced import ReducedGrid
from .mesh import Topology, BC_NONE, BC_FARFIELD, BC_WALL
from .kinetic import KineticInputs, sweep, wall_density, wall_kinetic_flux
from .macro import (MacroGeometry, primitives, cell_gradients, nsf, macro_solve, boundary_values, lsq_grad,
                    wall_nsf_flux)


def residual_eps(Wn, Wp, vol):
    """Convergence criterion of Sec. 4: max over W in {rho, u, T} of
    sqrt(sum (W^n - W^{n-1})^2 Omega / sum (W^{n-1})^2 Omega).  The velocity
    is taken as one vector quantity (|du|^2 over |u|^2); a quantity whose
    denominator is exactly zero (a gas initially at rest) is left out."""
    out = [0.0]
    for sl in (slice(0, 1), slice(1, 4), slice(4, 5)):
        num = np.sum(np.sum((Wn[:, sl] - Wp[:, sl]) ** 2, axis=1) * vol)
        den = np.sum(np.sum(Wp[:, sl] ** 2, axis=1) * vol)
        if den > 0.0:
            out.append(np.sqrt(num / den))
    return max(out)


def prim_to_U(W):
    U = np.zeros_like(W)
    for c in range(W.shape[0]):
        U[c] = M.conserved_from_primitive(W[c, 0], W[c, 1:4], W[c, 4])
    return U


def U_to_prim(U):
    rho, u, T = primitives(U)
    return np.concatenate([rho[:, None], u, T[:, None]], axis=1)


class OracleSolver:
    def __init__(self, case, flags_override=None):
        self.case = case
        self.topo = Topology(case.mesh)
        self.geo = MacroGeometry(self.topo)
        if getattr(case.vgrid, "reduced", False):   # 2D flow: xi_z integrated out (oracle.reduced)
            self.vg = ReducedGrid(case.vgrid.n, case.vgrid.lo, case.vgrid.hi)
        else:
            self.vg = M.VelocityGrid(case.vgrid.n, case.vgrid.lo, case.vgrid.hi)
        self.mu0 = M.mu0_from_kn(case.Kn)
        self.omega = case.omega
        self.bc_state = np.array(case.mesh.bc_state, dtype=np.float64)
        self.W = np.array(case.W0, dtype=np.float64)       # [N, 5] rho, u, T
        self.N = self.topo.ncell
        self.f = np.zeros((self.N, self.vg.nv))
        self.dvm = np.zeros(self.N, dtype=bool)
        self.flags_override = flags_override
        self.eps_history = []
        self.W_history = []
        self.kn_gll = np.zeros(self.N)
        self.hot_sigma = np.zeros((self.N, 3, 3))
        self.hot_q = np.zeros((self.N, 3))
        self.iteration = 0
        self.presolve_blocks = 0

    # ----------------------------------------------------------------- helpers
    def gradients(self, W):
        rho, u, T = W[:, 0], W[:, 1:4], W[:, 4]
        return cell_gradients(self.geo, self.bc_state, rho, u, T)

    def nsf_field(self, W):
        gu, gT = self.gradients(W)
        mu = M.viscosity(W[:, 4], self.mu0, self.omega)
        return nsf(mu, gu, gT)

    def kn_gll_field(self, W):
        """Eq. Kn_Gll: lambda * max(|grad rho|/rho, |grad U|/U, |grad T|/T) with
        lambda = mu(T)/p sqrt(pi T / 2) (the local analogue of the Kn
        definition) and U divided by max(U, a), a the sound speed, so that
        stagnation points (U -> 0) stay finite."""
        rho, u, T = W[:, 0], W[:, 1:4], W[:, 4]
        U = np.linalg.norm(u, axis=1)
        bv = boundary_values(self.geo, self.bc_state, rho, u, T)
        g_rho = lsq_grad(self.geo, rho, bv["rho"])
        g_U = lsq_grad(self.geo, U, bv["U"])
        g_T = lsq_grad(self.geo, T, bv["T"])
        a = np.sqrt(M.GAMMA * T)
        lam = M.viscosity(T, self.mu0, self.omega) / (rho * T) * np.sqrt(np.pi * T / 2.0)
        r = np.maximum(np.maximum(np.linalg.norm(g_rho, axis=1) / rho,
                                  np.linalg.norm(g_U, axis=1) / np.maximum(U, a)),
                       np.linalg.norm(g_T, axis=1) / T)
        return lam * r

    def region(self, W):
        """DVM-region rule of Sec. 3.2: 1 where Kn_Gll >= Kn_ref, plus the
        wall_layers cell layers next to a wall (Sec. 4.4)."""
        if self.flags_override is not None:
            return np.array(self.flags_override, dtype=bool)
        self.kn_gll = self.kn_gll_field(W)
        flag = self.kn_gll >= self.case.Kn_ref
        mesh = self.case.mesh
        if self.case.wall_layers > 0:
            for d in range(3):
                for hi in (0, 1):
                    if mesh.bc_type[2 * d + hi] != BC_WALL:
                        continue
                    for c in range(self.N):
                        m = self.topo.ijk(c)[d]
                        dist = m if hi == 0 else self.topo.n[d] - 1 - m
                        if dist < self.case.wall_layers:
                            flag[c] = True
        return flag

    def seed_vdf(self, cells, W):
        """Grad-13 VDF (Eq. G13_VDF) from W and its NSF stress / heat flux,
        conservation-corrected to W, for cells that enter the DVM region."""
        sig, q = self.nsf_field(W)
        for c in cells:
            rho, u, T = W[c, 0], W[c, 1:4], W[c, 4]
            g13 = self.vg.grad13(rho, u, T, sig[c], q[c])
            Mx = self.vg.maxwellian(rho, u, T)
            self.f[c] = self.vg.conservation_correct(g13, Mx, M.conserved_from_primitive(rho, u, T))

    def set_region(self, new_flags, W):
        entering = [c for c in range(self.N) if new_flags[c] and not self.dvm[c]]
        leaving = [c for c in range(self.N) if self.dvm[c] and not new_flags[c]]
        for c in leaving:
            self.f[c] = 0.0
        self.dvm = np.array(new_flags, dtype=bool)
        if entering:
            self.seed_vdf(entering, W)

    # ----------------------------------------------------------------- phases
    def presolve(self):
        """Sec. 3.4 Step 1: the macroscopic equations (HoT = 0) until the
        criterion of Sec. 4 holds between blocks of macro_steps pseudo-steps."""
        zs = np.zeros((self.N, 3, 3)); zq = np.zeros((self.N, 3))
        U = prim_to_U(self.W)
        for b in range(self.case.presolve_max_blocks):
            Wp = U_to_prim(U)
            U = macro_solve(self.geo, self.bc_state, U, zs, zq, self.mu0, self.omega,
                            self.case.cfl, self.case.k_sub, self.case.macro_steps)
            self.presolve_blocks = b + 1
            if residual_eps(U_to_prim(U), Wp, self.topo.vol) < self.case.tol:
                break
        self.W = U_to_prim(U)

    def initialise(self):
        # Sec. 3.4 Step 1: the initial field from the macroscopic equations (also
        # used to start an all-kinetic run when presolve blocks are requested)
        if self.case.presolve_max_blocks > 0:
            self.presolve()
        if self.case.adaptive:
            self.set_region(self.region(self.W), self.W)
        else:
            self.dvm[:] = True
            for c in range(self.N):
                rho, u, T = self.W[c, 0], self.W[c, 1:4], self.W[c, 4]
                self.f[c] = self.vg.corrected_maxwellian(rho, u, T)

    def kinetic_inputs(self):
        W = self.W
        vg = self.vg
        gt, tau, ghost, ff, mw = {}, {}, {}, {}, {}
        for c in range(self.N):
            if not self.dvm[c]:
                continue
            rho, u, T = W[c, 0], W[c, 1:4], W[c, 4]
            q = vg.heat_flux_about(self.f[c], u)
            gt[c] = vg.corrected_shakhov(rho, u, T, q)
            tau[c] = M.viscosity(T, self.mu0, self.omega) / (rho * T)
        need = set()
        for c in range(self.N):
            if self.dvm[c]:
                for sd in self.topo.sides[c]:
                    if sd.nbr >= 0 and not self.dvm[sd.nbr]:
                        need.add(sd.nbr)
        if need:
            sig, qn = self.nsf_field(W)
            for c in need:
                rho, u, T = W[c, 0], W[c, 1:4], W[c, 4]
                g13 = vg.grad13(rho, u, T, sig[c], qn[c])
                Mx = vg.maxwellian(rho, u, T)
                ghost[c] = vg.conservation_correct(g13, Mx, M.conserved_from_primitive(rho, u, T))
        for s in range(6):
            st = self.bc_state[s]
            if self.case.mesh.bc_type[s] == BC_FARFIELD:
                ff[s] = vg.corrected_maxwellian(st[0], st[1:4], st[4])
            elif self.case.mesh.bc_type[s] == BC_WALL:
                mw[s] = vg.maxwellian(1.0, np.zeros(3), st[4])
        return KineticInputs(gt, tau, ghost, ff, mw)

    def wall_correction(self, W_half, mw):
        """Per wall face (order of the wall faces of the macro geometry): for a
        DVM cell, the kinetic wall flux of f^{n+1/2} minus the NSF wall flux at
        W^{n+1/2}; zero for NS cells.  Added to the NSF wall flux inside the
        synthetic solve."""
        geo = self.geo
        idx = np.nonzero(geo.bT == BC_WALL)[0]
        corr = np.zeros((len(idx), 5))
        if len(idx) == 0:
            return corr
        gu, gT = self.gradients(W_half)
        F_nsf = wall_nsf_flux(geo, self.bc_state, W_half[:, 0], W_half[:, 1:4], W_half[:, 4], gu, gT,
                              self.mu0, self.omega)
        for r, f_i in enumerate(idx):
            c = geo.bC[f_i]
            if self.dvm[c]:
                F_kin = wall_kinetic_flux(self.f[c], geo.bS[f_i], mw[geo.bSide[f_i]], self.vg)
                corr[r] = F_kin - F_nsf[r]
        return corr

    def wall_loads(self):
        """Per cell, per unit wall area: [heat flux into the wall, wall pressure,
        wall shear stress (3)], 0 without wall sides.  Each wall side's flux
        F (mass, momentum, energy through its outward area vector S) is carried
        by the current distribution for a DVM cell (outgoing half of f,
        re-emitted rho_w M(0, T_w) with zero net mass flux) and by the NSF wall
        flux at the current state for an NS cell.  The momentum flux is the
        force on the wall: pressure = F_m . n, shear = F_m - (F_m . n) n with
        n = S/|S|; sums over the cell's wall sides divided by their area."""
        geo = self.geo
        idx = np.nonzero(geo.bT == BC_WALL)[0]
        num = np.zeros((self.N, 5)); area = np.zeros(self.N)
        if len(idx) == 0:
            return num
        gu, gT = self.gradients(self.W)
        F_nsf = wall_nsf_flux(geo, self.bc_state, self.W[:, 0], self.W[:, 1:4], self.W[:, 4], gu, gT,
                              self.mu0, self.omega)
        for r, f_i in enumerate(idx):
            c = geo.bC[f_i]
            if self.dvm[c]:
                Mw = self.vg.maxwellian(1.0, np.zeros(3), self.bc_state[geo.bSide[f_i], 4])
                F = wall_kinetic_flux(self.f[c], geo.bS[f_i], Mw, self.vg)
            else:
                F = F_nsf[r]
            n = geo.bS[f_i] / geo.bSabs[f_i]
            Fn = np.dot(F[1:4], n)
            num[c, 0] += F[4]
            num[c, 1] += Fn
            num[c, 2:5] += F[1:4] - Fn * n
            area[c] += geo.bSabs[f_i]
        has = area > 0
        return np.where(has[:, None], num / np.where(has, area, 1.0)[:, None], 0.0)

    def wall_heat_flux(self):
        """Heat flux into the wall per unit area, per cell (0 without wall
        sides): the first column of wall_loads."""
        return self.wall_loads()[:, 0]

    def constitutive(self):
        """Eq. full_constitutive at the current state: sigma = sigma_NSF(W) +
        HoT_sigma and q = q_NSF(W) + HoT_q, with the HoT of the last iteration
        (zero in NS cells and before the first iteration) -- the stress and heat
        flux of the synthetic equations, equal to the kinetic moments at a
        converged state."""
        sig_n, q_n = self.nsf_field(self.W)
        return sig_n + self.hot_sigma, q_n + self.hot_q

    def step(self):
        """One GSIS iteration; returns epsilon."""
        case = self.case
        if case.adaptive and self.iteration == case.adapt_every and self.flags_override is None:
            self.set_region(self.region(self.W), self.W)
        vg = self.vg
        inp = self.kinetic_inputs()
        sweep(self.topo, vg, self.f, self.dvm, inp)
        # moments of f^{n+1/2}
        W_half = self.W.copy()
        sig_k = np.zeros((self.N, 3, 3)); q_k = np.zeros((self.N, 3))
        for c in range(self.N):
            if self.dvm[c]:
                rho, u, T, sig, q = vg.moments(self.f[c])
                W_half[c] = [rho, u[0], u[1], u[2], T]
                sig_k[c] = sig; q_k[c] = q
        sig_n, q_n = self.nsf_field(W_half)
        self.hot_sigma = np.where(self.dvm[:, None, None], sig_k - sig_n, 0.0)
        self.hot_q = np.where(self.dvm[:, None], q_k - q_n, 0.0)
        self.W_half = W_half
        bcorr = np.zeros((len(self.geo.bC), 5))
        bcorr[self.geo.bT == BC_WALL] = self.wall_correction(W_half, inp.mw)
        U = macro_solve(self.geo, self.bc_state, prim_to_U(W_half), self.hot_sigma, self.hot_q,
                        self.mu0, self.omega, case.cfl, case.k_sub, case.macro_steps,
                        case.dt, prim_to_U(self.W), bcorr)
        W_new = U_to_prim(U)
        if case.relax != 1.0:
            W_new = W_half + case.relax * (W_new - W_half)
        for c in range(self.N):
            if self.dvm[c]:
                a = vg.corrected_maxwellian(W_new[c, 0], W_new[c, 1:4], W_new[c, 4])
                b = vg.corrected_maxwellian(W_half[c, 0], W_half[c, 1:4], W_half[c, 4])
                self.f[c] = self.f[c] + a - b
        eps = residual_eps(W_new, self.W, self.topo.vol)
        self.W = W_new
        self.eps_history.append(eps)
        self.W_history.append(W_new.copy())
        self.iteration += 1
        return eps

    def run(self, iterations=None):
        self.initialise()
        n = self.case.iterations if iterations is None else iterations
        for _ in range(n):
            self.step()
        return self
