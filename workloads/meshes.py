"""Structured finite-volume meshes (geometry only).

A mesh is an (ni, nj, nk) block of hexahedral cells indexed (i, j, k) with i
fastest: the flat cell index is c = i + ni * (j + nj * k).  For each index
direction d the faces normal to it are stored as area vectors S (magnitude =
face area, direction = +d) and face centres, in arrays shaped [k, j, i, 3]
with one extra face along d.  Six boundary sides (i-lo, i-hi, j-lo, j-hi,
k-lo, k-hi) carry a type and a state (rho, ux, uy, uz, T); for a wall the
state's T entry is the wall temperature.

Face area vectors are exact vector areas of the (bilinear) faces, so for every
closed cell the outward area vectors sum to zero up to rounding.
"""
from dataclasses import dataclass, field
import numpy as np

BC_NONE = 0       # zero-area side (2D/1D extrusion sides, polar axis): no flux
BC_FARFIELD = 1   # far field / inflow / outflow with a prescribed state
BC_WALL = 2       # diffuse isothermal wall at rest (state[4] = T_wall)
BC_PERIODIC = 3   # periodic wrap in this index direction


@dataclass
class Mesh:
    ni: int
    nj: int
    nk: int
    dim: int                    # number of spatial directions with gradients (1, 2, 3)
    centers: np.ndarray         # [nk, nj, ni, 3]
    volumes: np.ndarray         # [nk, nj, ni]
    S: list                     # S[d]: area vectors, shapes [nk,nj,ni+1,3], [nk,nj+1,ni,3], [nk+1,nj,ni,3]
    xf: list                    # face centres, same shapes as S
    bc_type: np.ndarray         # int32[6]
    bc_state: np.ndarray        # float64[6, 5]  (rho, ux, uy, uz, T)
    name: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def ncell(self):
        return self.ni * self.nj * self.nk

    def flat(self, a):
        """Cell array [nk, nj, ni, ...] -> [ncell, ...] with i fastest."""
        return np.ascontiguousarray(a.reshape((self.ncell,) + a.shape[3:]))


def _bc(types, states=None):
    t = np.asarray(types, dtype=np.int32)
    s = np.zeros((6, 5)) if states is None else np.asarray(states, dtype=np.float64)
    return t, s


def cartesian_1d(n, x0, x1, bc_lo_state, bc_hi_state):
    """Uniform 1D mesh of n cells on [x0, x1] with unit cross-section.

    The j and k sides are zero-flux (BC_NONE); both x ends are far-field
    boundaries with the given (rho, ux, uy, uz, T) states.
    """
    return cartesian_2d(n, 1, x0, x1, 0.0, 1.0, dim=1,
                        bc_types=[BC_FARFIELD, BC_FARFIELD, BC_NONE, BC_NONE, BC_NONE, BC_NONE],
                        bc_states=[bc_lo_state, bc_hi_state] + [[0.0] * 5] * 4, name=f"shock1d_{n}")


def cartesian_2d(ni, nj, x0, x1, y0, y1, dim, bc_types, bc_states, name="cart"):
    """Uniform Cartesian block (unit depth in z)."""
    xs = np.linspace(x0, x1, ni + 1)
    ys = np.linspace(y0, y1, nj + 1)
    zs = np.array([0.0, 1.0])
    return _hexa_block(_tensor_vertices(xs, ys, zs), dim, bc_types, bc_states, name)


def _tensor_vertices(xs, ys, zs):
    X, Y, Z = np.meshgrid(xs, ys, zs, indexing="ij")
    P = np.stack([X, Y, Z], axis=-1)            # [ni+1, nj+1, nk+1, 3]
    return np.ascontiguousarray(P.transpose(2, 1, 0, 3))   # [nk+1, nj+1, ni+1, 3]


def _quad_area(a, b, c, d):
    """Vector area of the bilinear quadrilateral a-b-c-d (exact)."""
    return 0.5 * np.cross(c - a, d - b)


def _hexa_block(P, dim, bc_types, bc_states, name, orient=None):
    """Build a Mesh from a vertex block P[nk+1, nj+1, ni+1, 3].

    Faces normal to i join vertices (j,k),(j+1,k),(j+1,k+1),(j,k+1) at fixed i;
    similarly for j and k.  Each area vector is oriented along +d using the
    vertex-block direction (difference of the adjacent vertex layers), or by
    orient(d, face_centre) when the block degenerates (poles).
    """
    nk, nj, ni = P.shape[0] - 1, P.shape[1] - 1, P.shape[2] - 1
    # i-faces: index [k, j, i] for i in 0..ni
    a = P[:-1, :-1, :]; b = P[:-1, 1:, :]; c = P[1:, 1:, :]; d = P[1:, :-1, :]
    Si = _quad_area(a, b, c, d)
    xi_f = 0.25 * (a + b + c + d)
    # j-faces: [k, j, i] for j in 0..nj ; vertices (i,k),(i+1,k),(i+1,k+1),(i,k+1)
    a = P[:-1, :, :-1]; b = P[:-1, :, 1:]; c = P[1:, :, 1:]; d = P[1:, :, :-1]
    Sj = _quad_area(a, b, c, d)
    xj_f = 0.25 * (a + b + c + d)
    # k-faces: [k, j, i] for k in 0..nk ; vertices (i,j),(i+1,j),(i+1,j+1),(i,j+1)
    a = P[:, :-1, :-1]; b = P[:, :-1, 1:]; c = P[:, 1:, 1:]; d = P[:, 1:, :-1]
    Sk = _quad_area(a, b, c, d)
    xk_f = 0.25 * (a + b + c + d)

    # orientation along +d from the mean edge direction of the vertex block
    def orient_dir(S, xf, d):
        if d == 0:
            e = P[:, :, 1:] - P[:, :, :-1]                        # [nk+1, nj+1, ni, 3]
            e = 0.25 * (e[:-1, :-1] + e[1:, :-1] + e[:-1, 1:] + e[1:, 1:])   # [nk, nj, ni, 3]
            e = np.concatenate([e, e[:, :, -1:]], axis=2)
        elif d == 1:
            e = P[:, 1:, :] - P[:, :-1, :]                        # [nk+1, nj, ni+1, 3]
            e = 0.25 * (e[:-1, :, :-1] + e[1:, :, :-1] + e[:-1, :, 1:] + e[1:, :, 1:])
            e = np.concatenate([e, e[:, -1:, :]], axis=1)
        else:
            e = P[1:, :, :] - P[:-1, :, :]
            e = 0.25 * (e[:, :-1, :-1] + e[:, 1:, :-1] + e[:, :-1, 1:] + e[:, 1:, 1:])
            e = np.concatenate([e, e[-1:, :, :]], axis=0)
        if orient is not None:
            e = orient(d, xf)
        sgn = np.sign(np.einsum("...k,...k->...", S, e))
        sgn[sgn == 0] = 1.0
        return S * sgn[..., None]

    Si = orient_dir(Si, xi_f, 0)
    Sj = orient_dir(Sj, xj_f, 1)
    Sk = orient_dir(Sk, xk_f, 2)

    # volume from the divergence theorem, V = (1/3) sum_F x_F . S_F,out
    def fx(S, X):
        return np.einsum("...k,...k->...", S, X)
    fi = fx(Si, xi_f); fj = fx(Sj, xj_f); fk = fx(Sk, xk_f)
    vol = (fi[:, :, 1:] - fi[:, :, :-1] + fj[:, 1:, :] - fj[:, :-1, :] + fk[1:] - fk[:-1]) / 3.0
    cen = 0.125 * (P[:-1, :-1, :-1] + P[:-1, :-1, 1:] + P[:-1, 1:, :-1] + P[:-1, 1:, 1:]
                   + P[1:, :-1, :-1] + P[1:, :-1, 1:] + P[1:, 1:, :-1] + P[1:, 1:, 1:])
    t, s = _bc(bc_types, bc_states)
    return Mesh(ni, nj, nk, dim, np.ascontiguousarray(cen), np.ascontiguousarray(vol),
                [np.ascontiguousarray(Si), np.ascontiguousarray(Sj), np.ascontiguousarray(Sk)],
                [np.ascontiguousarray(xi_f), np.ascontiguousarray(xj_f), np.ascontiguousarray(xk_f)],
                t, s, name)


def geometric_radii(n, r_in, r_out, dr0):
    """n radial cells from r_in to r_out, first cell dr0, constant growth ratio."""
    if abs(dr0 * n - (r_out - r_in)) < 1e-14:
        return np.linspace(r_in, r_out, n + 1)
    L = r_out - r_in
    lo, hi = 1.0 + 1e-12, 2.0
    if dr0 * n > L:
        lo, hi = 1e-6, 1.0 - 1e-12
    for _ in range(200):
        s = 0.5 * (lo + hi)
        tot = dr0 * (s ** n - 1.0) / (s - 1.0)
        if (tot > L) == (dr0 * n < L):
            hi = s
        else:
            lo = s
    s = 0.5 * (lo + hi)
    r = r_in + dr0 * (s ** np.arange(n + 1) - 1.0) / (s - 1.0)
    r[-1] = r_out
    return r


def cylinder_ogrid(n_r, n_theta, r_in, r_out, dr0, wall_T, farfield_state):
    """Body-fitted O-grid around a circular cylinder (unit depth in z).

    i runs radially (i-lo is the diffuse wall, i-hi the far field), j runs
    around the body and is periodic, k is the extrusion direction (zero flux).
    """
    r = geometric_radii(n_r, r_in, r_out, dr0)
    th = 2.0 * np.pi * np.arange(n_theta + 1) / n_theta
    zs = np.array([0.0, 1.0])
    R, TH, Z = np.meshgrid(r, th, zs, indexing="ij")
    P = np.stack([R * np.cos(TH), R * np.sin(TH), Z], axis=-1).transpose(2, 1, 0, 3)
    P = np.ascontiguousarray(P)
    ff = list(farfield_state)
    states = [[0, 0, 0, 0, wall_T], ff, [0] * 5, [0] * 5, [0] * 5, [0] * 5]
    m = _hexa_block(P, 2, [BC_WALL, BC_FARFIELD, BC_PERIODIC, BC_PERIODIC, BC_NONE, BC_NONE],
                    states, f"cylinder_{n_r}x{n_theta}")
    m.extra["radii"] = r
    return m


def sphere_ogrid(n_r, n_pol, n_az, r_in, r_out, dr0, wall_T, farfield_state):
    """Structured spherical O-grid: i radial (wall at i-lo), j polar angle in
    [0, pi] about the z axis (zero-area faces on the axis), k azimuth (periodic).
    The free stream runs along +x, so the stagnation line lies on the equator."""
    r = geometric_radii(n_r, r_in, r_out, dr0)
    th = np.pi * np.arange(n_pol + 1) / n_pol
    ph = 2.0 * np.pi * np.arange(n_az + 1) / n_az
    R, TH, PH = np.meshgrid(r, th, ph, indexing="ij")
    X = R * np.sin(TH) * np.cos(PH)
    Y = R * np.sin(TH) * np.sin(PH)
    Zc = R * np.cos(TH)
    P = np.ascontiguousarray(np.stack([X, Y, Zc], axis=-1).transpose(2, 1, 0, 3))
    # exact axis points (sin(pi) is not exactly 0 in floating point)
    P[:, 0, :, 0:2] = 0.0
    P[:, -1, :, 0:2] = 0.0

    def orient(d, xf):
        x, y, z = xf[..., 0], xf[..., 1], xf[..., 2]
        rho_xy = np.hypot(x, y)
        rr = np.sqrt(x * x + y * y + z * z)
        phi = np.arctan2(y, x)
        theta = np.arctan2(rho_xy, z)
        if d == 0:
            return xf / rr[..., None]
        if d == 1:
            return np.stack([np.cos(theta) * np.cos(phi), np.cos(theta) * np.sin(phi), -np.sin(theta)], -1)
        return np.stack([-np.sin(phi), np.cos(phi), np.zeros_like(phi)], -1)

    ff = list(farfield_state)
    states = [[0, 0, 0, 0, wall_T], ff, [0] * 5, [0] * 5, [0] * 5, [0] * 5]
    m = _hexa_block(P, 3, [BC_WALL, BC_FARFIELD, BC_NONE, BC_NONE, BC_PERIODIC, BC_PERIODIC],
                    states, f"sphere_{n_r}x{n_pol}x{n_az}", orient=orient)
    # the axis faces are degenerate; make their area exactly zero
    m.S[1][:, 0, :, :] = 0.0
    m.S[1][:, -1, :, :] = 0.0
    m.extra["radii"] = r
    return m
