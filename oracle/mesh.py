"""Structured-mesh connectivity and least-squares gradients (oracle; test
infrastructure only).

Cells are (i, j, k) with flat index c = i + ni (j + nj k).  A cell has six
sides (d, s) for direction d in {0,1,2} and s = -1 (low) / +1 (high).  Across a
side lies either another cell (interior, or wrapped in a periodic direction)
or a boundary of type NONE / FARFIELD / WALL.  In a periodic direction of n
cells the face between cell n-1 and cell 0 is face 0 of the stored face array
(the stored face n is not used).
"""
from dataclasses import dataclass
import numpy as np

BC_NONE, BC_FARFIELD, BC_WALL, BC_PERIODIC = 0, 1, 2, 3


@dataclass
class Side:
    d: int
    s: int                 # -1 low side, +1 high side
    S_out: np.ndarray      # outward area vector (3,)
    xf: np.ndarray         # face centre
    nbr: int               # neighbour flat cell index, or -1 for a boundary
    bc: int                # boundary type if nbr == -1, else BC_PERIODIC/-1
    bc_side: int           # 0..5 boundary side index (2d + (s>0)) if boundary


class Topology:
    def __init__(self, mesh):
        self.mesh = mesh
        self.ni, self.nj, self.nk = mesh.ni, mesh.nj, mesh.nk
        self.n = (mesh.ni, mesh.nj, mesh.nk)
        self.ncell = mesh.ncell
        self.dim = mesh.dim
        self.centers = mesh.flat(mesh.centers)
        self.vol = mesh.flat(mesh.volumes)
        self.periodic = [mesh.bc_type[2 * d] == BC_PERIODIC for d in range(3)]
        for d in range(3):
            if self.periodic[d]:
                assert mesh.bc_type[2 * d + 1] == BC_PERIODIC and self.n[d] >= 3
        self.sides = [self._cell_sides(c) for c in range(self.ncell)]

    def ijk(self, c):
        i = c % self.ni
        j = (c // self.ni) % self.nj
        k = c // (self.ni * self.nj)
        return i, j, k

    def flat(self, i, j, k):
        return i + self.ni * (j + self.nj * k)

    def step(self, c, d, s):
        """Cell index one step along (d, s), or -1 at a non-periodic boundary."""
        idx = list(self.ijk(c))
        m = idx[d] + s
        if m < 0 or m >= self.n[d]:
            if not self.periodic[d]:
                return -1
            m %= self.n[d]
        idx[d] = m
        return self.flat(*idx)

    def _face(self, d, i, j, k, face_index):
        idx = [i, j, k]
        idx[d] = face_index
        return self.mesh.S[d][idx[2], idx[1], idx[0]], self.mesh.xf[d][idx[2], idx[1], idx[0]]

    def _cell_sides(self, c):
        i, j, k = self.ijk(c)
        out = []
        for d in range(3):
            m = (i, j, k)[d]
            for s in (-1, 1):
                if s < 0:
                    fi = m
                else:
                    fi = m + 1
                    if self.periodic[d] and fi == self.n[d]:
                        fi = 0
                S, xf = self._face(d, i, j, k, fi)
                S_out = S * s
                nb = self.step(c, d, s)
                bs = 2 * d + (1 if s > 0 else 0)
                bc = -1 if nb >= 0 else int(self.mesh.bc_type[bs])
                out.append(Side(d, s, np.array(S_out, dtype=np.float64), np.array(xf), nb, bc, bs))
        return out

    def hyperplane(self, c):
        i, j, k = self.ijk(c)
        return i + j + k

    def interior_faces(self):
        """Each interior (or periodic) face once: (L, R, S pointing L->R)."""
        L, R, S = [], [], []
        for c in range(self.ncell):
            for sd in self.sides[c]:
                if sd.s > 0 and sd.nbr >= 0:
                    L.append(c); R.append(sd.nbr); S.append(sd.S_out)
        return np.array(L, dtype=np.int64), np.array(R, dtype=np.int64), np.array(S)

    def boundary_faces(self):
        """Each FARFIELD/WALL boundary face: (cell, outward S, face centre, side index, type)."""
        C, S, X, B, T = [], [], [], [], []
        for c in range(self.ncell):
            for sd in self.sides[c]:
                if sd.nbr < 0 and sd.bc in (BC_FARFIELD, BC_WALL):
                    C.append(c); S.append(sd.S_out); X.append(sd.xf); B.append(sd.bc_side); T.append(sd.bc)
        return (np.array(C, dtype=np.int64), np.array(S).reshape(-1, 3), np.array(X).reshape(-1, 3),
                np.array(B, dtype=np.int64), np.array(T, dtype=np.int64))


def lsq_gradient(topo, phi, bvalue):
    """Unweighted least-squares cell gradient (Sec. 3.4, Step 2 names the least
    squares method; the stencil is the reading taken: the face neighbours, plus
    the boundary face centre with its boundary value on FARFIELD/WALL sides).

    phi: [ncell] cell values.  bvalue(c, side) -> boundary value of phi.
    Returns [ncell, 3]; components beyond the mesh dimension are zero.
    """
    dim = topo.dim
    g = np.zeros((topo.ncell, 3))
    for c in range(topo.ncell):
        rows, rhs = [], []
        for sd in topo.sides[c]:
            if sd.nbr >= 0:
                rows.append(topo.centers[sd.nbr] - topo.centers[c])
                rhs.append(phi[sd.nbr] - phi[c])
            elif sd.bc in (BC_FARFIELD, BC_WALL):
                rows.append(sd.xf - topo.centers[c])
                rhs.append(bvalue(c, sd) - phi[c])
        A = np.array(rows)[:, :dim]
        b = np.array(rhs)
        G = A.T @ A
        g[c, :dim] = np.linalg.solve(G, A.T @ b)
    return g
