"""Unstructured meshes for the oracle (test infrastructure only).

The paper's three-dimensional runs (Secs. 4.3, 4.4) use unstructured spatial
meshes; it describes neither their data structures nor their reconstruction.
This module gives the oracle polygon meshes (2D, unit depth in z, like the
structured 2D meshes) and convex polyhedral meshes (3D: tetrahedra, pyramids,
prisms, hexahedra) with the interface the transport sweep of
oracle.kinetic and the synthetic solve of oracle.macro use, so that the
whole GSIS iteration of oracle.gsis runs on them unchanged.  Readings:

* face values are first order (the upwind cell value): index-space slopes do
  not exist on such a mesh, and the paper does not state the unstructured
  reconstruction; the synthetic solve's splitting is first order too;
* the Gauss-Seidel order is by a per-cell key (default x + y (+ z) of the
  centroid, i.e. the diagonal hyperplanes of a square or cubic structured grid); cells with
  nearly equal keys are not face neighbours on the meshes used here, so the
  order inside such a group does not change the result;
* the wall layers of the region rule (Sec. 4.4) are the cells within
  `wall_layers` face-neighbour steps of a wall face.

Boundary faces carry a tag 0..5 that indexes bc_type / bc_state, as the six
sides of a structured block do.
"""
from dataclasses import dataclass
import numpy as np

from .mesh import Side, BC_NONE, BC_FARFIELD, BC_WALL
from .macro import MacroGeometry
from .gsis import OracleSolver
from .reduced import ReducedGrid
from .hybrid import HybridGrid
from . import model as M


@dataclass
class PolygonMesh:
    """vertices [nV, 2]; cells: vertex-index lists in counter-clockwise order
    (3 to 6 vertices); boundary: {(a, b) with a < b: tag} for every edge that
    belongs to one cell only; bc_type [6], bc_state [6][5] per tag; W0 [N, 5];
    key: optional per-cell sweep-order key."""
    vertices: np.ndarray
    cells: list
    boundary: dict
    bc_type: list
    bc_state: np.ndarray
    W0: np.ndarray = None
    key: np.ndarray = None
    dim: int = 2

    @property
    def ncell(self):
        return len(self.cells)


def polygon_geometry(P):
    """Area and centroid of a simple polygon with counter-clockwise vertices P [m, 2]."""
    x, y = P[:, 0], P[:, 1]
    xn, yn = np.roll(x, -1), np.roll(y, -1)
    cr = x * yn - xn * y
    A = 0.5 * np.sum(cr)
    cx = np.sum((x + xn) * cr) / (6.0 * A)
    cy = np.sum((y + yn) * cr) / (6.0 * A)
    return A, np.array([cx, cy])


class _FaceTopology:
    """The interface of oracle.mesh.Topology built from per-cell face lists:
    sides with outward area vectors, face centres, neighbours across shared
    faces (matched by their vertex sets) and tagged boundary faces; no
    index-space steps (step() is always -1, so face values are first order)."""

    def _build(self, faces, boundary, bc_type, key):
        # faces[c]: list of (vertex-set id, outward S (3,), face centre (3,))
        owner = {}
        for c, fl in enumerate(faces):
            for fid, _, _ in fl:
                owner.setdefault(fid, []).append(c)
        self.sides = []
        for c, fl in enumerate(faces):
            sides = []
            for fid, S, xf in fl:
                own = owner[fid]
                nb = [o for o in own if o != c]
                if nb:
                    assert len(own) == 2
                    n = nb[0]
                    sides.append(Side(0, 1 if n > c else -1, S, xf, n, -1, -1))
                else:
                    tag = int(boundary[fid])
                    sides.append(Side(0, 1, S, xf, -1, int(bc_type[tag]), tag))
            assert len(sides) <= 6
            self.sides.append(sides)
        self.key = (np.asarray(key, dtype=np.float64) if key is not None
                    else np.sum(self.centers[:, :self.dim], axis=1))

    def step(self, c, d, s):
        return -1

    def hyperplane(self, c):
        return self.key[c]

    def interior_faces(self):
        L, R, S = [], [], []
        for c in range(self.ncell):
            for sd in self.sides[c]:
                if sd.s > 0 and sd.nbr >= 0:
                    L.append(c); R.append(sd.nbr); S.append(sd.S_out)
        return np.array(L, dtype=np.int64), np.array(R, dtype=np.int64), np.array(S)

    def boundary_faces(self):
        C, S, X, B, T = [], [], [], [], []
        for c in range(self.ncell):
            for sd in self.sides[c]:
                if sd.nbr < 0 and sd.bc in (BC_FARFIELD, BC_WALL):
                    C.append(c); S.append(sd.S_out); X.append(sd.xf); B.append(sd.bc_side); T.append(sd.bc)
        return (np.array(C, dtype=np.int64), np.array(S).reshape(-1, 3), np.array(X).reshape(-1, 3),
                np.array(B, dtype=np.int64), np.array(T, dtype=np.int64))


class UnstructuredTopology(_FaceTopology):
    """A PolygonMesh: area vectors (dy, -dx, 0) of each counter-clockwise edge
    (unit depth), edge midpoints, neighbours across shared edges."""

    def __init__(self, mesh):
        self.mesh = mesh
        self.ncell = mesh.ncell
        self.dim = 2
        self.n = (self.ncell, 1, 1)
        V = np.asarray(mesh.vertices, dtype=np.float64)
        self.vol = np.zeros(self.ncell)
        self.centers = np.zeros((self.ncell, 3))
        faces = []
        for c, cell in enumerate(mesh.cells):
            assert 3 <= len(cell) <= 6
            A, ctr = polygon_geometry(V[cell])
            assert A > 0.0, "cell %d is not counter-clockwise" % c
            self.vol[c] = A
            self.centers[c] = [ctr[0], ctr[1], 0.5]
            fl = []
            for a, b in zip(cell, cell[1:] + cell[:1]):
                d = V[b] - V[a]
                fl.append(((min(a, b), max(a, b)), np.array([d[1], -d[0], 0.0]),
                           np.array([0.5 * (V[a, 0] + V[b, 0]), 0.5 * (V[a, 1] + V[b, 1]), 0.5])))
            faces.append(fl)
        self._build(faces, mesh.boundary, mesh.bc_type, mesh.key)


@dataclass
class PolyhedralMesh:
    """vertices [nV, 3]; cells: lists of faces, each face a vertex-index list
    in cyclic order (either orientation: faces are turned outward from the
    cell's vertex mean; convex cells), 4 to 6 faces per cell; boundary:
    {sorted vertex tuple of a face: tag} for every face of one cell only;
    bc_type [6], bc_state [6][5] per tag; W0 [N, 5]; key as for PolygonMesh."""
    vertices: np.ndarray
    cells: list
    boundary: dict
    bc_type: list
    bc_state: np.ndarray
    W0: np.ndarray = None
    key: np.ndarray = None
    dim: int = 3

    @property
    def ncell(self):
        return len(self.cells)


def face_vector_area(Vf):
    """Vector area and centroid of a planar polygon Vf [m, 3] in the given
    cyclic order: fan of triangles from the vertex mean (the vector area of a
    closed polygon does not depend on the fan point)."""
    p = Vf.mean(axis=0)
    S = np.zeros(3)
    num = np.zeros(3)
    m = len(Vf)
    tri = []
    for i in range(m):
        s = 0.5 * np.cross(Vf[i] - p, Vf[(i + 1) % m] - p)
        S += s
        tri.append((s, (p + Vf[i] + Vf[(i + 1) % m]) / 3.0))
    n = S / np.linalg.norm(S)
    A = 0.0
    for s, c in tri:
        a = np.dot(s, n)
        A += a
        num += a * c
    return S, num / A


def polyhedron_geometry(V, faces):
    """Volume and centroid of a convex polyhedron (faces as vertex-index lists,
    turned outward): tetrahedra from the vertex mean to the fan triangles of
    each face."""
    p = V[sorted({v for f in faces for v in f})].mean(axis=0)
    vol, num = 0.0, np.zeros(3)
    for f in faces:
        Vf = V[f]
        fc = Vf.mean(axis=0)
        for i in range(len(f)):
            a, b = Vf[i], Vf[(i + 1) % len(f)]
            v = np.dot(fc - p, np.cross(a - p, b - p)) / 6.0
            vol += v
            num += v * (p + fc + a + b) / 4.0
    return vol, num / vol


class PolyhedralTopology(_FaceTopology):
    """A PolyhedralMesh: outward vector areas and centroids of the faces,
    neighbours across shared faces."""

    def __init__(self, mesh):
        self.mesh = mesh
        self.ncell = mesh.ncell
        self.dim = 3
        self.n = (self.ncell, 1, 1)
        V = np.asarray(mesh.vertices, dtype=np.float64)
        self.vol = np.zeros(self.ncell)
        self.centers = np.zeros((self.ncell, 3))
        faces = []
        for c, cell in enumerate(mesh.cells):
            assert 4 <= len(cell) <= 6
            p = V[sorted({v for f in cell for v in f})].mean(axis=0)
            oriented, fl = [], []
            for f in cell:
                S, xf = face_vector_area(V[f])
                if np.dot(S, xf - p) < 0.0:
                    f = list(f)[::-1]
                    S = -S
                oriented.append(list(f))
                fl.append((tuple(sorted(f)), S, xf))
            vol, ctr = polyhedron_geometry(V, oriented)
            assert vol > 0.0
            self.vol[c] = vol
            self.centers[c] = ctr
            faces.append(fl)
        self._build(faces, mesh.boundary, mesh.bc_type, mesh.key)


def topology_of(mesh):
    """The face topology of a PolygonMesh or a PolyhedralMesh."""
    return PolyhedralTopology(mesh) if isinstance(mesh, PolyhedralMesh) else UnstructuredTopology(mesh)


class UnstructuredGeometry(MacroGeometry):
    """oracle.macro.MacroGeometry on an UnstructuredTopology, without the
    index-space neighbour table (first-order face states)."""

    def __init__(self, topo):
        super().__init__(topo)
        self.nb[:] = -1


class UnstructuredSolver(OracleSolver):
    """oracle.gsis.OracleSolver on a PolygonMesh or a PolyhedralMesh (case.mesh)
    with a uniform, reduced or hybrid velocity grid (case.vgrid may be a
    HybridGrid)."""

    def __init__(self, case, flags_override=None):
        self.case = case
        self.topo = topology_of(case.mesh)
        self.geo = UnstructuredGeometry(self.topo)
        if isinstance(case.vgrid, HybridGrid):
            self.vg = case.vgrid
        elif getattr(case.vgrid, "reduced", False):
            self.vg = ReducedGrid(case.vgrid.n, case.vgrid.lo, case.vgrid.hi)
        else:
            self.vg = M.VelocityGrid(case.vgrid.n, case.vgrid.lo, case.vgrid.hi)
        self.mu0 = M.mu0_from_kn(case.Kn)
        self.omega = case.omega
        self.bc_state = np.array(case.mesh.bc_state, dtype=np.float64)
        self.W = np.array(case.W0, dtype=np.float64)
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

    def region(self, W):
        """Kn_Gll >= Kn_ref, plus the cells within wall_layers face-neighbour
        steps of a wall face."""
        if self.flags_override is not None:
            return np.array(self.flags_override, dtype=bool)
        self.kn_gll = self.kn_gll_field(W)
        return (self.kn_gll >= self.case.Kn_ref) | wall_layer_flags(self.topo, self.case.wall_layers)


def wall_layer_flags(topo, layers):
    """Cells within `layers` face-neighbour steps of a wall face (the first
    layer touches the wall)."""
    flag = np.zeros(topo.ncell, dtype=bool)
    front = [c for c in range(topo.ncell) if any(sd.bc == BC_WALL for sd in topo.sides[c])]
    seen = set(front)
    for _ in range(layers):
        nxt = []
        for c in front:
            flag[c] = True
            for sd in topo.sides[c]:
                if sd.nbr >= 0 and sd.nbr not in seen:
                    seen.add(sd.nbr); nxt.append(sd.nbr)
        front = nxt
    return flag
