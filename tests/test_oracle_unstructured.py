"""Pins of the unstructured-mesh and hybrid-velocity-grid oracle
(oracle.unstructured, oracle.hybrid; CPU only).

* The hybrid grid with uniform partitions is the uniform midpoint grid of
  oracle.model (every distribution and moment); with stretched partitions
  its discrete Maxwellian moments converge to the closed forms, its
  corrected distributions conserve exactly, the Shakhov heat flux is
  (1 - Pr) q and a Grad-13 distribution carries its stress and heat flux.
* Polygon geometry: areas and centroids in closed form, closed cells, least
  squares exact for linear fields on triangles.
* Polyhedra: tetrahedron and box closed forms; a conforming tetrahedral split
  of a box gives closed, outward cells and exact least squares.
* A square structured grid given as polygons, and a cubic one given as
  hexahedra, run the GSIS iteration of the structured oracle with first-order
  faces (same values); a uniform stream is a fixed point of the iteration on
  triangles and on tetrahedra (with a hybrid grid it moves by the
  second-order quadrature error); a heated channel on triangles with a
  hybrid grid and an adaptive region keeps Eq. updatef's conservation.
"""
import numpy as np
import pytest

from workloads.cases import Case, VGrid
from workloads.meshes import cartesian_2d, BC_FARFIELD, BC_WALL, BC_NONE
from oracle import model as M
from oracle.hybrid import HybridGrid, stretched_edges
from oracle.unstructured import PolygonMesh, UnstructuredTopology, UnstructuredGeometry, UnstructuredSolver, \
    polygon_geometry
from oracle.macro import lsq_grad
from oracle.gsis import OracleSolver

STATE = dict(rho=1.3, u=np.array([0.4, -0.25, 0.15]), T=1.6)
SIGMA = np.array([[0.05, -0.02, 0.01], [-0.02, -0.03, 0.005], [0.01, 0.005, -0.02]])
Q = np.array([0.07, -0.04, 0.03])


# ----------------------------------------------------------------------------- hybrid velocity grid
def test_uniform_hybrid_grid_is_the_midpoint_grid():
    n, lo, hi = (10, 8, 6), (-7.0, -6.0, -5.0), (8.0, 6.0, 7.0)
    g = M.VelocityGrid(n, lo, hi)
    h = HybridGrid(*[np.linspace(lo[d], hi[d], n[d] + 1) for d in range(3)])
    assert np.allclose(h.xi, g.xi, rtol=0, atol=1e-14) and np.allclose(h.wv, g.w, rtol=1e-14)
    s = STATE
    for fg, fh in ((g.corrected_maxwellian(s["rho"], s["u"], s["T"]), h.corrected_maxwellian(s["rho"], s["u"], s["T"])),
                   (g.corrected_shakhov(s["rho"], s["u"], s["T"], Q), h.corrected_shakhov(s["rho"], s["u"], s["T"], Q))):
        assert np.max(np.abs(fg - fh)) < 1e-13 * np.max(fg)
    f = g.grad13(s["rho"], s["u"], s["T"], SIGMA, Q)
    for a, b in zip(g.moments(f), h.moments(f)):
        assert np.allclose(a, b, rtol=1e-12, atol=1e-14)


def _stretched(n=36, ratio=1.08, box=10.0, centre=(0.3, -0.2, 0.1)):
    return HybridGrid(*[stretched_edges(-box, box, n, centre[d], ratio) for d in range(3)])


def test_stretched_partition():
    e = stretched_edges(-10.0, 10.0, 36, 0.3, 1.08)
    w = np.diff(e)
    assert len(e) == 37 and e[0] == -10.0 and abs(e[-1] - 10.0) < 1e-12 and np.any(np.abs(e - 0.3) < 1e-12)
    assert w.max() / w.min() > 3.0          # genuinely non-uniform: fine near the centre, coarse in the tails


def _errors(h):
    """Errors of the discrete moments against their closed forms: mass,
    velocity, temperature of a Maxwellian; heat flux (1 - Pr) q = q/3 of the
    corrected Shakhov form; stress and heat flux of a Grad-13 distribution."""
    s = STATE
    rho, u, T = s["rho"], s["u"], s["T"]
    r, uu, TT, _, _ = h.moments(h.maxwellian(rho, u, T))
    qs = h.heat_flux_about(h.corrected_shakhov(rho, u, T, Q), u)
    _, _, _, sg, q = h.moments(h.grad13(rho, u, T, SIGMA, Q))
    return np.array([abs(r / rho - 1), np.max(np.abs(uu - u)), abs(TT / T - 1), np.max(np.abs(qs - Q / 3.0)),
                     np.max(np.abs(sg - SIGMA)), np.max(np.abs(q - Q))])


def test_stretched_hybrid_grid_moments_and_conservation():
    """On a grid whose cells are 4 times wider in the tails than at the
    centre the midpoint rule is second order: halving every cell (twice the
    cells, the square root of the growth ratio) divides each error against
    the closed forms by about 4.  The corrected forms conserve exactly."""
    e1 = _errors(_stretched(36, 1.08))
    e2 = _errors(_stretched(72, 1.08 ** 0.5))
    assert np.all(e1 / e2 > 3.0) and np.all(e2 < 2e-3)
    h = _stretched()
    s = STATE
    U = M.conserved_from_primitive(s["rho"], s["u"], s["T"])
    for f in (h.corrected_maxwellian(s["rho"], s["u"], s["T"]), h.corrected_shakhov(s["rho"], s["u"], s["T"], Q)):
        assert np.max(np.abs(h.conserved(f) - U)) < 1e-13 * np.max(np.abs(U))
    assert np.max(np.abs(h.conserved(h.maxwellian(s["rho"], s["u"], s["T"])) - U)) > 1e-4   # not trivial


# ----------------------------------------------------------------------------- polygon geometry
def _quad_mesh(ni, nj, x0, x1, y0, y1, tags, bc_type, bc_state, triangles=False):
    """Structured vertices (i, j) -> i + (ni+1) j; quads (or two triangles
    each) in the flat order c = i + ni j; boundary tags (x-lo, x-hi, y-lo,
    y-hi) as the sides of a structured block."""
    xs, ys = np.linspace(x0, x1, ni + 1), np.linspace(y0, y1, nj + 1)
    V = np.array([[x, y] for y in ys for x in xs])
    vid = lambda i, j: i + (ni + 1) * j
    cells = []
    for j in range(nj):
        for i in range(ni):
            a, b, c, d = vid(i, j), vid(i + 1, j), vid(i + 1, j + 1), vid(i, j + 1)
            cells += [[a, b, c], [a, c, d]] if triangles else [[a, b, c, d]]
    bnd = {}
    for i in range(ni):
        bnd[tuple(sorted((vid(i, 0), vid(i + 1, 0))))] = tags[2]
        bnd[tuple(sorted((vid(i, nj), vid(i + 1, nj))))] = tags[3]
    for j in range(nj):
        bnd[tuple(sorted((vid(0, j), vid(0, j + 1))))] = tags[0]
        bnd[tuple(sorted((vid(ni, j), vid(ni, j + 1))))] = tags[1]
    return PolygonMesh(V, cells, bnd, list(bc_type), np.asarray(bc_state, dtype=np.float64))


FF_STATES = [[1.0, 0.3, 0.1, 0.0, 1.0]] * 6


def test_polygon_geometry_closed_forms():
    A, c = polygon_geometry(np.array([[0.0, 0.0], [2.0, 0.0], [0.0, 1.0]]))
    assert abs(A - 1.0) < 1e-15 and np.allclose(c, [2.0 / 3.0, 1.0 / 3.0])
    m = _quad_mesh(5, 4, 0.0, 1.5, -0.5, 0.7, (0, 1, 2, 3), [BC_FARFIELD] * 4 + [BC_NONE] * 2, FF_STATES,
                   triangles=True)
    t = UnstructuredTopology(m)
    assert abs(np.sum(t.vol) - 1.5 * 1.2) < 1e-13
    for c in range(t.ncell):
        assert np.max(np.abs(sum(sd.S_out for sd in t.sides[c]))) < 1e-15      # closed cells
        for sd in t.sides[c]:
            assert np.dot(sd.S_out[:2], sd.xf[:2] - t.centers[c, :2]) > 0       # outward


def test_least_squares_gradient_exact_for_linear_fields_on_triangles():
    m = _quad_mesh(5, 4, 0.0, 1.5, -0.5, 0.7, (0, 1, 2, 3), [BC_FARFIELD] * 4 + [BC_NONE] * 2, FF_STATES,
                   triangles=True)
    t = UnstructuredTopology(m)
    geo = UnstructuredGeometry(t)
    lin = lambda p: 0.7 - 1.3 * p[..., 0] + 2.1 * p[..., 1]
    phi = lin(t.centers)
    bv = np.zeros((t.ncell, 6))
    for c in range(t.ncell):
        for si, sd in enumerate(t.sides[c]):
            bv[c, si] = lin(sd.xf)
    g = lsq_grad(geo, phi, bv)
    assert np.allclose(g[:, 0], -1.3, atol=1e-12) and np.allclose(g[:, 1], 2.1, atol=1e-12)
    assert np.all(geo.nb == -1)


# ----------------------------------------------------------------------------- GSIS iteration
def _channel(unstructured, triangles=False, vgrid=None):
    """Channel flow between two diffuse walls at T_w = 1.5 (y = 0, 1) with
    far-field ends (x = 0, 1.5), square cells of 1/4, gas entering at
    u = (0.6, 0, 0): wall heating and shear make every term of the
    iteration act."""
    W_in = [1.0, 0.6, 0.0, 0.0, 1.0]
    W_out = [1.0, 0.6, 0.0, 0.0, 1.0]
    wall = [1.0, 0.0, 0.0, 0.0, 1.5]
    bc_type = [BC_FARFIELD, BC_FARFIELD, BC_WALL, BC_WALL, BC_NONE, BC_NONE]
    bc_state = [W_in, W_out, wall, wall, [0.0] * 5, [0.0] * 5]
    if unstructured:
        mesh = _quad_mesh(6, 4, 0.0, 1.5, 0.0, 1.0, (0, 1, 2, 3), bc_type, bc_state, triangles=triangles)
        n = mesh.ncell
    else:
        mesh = cartesian_2d(6, 4, 0.0, 1.5, 0.0, 1.0, dim=2, bc_types=bc_type, bc_states=bc_state)
        n = mesh.ncell
    vg = vgrid or VGrid((10, 10, 6), (-7.0, -7.0, -6.0), (8.0, 7.0, 6.0))
    W0 = np.tile(W_in, (n, 1))
    return Case("channel", mesh, vg, W0, Kn=0.1, adaptive=False, macro_steps=10, cfl=5.0, k_sub=2,
                iterations=2, presolve_max_blocks=0, dt=0.5)


def test_square_polygons_run_the_structured_iteration(monkeypatch):
    """The structured grid given as polygons (same cell order) and the
    structured oracle, both with first-order faces in the kinetic step and
    the synthetic solve: two GSIS iterations give the same states and VDFs
    (sums in a different order only)."""
    from oracle import kinetic as K, macro as Mac
    monkeypatch.setattr(K, "slope", lambda *a: 0.0)
    monkeypatch.setattr(Mac, "minmod", lambda a, b: np.zeros_like(a))
    o = OracleSolver(_channel(False)).run(2)
    u = UnstructuredSolver(_channel(True)).run(2)
    assert np.max(np.abs(o.W - o.W_history[0])) > 1e-3          # the state moved
    assert np.max(np.abs(u.W - o.W)) < 1e-12 * np.max(np.abs(o.W))
    assert np.max(np.abs(u.f - o.f)) < 1e-12 * np.max(np.abs(o.f))
    assert np.allclose(u.eps_history, o.eps_history, rtol=1e-10)
    assert np.allclose(u.wall_heat_flux(), o.wall_heat_flux(), rtol=1e-10, atol=1e-14)


def _uniform_stream(vgrid):
    W = [1.0, 0.4, -0.2, 0.0, 1.2]
    st = [W] * 4 + [[0.0] * 5] * 2
    mesh = _quad_mesh(5, 4, 0.0, 1.5, -0.5, 0.7, (0, 1, 2, 3), [BC_FARFIELD] * 4 + [BC_NONE] * 2, st,
                      triangles=True)
    case = Case("uniform", mesh, vgrid, np.tile(W, (mesh.ncell, 1)), Kn=0.1, adaptive=False, macro_steps=10,
                iterations=2, presolve_max_blocks=0)
    s = UnstructuredSolver(case).run(2)
    return np.max(np.abs(s.W - case.W0)), max(s.eps_history)


def test_uniform_stream_is_a_fixed_point_on_triangles():
    """Far field on every side with one state: on a triangle mesh with a
    velocity grid that resolves the Maxwellian (the midpoint rule is then
    spectrally accurate, so its discrete stress and heat flux vanish to
    rounding) the uniform stream stays uniform through the GSIS iteration."""
    dW, eps = _uniform_stream(VGrid((24, 24, 20), (-10.0,) * 3, (10.0,) * 3))
    assert dW < 1e-12 and eps < 1e-12


def test_uniform_stream_on_a_hybrid_grid_moves_at_quadrature_order():
    """On a stretched hybrid grid the corrected Maxwellian carries a stress
    and heat flux of the size of the (second-order) quadrature error, which
    the far-field faces pass on: the uniform stream moves by that much, and
    halving every velocity cell divides the move by about 4."""
    grids = []
    for k, r in ((1, 1.1), (2, 1.1 ** 0.5)):
        grids.append(HybridGrid(*[stretched_edges(-9.0, 9.0, n * k, c, r) for n, c in ((16, 0.4), (14, -0.2),
                                                                                        (10, 0.0))]))
    d1, _ = _uniform_stream(grids[0])
    d2, _ = _uniform_stream(grids[1])
    assert d1 < 1e-3 and d1 / d2 > 3.0


def test_heated_channel_on_triangles_with_a_hybrid_grid_converges():
    """The channel on a triangle mesh with a stretched hybrid grid, adaptive
    region with one wall layer: the iteration runs, every kinetic cell
    carries the new conserved moments after Eq. updatef, the residual falls,
    and the gas heats up at the walls."""
    hg = HybridGrid(*[stretched_edges(-8.0, 9.0, n, c, 1.1) for n, c in ((16, 0.6), (14, 0.0), (8, 0.0))])
    case = _channel(True, triangles=True, vgrid=hg)
    case.adaptive, case.Kn_ref, case.wall_layers, case.adapt_every = True, 1e9, 1, 1000
    s = UnstructuredSolver(case)
    s.initialise()
    touching = {c for c in range(s.N) if any(sd.bc == BC_WALL for sd in s.topo.sides[c])}
    assert set(np.nonzero(s.dvm)[0]) == touching and 0 < len(touching) < s.N   # one wall layer
    for _ in range(4):
        s.step()
        for c in np.nonzero(s.dvm)[0]:
            Uf = s.vg.conserved(s.f[c])
            Uw = M.conserved_from_primitive(s.W[c, 0], s.W[c, 1:4], s.W[c, 4])
            assert np.max(np.abs(Uf - Uw)) < 1e-12 * np.max(np.abs(Uw))
    e = s.eps_history
    assert e[-1] < e[0] and np.max(s.W[:, 4]) > 1.0 + 1e-3


# ----------------------------------------------------------------------------- 3D polyhedra
from oracle.unstructured import PolyhedralMesh, PolyhedralTopology, face_vector_area, polyhedron_geometry  # noqa: E402
from workloads.meshes import _hexa_block, _tensor_vertices  # noqa: E402


def _box_mesh(n, lo, hi, bc_type, bc_state, tets=False):
    """A box of n = (ni, nj, nk) cells as hexahedra (flat order c = i + ni (j +
    nj k), faces in the order x-lo, x-hi, y-lo, y-hi, z-lo, z-hi) or as six
    tetrahedra each (the split along each cube's main diagonal, conforming
    between neighbouring cubes); boundary tags 0..5 = x-lo .. z-hi."""
    ax = [np.linspace(lo[d], hi[d], n[d] + 1) for d in range(3)]
    V = np.array([[x, y, z] for z in ax[2] for y in ax[1] for x in ax[0]])
    vid = lambda i, j, k: i + (n[0] + 1) * (j + (n[1] + 1) * k)
    cells = []
    for k in range(n[2]):
        for j in range(n[1]):
            for i in range(n[0]):
                v = {(a, b, c): vid(i + a, j + b, k + c) for a in (0, 1) for b in (0, 1) for c in (0, 1)}
                if tets:
                    for perm in ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)):
                        path = [(0, 0, 0)]
                        for d in perm:
                            q = list(path[-1]); q[d] = 1; path.append(tuple(q))
                        t = [v[q] for q in path]
                        cells.append([[t[0], t[1], t[2]], [t[0], t[1], t[3]], [t[0], t[2], t[3]], [t[1], t[2], t[3]]])
                else:
                    cells.append([[v[0, 0, 0], v[0, 1, 0], v[0, 1, 1], v[0, 0, 1]],
                                  [v[1, 0, 0], v[1, 1, 0], v[1, 1, 1], v[1, 0, 1]],
                                  [v[0, 0, 0], v[1, 0, 0], v[1, 0, 1], v[0, 0, 1]],
                                  [v[0, 1, 0], v[1, 1, 0], v[1, 1, 1], v[0, 1, 1]],
                                  [v[0, 0, 0], v[1, 0, 0], v[1, 1, 0], v[0, 1, 0]],
                                  [v[0, 0, 1], v[1, 0, 1], v[1, 1, 1], v[0, 1, 1]]])
    count = {}
    for cell in cells:
        for f in cell:
            count[tuple(sorted(f))] = count.get(tuple(sorted(f)), 0) + 1
    bnd = {}
    for fid, m in count.items():
        if m == 1:
            P = V[list(fid)]
            for d in range(3):
                if np.all(np.abs(P[:, d] - lo[d]) < 1e-12):
                    bnd[fid] = 2 * d
                elif np.all(np.abs(P[:, d] - hi[d]) < 1e-12):
                    bnd[fid] = 2 * d + 1
    return PolyhedralMesh(V, cells, bnd, list(bc_type), np.asarray(bc_state, dtype=np.float64))


FF3 = [[1.0, 0.3, 0.1, -0.2, 1.0]] * 6


def test_polyhedron_geometry_closed_forms():
    V = np.array([[0.0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]])
    vol, c = polyhedron_geometry(V, [[0, 2, 1], [0, 1, 3], [0, 3, 2], [1, 2, 3]])
    assert abs(vol - 1.0 / 6.0) < 1e-15 and np.allclose(c, 0.25)
    S, xf = face_vector_area(np.array([[0.0, 0, 0], [2, 0, 0], [2, 3, 0], [0, 3, 0]]))
    assert np.allclose(S, [0, 0, 6.0]) and np.allclose(xf, [1.0, 1.5, 0.0])
    for tets in (False, True):
        m = _box_mesh((3, 2, 2), (0.0, -0.5, 0.2), (1.2, 0.3, 1.0), [BC_FARFIELD] * 6, FF3, tets=tets)
        t = PolyhedralTopology(m)
        assert t.ncell == 12 * (6 if tets else 1)
        assert abs(np.sum(t.vol) - 1.2 * 0.8 * 0.8) < 1e-13
        for c in range(t.ncell):
            assert np.max(np.abs(sum(sd.S_out for sd in t.sides[c]))) < 1e-15
            for sd in t.sides[c]:
                assert np.dot(sd.S_out, sd.xf - t.centers[c]) > 0
        assert len(m.boundary) == (2 * (6 + 6 + 4) if not tets else 2 * 2 * (6 + 6 + 4))


def test_least_squares_gradient_exact_for_linear_fields_on_tetrahedra():
    m = _box_mesh((3, 2, 2), (0.0, -0.5, 0.2), (1.2, 0.3, 1.0), [BC_FARFIELD] * 6, FF3, tets=True)
    t = PolyhedralTopology(m)
    geo = UnstructuredGeometry(t)
    lin = lambda p: 0.7 - 1.3 * p[..., 0] + 2.1 * p[..., 1] + 0.4 * p[..., 2]
    bv = np.zeros((t.ncell, 6))
    for c in range(t.ncell):
        for si, sd in enumerate(t.sides[c]):
            bv[c, si] = lin(sd.xf)
    g = lsq_grad(geo, lin(t.centers), bv)
    assert np.allclose(g, [-1.3, 2.1, 0.4], atol=1e-12)


def _box_case(poly, tets=False, vgrid=None):
    """Gas entering a box of cubic cells through the x ends, heated by
    diffuse walls at y = 0, 0.75 (T_w = 1.5); no flux through the z sides."""
    W_in = [1.0, 0.6, 0.0, 0.1, 1.0]
    wall = [1.0, 0.0, 0.0, 0.0, 1.5]
    bc_type = [BC_FARFIELD, BC_FARFIELD, BC_WALL, BC_WALL, BC_NONE, BC_NONE]
    bc_state = [W_in, W_in, wall, wall, [0.0] * 5, [0.0] * 5]
    n, lo, hi = (4, 3, 2), (0.0, 0.0, 0.0), (1.0, 0.75, 0.5)
    if poly:
        mesh = _box_mesh(n, lo, hi, bc_type, bc_state, tets=tets)
    else:
        ax = [np.linspace(lo[d], hi[d], n[d] + 1) for d in range(3)]
        mesh = _hexa_block(_tensor_vertices(*ax), 3, bc_type, bc_state, "box")
    vg = vgrid or VGrid((8, 8, 6), (-7.0, -7.0, -6.0), (8.0, 7.0, 6.0))
    return Case("box", mesh, vg, np.tile(W_in, (mesh.ncell, 1)), Kn=0.1, adaptive=False, macro_steps=8,
                cfl=5.0, k_sub=2, iterations=2, presolve_max_blocks=0, dt=0.5)


def test_hexahedra_run_the_structured_3d_iteration(monkeypatch):
    """A box of cubic cells given as hexahedra and as a structured block, both
    with first-order faces: two GSIS iterations give the same states and
    VDFs."""
    from oracle import kinetic as K, macro as Mac
    monkeypatch.setattr(K, "slope", lambda *a: 0.0)
    monkeypatch.setattr(Mac, "minmod", lambda a, b: np.zeros_like(a))
    o = OracleSolver(_box_case(False)).run(2)
    u = UnstructuredSolver(_box_case(True)).run(2)
    assert np.max(np.abs(o.W - o.W_history[0])) > 1e-3
    assert np.max(np.abs(u.W - o.W)) < 1e-12 * np.max(np.abs(o.W))
    assert np.max(np.abs(u.f - o.f)) < 1e-12 * np.max(np.abs(o.f))
    assert np.allclose(u.eps_history, o.eps_history, rtol=1e-10)


def test_uniform_stream_is_a_fixed_point_on_tetrahedra():
    """Far field on every side: a uniform stream (with all three velocity
    components) stays uniform on the tetrahedral split of a box, with a
    velocity grid that resolves its Maxwellian."""
    W = [1.0, 0.4, -0.2, 0.15, 1.2]
    mesh = _box_mesh((3, 2, 2), (0.0, -0.5, 0.2), (1.2, 0.3, 1.0), [BC_FARFIELD] * 6, [W] * 6, tets=True)
    case = Case("uniform3", mesh, VGrid((28, 28, 28), (-11.0,) * 3, (11.0,) * 3), np.tile(W, (mesh.ncell, 1)),
                Kn=0.1, adaptive=False, macro_steps=8, iterations=2, presolve_max_blocks=0)
    s = UnstructuredSolver(case).run(2)
    assert np.max(np.abs(s.W - case.W0)) < 1e-12 and max(s.eps_history) < 1e-12
