"""Sweep levels of unstructured meshes (gsis_sweep_levels, host code of the
library; CPU only): the hyperplanes of a structured grid, the two level
properties on a triangle mesh, the sequential Gauss-Seidel values when the
oracle's sweep visits the cells level by level, and the refusals."""
import numpy as np
import pytest

from paper_2501_02245_gb300 import gsis
from oracle.unstructured import UnstructuredTopology, UnstructuredSolver
from workloads.meshes import BC_FARFIELD, BC_NONE
from test_oracle_unstructured import _quad_mesh, _channel


@pytest.fixture(scope="module", autouse=True)
def _library():
    from paper_2501_02245_gb300 import build
    build.build()   # host code of the library: builds here without a GPU


def _adjacency(topo):
    return [[sd.nbr for sd in topo.sides[c] if sd.nbr >= 0] for c in range(topo.ncell)]


def test_levels_of_a_structured_grid_are_its_hyperplanes():
    ni, nj, nk = 5, 4, 3
    nb, key = [], []
    for k in range(nk):
        for j in range(nj):
            for i in range(ni):
                l = []
                for d, n in ((0, ni), (1, nj), (2, nk)):
                    idx = [i, j, k]
                    for s in (-1, 1):
                        m = idx[d] + s
                        if 0 <= m < n:
                            idx2 = list(idx); idx2[d] = m
                            l.append(idx2[0] + ni * (idx2[1] + nj * idx2[2]))
                nb.append(l)
                key.append(0.3 * i + 0.3 * j + 0.3 * k)
    lv, n = gsis.sweep_levels(nb, key)
    hp = [i + j + k for k in range(nk) for j in range(nj) for i in range(ni)]
    assert np.array_equal(lv, hp) and n == ni + nj + nk - 2


def test_level_properties_on_triangles():
    m = _quad_mesh(6, 5, 0.0, 1.5, -0.5, 0.7, (0, 1, 2, 3), [BC_FARFIELD] * 4 + [BC_NONE] * 2,
                   [[1.0, 0.3, 0.1, 0.0, 1.0]] * 6, triangles=True)
    t = UnstructuredTopology(m)
    adj = _adjacency(t)
    lv, n = gsis.sweep_levels(adj, t.key)
    order = sorted(range(t.ncell), key=lambda c: (t.key[c], c))
    rank = {c: r for r, c in enumerate(order)}
    for c in range(t.ncell):
        for nbr in adj[c]:
            assert lv[nbr] != lv[c]                                    # face neighbours never share a level
            assert (lv[nbr] < lv[c]) == (rank[nbr] < rank[c])           # earlier neighbours lie lower
    assert n == lv.max() + 1 and 1 < n < t.ncell                        # parallel work in the levels


def test_level_order_sweep_reproduces_the_sequential_sweep():
    """The oracle's Gauss-Seidel sweep visiting the cells level by level (cells
    of a level by index) gives bit for bit the values of its sequential
    sweep in key order, on a triangulated channel with walls."""
    seq = UnstructuredSolver(_channel(True, triangles=True)).run(2)
    lev = UnstructuredSolver(_channel(True, triangles=True))
    lv, _ = gsis.sweep_levels(_adjacency(lev.topo), lev.topo.key)
    lev.topo.hyperplane = lambda c: int(lv[c])
    order_seq = sorted(range(seq.N), key=lambda c: (seq.topo.key[c], c))
    order_lev = sorted(range(lev.N), key=lambda c: (lv[c], c))
    assert order_seq != order_lev                                       # a different visiting order
    lev.run(2)
    assert np.array_equal(lev.f, seq.f) and np.array_equal(lev.W, seq.W)


def test_refusals():
    ok = [[1], [0]]
    assert gsis.sweep_levels([], [])[1] == 0
    for nb, key in (([[1], []], [0.0, 1.0]),          # asymmetric
                    ([[0], []], [0.0, 1.0]),          # self-neighbour
                    ([[2], [0]], [0.0, 1.0]),         # out of range
                    (ok, [0.0, np.nan])):             # non-finite key
        with pytest.raises(gsis.GsisError):
            gsis.sweep_levels(nb, key)
    assert list(gsis.sweep_levels(ok, [1.0, 0.0])[0]) == [1, 0]


def test_levels_on_tetrahedra_reproduce_the_sequential_sweep():
    """The same two properties, and the level-by-level sweep equal bit for bit
    to the sequential one, on the tetrahedral split of a heated box."""
    from test_oracle_unstructured import _box_case
    seq = UnstructuredSolver(_box_case(True, tets=True)).run(2)
    lev = UnstructuredSolver(_box_case(True, tets=True))
    adj = _adjacency(lev.topo)
    lv, n = gsis.sweep_levels(adj, lev.topo.key)
    rank = {c: r for r, c in enumerate(sorted(range(lev.N), key=lambda c: (lev.topo.key[c], c)))}
    for c in range(lev.N):
        for nbr in adj[c]:
            assert lv[nbr] != lv[c] and (lv[nbr] < lv[c]) == (rank[nbr] < rank[c])
    assert 1 < n < lev.N
    lev.topo.hyperplane = lambda c: int(lv[c])
    lev.run(2)
    assert np.array_equal(lev.f, seq.f) and np.array_equal(lev.W, seq.W)
