"""Every tile shape of the kinetic sweep (register-stencil shapes and the
shared-memory hyperplane-window shapes) computes the same GSIS iterations:
each is forced in turn on a 2D O-grid whose velocity count leaves a ragged
last tile and whose periodic seam puts neighbours outside the hyperplane
window, and compared with the FP64 oracle (FP64 storage: the FP64 tolerance;
FP32 storage: the FP32 bound of the precision tests)."""
import numpy as np
import pytest

from workloads import cylinder_case
from helpers import run_oracle, w_rel_err, rel_err, RTOL_W

pytestmark = pytest.mark.gpu

TILES = {
    "f64": ["g2_v1_c2", "g1_v1_c2", "g4_v1_c1", "g2_v1_c1", "g8_v1_c1", "g16_v1_c1", "ring_w8_v32", "ring_w4_v32"],
    "f32": ["g8_v1_c1", "g4_v1_c1", "g8_v2_c1", "g4_v4_c1", "g8_v4_c1", "g4_v2_c2",
            "p8_v1_c1", "p4_v2_c1", "p8_v2_c1", "p4_v1_c1", "p5_v2_c1", "ring_w8_v32", "ring_w4_v32",
            "ring_w8_v64"],
}


def _case():
    case = cylinder_case(Ma=2.0, Kn=0.1, n_r=10, n_theta=16, nv=(14, 12, 6), adaptive=False, macro_steps=10,
                         cfl=5.0, k_sub=2, vbox=((-10, 10), (-9, 9), (-8, 8)), presolve_max_blocks=2)
    case.dt = 0.5
    return case


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_every_sweep_tile_matches_the_oracle(dtype):
    from paper_2501_02245_gb300 import Solver
    case = _case()
    n_iter = 2
    _, ho = run_oracle(case, n_iter)
    results = {}
    for tile in TILES[dtype]:
        s = Solver.from_case(case, vdf_dtype=dtype)
        s.set_sweep_tile(tile)
        assert tile in s.tuning_info()
        s.iterate(n_iter)
        W = s.W()
        s.close()
        results[tile] = W
        if dtype == "f64":
            assert w_rel_err(W, ho[-1]) < RTOL_W, "%s: %.3e" % (tile, w_rel_err(W, ho[-1]))
        else:
            e = max(rel_err(W[:, 0], ho[-1][:, 0]), rel_err(W[:, 4], ho[-1][:, 4]))
            assert e < 2e-5, "%s: %.3e" % (tile, e)
    ref = results[TILES[dtype][0]]
    for tile, W in results.items():
        assert w_rel_err(W, ref) <= (1e-12 if dtype == "f64" else 1e-5), tile
    if dtype == "f32":   # the packed pair update performs the same roundings as the single-velocity one
        for tile in ("p8_v1_c1", "p4_v2_c1", "p8_v2_c1", "p4_v1_c1", "p5_v2_c1"):
            assert np.array_equal(results[tile], ref), tile


def test_unknown_tile_is_rejected():
    from paper_2501_02245_gb300 import Solver, GsisError
    s = Solver.from_case(_case(), vdf_dtype="f64")
    with pytest.raises(GsisError):
        s.set_sweep_tile("no_such_tile")
    with pytest.raises(GsisError):
        s.set_sweep_tile("ring_w8_v64")   # FP64 has no 64-velocity window shape
    s.close()
    case = _case()
    case.vgrid = type(case.vgrid)((13, 12, 6), case.vgrid.lo, case.vgrid.hi)
    s = Solver.from_case(case, vdf_dtype="f32")
    with pytest.raises(GsisError):
        s.set_sweep_tile("p8_v1_c1")      # velocity pairs need an even nx
    s.close()
