"""Batched solves (gsis_iterate_batch): many independent 1D shocks with uneven
meshes, velocity grids and VDF storage types advanced together (one
persistent sweep launch, one fused synthetic-solve launch, one CUDA graph per
iteration, autotuned tile shape).

Checks: every solve of the batch agrees with the same solve iterated alone
through gsis_iterate (same kernels' arithmetic: agreement to within one
storage rounding unit of the solve's VDF type), and with the FP64 oracle
(FP64 solves within the FP64 tolerance, reduced-precision solves within the
bounds of the precision tests)."""
import numpy as np
import pytest

from workloads import shock_1d_case
from helpers import run_oracle, w_rel_err, rel_err, RTOL_W

pytestmark = pytest.mark.gpu

PREC_BOUND = {"f32": 2e-5, "bf16": 3.9e-3, "f16": 9.8e-4}
UNIT = {"f64": 1e-13, "f32": 2 ** -23, "bf16": 2 ** -8, "f16": 2 ** -10}


def _cases():
    specs = [  # (Ma, cells, velocity grid, dtype)
        (1.6, 23, (16, 8, 8), "f32"),
        (2.4, 37, (20, 10, 9), "bf16"),
        (2.0, 30, (18, 9, 8), "f64"),
        (3.1, 19, (24, 10, 10), "f16"),
    ]
    out = []
    for Ma, n, nv, dt in specs:
        c = shock_1d_case(Ma=Ma, n_cells=n, half_width=n / 4.0, nv=nv, vmax=8.0 + Ma, macro_steps=30)
        out.append((c, dt))
    return out


def test_batch_matches_single_solves_and_oracle():
    from paper_2501_02245_gb300 import Solver, iterate_batch, batch_info
    n_iter = 3
    cases = _cases()
    batch = [Solver.from_case(c, vdf_dtype=dt) for c, dt in cases]
    reps = iterate_batch(batch, n_iter)
    info = batch_info(batch)
    assert "items=" in info and "tile=" in info
    assert all(r["iterations"] == n_iter for r in reps)
    for (case, dt), sb, rep in zip(cases, batch, reps):
        single = Solver.from_case(case, vdf_dtype=dt)
        single.iterate(n_iter)
        Wb, Ws = sb.W(), single.W()
        single.close()
        assert w_rel_err(Wb, Ws) <= 4 * UNIT[dt], "%s batch vs single: %.3e" % (case.name, w_rel_err(Wb, Ws))
        _, ho = run_oracle(case, n_iter)
        Wo = ho[-1]
        if dt == "f64":
            assert w_rel_err(Wb, Wo) < RTOL_W
        else:
            e = max(rel_err(Wb[:, 0], Wo[:, 0]), rel_err(Wb[:, 4], Wo[:, 4]))
            assert e < PREC_BOUND[dt], "%s %s vs oracle: %.3e" % (case.name, dt, e)
        assert np.isfinite(rep["eps"]) and rep["n_dvm"] == case.mesh.ncell
    # a second call reuses the recorded graph and keeps advancing
    reps2 = iterate_batch(batch, 1)
    assert all(r["total_iterations"] == n_iter + 1 for r in reps2)
    for s in batch:
        s.close()


def test_batch_rerecords_after_a_solo_iteration():
    """Iterating one member alone swaps its state buffers; the next batched
    call must notice and record a fresh graph (results stay consistent with
    a solve that did the same sequence alone)."""
    from paper_2501_02245_gb300 import Solver, iterate_batch
    cases = _cases()[:2]
    batch = [Solver.from_case(c, vdf_dtype=dt) for c, dt in cases]
    iterate_batch(batch, 1)
    batch[0].iterate(1)
    iterate_batch(batch, 1)
    ref = Solver.from_case(cases[0][0], vdf_dtype=cases[0][1])
    ref.iterate(3)
    assert w_rel_err(batch[0].W(), ref.W()) <= 4 * UNIT[cases[0][1]]
    for s in batch + [ref]:
        s.close()


def test_batch_of_mixed_dimensions_matches_single_solves():
    """A batch with a 2D member runs every member in the 3-direction sweep
    kernel: the 1D shock and the 2D O-grid (walls, ghost sides, periodic seam)
    must still match the same solves iterated alone."""
    from paper_2501_02245_gb300 import Solver, iterate_batch
    from workloads import cylinder_case
    cyl = cylinder_case(Ma=2.0, Kn=0.1, n_r=8, n_theta=12, nv=(12, 10, 6), adaptive=False, macro_steps=10,
                        cfl=5.0, k_sub=2, vbox=((-10, 10), (-9, 9), (-8, 8)), presolve_max_blocks=2)
    cyl.dt = 0.5
    shock = shock_1d_case(Ma=1.8, n_cells=21, half_width=5.0, nv=(16, 8, 8), vmax=9.0, macro_steps=20)
    cases = [(shock, "f64"), (cyl, "f64"), (shock, "f32")]
    n_iter = 2
    batch = [Solver.from_case(c, vdf_dtype=dt) for c, dt in cases]
    iterate_batch(batch, n_iter)
    for (case, dt), sb in zip(cases, batch):
        single = Solver.from_case(case, vdf_dtype=dt)
        single.iterate(n_iter)
        e = w_rel_err(sb.W(), single.W())
        single.close()
        assert e <= 4 * UNIT[dt], "%s %s batch vs single: %.3e" % (case.name, dt, e)
    for s in batch:
        s.close()


@pytest.mark.parametrize("tile", ["pair1_cb1_w4", "pair2_cb1_w4", "pair1_cb1_w8", "vpt2_cb1_w4"])
def test_batch_velocity_pair_tiles(tile):
    """The persistent batched sweep on pairs of velocities (packed FP32
    arithmetic; FP32/BF16/FP16 members with even nx) forced by the test hook:
    every solve agrees with the same solve iterated alone within one storage
    rounding unit, with a ragged last item (nv not a multiple of 64)."""
    from paper_2501_02245_gb300 import Solver, iterate_batch, batch_info
    from paper_2501_02245_gb300.gsis import set_batch_tile
    specs = [(1.6, 23, (16, 8, 8), "f32"), (2.4, 37, (20, 10, 9), "bf16"), (3.1, 19, (24, 10, 10), "f16"),
             (2.0, 26, (18, 9, 7), "f32")]
    cases = []
    for Ma, n, nv, dt in specs:
        cases.append((shock_1d_case(Ma=Ma, n_cells=n, half_width=n / 4.0, nv=nv, vmax=8.0 + Ma, macro_steps=30), dt))
    set_batch_tile(tile)
    try:
        batch = [Solver.from_case(c, vdf_dtype=dt) for c, dt in cases]
        iterate_batch(batch, 3)
        assert "tile=" + tile in batch_info(batch)
    finally:
        set_batch_tile(None)
    for (case, dt), sb in zip(cases, batch):
        single = Solver.from_case(case, vdf_dtype=dt)
        single.iterate(3)
        e = w_rel_err(sb.W(), single.W())
        single.close()
        assert e <= 4 * UNIT[dt], "%s %s batch vs single: %.3e" % (case.name, dt, e)
    for s in batch:
        s.close()


def test_batch_pair_tile_refused_with_an_fp64_member():
    from paper_2501_02245_gb300 import Solver, iterate_batch, GsisError
    from paper_2501_02245_gb300.gsis import set_batch_tile
    set_batch_tile("pair1_cb1_w4")
    try:
        batch = [Solver.from_case(c, vdf_dtype=dt) for c, dt in _cases()]
        with pytest.raises(GsisError):
            iterate_batch(batch, 1)
        for s in batch:
            s.close()
    finally:
        set_batch_tile(None)
