"""The algorithmic constants bench.py reports its rooflines with, recomputed here from
their definitions (the oracle's flop count and the bytes a stage must move)."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_flops_per_cell_stage_matches_oracle_count():
    import af_inputs as ai
    import bench
    import oracle
    spec = ai.config2(256)
    st = [a.numpy() for a in ai.initial_state(spec)]
    fc = oracle.flop_count(spec, st, 1e-4)
    per_cell = (fc["add"] + fc["mul"] + fc["div"] + fc["exp"]) / spec.cells
    assert abs(per_cell - bench.FLOPS_PER_CELL_STAGE) < 0.01


def test_bytes_per_cell_stage():
    import bench
    # SSP-RK3 over three stages: stage 1 reads u0 and writes u1; stages 2 and 3 read the
    # stage input and u0 and write their output -> (2 + 3 + 3) / 3 arrays of each DoF
    # kind per stage; a cell owns 1 average + 3 point values.
    arrays = (2 + 3 + 3) / 3
    assert np.isclose(bench.BYTES_PER_CELL_STAGE["fp64"], round(arrays * 4 * 8, 2), atol=0.01)
    assert np.isclose(bench.BYTES_PER_CELL_STAGE["fp32_mixed"], round(arrays * (8 + 3 * 4), 2), atol=0.01)
    # SSP-RK(5,4): stage passes 2, 3, 3, 5 (reads U3, U0, U2, writes U1, U2), 3 over 5 stages
    arrays54 = (2 + 3 + 3 + 5 + 3) / 5
    assert np.isclose(bench.BYTES_PER_CELL_STAGE_RK54["fp64"], arrays54 * 4 * 8)
    assert np.isclose(bench.BYTES_PER_CELL_STAGE_RK54["fp32_mixed"], arrays54 * (8 + 3 * 4))


def test_flops_per_cell_stage_1d_match_oracle_count():
    import af_inputs as ai
    import bench
    import oracle
    for form in ("dc", "nodc"):
        spec = ai.evje_karlsen(65536, diffusion_form=form)
        st = [a.numpy() for a in ai.initial_state(spec)]
        fc = oracle.flop_count(spec, st, 0.3 * oracle.dt_cfl(spec, st[0]))
        per_cell = (fc["add"] + fc["mul"] + fc["div"] + fc["exp"]) / spec.cells
        assert abs(per_cell - bench.FLOPS_PER_CELL_STAGE_1D[form]) < 0.01


def test_bytes_per_cell_stage_1d():
    import bench
    arrays = (2 + 3 + 3) / 3     # SSP-RK3 state passes per stage; a cell owns ub and one point
    assert np.isclose(bench.BYTES_PER_CELL_STAGE_1D["fp64"], round(arrays * 2 * 8, 2), atol=0.01)
    assert np.isclose(bench.BYTES_PER_CELL_STAGE_1D["fp32_mixed"], arrays * (8 + 4))


def test_constants_3d():
    import af_inputs as ai
    import bench
    import oracle
    assert np.isclose(bench.BYTES_PER_CELL_STAGE_3D, round((2 + 3 + 3) / 3 * 8 * 8, 2), atol=0.01)
    spec = ai.pme_3d(24)
    st = [a.numpy() for a in ai.initial_state(spec, sub=2, order=3)]
    fc = oracle.flop_count(spec, st, 0.3 * oracle.dt_cfl(spec, st[0]))
    per_cell = (fc["add"] + fc["mul"] + fc["div"] + fc["exp"]) / spec.cells
    assert abs(per_cell - bench.FLOPS_PER_CELL_STAGE_3D) < 0.01
