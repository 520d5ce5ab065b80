"""Batched persistent execution (uneven instances, one launch per RK stage, graph
replay, autotuned tile shape) against single-mesh contexts and the oracle."""
import numpy as np
import pytest

import af_inputs as ai
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2510_11527_gb300 import build
    build.build()


def _structs(specs, prec, rk):
    from paper_2510_11527_gb300 import capi
    grids, fl, df, bd = [], [], [], []
    for s in specs:
        grids.append(capi.af_grid(2, s.nx, s.ny, s.x0, s.x1, s.y0, s.y1))
        f = capi.af_flux()
        f.kind = capi.FLUX[s.flux[0]]
        for k, v in enumerate(s.flux[1]):
            f.p[k] = v
        d = capi.af_diff()
        d.kind = capi.DIFF[s.diff[0]]
        for k, v in enumerate(s.diff[1]):
            d.p[k] = v
        fl.append(f)
        df.append(d)
        bd.append(capi.af_bounds_t(s.umin, s.umax, 0))
    opts = capi.af_opts(capi.PREC[prec], rk, 0.0, 0.0, 1, 0, 1.0)
    return grids, fl, df, bd, opts


def _instances(count=7, seed=3, nmax=130):
    return ai.batch_instances(count=count, seed=seed, nmin=20, nmax=nmax)


@pytest.mark.parametrize("prec", ["fp64", "fp32_mixed"])
@pytest.mark.parametrize("tile", [(32, 8), (64, 4), (16, 16)])
@pytest.mark.parametrize("rk", [3, 54])
def test_batch_bitwise_equals_single_mesh(prec, tile, rk):
    from paper_2510_11527_gb300 import Solver, capi
    inst = _instances()
    specs = [s for s, _ in inst]
    states = [[a.numpy() for a in ai.batch_state(s, m)] for s, m in inst]
    b = capi.af_batch_create(*_structs(specs, prec, rk))
    try:
        capi.af_batch_set_tile(b, *tile)
        for i, (s, st) in enumerate(zip(specs, states)):
            capi.af_batch_set_state(b, i, s.cells, *st)
        capi.af_batch_step(b, 3)
        capi.af_batch_sync(b)
        for i, (s, st) in enumerate(zip(specs, states)):
            got = capi.af_batch_get_state(b, i, s.cells)
            with Solver(s, precision=prec, rk=rk) as one:
                one.set_state(st)
                for _ in range(3):
                    one.step(0.0)
                want = one.get_state()
                tb, ts = capi.af_batch_time(b, i), one.time()
            scale = max(abs(s.umin), abs(s.umax))
            if rk == 3 and prec == "fp64":
                assert tb == ts
                for x, y in zip(got, want):
                    assert np.array_equal(x.reshape(y.shape), y)
            elif prec == "fp32_mixed":
                # the single-mesh FP32-mixed stage is the column-marching kernel, the
                # batch runs the tile kernel: the same arithmetic in another order,
                # agreement within the FP32 stencils' rounding
                assert tb == pytest.approx(ts, rel=2e-6)
                for x, y in zip(got, want):
                    assert np.max(np.abs(x.reshape(y.shape) - y)) <= 2e-6 * scale
            else:
                # separate compilations of the same tile code may contract a few
                # multiply-adds differently: agreement to a few ulp of the arithmetic
                tol = 2e-15 if prec == "fp64" else 2e-6
                assert tb == pytest.approx(ts, rel=tol)
                for x, y in zip(got, want):
                    assert np.max(np.abs(x.reshape(y.shape) - y)) <= tol * scale
            lo, hi = capi.af_batch_bounds(b, i)
            assert lo >= s.umin and hi <= s.umax
        assert capi.af_batch_stats(b)["errors"] == 0
    finally:
        capi.af_batch_destroy(b)


def test_batch_matches_oracle_fp64():
    from paper_2510_11527_gb300 import capi
    inst = _instances(count=4, seed=9, nmax=60)
    specs = [s for s, _ in inst]
    states = [[a.numpy() for a in ai.batch_state(s, m)] for s, m in inst]
    b = capi.af_batch_create(*_structs(specs, "fp64", 3))
    try:
        for i, (s, st) in enumerate(zip(specs, states)):
            capi.af_batch_set_state(b, i, s.cells, *st)
        capi.af_batch_step(b, 2)
        for i, (s, st) in enumerate(zip(specs, states)):
            ref = [a.copy() for a in st]
            for _ in range(2):
                ref, _ = oracle.step(s, 3, ref, oracle.dt_cfl(s, ref[0]))
            got = capi.af_batch_get_state(b, i, s.cells)
            err = max(np.max(np.abs(g.reshape(r.shape) - r)) for g, r in zip(got, ref))
            assert err <= 1e-12 * max(abs(s.umin), abs(s.umax))
            m0 = oracle.mass(s, st[0])
            assert abs(capi.af_batch_mass(b, i) - m0) <= 1e-14 * max(1.0, abs(m0))
    finally:
        capi.af_batch_destroy(b)


def test_autotune_restores_state_and_picks_a_built_shape():
    from paper_2510_11527_gb300 import capi
    inst = _instances(count=6, seed=5, nmax=200)
    specs = [s for s, _ in inst]
    states = [[a.numpy() for a in ai.batch_state(s, m)] for s, m in inst]
    outs = []
    for tune in (False, True):
        b = capi.af_batch_create(*_structs(specs, "fp32_mixed", 3))
        try:
            for i, (s, st) in enumerate(zip(specs, states)):
                capi.af_batch_set_state(b, i, s.cells, *st)
            if tune:
                shape = capi.af_batch_autotune(b)
                assert shape in [(32, 8), (64, 4), (16, 16)]
                assert capi.af_batch_info(b)["tile"] == shape
                assert capi.af_batch_time(b, 0) == 0.0
            capi.af_batch_step(b, 2)
            outs.append([capi.af_batch_get_state(b, i, s.cells) for i, s in enumerate(specs)])
        finally:
            capi.af_batch_destroy(b)
    # the tile shapes are separate compilations of the same FP32 tile code, which may
    # contract a few multiply-adds differently: agreement to the FP32 stencils' rounding
    for a, c in zip(outs[0], outs[1]):
        for x, y in zip(a, c):
            assert np.max(np.abs(x - y)) <= 2e-6


def test_batch_rejects_mixed_flux_kinds_and_blend():
    from paper_2510_11527_gb300 import capi
    s1 = ai.config2(16)
    s2 = ai.Spec(dim=2, nx=16, ny=16, flux=("linear", (1.0, 1.0)), diff=("const", (0.01,)), umin=-1, umax=1)
    with pytest.raises(capi.AfError) as ei:
        capi.af_batch_create(*_structs([s1, s2], "fp64", 3))
    assert ei.value.status == capi.AF_E_ARG
    # the external indicator comes from an attached network: none attached, no step
    g, f, d, b, o = _structs([s1], "fp64", 3)
    o.blend = 2
    bt = capi.af_batch_create(g, f, d, b, o)
    try:
        for call in (lambda: capi.af_batch_step(bt, 1), lambda: capi.af_batch_autotune(bt)):
            with pytest.raises(capi.AfError) as ei:
                call()
            assert ei.value.status == capi.AF_E_STATE
    finally:
        capi.af_batch_destroy(bt)
    # a network needs a batch created for it
    o.blend = 1
    bt = capi.af_batch_create(g, f, d, b, o)
    net = capi.af_mlp_create()
    try:
        with pytest.raises(capi.AfError) as ei:
            capi.af_batch_set_mlp(bt, net)
        assert ei.value.status == capi.AF_E_STATE
    finally:
        capi.af_batch_destroy(bt)
        capi.af_mlp_destroy(net)


@pytest.mark.parametrize("prec", ["fp64", "fp32_mixed"])
def test_batch_plain_blend_matches_single_mesh_and_oracle(prec):
    """The smoothness-indicator blend (Section 5.1.3) in the batch path: instances of
    uneven size with gamma = 1 agree with single-mesh contexts (FP64 within 1e-12; FP32-mixed
    bit for bit: the batch runs the single mesh's column-marching blend) and, in FP64, with
    the oracle."""
    from paper_2510_11527_gb300 import Solver, capi
    inst = _instances(count=5, seed=11, nmax=90)
    specs = []
    for s, _ in inst:
        s.blend = "plain"
        specs.append(s)
    states = [[a.numpy() for a in ai.batch_state(s, m)] for s, (_, m) in zip(specs, inst)]
    g, f, d, bd, o = _structs(specs, prec, 3)
    o.blend = 1
    b = capi.af_batch_create(g, f, d, bd, o)
    try:
        for i, (s, st) in enumerate(zip(specs, states)):
            capi.af_batch_set_state(b, i, s.cells, *st)
        capi.af_batch_step(b, 2)
        capi.af_batch_sync(b)
        assert capi.af_batch_stats(b)["errors"] == 0
        for i, (s, st) in enumerate(zip(specs, states)):
            got = capi.af_batch_get_state(b, i, s.cells)
            with Solver(s, precision=prec, rk=3) as one:
                one.set_state(st)
                for _ in range(2):
                    one.step(0.0)
                want = one.get_state()
            tol = 1e-12 if prec == "fp64" else 0.0   # FP32-mixed: the single mesh's column-marching arithmetic
            for x, y in zip(got, want):
                assert np.max(np.abs(x.reshape(y.shape) - y)) <= tol
            if prec == "fp64":
                ref = [a.copy() for a in st]
                for _ in range(2):
                    ref, _ = oracle.step(s, 3, ref, oracle.dt_cfl(s, ref[0]))
                assert max(np.max(np.abs(x.reshape(r.shape) - r)) for x, r in zip(got, ref)) <= 1e-12
    finally:
        capi.af_batch_destroy(b)


@pytest.mark.parametrize("prec", ["fp64", "fp32_mixed"])
def test_batch_learned_blend_matches_single_mesh(prec):
    """The learned indicator in the batch path: one launch per stage forms s for every
    instance (uneven sizes, ragged 32 x 8 tiles) with the network, then the blended
    stage reads it. Each instance agrees with a single-mesh context running the same
    network (FP64 within 1e-12, FP32-mixed bit for bit), the indicator is
    the network's (the result differs from the plain blend's), and detaching the
    network stops the batch."""
    from paper_2510_11527_gb300 import Solver, capi
    inst = _instances(count=5, seed=17, nmax=90)
    specs = [s for s, _ in inst]
    states = [[a.numpy() for a in ai.batch_state(s, m)] for s, m in inst]
    net = capi.af_mlp_create()
    capi.af_mlp_set_params(net, ai.mlp_init_params(6))
    finals = {}
    try:
        for mode in (2, 1):
            g, f, d, bd, o = _structs(specs, prec, 3)
            o.blend = mode
            b = capi.af_batch_create(g, f, d, bd, o)
            try:
                if mode == 2:
                    capi.af_batch_set_mlp(b, net)
                for i, (s, st) in enumerate(zip(specs, states)):
                    capi.af_batch_set_state(b, i, s.cells, *st)
                capi.af_batch_step(b, 2)
                capi.af_batch_sync(b)
                assert capi.af_batch_stats(b)["errors"] == 0
                finals[mode] = [capi.af_batch_get_state(b, i, s.cells) for i, s in enumerate(specs)]
                if mode == 2:
                    capi.af_batch_set_mlp(b, None)
                    with pytest.raises(capi.AfError) as ei:
                        capi.af_batch_step(b, 1)
                    assert ei.value.status == capi.AF_E_STATE
            finally:
                capi.af_batch_destroy(b)
        tol = 1e-12 if prec == "fp64" else 0.0   # FP32-mixed: the single mesh's column-marching arithmetic
        moved = 0.0
        for i, (s, st) in enumerate(zip(specs, states)):
            s.blend = "external"
            with Solver(s, precision=prec, rk=3) as one:
                capi.af_set_mlp(one.ctx, net)
                one.set_state(st)
                for _ in range(2):
                    one.step(0.0)
                want = one.get_state()
            for x, y in zip(finals[2][i], want):
                assert np.max(np.abs(x.reshape(y.shape) - y)) <= tol
            moved = max(moved, float(np.max(np.abs(finals[2][i][0] - finals[1][i][0]))))
        assert moved > 1e-10
    finally:
        capi.af_mlp_destroy(net)


def test_batch_cfl_interior_extrema_bl():
    """Per-instance device dt of Buckley-Leverett instances on 0/1 patterns, where the
    wave speed of every face comes from an interior extremum of f_l', equals the
    oracle's CFL step."""
    from paper_2510_11527_gb300 import capi
    specs, states = [], []
    for k, (nx, ny) in enumerate([(40, 24), (33, 17)]):
        s = ai.Spec(dim=2, nx=nx, ny=ny, x0=0.0, x1=1.3, y0=0.0, y1=0.9, flux=("bl", (5.0,)),
                    diff=("cubic", (0.0, 0.02, -0.04 / 3)), umin=0.0, umax=1.0)
        j, i = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
        ub = ((i + j) % 2 if k == 0 else i % 2).astype(np.float64)
        specs.append(s)
        states.append([ub, np.zeros_like(ub), np.zeros_like(ub), np.zeros_like(ub)])
    b = capi.af_batch_create(*_structs(specs, "fp64", 3))
    try:
        for i, (s, st) in enumerate(zip(specs, states)):
            capi.af_batch_set_state(b, i, s.cells, *st)
        capi.af_batch_step(b, 1)
        capi.af_batch_sync(b)
        for i, (s, st) in enumerate(zip(specs, states)):
            assert capi.af_batch_time(b, i) == pytest.approx(oracle.dt_cfl(s, st[0]), rel=1e-14)
    finally:
        capi.af_batch_destroy(b)


@pytest.mark.parametrize("prec", ["fp64", "fp32_mixed"])
def test_batch_tiny_and_ragged_meshes_equal_single_mesh(prec):
    """Meshes smaller than the halo (1x1, 3x2), ragged tile edges (5x7, 33x9) and a
    non-square mesh in one batch, with and without a diffusion term: SSP-RK3 steps agree
    with single-mesh contexts, bit for bit in FP64 (the periodic wrap takes its modulo
    path for the smallest ones)."""
    from paper_2510_11527_gb300 import Solver, capi
    sizes = [(1, 1), (3, 2), (5, 7), (33, 9), (40, 17)]
    specs, states = [], []
    for k, (nx, ny) in enumerate(sizes):
        # every other instance without a diffusion term (face limiter factor 4, not 12)
        s = ai.Spec(dim=2, nx=nx, ny=ny, x0=0.0, x1=0.1 * nx, y0=0.0, y1=0.1 * ny, flux=("burgers", (0.5,)),
                    diff=("pwl", (0.03, 0.25, 0.03, 0.75)) if k % 2 == 0 else ("none", ()), umin=0.0, umax=1.0)
        specs.append(s)
        states.append([a.numpy() for a in ai.random_state_2d(s, seed=40 + k)])
    b = capi.af_batch_create(*_structs(specs, prec, 3))
    try:
        for i, (s, st) in enumerate(zip(specs, states)):
            capi.af_batch_set_state(b, i, s.cells, *st)
        capi.af_batch_step(b, 2)
        capi.af_batch_sync(b)
        for i, (s, st) in enumerate(zip(specs, states)):
            got = capi.af_batch_get_state(b, i, s.cells)
            with Solver(s, precision=prec, rk=3) as one:
                one.set_state(st)
                for _ in range(2):
                    one.step(0.0)
                want = one.get_state()
                if prec == "fp64":
                    assert capi.af_batch_time(b, i) == one.time()
                else:
                    assert capi.af_batch_time(b, i) == pytest.approx(one.time(), rel=2e-6)
            for x, y in zip(got, want):
                if prec == "fp64":
                    assert np.array_equal(x.reshape(y.shape), y)
                else:   # column-marching single-mesh kernel vs the batch's tile kernel
                    assert np.max(np.abs(x.reshape(y.shape) - y)) <= 2e-6 * max(abs(s.umin), abs(s.umax))
        assert capi.af_batch_stats(b)["errors"] == 0
    finally:
        capi.af_batch_destroy(b)
