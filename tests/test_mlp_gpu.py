"""Learned smoothness indicator on the GPU against the FP64 reference (oracle/mlp.py):
features and labels, tensor-core inference, the fused indicator, gradients, one Adam
step; then training on method-labelled data and what the trained network gains over
the method without a blend."""
import math

import numpy as np
import pytest
import torch

import af_inputs as ai
import oracle
from oracle import mlp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2510_11527_gb300 import build
    build.build()


def _ctx_with_state(spec, state, prec="fp64"):
    from paper_2510_11527_gb300 import Solver
    s = Solver(spec, precision=prec)
    s.set_state(state)
    return s


def _net(seed=4):
    from paper_2510_11527_gb300 import capi
    net = capi.af_mlp_create()
    p = ai.mlp_init_params(seed)
    capi.af_mlp_set_params(net, p)
    return net, p


def test_features_and_labels_match_reference():
    from paper_2510_11527_gb300 import capi
    spec = ai.Spec(dim=2, nx=40, ny=30, flux=("burgers", (0.5,)), diff=("pwl", (0.0, 0.0, 0.1, 0.5)),
                   umin=-1.0, umax=1.0, blend="external")
    st = [a.numpy() for a in ai.random_state_2d(spec, seed=3, lo=-1, hi=1)]
    with _ctx_with_state(spec, st) as s:
        feat = torch.empty((spec.cells, 21), dtype=torch.float32, device="cuda")
        lab = torch.empty(spec.cells, dtype=torch.float32, device="cuda")
        capi.af_mlp_features(s.ctx, feat.data_ptr(), lab.data_ptr())
        torch.cuda.synchronize()
    ref_f = mlp.features(*st)
    ref_l = mlp.plain_label(st[0])
    assert np.max(np.abs(feat.cpu().numpy() - ref_f)) <= 1e-6
    np.testing.assert_allclose(lab.cpu().numpy(), ref_l, rtol=1e-6, atol=1e-7)


def _ref_forward(p, x32):
    return mlp.forward(mlp.unpack(p.astype(np.float64)), x32.astype(np.float64), quantize=True)[0]


# one FP32 ulp at 1: a full ulp per operation, since the order and rounding of the tensor
# cores' FP32 accumulation are not specified
_U = 2.0 ** -23


def _tc_bound(p, x, eps_x=0.0):
    """Per-row bound on |GPU - reference| of the network output, from the arithmetic.

    The reference sums exactly; the GPU rounds the same bf16 inputs and weights, adds
    bf16 x bf16 products (exact in FP32) in FP32, rounds h1 to bf16 and evaluates the
    output layer and softplus in FP32. With x off by at most eps_x (features formed on
    the GPU), the GPU's bf16 input lies between bf16(x - eps_x) and bf16(x + eps_x).
    Layer 1's pre-activation is then within e1 = |W1q| dx + (n+2) u (|W1q| |xq| + |b1|)
    of the reference's, so both roundings of relu(z1) to bf16 lie between
    bf16(relu(z1 -+ e1)): a rounding that can flip contributes its full bf16 step. The
    same accumulation bound follows through layer 2 (relu is 1-Lipschitz), the output
    layer and softplus (1-Lipschitz; a few FP32 ulps of its value)."""
    P = mlp.unpack(p.astype(np.float64))
    W1q, W2q = mlp.bf16(P["W1"]), mlp.bf16(P["W2"])
    b1, b2, w3, b3 = P["b1"], P["b2"], P["w3"], float(P["b3"][0])
    x = x.astype(np.float64)
    xq = mlp.bf16(x)
    dx = (mlp.bf16(x + eps_x) - mlp.bf16(x - eps_x)) if eps_x > 0 else np.zeros_like(x)
    A1, A2 = np.abs(W1q), np.abs(W2q)
    z1 = xq @ W1q.T + b1
    e1 = dx @ A1.T + (mlp.NIN + 2) * _U * ((np.abs(xq) + dx) @ A1.T + np.abs(b1))
    h_lo, h_hi = mlp.bf16(np.maximum(z1 - e1, 0.0)), mlp.bf16(np.maximum(z1 + e1, 0.0))
    z2 = mlp.bf16(np.maximum(z1, 0.0)) @ W2q.T + b2
    e2 = (h_hi - h_lo) @ A2.T + (mlp.NH + 2) * _U * (h_hi @ A2.T + np.abs(b2))
    e3 = e2 @ np.abs(w3) + (mlp.NH + 4) * _U * ((np.maximum(z2, 0.0) + e2) @ np.abs(w3) + abs(b3))
    out = mlp.forward(P, x, quantize=True)[0]
    return e3 + 8 * _U * np.abs(out) + 1e-8


def test_tensor_core_inference_matches_reference():
    from paper_2510_11527_gb300 import capi
    rng = np.random.default_rng(0)
    net, p = _net()
    try:
        x = rng.normal(0, 0.6, (5000, 21)).astype(np.float32)
        xd = torch.from_numpy(x).cuda()
        out = torch.empty(5000, dtype=torch.float32, device="cuda")
        capi.af_mlp_infer(net, xd.data_ptr(), 5000, out.data_ptr())
        got = out.cpu().numpy()
        want = _ref_forward(p, x)
        err = np.abs(got - want)
        # FP32 accumulation on the tensor cores vs exact sums; a bf16 rounding of a
        # hidden activation can flip when its FP32 sum lands near a rounding boundary:
        # every row within the bound its arithmetic allows
        bound = _tc_bound(p, x)
        assert np.quantile(err, 0.999) <= 1e-4 * (1 + np.abs(want)).max()
        assert np.all(err <= bound), float(np.max(err / bound))
        assert np.median(bound) <= 1e-3
    finally:
        capi.af_mlp_destroy(net)


def test_fused_indicator_matches_reference():
    from paper_2510_11527_gb300 import capi
    spec = ai.Spec(dim=2, nx=70, ny=45, flux=("bl", (5.0,)), diff=("cubic", (0.0, 0.02, -0.04 / 3)),
                   umin=0.0, umax=1.0, blend="external")
    st = [a.numpy() for a in ai.random_piecewise(spec, seed=11)]
    net, p = _net(7)
    try:
        for prec in ("fp64", "fp32_mixed"):
            with _ctx_with_state(spec, st, prec) as s:
                sd = torch.empty(spec.cells, dtype=torch.float64, device="cuda")
                capi.af_mlp_indicator(net, s.ctx, sd.data_ptr())
                got = sd.cpu().numpy()
            x32 = mlp.features(*st).astype(np.float32)
            want = _ref_forward(p, x32)
            err = np.abs(got - want)
            # the GPU's features are within 1e-6 of the reference's (FP32 arithmetic on
            # values of magnitude <= 2); 2e-6 leaves room for the FP32-mixed state
            bound = _tc_bound(p, x32, eps_x=2e-6)
            assert np.quantile(err, 0.999) <= 1e-4 * (1 + np.abs(want)).max()
            assert np.all(err <= bound), float(np.max(err / bound))
    finally:
        capi.af_mlp_destroy(net)


def test_gradient_and_adam_step_match_reference():
    from paper_2510_11527_gb300 import capi
    rng = np.random.default_rng(5)
    n = 3000
    x = rng.normal(0, 0.6, (n, 21)).astype(np.float32)
    y = rng.uniform(0, 1, n).astype(np.float32)
    net, p = _net(9)
    try:
        xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
        g, loss = capi.af_mlp_grad(net, xd.data_ptr(), yd.data_ptr(), n)
        P = mlp.unpack(p.astype(np.float64))
        lref, gref = mlp.loss_and_grad(P, x.astype(np.float64), y.astype(np.float64), quantize=True)
        gref = mlp.pack(gref)
        assert loss == pytest.approx(lref, rel=1e-4)
        assert np.max(np.abs(g - gref)) <= 1e-4 * np.max(np.abs(gref))
        # one Adam step on the same rows in order
        lr = 1e-3
        capi.af_mlp_train(net, xd.data_ptr(), yd.data_ptr(), n, n, 1, lr, 0)
        p1 = capi.af_mlp_get_params(net)
        pref, _, _ = mlp.adam(p.astype(np.float64), gref, np.zeros_like(gref), np.zeros_like(gref), 1, lr)
        # the first Adam step moves each parameter by ~lr sign(g): compare where |g| is
        # not tiny (the sign of a ~0 gradient is rounding noise)
        big = np.abs(gref) > 1e-3 * np.max(np.abs(gref))
        np.testing.assert_allclose(p1[big], pref[big], rtol=0, atol=1e-6)
    finally:
        capi.af_mlp_destroy(net)


def _training_data(count=8, n=128, steps=4):
    """Method-labelled patches: random piecewise-constant fields advanced a few steps by
    the plain method (Buckley-Leverett, FP32-mixed, plain blend)."""
    from paper_2510_11527_gb300 import Solver, capi
    feats, labels = [], []
    for k in range(count):
        spec = ai.config5(n)
        spec.blend = "plain"
        st = [a.numpy() for a in ai.random_piecewise(spec, seed=100 + k)]
        with Solver(spec, precision="fp32_mixed") as s:
            s.set_state(st)
            for _ in range(steps):
                s.step(0.0)
            spec_e = ai.config5(n)
            spec_e.blend = "external"
            f = torch.empty((spec.cells, 21), dtype=torch.float32, device="cuda")
            l = torch.empty(spec.cells, dtype=torch.float32, device="cuda")
            capi.af_mlp_features(s.ctx, f.data_ptr(), l.data_ptr())
        feats.append(f)
        labels.append(l)
    return torch.cat(feats), torch.cat(labels)


@pytest.fixture(scope="module")
def trained():
    from paper_2510_11527_gb300 import capi
    X, Y = _training_data()
    net, _ = _net(1)
    l0 = capi.af_mlp_train(net, X.data_ptr(), Y.data_ptr(), X.shape[0], 4096, 1, 1e-3, 7)
    l1 = capi.af_mlp_train(net, X.data_ptr(), Y.data_ptr(), X.shape[0], 4096, 1500, 3e-3, 8)
    yield net, l0, l1, (X, Y)
    capi.af_mlp_destroy(net)


def test_training_reduces_loss(trained):
    net, l0, l1, _ = trained
    assert l1 < 0.2 * l0


def _tv(a):
    return float(np.sum(np.abs(np.diff(a, axis=0))) + np.sum(np.abs(np.diff(a, axis=1))))


def test_learned_blend_gain_over_no_blend(trained):
    """Buckley-Leverett disc (the paper's Example 6.7 setting, periodic), 128^2, FP32-mixed.
    The plain smoothness indicator is the reference: the learned blend must move the
    solution toward the plain-blend solution and reduce the oscillation (total variation
    growth) of the method without a blend; bounds and conservation hold in every case."""
    from paper_2510_11527_gb300 import Solver, capi
    net = trained[0]
    res = {}
    for mode in ("off", "plain", "learned"):
        spec = ai.config5(128)
        spec.blend = "external" if mode == "learned" else mode
        st = [a.numpy() for a in ai.initial_state(spec)]
        with Solver(spec, precision="fp32_mixed") as s:
            if mode == "learned":
                capi.af_set_mlp(s.ctx, net)
            s.set_state(st)
            m0 = s.mass()
            for _ in range(60):
                s.step(0.0)
            out = s.get_state()
            lo, hi = s.bounds()
            stats = s.stats()
            assert lo >= 0.0 and hi <= 1.0 and stats["errors"] == 0
            assert abs(s.mass() - m0) <= 1e-12 + stats["mass_adjust"]
        res[mode] = out[0]
    d_off = np.mean(np.abs(res["off"] - res["plain"]))
    d_learn = np.mean(np.abs(res["learned"] - res["plain"]))
    assert d_learn < 0.5 * d_off
    assert _tv(res["learned"]) < _tv(res["off"])
