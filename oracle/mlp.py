"""FP64 reference of the learned smoothness indicator (test infrastructure only).

The indicator network stands in for the smoothness indicator s of the blend in
Section 5.1.3 (applied direction by direction in 2D, Section 5.2): it maps a
normalised 21-value patch of cell averages and point values around a cell to s >= 0,
which then replaces s in theta^{c,s} = exp(-gamma s_face) and theta^{d,s} = exp(-gamma s).
The limiter and the projection still follow, so bounds and conservation do not depend
on the network.

Patch of cell (i, j): 13 cell averages ub(i+a, j+b) for (a, b) in PATCH_UB, then the 8
point values of the cell's closure V(i-1,j-1), V(i,j-1), V(i-1,j), V(i,j), X(i-1,j),
X(i,j), Y(i,j-1), Y(i,j). Features: (v_k - ub(i,j)) / (max_k |v_k| + 1e-13).

Label (training target): the plain indicator of Section 5.1.3, max(s_1, s_2) with
s_l = (s~_{l,-1} + 4 s~_l + s~_{l,+1}) / 6 and s~ = |u_- - 2u + u_+| / (|u_-| + 2|u| +
|u_+| + 1e-13) along direction l.

Network 21 -> 32 -> 32 -> 1: h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2),
s = softplus(w3 . h2 + b3). With quantize=True the two tensor-core layers see bf16
inputs and bf16 weights (round to nearest even), as on the GPU; sums are exact here
(FP64). Gradients pass straight through the rounding.
"""
import numpy as np

PATCH_UB = [(-1, -1), (0, -1), (1, -1), (-1, 0), (0, 0), (1, 0), (-1, 1), (0, 1), (1, 1),
            (-2, 0), (2, 0), (0, -2), (0, 2)]
NIN, NH = 21, 32
PARAM_SHAPES = [("W1", (NH, NIN)), ("b1", (NH,)), ("W2", (NH, NH)), ("b2", (NH,)), ("w3", (NH,)), ("b3", (1,))]
NPARAM = sum(int(np.prod(s)) for _, s in PARAM_SHAPES)


def unpack(flat):
    out, k = {}, 0
    for name, shape in PARAM_SHAPES:
        n = int(np.prod(shape))
        out[name] = np.asarray(flat[k:k + n], dtype=np.float64).reshape(shape)
        k += n
    return out


def pack(p):
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel() for name, _ in PARAM_SHAPES])


def bf16(x):
    """Round to bfloat16 (round to nearest even) through float32, as the GPU does."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _sh(a, di, dj):
    """a shifted so that result[j, i] = a[j + dj, i + di] (periodic)."""
    return np.roll(np.roll(a, -dj, axis=0), -di, axis=1)


def features(ub, V, X, Y):
    """(ny*nx, 21) normalised patches, row-major cells."""
    vals = [_sh(ub, a, b) for a, b in PATCH_UB]
    vals += [_sh(V, -1, -1), _sh(V, 0, -1), _sh(V, -1, 0), V, _sh(X, -1, 0), X, _sh(Y, 0, -1), Y]
    P = np.stack([np.asarray(v, dtype=np.float64) for v in vals], axis=-1)
    scale = np.max(np.abs(P), axis=-1, keepdims=True) + 1e-13
    return ((P - np.asarray(ub, dtype=np.float64)[..., None]) / scale).reshape(-1, NIN)


def plain_label(ub):
    """max(s_1, s_2) of the plain smoothness indicator, per cell (row-major)."""
    u = np.asarray(ub, dtype=np.float64)

    def st(um, uc, up):
        return np.abs(um - 2 * uc + up) / (np.abs(um) + 2 * np.abs(uc) + np.abs(up) + 1e-13)

    s1t = st(_sh(u, -1, 0), u, _sh(u, 1, 0))
    s2t = st(_sh(u, 0, -1), u, _sh(u, 0, 1))
    s1 = (_sh(s1t, -1, 0) + 4 * s1t + _sh(s1t, 1, 0)) / 6
    s2 = (_sh(s2t, 0, -1) + 4 * s2t + _sh(s2t, 0, 1)) / 6
    return np.maximum(s1, s2).ravel()


def softplus(z):
    return np.where(z > 20, z, np.log1p(np.exp(np.minimum(z, 20))))


def forward(p, x, quantize=True):
    q = bf16 if quantize else (lambda a: np.asarray(a, dtype=np.float64))
    xq = q(x)
    z1 = xq @ q(p["W1"]).T + p["b1"]
    h1 = np.maximum(z1, 0.0)
    h1q = q(h1)
    z2 = h1q @ q(p["W2"]).T + p["b2"]
    h2 = np.maximum(z2, 0.0)
    z3 = h2 @ p["w3"] + p["b3"][0]
    return softplus(z3), dict(xq=xq, z1=z1, h1q=h1q, z2=z2, h2=h2, z3=z3)


def loss_and_grad(p, x, y, quantize=True):
    """Mean squared error and its gradient w.r.t. the (unrounded) parameters."""
    out, c = forward(p, x, quantize)
    q = bf16 if quantize else (lambda a: np.asarray(a, dtype=np.float64))
    B = x.shape[0]
    r = out - y
    loss = np.mean(r * r)
    dz3 = (2.0 / B) * r / (1.0 + np.exp(-c["z3"]))           # softplus' = sigmoid
    g = {"w3": c["h2"].T @ dz3, "b3": np.array([dz3.sum()])}
    dz2 = np.outer(dz3, p["w3"]) * (c["z2"] > 0)
    g["W2"] = dz2.T @ c["h1q"]
    g["b2"] = dz2.sum(axis=0)
    dz1 = (dz2 @ q(p["W2"])) * (c["z1"] > 0)
    g["W1"] = dz1.T @ c["xq"]
    g["b1"] = dz1.sum(axis=0)
    return loss, g


def adam(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step on flat arrays (returns new p, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def init_params(seed):
    rng = np.random.default_rng(seed)
    return {"W1": rng.normal(0, np.sqrt(2.0 / NIN), (NH, NIN)), "b1": np.zeros(NH),
            "W2": rng.normal(0, np.sqrt(2.0 / NH), (NH, NH)), "b2": np.zeros(NH),
            "w3": rng.normal(0, np.sqrt(1.0 / NH), NH), "b3": np.array([-2.0])}
