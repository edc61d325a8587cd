"""Oracle of the learned smoothing proposal: features, MLP, loss, gradients, AdamW.

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers; the library never imports
this module and this module never imports the library.

The learned proposal predicts, from a point's stencil and constraint box, where
the plain smoother (Eq. 1, Sec. 2.2) puts the point after the full iteration
count; a few plain correction sweeps and the box clamp follow.  The model is a
multilayer perceptron 32 -> 64 -> 64 -> 3 with ReLU, BF16 weights and
activations, FP32 accumulation and biases, trained by AdamW on the mean squared
error of the offset.  This module writes each step out plainly in FP64 with
numpy; where the kernels round to BF16 it rounds too (round to nearest, ties to
even) so that both sides take the same decisions.

Features of point i (32 slots; every value is exact in BF16):
    0-2    s_i = sum of the unit steps u_f over the faces f of i's stencil
    3      n_i = number of stencil neighbours
    4-9    p_f = 1 if face f (-x, +x, -y, +y, -z, +z) has a neighbour, else 0
    10-27  s_j of the neighbour j across face f (slots 10 + 3f .. 12 + 3f), 0 if none
    28     h = half the constraint distance (box half-width, voxel units), rounded to BF16
    29-31  0
Parameters (flat, in this order): W1 [64][32], b1 [64], W2 [64][64], b2 [64],
W3 [3][64], b3 [3] -- 6467 values; the weights act as y = W x + b.
"""
from __future__ import annotations

import numpy as np

N_IN, N_HID, N_OUT, N_FEAT = 32, 64, 3, 32
SIZES = (("W1", (N_HID, N_IN)), ("b1", (N_HID,)), ("W2", (N_HID, N_HID)), ("b2", (N_HID,)),
         ("W3", (N_OUT, N_HID)), ("b3", (N_OUT,)))
N_PARAMS = sum(int(np.prod(s)) for _, s in SIZES)
WEIGHTS = ("W1", "W2", "W3")

# unit step towards the neighbour across face f, faces in stencil order
UNIT = np.array([[-1, 0, 0], [1, 0, 0], [0, -1, 0], [0, 1, 0], [0, 0, -1], [0, 0, 1]], dtype=np.float64)


def bf16(x):
    """Round to the nearest BF16 value (8 significant bits, FP32's exponent range), ties to even."""
    x = np.asarray(x, dtype=np.float64)
    _, e = np.frexp(x)                               # x = m * 2^e, 0.5 <= |m| < 1
    q = np.ldexp(1.0, np.maximum(e, -125) - 8)       # spacing of BF16 values near x (subnormals below 2^-126)
    return np.rint(x / q) * q


def unpack(params):
    """Flat parameter vector -> dict of FP64 arrays."""
    p = np.asarray(params, dtype=np.float64)
    if p.size != N_PARAMS:
        raise ValueError(f"expected {N_PARAMS} parameters")
    out, at = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = p[at:at + n].reshape(shape)
        at += n
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in SIZES])


def init_params(seed):
    """He-uniform weights (bound sqrt(6 / fan_in)), zero biases, rounded to FP32; numpy's PCG64 stream."""
    rng = np.random.default_rng(seed)
    d = {}
    for name, shape in SIZES:
        if name in WEIGHTS:
            bound = np.sqrt(6.0 / shape[1])
            d[name] = rng.uniform(-bound, bound, size=shape)
        else:
            d[name] = np.zeros(shape)
    return pack(d).astype(np.float32)


def features(stencil_offsets, stencil_ids, face_masks, constraint_distance):
    """(n, 32) features of every point of a mesh from its stencil (face order -x, +x, -y, +y, -z, +z)."""
    so = np.asarray(stencil_offsets, dtype=np.int64)
    ids = np.asarray(stencil_ids, dtype=np.int64)
    fm = np.asarray(face_masks, dtype=np.int64)
    n = fm.size
    p = ((fm[:, None] >> np.arange(6)[None, :]) & 1).astype(np.float64)   # (n, 6)
    s = p @ UNIT                                                           # (n, 3)
    x = np.zeros((n, N_FEAT))
    x[:, 0:3] = s
    x[:, 3] = p.sum(axis=1)
    x[:, 4:10] = p
    for i in range(n):
        k = so[i]
        for f in range(6):
            if p[i, f]:
                j = ids[k]
                k += 1
                x[i, 10 + 3 * f:13 + 3 * f] = s[j]
    x[:, 28] = bf16(0.5 * float(np.float32(constraint_distance)))
    return x


def forward(params, X, exact=False):
    """y = W3 r(W2 r(W1 x + b1) + b2) + b3, r = ReLU, for the rows of X.

    Unless `exact`, the weights and the hidden activations are rounded to BF16 as
    the kernels hold them.  Returns (y, cache)."""
    P = unpack(params)
    rnd = (lambda v: v) if exact else bf16
    W1, W2, W3 = rnd(P["W1"]), rnd(P["W2"]), rnd(P["W3"])
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ W1.T + P["b1"]
    h1 = rnd(np.maximum(z1, 0.0))
    z2 = h1 @ W2.T + P["b2"]
    h2 = rnd(np.maximum(z2, 0.0))
    y = h2 @ W3.T + P["b3"]
    return y, {"X": X, "h1": h1, "h2": h2, "W1": W1, "W2": W2, "W3": W3}


def loss_and_grad(params, X, T, exact=False):
    """Mean squared error over the N x 3 outputs and its gradient w.r.t. the flat parameters.

    The gradient flows through the BF16 weights onto the master values unchanged;
    unless `exact`, the output gradient and the hidden-layer gradients are
    rounded to BF16 before each product, as in the kernels."""
    rnd = (lambda v: v) if exact else bf16
    y, c = forward(params, X, exact)
    T = np.asarray(T, dtype=np.float64)
    n = y.shape[0]
    loss = float(np.mean((y - T) ** 2)) if n else 0.0
    dy = rnd(2.0 * (y - T) / (3.0 * n))                  # dL/dy
    g = {"W3": dy.T @ c["h2"], "b3": dy.sum(axis=0)}
    dz2 = rnd((dy @ c["W3"]) * (c["h2"] > 0))          # through ReLU: h > 0 exactly where z > 0
    g["W2"], g["b2"] = dz2.T @ c["h1"], dz2.sum(axis=0)
    dz1 = rnd((dz2 @ c["W2"]) * (c["h1"] > 0))
    g["W1"], g["b1"] = dz1.T @ c["X"], dz1.sum(axis=0)
    return loss, pack(g)


def weight_mask():
    """1 for the entries of W1, W2, W3 (decayed by AdamW), 0 for the biases."""
    return pack({name: (np.ones(shape) if name in WEIGHTS else np.zeros(shape)) for name, shape in SIZES})


def adamw(params, grads, m, v, t, lr, weight_decay, beta1=0.9, beta2=0.999, eps=1e-8):
    """One AdamW step (Adam moments with bias correction, decoupled weight decay on the weights only).

    `t` is the number of this step, starting at 1.  Returns (params, m, v)."""
    p = np.asarray(params, dtype=np.float64)
    g = np.asarray(grads, dtype=np.float64)
    m = beta1 * np.asarray(m, dtype=np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, dtype=np.float64) + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    p = p - lr * (mhat / (np.sqrt(vhat) + eps) + weight_decay * weight_mask() * p)
    return p, m, v


def smooth_from(stencil_offsets, stencil_ids, face_masks, o0, iterations, relaxation, constraint_distance,
                sphere=False):
    """Jacobi sweeps of Eq. 1 starting from the offsets o0 (n, 3), voxel units, FP64.

    Each sweep reads every offset from the previous buffer (the double buffer of
    Sec. 2.4): o_i <- clamp(o_i + lambda / N_i * sum_j (u_ij + o_j - o_i)), the
    clamp a box of half-width d/2 per axis or (sphere) a ball of radius d/2."""
    so = np.asarray(stencil_offsets, dtype=np.int64)
    ids = np.asarray(stencil_ids, dtype=np.int64)
    fm = np.asarray(face_masks, dtype=np.int64)
    n = fm.size
    h = 0.5 * float(np.float32(constraint_distance))
    lam = float(np.float32(relaxation))
    # (point, neighbour, unit step) triples in stencil order
    rows, cols, steps = [], [], []
    for i in range(n):
        k = so[i]
        for f in range(6):
            if (fm[i] >> f) & 1:
                rows.append(i)
                cols.append(ids[k])
                steps.append(UNIT[f])
                k += 1
    rows, cols = np.array(rows, dtype=np.int64), np.array(cols, dtype=np.int64)
    steps = np.array(steps, dtype=np.float64).reshape(-1, 3)
    deg = np.bincount(rows, minlength=n).astype(np.float64)
    o = np.array(o0, dtype=np.float64).reshape(n, 3)
    for _ in range(int(iterations)):
        acc = np.zeros((n, 3))
        np.add.at(acc, rows, steps + o[cols] - o[rows])
        scale = np.where(deg > 0, lam / np.maximum(deg, 1.0), 0.0)
        new = o + scale[:, None] * acc
        if sphere:
            r = np.sqrt((new * new).sum(axis=1))
            f = np.where(r > h, h / np.where(r > 0, r, 1.0), 1.0)
            new = new * f[:, None]
        else:
            new = np.clip(new, -h, h)
        o = new
    return o
