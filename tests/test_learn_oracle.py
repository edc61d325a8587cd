"""Pins of the learned-proposal oracle (oracle/learn.py) against independent facts.

* BF16 rounding: hand-picked values and torch's own float32 -> bfloat16 cast.
* Features: the unit-voxel example worked out by hand, and a second construction
  of the neighbour blocks from the cell grid (not from the stencil ids).
* Forward pass: the composed affine map when no ReLU is active, and exactness of
  the BF16 mode on operands that BF16 holds exactly.
* Gradients: central finite differences of the exact-mode loss.
* AdamW: the closed form of the first step and a scalar worked by hand.
"""
import numpy as np
import pytest

import oracle
from oracle import learn


# ------------------------------------------------------------------ bf16
def test_bf16_hand_values():
    one = 1.0
    ulp = 2.0 ** -7                                   # spacing of BF16 values in [1, 2)
    cases = {
        one: one,
        one + ulp / 2: one,                           # tie -> even (1.0)
        one + 3 * ulp / 2: one + 2 * ulp,             # tie -> even (1 + 2 ulp)
        one + ulp / 2 + 1e-9: one + ulp,              # above the tie
        -3.0: -3.0,
        0.1: 0.10009765625,                           # 0x3DCD
        65504.0: 65536.0,
        0.0: 0.0,
        2.0 ** -130: 2.0 ** -130,                     # subnormal, representable
        2.0 ** -134: 0.0,                             # half the smallest subnormal: tie -> 0
    }
    for x, want in cases.items():
        assert learn.bf16(x) == want, (x, learn.bf16(x), want)


def test_bf16_matches_torch_on_float32_inputs():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = (rng.standard_normal(20000) * np.exp(rng.uniform(-30, 30, 20000))).astype(np.float32)
    x[:100] = (1.0 + (np.arange(100) + 0.5) * 2.0 ** -7).astype(np.float32)   # exact ties
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(learn.bf16(x.astype(np.float64)), want)


# -------------------------------------------------------------- features
def _unit_voxel_mesh():
    lab = np.zeros((3, 3, 3), dtype=np.uint16)
    lab[1, 1, 1] = 7
    return oracle.extract(lab)


def test_features_unit_voxel_by_hand():
    m = _unit_voxel_mesh()
    X = learn.features(m.stencil_offsets, m.stencil_ids, m.face_masks, 1.0)
    assert X.shape == (8, 32)
    # point 0 is cell (0,0,0): neighbours across +x, +y, +z (cells (1,0,0), (0,1,0), (0,0,1))
    want0 = np.zeros(32)
    want0[0:3] = (1, 1, 1)
    want0[3] = 3
    want0[4:10] = (0, 1, 0, 1, 0, 1)
    want0[13:16] = (-1, 1, 1)   # +x neighbour, cell (1,0,0): faces -x, +y, +z
    want0[19:22] = (1, -1, 1)   # +y neighbour, cell (0,1,0): faces +x, -y, +z
    want0[25:28] = (1, 1, -1)   # +z neighbour, cell (0,0,1): faces +x, +y, -z
    want0[28] = 0.5
    np.testing.assert_array_equal(X[0], want0)
    # point 7 is cell (1,1,1): neighbours across -x, -y, -z
    want7 = np.zeros(32)
    want7[0:3] = (-1, -1, -1)
    want7[3] = 3
    want7[4:10] = (1, 0, 1, 0, 1, 0)
    want7[10:13] = (1, -1, -1)  # -x neighbour, cell (0,1,1): faces +x, -y, -z
    want7[16:19] = (-1, 1, -1)  # -y neighbour, cell (1,0,1)
    want7[22:25] = (-1, -1, 1)  # -z neighbour, cell (1,1,0)
    want7[28] = 0.5
    np.testing.assert_array_equal(X[7], want7)


def _features_from_cells(m, d):
    """Neighbour blocks found by looking the face-adjacent cell up in the cell grid."""
    cells = np.asarray(m.cells, dtype=np.int64)
    where = {tuple(c): i for i, c in enumerate(cells)}
    fm = np.asarray(m.face_masks, dtype=np.int64)
    n = fm.size
    X = np.zeros((n, 32))
    unit = [(-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)]

    def s_of(i):
        return np.sum([unit[f] for f in range(6) if (fm[i] >> f) & 1], axis=0) if fm[i] else np.zeros(3)

    for i in range(n):
        X[i, 0:3] = s_of(i)
        X[i, 3] = bin(int(fm[i])).count("1")
        for f in range(6):
            if (fm[i] >> f) & 1:
                X[i, 4 + f] = 1
                j = where[tuple(cells[i] + np.array(unit[f]))]
                X[i, 10 + 3 * f:13 + 3 * f] = s_of(j)
        X[i, 28] = learn.bf16(d / 2)
    return X


@pytest.mark.parametrize("seed", [1, 2])
def test_features_match_cell_grid_construction(seed):
    rng = np.random.default_rng(seed)
    lab = rng.integers(0, 3, size=(7, 8, 9)).astype(np.uint8)
    m = oracle.extract(lab)
    X = learn.features(m.stencil_offsets, m.stencil_ids, m.face_masks, 0.7)
    np.testing.assert_array_equal(X, _features_from_cells(m, 0.7))
    assert np.all(learn.bf16(X) == X)                 # every feature is exact in BF16


# ----------------------------------------------------------------- forward
def test_forward_without_relu_is_the_composed_affine_map():
    rng = np.random.default_rng(3)
    d = {name: rng.standard_normal(shape) * 0.1 for name, shape in learn.SIZES}
    d["b1"] = np.full(64, 50.0)                        # keeps every hidden pre-activation positive
    d["b2"] = np.full(64, 50.0)
    d["W2"] = np.abs(d["W2"])
    p = learn.pack(d)
    X = rng.uniform(-1, 1, size=(20, 32))
    y, _ = learn.forward(p, X, exact=True)
    A = d["W3"] @ d["W2"] @ d["W1"]
    c = d["W3"] @ (d["W2"] @ d["b1"] + d["b2"]) + d["b3"]
    np.testing.assert_allclose(y, X @ A.T + c, rtol=1e-12, atol=1e-12)


def test_forward_bf16_mode_is_exact_on_representable_operands():
    # sparse small weights keep every hidden value on a coarse grid that BF16 holds exactly
    rng = np.random.default_rng(4)
    d = {name: np.zeros(shape) for name, shape in learn.SIZES}
    for r in range(64):
        d["W1"][r, rng.choice(32, 3, replace=False)] = rng.choice([-1.0, -0.5, 0.5, 1.0], 3)
        d["W2"][r, rng.choice(64, 2, replace=False)] = rng.choice([-1.0, 1.0], 2)
    d["b1"] = rng.integers(-4, 5, 64) * 0.25
    d["b2"] = rng.integers(-4, 5, 64) * 0.25
    d["W3"] = rng.standard_normal((3, 64))
    d["b3"] = rng.standard_normal(3)
    p = learn.pack(d)
    X = rng.integers(-3, 4, size=(30, 32)).astype(np.float64)
    y_b, c = learn.forward(p, X)
    y_e, _ = learn.forward(p, X, exact=True)
    assert np.all(learn.bf16(c["h1"]) == c["h1"]) and np.all(learn.bf16(c["h2"]) == c["h2"])
    assert np.all(learn.bf16(d["W3"]) != d["W3"])    # W3 is rounded in BF16 mode ...
    d["W3"] = learn.bf16(d["W3"])                      # ... and nothing else is
    y_e, _ = learn.forward(learn.pack(d), X, exact=True)
    np.testing.assert_array_equal(y_b, y_e)


def test_relu_zeroes_negative_units():
    d = {name: np.zeros(shape) for name, shape in learn.SIZES}
    d["W1"][0, 0] = 1.0                                # unit 0 of layer 1 copies x0
    d["W2"][0, 0] = 1.0                                # unit 0 of layer 2 copies it again
    d["W3"][0, 0] = 2.0
    d["b3"][:] = (0.5, -1.0, 0.0)
    X = np.zeros((2, 32))
    X[0, 0], X[1, 0] = 3.0, -3.0
    y, _ = learn.forward(learn.pack(d), X)
    np.testing.assert_array_equal(y, [[6.5, -1.0, 0.0], [0.5, -1.0, 0.0]])


# ---------------------------------------------------------------- gradient
def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(5)
    p = learn.init_params(11).astype(np.float64)
    p[learn.pack({n: (np.ones(s) if n.startswith("b") else np.zeros(s)) for n, s in learn.SIZES}) > 0] = \
        rng.uniform(-0.1, 0.1, 64 + 64 + 3)
    X = rng.uniform(-2, 2, size=(12, 32))
    T = rng.uniform(-0.5, 0.5, size=(12, 3))
    _, g = learn.loss_and_grad(p, X, T, exact=True)
    idx = rng.choice(learn.N_PARAMS, 300, replace=False)
    eps = 1e-6
    for k in idx:
        e = np.zeros(learn.N_PARAMS)
        e[k] = eps
        lp, _ = learn.loss_and_grad(p + e, X, T, exact=True)
        lm, _ = learn.loss_and_grad(p - e, X, T, exact=True)
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)), (k, fd, g[k])


def test_gradient_of_a_perfect_fit_is_zero():
    rng = np.random.default_rng(6)
    p = learn.init_params(3)
    X = rng.integers(-3, 4, size=(9, 32)).astype(np.float64)
    y, _ = learn.forward(p, X)
    loss, g = learn.loss_and_grad(p, X, y)
    assert loss == 0.0 and np.all(g == 0.0)


# ------------------------------------------------------------------- AdamW
def test_adamw_first_step_closed_form():
    rng = np.random.default_rng(7)
    p = rng.standard_normal(learn.N_PARAMS)
    g = rng.standard_normal(learn.N_PARAMS)
    lr, wd, eps = 1e-3, 0.01, 1e-8
    p1, m1, v1 = learn.adamw(p, g, np.zeros_like(p), np.zeros_like(p), 1, lr, wd, eps=eps)
    # after one step the bias-corrected moments are g and g^2
    np.testing.assert_allclose(m1, 0.1 * g, rtol=1e-14)
    np.testing.assert_allclose(v1, 0.001 * g * g, rtol=1e-14)
    wmask = learn.weight_mask()
    want = p - lr * (g / (np.abs(g) + eps) + wd * wmask * p)
    np.testing.assert_allclose(p1, want, rtol=1e-12, atol=1e-15)
    assert wmask.sum() == 64 * 32 + 64 * 64 + 3 * 64


def test_adamw_two_scalar_steps_by_hand():
    n = learn.N_PARAMS
    k = 0                                              # an entry of W1 (decayed)
    p, m, v = np.zeros(n), np.zeros(n), np.zeros(n)
    p[k] = 1.0
    g1, g2 = np.zeros(n), np.zeros(n)
    g1[k], g2[k] = 0.5, -0.25
    p, m, v = learn.adamw(p, g1, m, v, 1, 0.1, 0.5, eps=0.0)
    # m = 0.05, v = 0.00025; mhat = 0.5, vhat = 0.25 -> step 1; decay 0.5 * 1
    assert p[k] == pytest.approx(1.0 - 0.1 * (1.0 + 0.5), abs=1e-15)
    p, m, v = learn.adamw(p, g2, m, v, 2, 0.1, 0.5, eps=0.0)
    m2 = 0.9 * 0.05 + 0.1 * -0.25                       # 0.02
    v2 = 0.999 * 0.00025 + 0.001 * 0.0625               # 0.00031225
    mhat, vhat = m2 / (1 - 0.81), v2 / (1 - 0.999 ** 2)
    want = 0.85 - 0.1 * (mhat / np.sqrt(vhat) + 0.5 * 0.85)
    assert p[k] == pytest.approx(want, abs=1e-14)


# ------------------------------------------------- smoothing from given offsets
@pytest.mark.parametrize("sphere", [False, True])
def test_smooth_from_zero_matches_the_c_oracle(sphere):
    rng = np.random.default_rng(8)
    lab = rng.integers(0, 3, size=(8, 9, 10)).astype(np.uint16)
    m = oracle.extract(lab, spacing=(1.0, 2.0, 0.5))
    off, _ = oracle.smooth(m, spacing=(1.0, 2.0, 0.5), iterations=7, relaxation=0.5, constraint=0.75, sphere=sphere)
    o = learn.smooth_from(m.stencil_offsets, m.stencil_ids, m.face_masks, np.zeros((m.n_points, 3)), 7, 0.5, 0.75,
                          sphere=sphere)
    np.testing.assert_allclose(o, off, rtol=0, atol=1e-12)


def test_smooth_from_splits_into_consecutive_runs():
    rng = np.random.default_rng(9)
    lab = rng.integers(0, 2, size=(7, 7, 7)).astype(np.uint8)
    m = oracle.extract(lab)
    args = (m.stencil_offsets, m.stencil_ids, m.face_masks)
    o5 = learn.smooth_from(*args, np.zeros((m.n_points, 3)), 5, 0.4, 1.0)
    o2 = learn.smooth_from(*args, np.zeros((m.n_points, 3)), 2, 0.4, 1.0)
    o23 = learn.smooth_from(*args, o2, 3, 0.4, 1.0)
    np.testing.assert_allclose(o23, o5, rtol=0, atol=1e-15)
