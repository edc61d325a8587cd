"""Learned smoothing proposal: CUDA path vs the FP64 oracle (oracle/learn.py), through the C ABI.

* Features are exact small integers (and d/2 in BF16): bit-exact.
* Forward pass: both sides round weights and hidden activations to BF16; they
  differ by FP32 vs FP64 accumulation, which can move a hidden value across a
  BF16 rounding boundary.  Such a flip changes that value by at most one BF16
  ulp (2^-7 of it), so each output is bounded by
  2^-7 * sum_k |W3_ck| (|h2_k| + 2 sum_j |W2_kj| |h1_j|) (+1e-5), and nearly all
  outputs must agree to 1e-5.
* Gradient and AdamW: FP32 sums of BF16 products against FP64 sums; the
  gradient within 2% of its largest entry everywhere and 1e-3 relative for most
  entries, AdamW within 1e-5 relative.
* Proposal + corrections: the proposal within the forward bound; a correction
  sweep does not grow a max-norm difference (convex combination, then a
  1-Lipschitz clamp), so the same bound holds after the sweeps.
"""
import numpy as np
import pytest

import oracle
import sn_synth
from oracle import learn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2401_14906_gb300 import build
    build.build()


def _sn():
    from paper_2401_14906_gb300 import sn
    return sn


def _dev_labels(labels):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(labels).view(
        {1: np.uint8, 2: np.int16, 4: np.int32}[labels.dtype.itemsize])).cuda()
    return t.view({1: torch.uint8, 2: torch.uint16, 4: torch.uint32}[labels.dtype.itemsize])


def _bits_to_float(x16):
    """int16 tensor of BF16 bit patterns -> float64 numpy array."""
    u = x16.cpu().numpy().view(np.uint16).astype(np.uint32) << 16
    return u.view(np.float32).astype(np.float64)


def _float_to_bits(x):
    """float64 array of BF16-exact values -> int16 device tensor of BF16 bits."""
    import torch
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    assert np.all(learn.bf16(f.astype(np.float64)) == f)
    b = (f.view(np.uint32) >> 16).astype(np.uint16).view(np.int16)
    return torch.from_numpy(b).cuda()


def _maps():
    rng = np.random.default_rng(21)
    small = rng.integers(0, 3, size=(13, 17, 40)).astype(np.uint8)
    w = sn_synth.config1()
    return [("random_u8", small, (1.0, 1.0, 1.0)), ("config1", w.labels, w.spacing)]


def _params(seed):
    p = learn.init_params(seed).astype(np.float64)
    rng = np.random.default_rng(seed + 100)
    bias = learn.weight_mask() == 0
    p[bias] = rng.uniform(-0.2, 0.2, int(bias.sum()))
    return p.astype(np.float32)


def _forward_bound(params, X):
    y, c = learn.forward(params, X)
    W2, W3 = np.abs(c["W2"]), np.abs(c["W3"])
    inner = np.abs(c["h2"]) + 2.0 * (np.abs(c["h1"]) @ W2.T)
    return y, 2.0 ** -7 * (inner @ W3.T) + 1e-5


# ---------------------------------------------------------------- features
@pytest.mark.parametrize("case", range(2))
@pytest.mark.parametrize("d", [1.0, 0.7])
def test_features_bit_exact(case, d):
    sn = _sn()
    name, lab, sp = _maps()[case]
    ref = oracle.extract(lab, spacing=sp)
    want = learn.features(ref.stencil_offsets, ref.stencil_ids, ref.face_masks, d)
    m = sn.sn_extract(_dev_labels(lab), sp)
    got = _bits_to_float(sn.sn_learn_features(m, d))
    m.free()
    np.testing.assert_array_equal(got, want)


# ----------------------------------------------------------------- forward
@pytest.mark.parametrize("n", [1, 15, 16, 17, 64, 1000, 4099])
def test_forward_matches_oracle(n):
    sn = _sn()
    rng = np.random.default_rng(n)
    X = rng.integers(-6, 7, size=(n, 32)).astype(np.float64)
    X[:, 28] = 0.5
    p = _params(3)
    L = sn.sn_learner_create()
    sn.sn_learner_set_params(L, p)
    y = sn.sn_learn_forward(L, _float_to_bits(X)).cpu().numpy().astype(np.float64)
    want, bound = _forward_bound(p, X)
    err = np.abs(y - want)
    assert np.all(err <= bound), (err - bound).max()
    assert np.mean(err <= 1e-5 * (1 + np.abs(want))) >= 0.99
    L.free()


def test_params_round_trip():
    sn = _sn()
    p = _params(4)
    L = sn.sn_learner_create()
    sn.sn_learner_set_params(L, p)
    np.testing.assert_array_equal(sn.sn_learner_get_params(L), p)
    L.free()


# ---------------------------------------------------------------- gradient
@pytest.mark.parametrize("n", [16, 100, 1000, 3000])
def test_gradient_matches_oracle(n):
    import torch
    sn = _sn()
    rng = np.random.default_rng(n + 7)
    X = rng.integers(-6, 7, size=(n, 32)).astype(np.float64)
    X[:, 28] = 0.5
    T = rng.uniform(-0.5, 0.5, size=(n, 3)).astype(np.float32)
    p = _params(5)
    L = sn.sn_learner_create()
    sn.sn_learner_set_params(L, p)
    g, sse = sn.sn_learn_gradient(L, _float_to_bits(X), torch.from_numpy(T).cuda())
    g = g.cpu().numpy().astype(np.float64)
    loss, want = learn.loss_and_grad(p, X, T.astype(np.float64))
    assert float(sse.item()) / (3 * n) == pytest.approx(loss, rel=1e-4)
    scale = np.abs(want).max()
    assert np.abs(g - want).max() <= 0.02 * scale
    big = np.abs(want) > 1e-3 * scale
    rel = np.abs(g - want)[big] / np.abs(want)[big]
    assert np.median(rel) <= 1e-3
    L.free()


# ------------------------------------------------------------------- AdamW
def test_adamw_steps_match_oracle():
    import torch
    sn = _sn()
    rng = np.random.default_rng(9)
    p = _params(6)
    L = sn.sn_learner_create()
    sn.sn_learner_set_params(L, p)
    want, m, v = p.astype(np.float64), np.zeros(learn.N_PARAMS), np.zeros(learn.N_PARAMS)
    for t in (1, 2, 3):
        g = rng.standard_normal(learn.N_PARAMS).astype(np.float32)
        sn.sn_learner_step(L, torch.from_numpy(g).cuda(), 1e-2, 0.05)
        want, m, v = learn.adamw(want, g.astype(np.float64), m, v, t, 1e-2, 0.05)
    got = sn.sn_learner_get_params(L).astype(np.float64)
    np.testing.assert_allclose(got, want, rtol=1e-5, atol=1e-6)
    L.free()


# --------------------------------------------------- training, proposal, corrections
def _trained_learner(lab, sp, epochs=40):
    sn = _sn()
    m = sn.sn_extract(_dev_labels(lab), sp)
    sn.sn_smooth(m, 16, 0.5, 1.0)
    L = sn.sn_learner_create()
    sn.sn_learner_set_params(L, learn.init_params(1))
    sn.sn_learner_add_examples(L, m, 1.0)
    assert sn.sn_learner_n_examples(L) == m.counts[0]
    first = sn.sn_learner_train(L, 1, 512, 3e-3, 1e-4, seed=5)
    last = sn.sn_learner_train(L, epochs, 512, 3e-3, 1e-4, seed=6)
    m.free()
    return L, first, last


def test_training_lowers_the_loss():
    w = sn_synth.config1()
    L, first, last = _trained_learner(w.labels, w.spacing)
    assert np.isfinite(last) and last < first
    L.free()


@pytest.mark.parametrize("engine", ["mma_sync", "tcgen05"])
@pytest.mark.parametrize("corrections", [0, 1, 2, 3])
@pytest.mark.parametrize("sphere", [False, True])
def test_learned_smoothing_matches_oracle(corrections, sphere, engine):
    sn = _sn()
    w = sn_synth.config1()
    sp = (1.0, 1.5, 0.75)
    ref = oracle.extract(w.labels, spacing=sp)
    p = _params(8)
    L = sn.sn_learner_create()
    sn.sn_learner_set_params(L, p)
    sn.sn_learner_set_engine(L, engine)
    m = sn.sn_extract(_dev_labels(w.labels), sp)
    sn.sn_smooth_learned(m, L, corrections, 0.5, 1.0, sphere=sphere)
    got = sn.sn_mesh_copy_to_host(m)
    m.free()
    L.free()
    X = learn.features(ref.stencil_offsets, ref.stencil_ids, ref.face_masks, 1.0)
    y, bound = _forward_bound(p, X)
    h = 0.5
    if sphere:
        r = np.sqrt((y * y).sum(axis=1))
        o0 = y * np.where(r > h, h / np.where(r > 0, r, 1.0), 1.0)[:, None]
    else:
        o0 = np.clip(y, -h, h)
    want = learn.smooth_from(ref.stencil_offsets, ref.stencil_ids, ref.face_masks, o0, corrections, 0.5, 1.0,
                             sphere=sphere)
    off = got["offsets"].astype(np.float64)
    tol = bound.max() + 1e-5
    assert np.abs(off - want).max() <= tol
    # every point in its constraint region
    if sphere:
        assert np.all(np.sqrt((off * off).sum(axis=1)) <= h * (1 + 1e-6))
    else:
        assert np.all(np.abs(off) <= h)
    # world positions: cell centre + spacing * offset, one FP32 rounding
    centre = ref.points                                # FP64 cell centres (unsmoothed oracle points)
    world = centre + np.array(sp) * off
    np.testing.assert_allclose(got["points"], world, rtol=0, atol=1e-5 * max(sp) + 1e-5)


@pytest.mark.parametrize("nx", [1, 3, 6, 11, 24, 40])
def test_engines_agree_on_ragged_tiles(nx):
    """Both engines on small random maps whose point counts fall on and between 128-point tiles."""
    sn = _sn()
    rng = np.random.default_rng(nx)
    lab = rng.integers(0, 3, size=(5, 7, nx)).astype(np.uint8)
    p = _params(9)
    outs = []
    for engine in ("mma_sync", "tcgen05"):
        L = sn.sn_learner_create()
        sn.sn_learner_set_params(L, p)
        sn.sn_learner_set_engine(L, engine)
        m = sn.sn_extract(_dev_labels(lab))
        sn.sn_smooth_learned(m, L, 0, 0.5, 1.0)
        outs.append(sn.sn_mesh_copy_to_host(m)["offsets"].astype(np.float64))
        m.free()
        L.free()
    ref = oracle.extract(lab)
    assert outs[0].shape == outs[1].shape == (ref.n_points, 3) and ref.n_points > 0
    X = learn.features(ref.stencil_offsets, ref.stencil_ids, ref.face_masks, 1.0)
    y, bound = _forward_bound(p, X)
    want = np.clip(y, -0.5, 0.5)
    for o in outs:
        assert np.all(np.abs(o - want) <= bound)


def test_unknown_engine_rejected():
    sn = _sn()
    L = sn.sn_learner_create()
    with pytest.raises(sn.SNError):
        sn.sn_learner_set_engine(L, 7)
    L.free()


@pytest.mark.parametrize("engine", ["mma_sync", "tcgen05"])
def test_degenerate_meshes(engine):
    """No points at all, and the 8 points of a single voxel (one partial tile of either engine)."""
    sn = _sn()
    L = sn.sn_learner_create()
    p = _params(10)
    sn.sn_learner_set_params(L, p)
    sn.sn_learner_set_engine(L, engine)
    empty = sn.sn_extract(_dev_labels(np.zeros((3, 4, 5), np.uint16)))
    sn.sn_smooth_learned(empty, L, 2, 0.5, 1.0)
    assert empty.counts == (0, 0, 0)
    empty.free()
    lab = np.zeros((3, 3, 3), np.uint16)
    lab[1, 1, 1] = 5
    m = sn.sn_extract(_dev_labels(lab))
    sn.sn_smooth_learned(m, L, 0, 0.5, 1.0)
    got = sn.sn_mesh_copy_to_host(m)["offsets"].astype(np.float64)
    m.free()
    L.free()
    ref = oracle.extract(lab)
    X = learn.features(ref.stencil_offsets, ref.stencil_ids, ref.face_masks, 1.0)
    y, bound = _forward_bound(p, X)
    assert got.shape == (8, 3)
    assert np.all(np.abs(got - np.clip(y, -0.5, 0.5)) <= bound)
