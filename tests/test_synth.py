"""The seeded input generators: deterministic, and the Voronoi bucket search is exact."""
import numpy as np

import sn_synth


def test_deterministic():
    a = sn_synth.config1().labels
    b = sn_synth.config1().labels
    assert a.dtype == np.uint16 and a.shape == (64, 64, 64)
    np.testing.assert_array_equal(a, b)
    assert set(np.unique(a).tolist()) <= {0, 1, 2, 3, 4}


def _brute_voronoi(dims, sx, sy, sz, zs):
    nx, ny, nz = dims
    z, y, x = np.mgrid[0:nz, 0:ny, 0:nx]
    best = np.full(x.shape, np.iinfo(np.int64).max)
    second = best.copy()
    arg = np.zeros(x.shape, dtype=np.int64)
    for s in range(len(sx)):
        d = (x - sx[s]) ** 2 + (y - sy[s]) ** 2 + (zs * (z - sz[s])) ** 2
        closer = d < best
        second = np.where(closer, best, np.minimum(second, d))
        arg = np.where(closer, s, arg)
        best = np.where(closer, d, best)
    return arg, best, second


def _seeds(n, dims, seed):
    r = sn_synth._SplitMix(seed)
    out = []
    for _ in range(n):
        out.append(tuple(r.below(d) for d in dims))
    return np.array(out)


def test_voronoi_bucket_search_exact():
    # the C generator draws seeds with the same splitmix64 stream as _SplitMix.below
    dims = (37, 29, 23)
    for n, seed in [(5, 11), (60, 12), (300, 13)]:
        lab = sn_synth.voronoi(dims, n, np.uint16, seed=seed)
        s = _seeds(n, dims, seed)
        arg, _, _ = _brute_voronoi(dims, s[:, 0], s[:, 1], s[:, 2], 1)
        np.testing.assert_array_equal(lab.astype(np.int64), arg + 1)


def test_connectome_gap_fraction_and_labels():
    # at this small size the integer thresholds step by more than the band
    a = sn_synth.connectome((96, 80, 40), n_seeds=300, zscale=4, seed=3)
    assert abs(float((a == 0).mean()) - 0.05) <= 0.015
    assert a.max() <= 300
    b = sn_synth.connectome((256, 256, 128), n_seeds=800, zscale=4, seed=3)
    assert abs(float((b == 0).mean()) - 0.05) <= 0.0025


def test_atlas_occupancy():
    a = sn_synth.atlas((96, 96, 96), n_seeds=20, seed=2)
    occ = float((a > 0).mean())
    assert abs(occ - 0.40) <= 0.005
    assert a.max() <= 20


def test_config5_params_ranges():
    for i in range(256):
        dims, dtype, kind, n, seed = sn_synth.config5_params(i)
        assert all(32 <= d <= 256 for d in dims)
        assert dtype in (np.uint8, np.uint16)
        assert kind in ("ellipsoids", "voronoi")
        assert 1 <= n <= 20 and seed == 5000 + i
