"""The r-ring lower bound on proposal error (tests/ring_bound.py), checked on small maps:

* the n-ring view of a point fixes its offset after n sweeps (the bound at r = n is
  rounding noise), so the bound is a property of the method, not of a model;
* the bound never grows with r (a finer partition has smaller classes);
* the hashed colour classes equal the classes of explicitly built view tuples for r <= 2;
* the per-face neighbour table reproduces the CSR stencil in face order.
"""
import numpy as np

import oracle
import sn_synth
from ring_bound import class_half_spread, face_neighbours, ring_bounds


def _mesh(seed=3, dims=(36, 32, 28)):
    lab = sn_synth.ellipsoids(dims, 4, 4.0, 12.0, np.uint16, seed=seed)
    return oracle.extract(lab)


def test_face_neighbours_follow_the_stencil():
    m = _mesh()
    nb = face_neighbours(m.stencil_offsets, m.stencil_ids, m.face_masks)
    for i in range(0, m.n_points, 97):
        ids = [int(j) for j in nb[i] if j >= 0]
        assert ids == list(m.stencil_ids[m.stencil_offsets[i]:m.stencil_offsets[i + 1]])
        assert bin(int(m.face_masks[i])).count("1") == len(ids)


def test_n_ring_fixes_the_result_and_the_bound_decreases():
    m = _mesh()
    n = 6
    off, _ = oracle.smooth(m, iterations=n, relaxation=0.5, constraint=1.0)
    rows = ring_bounds(m, off, n)
    lbs = [lb for _, lb, _ in rows]
    assert lbs[0] > 0.05          # the face mask alone does not fix the offset
    assert lbs[-1] < 1e-12        # the n-ring view does (up to rounding)
    assert all(b <= a + 1e-15 for a, b in zip(lbs, lbs[1:]))
    classes = [k for _, _, k in rows]
    assert all(b >= a for a, b in zip(classes, classes[1:]))


def test_hashed_classes_match_explicit_views():
    m = _mesh(seed=5, dims=(24, 22, 20))
    nb = face_neighbours(m.stencil_offsets, m.stencil_ids, m.face_masks)
    views = [int(v) for v in m.face_masks]
    # one column of targets per point id: each class's spread is zero iff the class is a single view
    for r in range(3):
        _, lb, k = ring_bounds(m, np.zeros((m.n_points, 1)), r)[-1]
        assert lb == 0.0
        assert k == len(set(views))
        views = [(views[i], tuple(views[j] if j >= 0 else None for j in nb[i])) for i in range(m.n_points)]


def test_half_spread_by_hand():
    colours = np.array([1, 1, 2, 2, 2], dtype=np.uint64)
    t = np.array([[0.0], [0.5], [1.0], [1.1], [0.9]])
    lb, k = class_half_spread(colours, t)
    assert k == 2 and abs(lb - 0.25) < 1e-15
