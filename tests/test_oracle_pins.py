"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these compares the oracle with itself: each check uses a hand-derived
fixture, a closed form, a topological invariant, or an independent construction
(``brute.py``).  A dropped edge term, a wrong sign or index, a transposed cell or
a wrong smoothing term fails at least one of them.
"""
import json
import os

import numpy as np
import pytest

import brute
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------ worked example
def test_unit_voxel_golden():
    g = json.load(open(os.path.join(GOLDEN, "unit_voxel.json")))
    lab = np.zeros(g["dims"][::-1], dtype=np.uint16)
    x, y, z = g["voxel"]
    lab[z, y, x] = g["label"]
    m = oracle.extract(lab)
    assert m.n_points == g["n_points"]
    np.testing.assert_array_equal(m.cells, np.array(g["cells_zyx_order"]))
    np.testing.assert_array_equal(m.points, np.array(g["points"]))
    np.testing.assert_array_equal(m.quads, np.array(g["quads"]))
    np.testing.assert_array_equal(m.quad_labels, np.array(g["quad_labels"]))
    np.testing.assert_array_equal(m.stencil_offsets, np.array(g["stencil_offsets"]))
    np.testing.assert_array_equal(m.stencil_ids, np.array(g["stencil_ids"]))
    for case in g["smoothing_cases"]:
        off, pts = oracle.smooth(m, iterations=case["iterations"], relaxation=case["relaxation"],
                                 constraint=case["constraint"])
        # distance of every point from the cube centre (1,1,1), per axis
        h = np.abs(pts - 1.0)
        np.testing.assert_allclose(h, case["h"], rtol=0, atol=1e-15)


# -------------------------------------------------- brute-force agreement
def _check_against_faces(lab, selected=None, background=0):
    m = oracle.extract(lab, selected=selected, background=background)
    fq = brute.face_quads(lab, selected, background)
    cells = brute.point_cells(fq)
    assert m.n_points == len(cells)
    if cells:
        np.testing.assert_array_equal(m.cells, np.array(cells, dtype=np.int32))
    assert m.n_quads == len(fq)
    for q in range(m.n_quads):
        key, cset, labs = fq[q]
        got = [tuple(int(v) for v in m.cells[p]) for p in m.quads[q]]
        assert frozenset(got) == cset, (q, key)
        assert tuple(int(v) for v in m.quad_labels[q]) == labs
        # the four cells form a cycle of unit steps ...
        for r in range(4):
            a, b = np.array(got[r]), np.array(got[(r + 1) % 4])
            assert np.abs(a - b).sum() == 1
        # ... oriented with the normal along +axis
        v = np.array(got, dtype=np.float64)
        n = np.cross(v[2] - v[0], v[3] - v[1])
        axis = key[3]
        assert n[axis] > 0 and abs(n[(axis + 1) % 3]) == 0 and abs(n[(axis + 2) % 3]) == 0
    # stencil: the face-neighbour 1-ring of the quad mesh, faces -x,+x,-y,+y,-z,+z
    ring = brute.one_ring(m.n_points, m.quads)
    order = {(-1, 0, 0): 0, (1, 0, 0): 1, (0, -1, 0): 2, (0, 1, 0): 3, (0, 0, -1): 4, (0, 0, 1): 5}
    for p in range(m.n_points):
        ids = m.stencil_ids[m.stencil_offsets[p]:m.stencil_offsets[p + 1]]
        assert set(int(i) for i in ids) == ring[p]
        faces = [order[tuple(int(t) for t in (m.cells[j] - m.cells[p]))] for j in ids]
        assert faces == sorted(faces)
        assert m.face_masks[p] == sum(1 << f for f in faces)
    return m


def test_all_two_label_2x2x2_maps():
    n = 0
    for lab in brute.all_maps((2, 2, 2), 2):
        _check_against_faces(lab)
        n += 1
    assert n == 256


def test_all_three_label_2x2x2_maps_sampled():
    maps = list(brute.all_maps((2, 2, 2), 3))
    assert len(maps) == 6561
    for lab in maps[::7]:
        _check_against_faces(lab)


@pytest.mark.parametrize("seed", range(12))
def test_random_small_maps(seed):
    rng = np.random.default_rng(seed)
    shape = tuple(int(s) for s in rng.integers(1, 7, size=3))
    nl = int(rng.integers(2, 9))
    dtype = [np.uint8, np.uint16, np.uint32][seed % 3]
    lab = rng.integers(0, nl, size=shape).astype(dtype)
    _check_against_faces(lab)


@pytest.mark.parametrize("seed", range(6))
def test_random_small_maps_selected(seed):
    rng = np.random.default_rng(100 + seed)
    shape = tuple(int(s) for s in rng.integers(2, 6, size=3))
    lab = rng.integers(0, 6, size=shape).astype(np.uint16)
    sel = sorted(set(int(v) for v in rng.integers(1, 6, size=2)))
    _check_against_faces(lab, selected=sel, background=0)


def test_max_label_values():
    for dtype in (np.uint8, np.uint16, np.uint32):
        top = np.iinfo(dtype).max
        lab = np.zeros((4, 4, 4), dtype=dtype)
        lab[1:3, 1:3, 1:3] = top
        lab[2, 2, 2] = top - 1
        m = _check_against_faces(lab)
        assert int(m.quad_labels.max()) == top


# ----------------------------------------------------- closed forms, counts
@pytest.mark.parametrize("abc", [(1, 1, 1), (2, 3, 4), (5, 1, 3), (7, 6, 2)])
def test_single_box_closed_form(abc):
    a, b, c = abc
    lab = np.zeros((c + 4, b + 5, a + 3), dtype=np.uint16)
    lab[2:2 + c, 2:2 + b, 1:1 + a] = 9
    m = oracle.extract(lab)
    s = a * b + b * c + c * a
    assert m.n_quads == 2 * s
    assert m.n_points == 2 * s + 2
    edges = brute.quad_edges(m.quads)
    assert len(edges) == 2 * m.n_quads
    assert all(v == 2 for v in edges.values())
    assert m.n_points - len(edges) + m.n_quads == 2


@pytest.mark.parametrize("r,centre", [(2.0, (5.0, 5.0, 5.0)), (3.3, (6.2, 5.7, 6.9)), (4.5, (7.5, 7.0, 7.25)),
                                      (5.9, (8.1, 8.4, 7.6))])
def test_digital_ball_euler_characteristic(r, centre):
    n = 16
    z, y, x = np.mgrid[0:n, 0:n, 0:n]
    d2 = (x - centre[0]) ** 2 + (y - centre[1]) ** 2 + (z - centre[2]) ** 2
    lab = (d2 <= r * r).astype(np.uint8) * 3
    m = oracle.extract(lab)
    edges = brute.quad_edges(m.quads)
    assert all(v == 2 for v in edges.values())
    assert m.n_points - len(edges) + m.n_quads == 2
    nq, npnt = brute.vectorised_counts(lab)
    assert (m.n_quads, m.n_points) == (nq, npnt)


def test_counts_match_vectorised_on_config1():
    import sn_synth
    w = sn_synth.config1()
    m = oracle.extract(w.labels)
    assert (m.n_quads, m.n_points) == brute.vectorised_counts(w.labels)
    # stencil entries = twice the number of unique quad edges (each edge joins two face neighbours)
    assert m.n_stencil == 2 * len(brute.quad_edges(m.quads))


def test_points_shared_between_objects():
    # two boxes of different labels touching along x: the shared wall is a single
    # layer of quads labelled (A, B), and its rim points are the same ids the
    # quads facing the background use
    lab = np.zeros((6, 6, 10), dtype=np.uint16)
    lab[1:5, 1:5, 1:5] = 4
    lab[1:5, 1:5, 5:9] = 8
    m = oracle.extract(lab)
    assert len({tuple(c) for c in m.cells.tolist()}) == m.n_points  # no duplicated points
    lp = [tuple(v) for v in m.quad_labels.tolist()]
    wall = [q for q in range(m.n_quads) if lp[q] == (4, 8)]
    assert len(wall) == 16
    wall_pts = set(int(p) for q in wall for p in m.quads[q])
    bg_pts = set(int(p) for q in range(m.n_quads) if 0 in lp[q] for p in m.quads[q])
    rim = wall_pts & bg_pts
    assert len(rim) == 16  # the 4x4 wall has 5x5 points; its 16 rim points are shared
    edges = brute.quad_edges(m.quads)
    # rim edges of the wall are shared by 3 quads (two background faces and the wall)
    assert sorted(set(edges.values())) == [2, 3]


def test_unselected_labels_merge_into_background():
    lab = np.zeros((5, 5, 8), dtype=np.uint16)
    lab[1:4, 1:4, 1:4] = 2
    lab[1:4, 1:4, 4:7] = 3  # not selected: behaves like background
    m = oracle.extract(lab, selected=[2], background=0)
    ref = np.where(lab == 3, 0, lab)
    m2 = oracle.extract(ref)
    np.testing.assert_array_equal(m.quads, m2.quads)
    np.testing.assert_array_equal(m.quad_labels, m2.quad_labels)
    # an unselected label next to background produces nothing
    only3 = oracle.extract(np.where(lab == 2, 0, lab), selected=[2], background=0)
    assert only3.n_points == 0 and only3.n_quads == 0


def test_degenerate_volumes():
    for shape in [(1, 1, 1), (1, 1, 5), (1, 4, 1), (2, 1, 1), (1, 2, 2)]:
        lab = np.arange(int(np.prod(shape)), dtype=np.uint16).reshape(shape) % 2
        _check_against_faces(lab)
    empty = oracle.extract(np.zeros((3, 4, 5), dtype=np.uint8))
    assert empty.n_points == 0 and empty.n_quads == 0 and empty.n_stencil == 0
    # checkerboard: every edge intersected
    z, y, x = np.mgrid[0:4, 0:3, 0:5]
    cb = ((x + y + z) % 2).astype(np.uint8)
    m = _check_against_faces(cb)
    assert m.n_quads == 4 * 3 * 4 + 4 * 2 * 5 + 3 * 3 * 5


# ---------------------------------------------------------------- smoothing
def _small_mesh(seed, shape=(5, 6, 7), nl=3):
    rng = np.random.default_rng(seed)
    lab = rng.integers(0, nl, size=shape).astype(np.uint16)
    return lab, oracle.extract(lab)


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("spacing", [(1.0, 1.0, 1.0), (1.0, 1.0, 4.0), (0.5, 2.0, 1.25)])
def test_smoothing_matches_dense_jacobi_in_world_units(seed, spacing):
    lab, m = _small_mesh(seed)
    origin = (-3.0, 2.5, 10.0)
    for it, lam, d in [(16, 0.5, 1.0), (7, 0.9, 0.6), (3, 0.25, 2.0)]:
        _, pts = oracle.smooth(m, spacing, origin, it, lam, d)
        ref = brute.dense_jacobi_world(m.cells, m.quads, spacing, origin, it, lam, d)
        np.testing.assert_allclose(pts, ref, rtol=0, atol=1e-11)


def test_smoothing_zero_iterations_and_zero_relaxation_give_centres():
    lab, m = _small_mesh(7)
    for it, lam in [(0, 0.5), (9, 0.0)]:
        off, pts = oracle.smooth(m, (1.0, 2.0, 3.0), (1.0, 1.0, 1.0), it, lam, 1.0)
        assert np.all(off == 0.0)
        np.testing.assert_array_equal(pts, 1.0 + np.array([1.0, 2.0, 3.0]) * (m.cells + 0.5))


def test_smoothing_stays_in_box():
    lab, m = _small_mesh(8, (8, 8, 8), 4)
    for d in (0.2, 1.0, 1.7):
        off, _ = oracle.smooth(m, iterations=20, relaxation=0.9, constraint=d)
        assert np.all(np.abs(off) <= 0.5 * d + 0.0)


def test_flat_interface_motion_spreads_one_ring_per_iteration():
    # a plane x = 4 across the whole volume: every point stays in the plane; the
    # points on the volume boundary lack a neighbour and move first, and with a
    # double buffer (Sec. 2.4) that motion reaches one more ring of points per
    # iteration, so after t iterations points >= t rings inside have not moved
    ny, nz = 12, 11
    lab = np.zeros((nz, ny, 9), dtype=np.uint16)
    lab[:, :, 4:] = 5
    m = oracle.extract(lab)
    assert np.all(m.cells[:, 0] == 3)
    cy, cz = m.cells[:, 1], m.cells[:, 2]
    ring = np.minimum.reduce([cy + 1, ny - 1 - cy, cz + 1, nz - 1 - cz])
    for t in (1, 2, 3, 4):
        off, _ = oracle.smooth(m, iterations=t, relaxation=0.5, constraint=1.0)
        assert np.all(off[:, 0] == 0.0)
        assert np.all(off[ring >= t] == 0.0)
        assert np.all(np.abs(off[ring == t - 1]).sum(axis=1) > 0.0)


# ------------------------------------------------------------ sphere constraint
def test_sphere_constraint_closed_form_unit_voxel():
    # every point moves along its cube diagonal: its per-axis distance h from the
    # cube centre obeys h' = max(h(1 - 2 lambda/3), 1/2 - d/(2 sqrt 3)) with the ball
    lab = np.zeros((3, 3, 3), dtype=np.uint16)
    lab[1, 1, 1] = 7
    m = oracle.extract(lab)
    for it, lam, d in [(16, 0.5, 1.0), (3, 0.5, 1.0), (6, 0.8, 0.4), (1, 0.5, 1.0)]:
        h = 0.5
        for _ in range(it):
            h = max(h * (1.0 - 2.0 * lam / 3.0), 0.5 - d / (2.0 * np.sqrt(3.0)))
        off, pts = oracle.smooth(m, iterations=it, relaxation=lam, constraint=d, sphere=True)
        np.testing.assert_allclose(np.abs(pts - 1.0), h, rtol=0, atol=1e-14)
        assert np.all(np.sqrt((off ** 2).sum(axis=1)) <= 0.5 * d + 1e-15)


@pytest.mark.parametrize("seed", range(3))
def test_sphere_smoothing_matches_dense_jacobi(seed):
    lab, m = _small_mesh(seed)
    for it, lam, d in [(16, 0.5, 1.0), (7, 0.9, 0.6)]:
        _, pts = oracle.smooth(m, (1.5, 1.5, 1.5), (2.0, -1.0, 0.5), it, lam, d, sphere=True)
        ref = brute.dense_jacobi_world(m.cells, m.quads, (1.5, 1.5, 1.5), (2.0, -1.0, 0.5), it, lam, d, sphere=True)
        np.testing.assert_allclose(pts, ref, rtol=0, atol=1e-11)


# ---------------------------------------------------------------- triangulation
def _quad_points(lift):
    # unit square in z = 0 with vertex `lift` raised to z = 1 (a folded quad)
    p = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0]], dtype=np.float32)
    p[lift, 2] = 1.0
    return p, np.array([[0, 1, 2, 3]], dtype=np.int32)


def test_triangulation_choices_on_folded_quads():
    # lifting v2 (or v0) lengthens diagonal v0-v2 (sqrt 3 vs sqrt 2); the split
    # along v1-v3 then has twice-area 1 + sqrt(3) = 2.732 < 2 sqrt(2) = 2.828 for
    # v0-v2, and normals at cosine 1/sqrt(3) = 0.577 > 1/2: every criterion picks
    # v1-v3.  Lifting v1 or v3 mirrors the quad and every criterion picks v0-v2.
    for lift, want_alt in [(2, True), (3, False), (0, True), (1, False)]:
        pts, quads = _quad_points(lift)
        for method in ("shortest", "min_area", "coplanar"):
            tris, alt, metric = oracle.triangulate(pts, quads, method)
            assert bool(alt[0]) == want_alt, (lift, method)
        tris, alt, _ = oracle.triangulate(pts, quads, "greedy")
        assert not alt[0] and tris.tolist() == [[0, 1, 2], [0, 2, 3]]
    pts, quads = _quad_points(2)
    _, _, metric = oracle.triangulate(pts, quads, "min_area")
    np.testing.assert_allclose(metric[0], [2.0 * np.sqrt(2.0), 1.0 + np.sqrt(3.0)], rtol=1e-6)
    _, _, metric = oracle.triangulate(pts, quads, "coplanar")
    np.testing.assert_allclose(metric[0], [0.5, 1 / np.sqrt(3.0)], rtol=1e-6)
    tris, _, _ = oracle.triangulate(pts, quads, "shortest")
    assert tris.tolist() == [[0, 1, 3], [1, 2, 3]]


@pytest.mark.parametrize("method", ["greedy", "shortest", "min_area", "coplanar"])
def test_triangulation_invariants(method):
    lab, m = _small_mesh(11, (7, 8, 9), 4)
    _, pts = oracle.smooth(m, iterations=8, relaxation=0.5, constraint=1.0)
    tris, alt, _ = oracle.triangulate(pts.astype(np.float32), m.quads, method)
    assert tris.shape == (2 * m.n_quads, 3)
    for q in range(m.n_quads):
        v = [int(x) for x in m.quads[q]]
        t0, t1 = [int(x) for x in tris[2 * q]], [int(x) for x in tris[2 * q + 1]]
        assert set(t0) | set(t1) == set(v)
        diag = set(t0) & set(t1)
        assert diag == ({v[1], v[3]} if alt[q] else {v[0], v[2]})
        # each triangle keeps the quad's cyclic order (hence its winding)
        for t in (t0, t1):
            k = [v.index(x) for x in t]
            assert k in ([0, 1, 2], [0, 2, 3], [0, 1, 3], [1, 2, 3])
    # on the unsmoothed mesh every triangle normal points along the quad's axis
    c = oracle.triangulate(m.points.astype(np.float32), m.quads, method)[0]
    p = m.points[c]
    n = np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0])
    axis_of = np.argmax(np.abs(n), axis=1)
    assert np.all(n[np.arange(len(n)), axis_of] > 0)
