"""Independent constructions used to pin the oracle (and, at large sizes, the GPU output).

Nothing here calls the oracle or the CUDA library.  Each function restates what
the paper defines in a different form from the oracle's cell-by-cell loops:

* ``face_quads``: the dual "voxel-face" view -- every pair of face-adjacent
  samples whose classes differ is one quad (Sec. 2.2), whose vertices are the
  four cells containing that sample pair's edge.
* ``vectorised_counts``: quad and point counts with numpy array slicing.
* ``dense_jacobi_world``: Eq. 1 as a dense matrix iteration in world units
  with the box constraint in world units (Sec. 2.2, 2.4).
"""
from __future__ import annotations

import itertools

import numpy as np


def classes(labels, selected=None, background=0):
    """kappa over the whole map: selected values keep their label, others become background."""
    lab = np.asarray(labels)
    if selected is None:
        return lab.astype(np.int64)
    keep = np.isin(lab, np.asarray(selected, dtype=lab.dtype))
    return np.where(keep, lab, background).astype(np.int64)


def face_quads(labels, selected=None, background=0):
    """List of (key, cells, (l0, l1)) for every label-differing face adjacency.

    key = (k, j, i, axis) of the first sample; cells = the 4 cells (cx, cy, cz)
    around the edge, as an unordered frozenset; labels along +axis.
    """
    kap = classes(labels, selected, background)
    nz, ny, nx = kap.shape
    out = []
    for axis in range(3):
        d = [0, 0, 0]
        d[axis] = 1
        for k in range(nz - d[2]):
            for j in range(ny - d[1]):
                for i in range(nx - d[0]):
                    a = kap[k, j, i]
                    b = kap[k + d[2], j + d[1], i + d[0]]
                    if a == b:
                        continue
                    x = (i, j, k)
                    others = [o for o in range(3) if o != axis]
                    cells = set()
                    for s0 in (0, 1):
                        for s1 in (0, 1):
                            c = list(x)
                            c[others[0]] -= s0
                            c[others[1]] -= s1
                            cells.add(tuple(c))
                    out.append(((k, j, i, axis), frozenset(cells), (int(a), int(b))))
    out.sort(key=lambda t: t[0])
    return out


def point_cells(quads):
    """Cells that carry a point = cells used by any quad, in (cz, cy, cx) order."""
    s = set()
    for _, cells, _ in quads:
        s |= cells
    return sorted(s, key=lambda c: (c[2], c[1], c[0]))


def vectorised_counts(labels, selected=None, background=0):
    """(n_quads, n_points) with numpy slicing, independent of any loop code."""
    kap = classes(labels, selected, background)
    cx = kap[:, :, 1:] != kap[:, :, :-1]
    cy = kap[:, 1:, :] != kap[:, :-1, :]
    cz = kap[1:, :, :] != kap[:-1, :, :]
    n_quads = int(cx.sum() + cy.sum() + cz.sum())
    nz, ny, nx = kap.shape
    # cell (c) of the padded grid [-1, N-1]^3 has index c+1; an edge with first
    # sample x touches the cells x - {0,1} along the two other axes
    has = np.zeros((nz + 1, ny + 1, nx + 1), dtype=bool)
    # x-edges: sample (k, j, i) -> cells (i, j-b, k-d): padded index (k+1-d, j+1-b, i+1)
    for b in (0, 1):
        for d in (0, 1):
            has[1 - d:nz + 1 - d, 1 - b:ny + 1 - b, 1:nx] |= cx
            has[1 - d:nz + 1 - d, 1:ny, 1 - b:nx + 1 - b] |= cy
            has[1:nz, 1 - d:ny + 1 - d, 1 - b:nx + 1 - b] |= cz
    return n_quads, int(has.sum())


def quad_edges(quads_ids):
    """Unique undirected quad edges and how many quads use each."""
    cnt = {}
    for q in quads_ids:
        for r in range(4):
            a, b = int(q[r]), int(q[(r + 1) % 4])
            e = (a, b) if a < b else (b, a)
            cnt[e] = cnt.get(e, 0) + 1
    return cnt


def one_ring(n_points, quads_ids):
    nb = [set() for _ in range(n_points)]
    for q in quads_ids:
        for r in range(4):
            a, b = int(q[r]), int(q[(r + 1) % 4])
            nb[a].add(b)
            nb[b].add(a)
    return nb


def dense_jacobi_world(cells, quads_ids, spacing, origin, iterations, relaxation, constraint, sphere=False):
    """Eq. 1 in world units with a dense adjacency matrix built from the quad edges.

    P <- clamp(P + lambda * (D^-1 A P - P)), box = cell centre +- (d/2)*spacing;
    with sphere=True (isotropic spacing only) the displacement from the centre is
    scaled back onto the ball of radius (d/2)*spacing when it leaves it.
    """
    cells = np.asarray(cells, dtype=np.float64)
    n = cells.shape[0]
    sp = np.asarray(spacing, dtype=np.float64)
    centre = np.asarray(origin, dtype=np.float64) + sp * (cells + 0.5)
    A = np.zeros((n, n))
    for q in quads_ids:
        for r in range(4):
            a, b = int(q[r]), int(q[(r + 1) % 4])
            A[a, b] = 1.0
            A[b, a] = 1.0
    deg = A.sum(axis=1)
    P = centre.copy()
    half = 0.5 * constraint * sp
    for _ in range(iterations):
        mean = (A @ P) / deg[:, None]
        P = P + relaxation * (mean - P)
        if sphere:
            disp = P - centre
            r = np.sqrt((disp ** 2).sum(axis=1))
            R = half[0]
            scale = np.where(r > R, R / np.where(r > 0, r, 1.0), 1.0)
            P = centre + disp * scale[:, None]
        else:
            P = np.minimum(np.maximum(P, centre - half), centre + half)
    return P


def all_maps(shape, n_labels):
    """Every map of the given shape over labels 0..n_labels-1."""
    n = int(np.prod(shape))
    for vals in itertools.product(range(n_labels), repeat=n):
        yield np.array(vals, dtype=np.uint8).reshape(shape)
