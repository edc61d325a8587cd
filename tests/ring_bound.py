"""Lower bound on the error of any smoothing proposal that sees only an r-ring.

After n Jacobi sweeps of Eq. 1 (Sec. 2.2, 2.4) from zero offsets, a point's
offset is a function of its n-ring: every sweep mixes in one more ring of face
neighbours, and the update of a point depends only on which faces of its cell
have neighbours (the unit steps, the stencil size) and on the neighbours'
offsets.  A predictor that reads less -- the r-ring view of a point, r < n --
must give the same answer to two points whose r-ring views are the same, so
within each class of points with equal views its largest error is at least half
the spread of their true offsets.  The largest such half-spread over all
classes is therefore a lower bound on the max-norm error of ANY predictor that
is a function of the r-ring view, however it is trained.

The r-ring view is computed by colour refinement over the face-labelled
stencil graph: colour_0 = the face mask; colour_{k+1} = a 64-bit hash of
(colour_k of the point, colour_k of its -x, +x, -y, +y, -z, +z neighbour or a
mark for an absent face).  Equal colour_r means equal r-ring views up to hash
collisions (which can only merge classes, i.e. make the bound larger; with 64
bits and a few million points none is expected).

Run as a script on the 512^3 atlas-like map to print the table for r = 0..n:
    python tests/ring_bound.py [--dims 512] [--iterations 16]
The oracle supplies the mesh and the FP64 offsets.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

_M1, _M2 = np.uint64(0xBF58476D1CE4E5B9), np.uint64(0x94D049BB133111EB)


def _mix(z):
    """splitmix64 finaliser on a uint64 array."""
    with np.errstate(over="ignore"):
        z = z + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def face_neighbours(stencil_offsets, stencil_ids, face_masks):
    """(n, 6) int64 neighbour id per face -x,+x,-y,+y,-z,+z, -1 where the face has none."""
    n = face_masks.shape[0]
    nb = np.full((n, 6), -1, dtype=np.int64)
    fm = face_masks.astype(np.int64)
    start = stencil_offsets[:-1].astype(np.int64)
    rank = np.zeros(n, dtype=np.int64)  # entries of lower faces already passed
    for f in range(6):
        has = ((fm >> f) & 1).astype(bool)
        nb[has, f] = stencil_ids[start[has] + rank[has]]
        rank += has
    return nb


def refine(colours, nb):
    """One refinement step: hash of the own colour and the six neighbour colours in face order."""
    h = _mix(colours)
    absent = np.uint64(0x5DEECE66D)
    with np.errstate(over="ignore"):
        for f in range(6):
            c = np.where(nb[:, f] >= 0, colours[np.maximum(nb[:, f], 0)], absent)
            h = _mix(h ^ (c + np.uint64(f + 1) * np.uint64(0x9E3779B97F4A7C15)))
    return h


def class_half_spread(colours, target):
    """Largest half-spread of `target` (n, 3) over the classes of equal colour, max over axes; and the
    number of classes."""
    _, inv = np.unique(colours, return_inverse=True)
    k = int(inv.max()) + 1 if inv.size else 0
    worst = 0.0
    for a in range(target.shape[1]):
        lo = np.full(k, np.inf)
        hi = np.full(k, -np.inf)
        np.minimum.at(lo, inv, target[:, a])
        np.maximum.at(hi, inv, target[:, a])
        worst = max(worst, float(((hi - lo) * 0.5).max()) if k else 0.0)
    return worst, k


def ring_bounds(mesh, target, r_max):
    """[(r, lower bound, classes)] for r = 0..r_max."""
    nb = face_neighbours(mesh.stencil_offsets, mesh.stencil_ids, mesh.face_masks)
    colours = _mix(mesh.face_masks.astype(np.uint64))
    out = []
    for r in range(r_max + 1):
        lb, k = class_half_spread(colours, target)
        out.append((r, lb, k))
        if r < r_max:
            colours = refine(colours, nb)
    return out


def main():
    import oracle
    import sn_synth
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--dims", type=int, default=512)
    ap.add_argument("--iterations", type=int, default=16)
    a = ap.parse_args()
    w = sn_synth.config2((a.dims,) * 3)
    mesh = oracle.extract(w.labels, w.spacing, w.origin)
    off, _ = oracle.smooth(mesh, w.spacing, w.origin, a.iterations, w.relaxation, w.constraint)
    rows = ring_bounds(mesh, off, a.iterations)
    print(json.dumps({"map": w.name, "dims": a.dims, "points": mesh.n_points, "iterations": a.iterations,
                      "rows": [{"r": r, "lower_bound_vox": lb, "classes": k} for r, lb, k in rows]}))


if __name__ == "__main__":
    main()
