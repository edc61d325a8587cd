"""z-slab decomposition of one label map over several ranks (one GPU each).

The paper leaves the regions open at the volume faces so that sub-volumes can
be processed separately and their meshes stitched (Sec. 4.2, Sec. 5).  Here
rank r owns

* the quads of the sample slices k in [k0, k1) (quads are ordered by their
  first sample, Sec. 2.3), and
* the points of the cell slices cz in [k0 - 1, k1 - 1) (the last rank also
  cz = nz - 1), since points are ordered by (cz, cy, cx).

Each rank extracts and smooths the sample slices [s0, s1) = [k0 - 1 - g,
k1 + g) (clipped to the volume) with g = iterations + 2 ghost slices on each
side.  A point's stencil reaches one cell slice up and down, so information
moves one cell slice per Jacobi sweep.  The cells at a cut face are wrong (they
see an open boundary that is not there), and their error moves inward by one
slice per sweep.  After n sweeps the owned cells are still n + 1 slices away
from any such error, so their offsets match the whole-volume run exactly.

The only exchange is an exclusive scan over the ranks of the owned (points,
quads, stencil entries): an allgather of three integers per rank.  Local
point ids then map to global canonical ids as follows:
* the owned slices keep their order;
* the halo cell slice below the owned range is the end of the previous rank's
  range;
* the halo cell slice above it is the start of the next rank's range.

A rank needs no data from its neighbours; the ghost slices are recomputed.
Since both halo slices sit right next to the owned run in the canonical order,
the whole id remap is one shift per rank (global = local - first owned local +
first global), which sn_slab_stitch applies on the device (the `device_*`
functions); `own`/`stitch` are the same steps on host arrays.
"""
from __future__ import annotations

import numpy as np


def slab_plan(nz: int, world: int, iterations: int):
    """Per rank: owned sample slices [k0, k1), owned cell slices [c0, c1), extracted sample slices [s0, s1)."""
    if world < 1 or nz < world:
        raise ValueError("need 1 <= world <= nz")
    g = int(iterations) + 2
    bounds = [nz * r // world for r in range(world + 1)]
    plan = []
    for r in range(world):
        k0, k1 = bounds[r], bounds[r + 1]
        c0 = k0 - 1
        c1 = k1 - 1 if r < world - 1 else nz
        plan.append({"rank": r, "k0": k0, "k1": k1, "c0": c0, "c1": c1,
                     "s0": max(0, k0 - 1 - g), "s1": min(nz, k1 + g)})
    return plan


def _slice_starts(cz, lo, hi):
    """First local id of each cell slice in [lo, hi] (ids are sorted by cz); entry hi + 1 - lo = end."""
    return np.searchsorted(cz, np.arange(lo, hi + 2), side="left")


def own(local, p):
    """The rank's owned part of a local slab mesh, with local ids (before the exchange).

    `local`: dict of host arrays from one slab -- points (n,3), offsets (n,3),
    cells (n,3) global (cx, cy, cz), quads (q,4), quad_labels (q,2),
    stencil_offsets (n+1,), stencil_ids (s,)."""
    cz = local["cells"][:, 2]
    st = _slice_starts(cz, p["c0"] - 1, p["c1"])      # slices c0-1 .. c1 (halos included)
    a, b = st[1], st[-2]                                # owned points [a, b)
    q = local["quads"]
    # a quad's first sample slice is the largest cz among its four cells
    qk = cz[q].max(axis=1) if q.size else np.zeros(0, np.int64)
    qa, qb = np.searchsorted(qk, p["k0"], "left"), np.searchsorted(qk, p["k1"], "left")
    so = local["stencil_offsets"]
    return {"a": int(a), "b": int(b), "qa": int(qa), "qb": int(qb),
            "below": int(st[1] - st[0]),                # points of the halo slice c0 - 1 in the slab
            "above_start": int(st[-2]),                 # first local id of the halo slice c1
            "n_points": int(b - a), "n_quads": int(qb - qa), "n_stencil": int(so[b] - so[a])}


def stitch(local, p, o, offsets_all):
    """Owned arrays with global ids.  `offsets_all[r]` = exclusive prefix of (points, quads, stencil) over ranks."""
    off_p, off_q, off_s = (int(v) for v in offsets_all[p["rank"]])
    a, b, qa, qb = o["a"], o["b"], o["qa"], o["qb"]

    def gid(ids):
        ids = np.asarray(ids, dtype=np.int64)
        out = ids - a + off_p                           # owned slices and the slice above keep their order
        below = ids < a                                 # the previous rank's last slice ends at off_p
        out[below] = off_p - (a - ids[below])
        return out

    so = local["stencil_offsets"]
    sids = local["stencil_ids"][so[a]:so[b]]
    return {
        "points": local["points"][a:b],
        "offsets": local["offsets"][a:b],
        "cells": local["cells"][a:b],
        "quads": gid(local["quads"][qa:qb]).astype(np.int32),
        "quad_labels": local["quad_labels"][qa:qb],
        "stencil_offsets": (so[a:b] - so[a] + off_s).astype(np.int64),
        "stencil_ids": gid(sids).astype(np.int32),
        "first_point": off_p, "first_quad": off_q, "first_stencil": off_s,
    }


def exclusive_offsets(counts_all):
    """(world, 3) owned counts -> (world, 3) exclusive prefix and the (3,) totals."""
    c = np.asarray(counts_all, dtype=np.int64).reshape(-1, 3)
    ex = np.zeros_like(c)
    ex[1:] = np.cumsum(c, axis=0)[:-1]
    return ex, c.sum(axis=0)


def run_rank(labels, spacing, origin, iterations, relaxation, constraint, rank, world, extract, allgather):
    """One rank's share of extract + smooth: its owned mesh part with global ids.

    `extract(sub_labels, spacing, sub_origin, z0, iterations, relaxation, constraint)` returns the
    local dict described in `own` with cells already in global coordinates (z0 = first sample
    slice of the slab); `allgather(np.int64[3]) -> np.int64[world, 3]` is the exchange."""
    p = slab_plan(labels.shape[0], world, iterations)[rank]
    s0, s1 = p["s0"], p["s1"]
    sub_origin = (origin[0], origin[1], origin[2] + s0 * spacing[2])
    local = extract(labels[s0:s1], spacing, sub_origin, s0, iterations, relaxation, constraint)
    o = own(local, p)
    counts_all = allgather(np.array([o["n_points"], o["n_quads"], o["n_stencil"]], dtype=np.int64))
    ex, totals = exclusive_offsets(counts_all)
    part = stitch(local, p, o, ex)
    part["totals"] = totals
    return part


def gpu_extract(sub_labels, spacing, sub_origin, z0, iterations, relaxation, constraint):
    """The per-rank extractor of the library: sn_extract + sn_smooth on this rank's GPU."""
    from . import sn
    m = sn.sn_extract(sub_labels, spacing, sub_origin)
    if iterations:
        sn.sn_smooth(m, iterations, relaxation, constraint)
    host = sn.sn_mesh_copy_to_host(m)
    cells = sn.sn_mesh_cells(m).cpu().numpy()
    cells[:, 2] += z0
    host["cells"] = cells
    m.free()
    return host


def torch_allgather(vec):
    """allgather of an int64[3] over the default torch.distributed group (NCCL or gloo)."""
    import torch
    import torch.distributed as dist
    backend = dist.get_backend()
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    t = torch.as_tensor(vec, dtype=torch.int64, device=dev)
    out = [torch.empty_like(t) for _ in range(dist.get_world_size())]
    dist.all_gather(out, t)
    return np.stack([x.cpu().numpy() for x in out])


# ------------------------------------------------------- device-resident path
def device_part(sub_labels, spacing, sub_origin, p, iterations, relaxation, constraint, stream=None):
    """Extract and smooth one rank's slab on its GPU and find its owned ranges (sn_slab_part_of).
    Returns (mesh, part); the mesh stays on the device."""
    from . import sn
    s0 = p["s0"]
    m = sn.sn_extract(sub_labels, spacing, sub_origin, stream=stream)
    if iterations:
        sn.sn_smooth(m, iterations, relaxation, constraint)
    part = sn.sn_slab_part_of(m, p["c0"] - s0, p["c1"] - s0, p["k0"] - s0, p["k1"] - s0)
    return m, part


def device_stitch(m, part, first, z0, stream=None):
    """The owned part of a slab mesh with global ids, as device tensors (sn_slab_stitch for the ids; the
    other arrays are copies of contiguous ranges of the mesh).  `first` = (first global point, first
    global quad, first global stencil entry) of this rank."""
    import torch

    from . import sn
    quads, so, si = sn.sn_slab_stitch(m, part, first[0], first[2], stream=stream)
    arr = sn.sn_mesh_device_arrays(m)
    a, b = part.first_point, part.first_point + part.n_points
    qa, qb = part.first_quad, part.first_quad + part.n_quads
    cells = sn.sn_mesh_cells(m)[a:b].clone()
    cells[:, 2] += z0
    lab = arr["quad_labels"]
    lab = lab.view({1: torch.uint8, 2: torch.int16, 4: torch.int32}[lab.element_size()])  # raw label bits
    return {"points": arr["points"][a:b].clone(), "offsets": arr["offsets"][a:b].clone(), "cells": cells,
            "quads": quads, "quad_labels": lab[qa:qb].clone(), "stencil_offsets": so,
            "stencil_ids": si, "first_point": int(first[0]), "first_quad": int(first[1]),
            "first_stencil": int(first[2])}


def device_assemble(parts, totals):
    """The global mesh (device tensors) from the ranks' device parts in rank order (one GPU)."""
    import torch
    out = {k: torch.cat([p[k] for p in parts]) for k in
           ("points", "offsets", "cells", "quads", "quad_labels", "stencil_ids")}
    out["stencil_offsets"] = torch.cat([p["stencil_offsets"] for p in parts] +
                                       [torch.tensor([int(totals[2])], dtype=torch.int64, device="cuda")])
    return out


def run_rank_device(labels_dev, spacing, origin, iterations, relaxation, constraint, rank, world, nz,
                    allgather, stream=None):
    """One rank's share on its GPU with the slab labels already on the device: extract, smooth, count
    exchange (`allgather`), stitch.  `labels_dev` holds sample slices [s0, s1) of the plan.  Returns the
    owned part (device tensors) and the totals."""
    p = slab_plan(nz, world, iterations)[rank]
    sub_origin = (origin[0], origin[1], origin[2] + p["s0"] * spacing[2])
    m, part = device_part(labels_dev, spacing, sub_origin, p, iterations, relaxation, constraint, stream)
    counts_all = allgather(np.array([part.n_points, part.n_quads, part.n_stencil], dtype=np.int64))
    ex, totals = exclusive_offsets(counts_all)
    out = device_stitch(m, part, ex[rank], p["s0"], stream)
    m.free()
    return out, totals


def emulate_device(labels, spacing, origin, iterations, relaxation, constraint, world):
    """All ranks in one process on one GPU through the device path; returns the global mesh as host
    arrays."""
    nz = labels.shape[0]
    plan = slab_plan(nz, world, iterations)
    meshes = []
    for p in plan:
        sub_origin = (origin[0], origin[1], origin[2] + p["s0"] * spacing[2])
        meshes.append(device_part(np.ascontiguousarray(labels[p["s0"]:p["s1"]]), spacing, sub_origin, p,
                                  iterations, relaxation, constraint))
    counts = np.array([[pt.n_points, pt.n_quads, pt.n_stencil] for _, pt in meshes], dtype=np.int64)
    ex, totals = exclusive_offsets(counts)
    parts = [device_stitch(m, pt, ex[r], plan[r]["s0"]) for r, (m, pt) in enumerate(meshes)]
    for m, _ in meshes:
        m.free()
    out = device_assemble(parts, totals)
    host = {k: v.cpu().numpy() for k, v in out.items()}
    ldt = {1: np.uint8, 2: np.uint16, 4: np.uint32}[labels.dtype.itemsize]
    host["quad_labels"] = host["quad_labels"].view(ldt)
    return host


def assemble(parts):
    """The global mesh from the ranks' parts (in rank order)."""
    tot = parts[0]["totals"]
    so = np.concatenate([p["stencil_offsets"] for p in parts] + [np.array([tot[2]], dtype=np.int64)])
    out = {k: np.concatenate([p[k] for p in parts]) for k in
           ("points", "offsets", "cells", "quads", "quad_labels", "stencil_ids")}
    out["stencil_offsets"] = so
    return out


def emulate(labels, spacing, origin, iterations, relaxation, constraint, world, extract=gpu_extract):
    """All ranks of the decomposition in one process (the allgather becomes a list); returns the global mesh."""
    nz = labels.shape[0]
    plan = slab_plan(nz, world, iterations)
    locs, owns = [], []
    for p in plan:
        s0, s1 = p["s0"], p["s1"]
        sub_origin = (origin[0], origin[1], origin[2] + s0 * spacing[2])
        loc = extract(labels[s0:s1], spacing, sub_origin, s0, iterations, relaxation, constraint)
        locs.append(loc)
        owns.append(own(loc, p))
    counts = np.array([[o["n_points"], o["n_quads"], o["n_stencil"]] for o in owns], dtype=np.int64)
    ex, totals = exclusive_offsets(counts)
    parts = []
    for p, loc, o in zip(plan, locs, owns):
        part = stitch(loc, p, o, ex)
        part["totals"] = totals
        parts.append(part)
    return assemble(parts)
