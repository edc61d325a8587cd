"""Per-rank extractor backed by the oracle, for testing the slab decomposition on the CPU."""
import numpy as np

import oracle


def oracle_extract(sub_labels, spacing, sub_origin, z0, iterations, relaxation, constraint):
    lab = np.ascontiguousarray(sub_labels)
    m = oracle.extract(lab, spacing, sub_origin)
    off, pts = oracle.smooth(m, spacing, sub_origin, iterations, relaxation, constraint)
    cells = m.cells.astype(np.int64).copy()
    cells[:, 2] += z0
    return {"points": pts, "offsets": off, "cells": cells, "quads": m.quads, "quad_labels": m.quad_labels,
            "stencil_offsets": m.stencil_offsets, "stencil_ids": m.stencil_ids}


def oracle_whole(labels, spacing, origin, iterations, relaxation, constraint):
    m = oracle.extract(labels, spacing, origin)
    off, pts = oracle.smooth(m, spacing, origin, iterations, relaxation, constraint)
    return {"points": pts, "offsets": off, "cells": m.cells.astype(np.int64), "quads": m.quads,
            "quad_labels": m.quad_labels, "stencil_offsets": m.stencil_offsets, "stencil_ids": m.stencil_ids}


def assert_same(a, b, float_tol=0.0):
    """Integer arrays exactly; offsets and world points exactly, or within `float_tol` (absolute) where the
    per-rank extractor works in absolute world coordinates (the oracle), whose rounding depends on the
    slab's origin."""
    for k in ("cells", "quads", "quad_labels", "stencil_offsets", "stencil_ids"):
        np.testing.assert_array_equal(np.asarray(a[k]), np.asarray(b[k]), err_msg=k)
    for k in ("offsets", "points"):
        x, y = np.asarray(a[k]), np.asarray(b[k])
        if float_tol == 0.0:
            np.testing.assert_array_equal(x, y, err_msg=k)
        else:
            assert x.shape == y.shape and np.abs(x - y).max(initial=0.0) <= float_tol, k
