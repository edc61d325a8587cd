"""Seeded synthetic label maps shared by the tests, the benchmark and the oracle runs.

This module only paints label values; it holds none of the surface-extraction or
smoothing arithmetic.  The native part (``sn_synth.c``) is compiled on first use
with gcc (``-ffp-contract=off`` so that maps are bit-identical on x86-64 and
aarch64).  Arrays are numpy arrays of shape ``(nz, ny, nx)`` in C order, i.e. x is
the fastest-varying index, as in the paper's data layout (Sec. 2.1).

Workload recipes (stand-ins for the paper's datasets of Sec. 4.1, which are not
available here):

* ``config1``  64^3 uint16, 4 random ellipsoids (radii 6-20, later labels overwrite
  earlier), background 0, seed 1.
* ``config2``  512^3 uint16 atlas-like map (Torso stand-in, 93 labels): Voronoi
  partition of 93 seeds inside a noise-perturbed ellipsoid blob occupying 40% of
  the volume, rest background 0, seed 2.
* ``config3``  1024x1024x512 uint32 connectomics-like map (connectome stand-in):
  50,000 Voronoi cells with sample spacing (1,1,4) and 5% background gaps along
  cell faces, seed 3.
* ``config3_slab``  1024x1024x64 uint32 with the connectome's cell density (for
  profiler captures of the same kernels at a few GB of device memory).
* ``config5_maps``  256 maps of uneven sizes (edges 32-256), uint8/uint16, 1-20
  ellipsoid or Voronoi labels, seeds 5000-5255.
* ``config4_train_map``  256^3 uint16 training maps (alternating Voronoi with
  20-93 seeds and 1-20 ellipsoids), seeds 1000-1199.
* ``paper_synthetic``  512^3 uint16, 128 overlapping spheres (the paper's
  "Synthetic" dataset description).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sn_synth.c")
_LIBDIR = os.path.join(_HERE, "lib")
_LIB = os.path.join(_LIBDIR, "libsn_synth.so")
_lock = threading.Lock()
_lib = None

_TYPE = {np.dtype(np.uint8): 1, np.dtype(np.uint16): 2, np.dtype(np.uint32): 4}


def build(force: bool = False) -> str:
    """Compile libsn_synth.so next to this file (no-op when up to date)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp.%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-o", tmp, _SRC, "-lpthread", "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, u64, u32, dbl, vp = (ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32,
                                      ctypes.c_double, ctypes.c_void_p)
            lib.sn_synth_ellipsoids.argtypes = [vp, ctypes.c_int, i64, i64, i64, ctypes.c_int, dbl, dbl,
                                                u32, u32, u64]
            lib.sn_synth_spheres.argtypes = lib.sn_synth_ellipsoids.argtypes
            lib.sn_synth_atlas.argtypes = [vp, ctypes.c_int, i64, i64, i64, ctypes.c_int, dbl, dbl, dbl,
                                           dbl, dbl, dbl, ctypes.c_int, u64, ctypes.c_int,
                                           ctypes.POINTER(dbl)]
            lib.sn_synth_voronoi.argtypes = [vp, ctypes.c_int, i64, i64, i64, ctypes.c_int, u32, u64,
                                             ctypes.c_int]
            lib.sn_synth_connectome.argtypes = [vp, i64, i64, i64, ctypes.c_int, i64, dbl, dbl, u64,
                                                ctypes.c_int, ctypes.POINTER(i64)]
            for f in ("sn_synth_ellipsoids", "sn_synth_spheres", "sn_synth_atlas", "sn_synth_voronoi",
                      "sn_synth_connectome"):
                getattr(lib, f).restype = ctypes.c_int
            _lib = lib
    return _lib


def _threads(n):
    return int(n) if n else max(1, min(64, os.cpu_count() or 1))


def _empty(dims, dtype):
    nx, ny, nz = (int(d) for d in dims)
    return np.empty((nz, ny, nx), dtype=np.dtype(dtype))


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"{what} failed with code {rc}")


def ellipsoids(dims, n_labels, rmin, rmax, dtype=np.uint16, seed=1, first_label=1, background=0):
    a = _empty(dims, dtype)
    _check(_load().sn_synth_ellipsoids(a.ctypes.data, _TYPE[a.dtype], dims[0], dims[1], dims[2],
                                       int(n_labels), float(rmin), float(rmax), int(first_label),
                                       int(background), int(seed)), "sn_synth_ellipsoids")
    return a


def spheres(dims, n_spheres, rmin, rmax, dtype=np.uint16, seed=1, first_label=1, background=0):
    a = _empty(dims, dtype)
    _check(_load().sn_synth_spheres(a.ctypes.data, _TYPE[a.dtype], dims[0], dims[1], dims[2],
                                    int(n_spheres), float(rmin), float(rmax), int(first_label),
                                    int(background), int(seed)), "sn_synth_spheres")
    return a


def atlas(dims, n_seeds=93, occupancy=0.40, tol=0.005, semi=(0.45, 0.40, 0.38), amp=0.15, lattice=8,
          dtype=np.uint16, seed=2, threads=None):
    a = _empty(dims, dtype)
    t = ctypes.c_double(0.0)
    _check(_load().sn_synth_atlas(a.ctypes.data, _TYPE[a.dtype], dims[0], dims[1], dims[2], int(n_seeds),
                                  float(occupancy), float(tol), float(semi[0]), float(semi[1]),
                                  float(semi[2]), float(amp), int(lattice), int(seed), _threads(threads),
                                  ctypes.byref(t)), "sn_synth_atlas")
    return a


def voronoi(dims, n_seeds, dtype=np.uint16, seed=1, first_label=1, threads=None):
    a = _empty(dims, dtype)
    _check(_load().sn_synth_voronoi(a.ctypes.data, _TYPE[a.dtype], dims[0], dims[1], dims[2], int(n_seeds),
                                    int(first_label), int(seed), _threads(threads)), "sn_synth_voronoi")
    return a


def connectome(dims, n_seeds=50000, zscale=4, gap=0.05, tol=0.0025, seed=3, threads=None):
    a = _empty(dims, np.uint32)
    tau = ctypes.c_int64(0)
    _check(_load().sn_synth_connectome(a.ctypes.data, dims[0], dims[1], dims[2], int(n_seeds), int(zscale),
                                       float(gap), float(tol), int(seed), _threads(threads),
                                       ctypes.byref(tau)), "sn_synth_connectome")
    return a


# ----------------------------------------------------------------- workloads
class Workload:
    """One synthetic workload: the label map plus the extraction/smoothing parameters."""

    def __init__(self, name, labels, spacing=(1.0, 1.0, 1.0), origin=(0.0, 0.0, 0.0), iterations=16,
                 relaxation=0.5, constraint=1.0, selected=None, background=0):
        self.name = name
        self.labels = labels
        self.spacing = tuple(float(s) for s in spacing)
        self.origin = tuple(float(o) for o in origin)
        self.iterations = int(iterations)
        self.relaxation = float(relaxation)
        self.constraint = float(constraint)
        self.selected = selected
        self.background = int(background)

    @property
    def dims(self):
        nz, ny, nx = self.labels.shape
        return (nx, ny, nz)

    @property
    def voxels(self):
        return int(self.labels.size)


def config1():
    """64^3 uint16, 4 ellipsoids, all labels, 16 iterations, relaxation 0.5, constraint 1."""
    return Workload("c1_64cube_u16_4ellipsoids", ellipsoids((64, 64, 64), 4, 6.0, 20.0, np.uint16, seed=1))


def config2(dims=(512, 512, 512)):
    """512^3 uint16 atlas-like map, 93 Voronoi labels in a 40% blob, 16 iterations."""
    return Workload("c2_512cube_u16_atlas93", atlas(dims, 93, seed=2))


def config3(dims=(1024, 1024, 512), n_seeds=50000):
    """1024x1024x512 uint32 connectomics-like map, 50k cells, spacing (1,1,4), 8 iterations."""
    return Workload("c3_1024x1024x512_u32_connectome", connectome(dims, n_seeds, 4, seed=3),
                    spacing=(1.0, 1.0, 4.0), iterations=8)


def config3_slab(nz=64):
    """A slab of the connectomics-like map's shape: 1024x1024xnz uint32 with the same cell density
    (50,000 * nz / 512 cells), spacing (1,1,4), 8 iterations -- small enough for a profiler capture."""
    return Workload("c3slab_1024x1024x%d_u32_connectome" % nz,
                    connectome((1024, 1024, nz), max(1, 50000 * nz // 512), 4, seed=3),
                    spacing=(1.0, 1.0, 4.0), iterations=8)


def paper_synthetic(dims=(512, 512, 512), n_spheres=128, seed=7):
    """The paper's Synthetic dataset shape: 512^3 uint16 with 128 overlapping spheres."""
    r = min(dims) / 512.0
    return Workload("paper_synthetic_512cube_u16_128spheres",
                    spheres(dims, n_spheres, 20.0 * r, 60.0 * r, np.uint16, seed=seed))


class _SplitMix:
    """splitmix64 in pure Python, used to draw per-map parameters."""

    def __init__(self, seed):
        self.s = int(seed) & 0xFFFFFFFFFFFFFFFF

    def next(self):
        self.s = (self.s + 0x9E3779B97F4A7C15) & 0xFFFFFFFFFFFFFFFF
        z = self.s
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & 0xFFFFFFFFFFFFFFFF
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & 0xFFFFFFFFFFFFFFFF
        return z ^ (z >> 31)

    def below(self, n):
        return (self.next() * n) >> 64


def config5_params(index):
    """Parameters of batched map `index` (0..255): dims, dtype, kind, n_labels, seed."""
    seed = 5000 + int(index)
    r = _SplitMix(seed)
    dims = tuple(32 + r.below(225) for _ in range(3))
    dtype = np.uint8 if r.below(2) == 0 else np.uint16
    kind = "ellipsoids" if r.below(2) == 0 else "voronoi"
    n_labels = 1 + r.below(20)
    return dims, dtype, kind, n_labels, seed


def config5_map(index):
    dims, dtype, kind, n, seed = config5_params(index)
    if kind == "ellipsoids":
        m = min(dims)
        lab = ellipsoids(dims, n, 0.08 * m, 0.30 * m, dtype, seed=seed)
    else:
        lab = voronoi(dims, n, dtype, seed=seed)
    return Workload(f"c5_map{index}_{kind}", lab)


def config5_maps(count=256):
    return [config5_map(i) for i in range(count)]


def config4_train_map(index, dims=(256, 256, 256)):
    """Training map `index` (0..199): even indices Voronoi (20-93 seeds), odd ellipsoids (1-20)."""
    seed = 1000 + int(index)
    r = _SplitMix(seed)
    if index % 2 == 0:
        lab = voronoi(dims, 20 + r.below(74), np.uint16, seed=seed)
    else:
        m = min(dims)
        lab = ellipsoids(dims, 1 + r.below(20), 0.08 * m, 0.30 * m, np.uint16, seed=seed)
    return Workload(f"c4_train{index}", lab)


def map_sha256(a):
    import hashlib
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()
