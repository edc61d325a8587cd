"""GB300 (sm_103a) SurfaceNets: shared quad-mesh extraction from label maps and
constrained smoothing (arXiv 2401.14906), as hand-written CUDA kernels behind a
C ABI (include/sn.h).  ``sn`` is the Python binding; ``build`` compiles libsn.so.
"""
from . import sn  # noqa: F401
from .sn import (Mesh, SNError, sn_extract, sn_mesh_copy_to_host, sn_mesh_counts,  # noqa: F401
                 sn_mesh_device_arrays, sn_smooth)
