"""GB300 (sm_103a) spherical harmonic transforms after arXiv:1106.0159.

``Plan`` (in ``sht``) wraps the C ABI of ``include/sht.h``; the CUDA library
is built in-tree by ``_build.build()`` and loaded on first use.
"""
from .sht import (GRID_CUSTOM, GRID_GAUSS_LEGENDRE, GRID_HEALPIX, Plan, ShtError, alm_index,  # noqa: F401
                  gauss_legendre_geometry, healpix_geometry, nalm)
