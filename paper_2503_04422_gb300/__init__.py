"""GB300-native PDX vector search: PDX layout, PDXearch, PDX-BOND, ADSampling
and BSA pruning as sm_103a CUDA kernels behind a C ABI (include/pdx.h).

``paper_2503_04422_gb300.pdx`` is the Python binding (same function names as
the C ABI); ``paper_2503_04422_gb300.build`` compiles the library in-tree.
"""
from .pdx import (Index, PdxError, pdx_build_layout, pdx_free, pdx_ivf_build, pdx_last_error,  # noqa: F401
                  pdx_search_exact, pdx_search_ivf, search_opts)
