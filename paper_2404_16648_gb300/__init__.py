"""GB300-native tree-based dGSEM (arXiv 2404.16648 hot path): CUDA kernels behind a C ABI."""
from .dg import (DG_FP32_PERT, DG_FP64, Batch, DGError, EXPORTED, LIB_PATH, Forest, Mesh, adapt_initial,
                 load_library, make_desc, probe_fma_rate, sphere_geometry, sphere_transfer)

__all__ = ["Mesh", "Forest", "Batch", "DGError", "load_library", "adapt_initial", "LIB_PATH", "EXPORTED",
           "DG_FP64", "DG_FP32_PERT", "make_desc", "probe_fma_rate", "sphere_geometry", "sphere_transfer"]
