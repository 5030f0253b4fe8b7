"""GB300 (sm_103a) Canonical Variates Analysis for multispectral manuscript
images (arXiv 1612.06457): CUDA fit (exact class moments on the tensor cores,
double-float eigensolve on one CTA) and fused projection + 8-bit rescale, with
the FP64 form, the batched form for many pages, the third rescale, 16-bit
images, principal components, Section 3's indices and the colour composite,
behind a C ABI (``include/cva.h``) with a thin ctypes binding.
"""
from ._build import build as _build_lib
from ._lib import *  # noqa: F401,F403
from ._lib import Model, CvaError, load, library_path, SIGNATURES  # noqa: F401


def build(force: bool = False) -> str:
    """Compile the CUDA library for sm_103a and return its path."""
    return _build_lib(force=force)
