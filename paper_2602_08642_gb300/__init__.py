"""GB300-native sub-1-spp adaptive sampling and gather-pyramid reconstruction.

After "Forget Superresolution, Sample Adaptively (when Path Tracing)"
(arXiv 2602.08642).  The compute path is the CUDA library ``_build/libspp.so``
(C ABI in ``include/spp.h``, hand-written sm_103a kernels); this package is
its thin Python binding (``_binding``) and a per-frame buffer driver
(``pipeline``).  Importing the package fails when the library is missing: there is no CPU
fallback.
"""
from . import _binding as binding  # noqa: F401  (raises ImportError if libspp.so is missing)
from ._binding import (  # noqa: F401
    SppError, check, make_params, make_tonemap, spp_abi_version, spp_alloc_sample_map,
    spp_alloc_sample_map_static,
    spp_alloc_workspace_bytes, spp_clear_status, spp_get_status, spp_launch_count,
    spp_reconstruct_frame, spp_reconstruct_level, spp_reconstruct_workspace_bytes,
    spp_warp_previous,
    spp_render_synthetic, spp_splat_samples, spp_strerror)
from .pipeline import Frame, default_capacity, logit_channels  # noqa: F401
from . import autograd  # noqa: F401,E402
