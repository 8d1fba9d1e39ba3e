"""librearr: GB300 (sm_103a) kernels for the data-rearrangement operations of
arXiv:1011.3583 (permute, reorder by an index sequence, interlace and
de-interlace, and the generic 2-D stencil), behind a C ABI
(include/librearr*.h) with this thin binding."""
from .librearr import (  # noqa: F401
    EINVAL, Arena, OpSpec, Server, batch_noalloc, tuning_load,
    MAX_K, MAX_RANK, Plan, PermuteInfo, RearrError, deinterlace, describe_permute, interlace, launch_count,
    lib_path, load, memcpy_d2d, permute, reorder, reorder64, reorder_nm, scatter, scatter64, selftest_host,
    status_str, STENCIL_CLAMP, STENCIL_ZERO, describe_stencil, stencil2d, wait_timeouts, inject_wait_timeout,
    Pipeline, check_indices, reorder_checked, ERANGE,
    DistPlan, dist_permute_plan, dist_permute_pack, dist_permute_unpack, describe_reorder_nm,
    describe_reorder,
)
from .dist import dist_permute  # noqa: F401
