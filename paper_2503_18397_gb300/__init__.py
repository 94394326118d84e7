"""GB300-native epsilon-cost-sharded static functions (VFunc) and filters (VFilter).

Thin Python binding of the C ABI in ``include/vfunc.h`` (``libvfunc.so``):
argument marshalling only; every step runs in the CUDA kernels of the library.
PyTorch provides device memory and streams.
"""
from ._binding import (  # noqa: F401
    FILTER,
    FUNC,
    KEYS_BYTES,
    KEYS_U64,
    MODE_AUTO,
    MODE_FUSE,
    MODE_LGE,
    REGIME_FUSE,
    REGIME_LGE,
    SOLVER_FLOW,
    SOLVER_ROUNDS,
    VFError,
    VfInfo,
    VfParams,
    Structure,
    lib,
    lib_path,
    VfBatchItem,
    VfBatchOpts,
    vf_batch_opts_default,
    vf_build,
    vf_build_batch,
    vf_tune_batch,
    vf_build_static,
    vf_export,
    vf_free,
    vf_get_info,
    vf_params_default,
    vf_plan,
    vf_query,
    vf_query_batch,
    VfQueryReq,
    vf_signatures,
    vf_timing_enable,
    vf_timing_read,
    PHASES,
)
