"""GB300-native nested Krylov sign function for the overlap operator.

The compute path is libov (hand-written sm_103a CUDA behind the C-ABI in
include/ov.h); this package is its thin Python binding. See binding.py.
"""
from .binding import (  # noqa: F401
    Overlap,
    OvError,
    ov_apply,
    ov_batch_create,
    ov_batch_sign_apply,
    ov_create,
    ov_deflate,
    ov_get_deflation,
    ov_default_opts,
    ov_get_coefficients,
    ov_mlp_forward,
    ov_mlp_loss_grad,
    ov_mlp_train,
    ov_set_sizer,
    ov_destroy,
    ov_get_stats,
    ov_reset_stats,
    ov_inner_sign,
    ov_rh_sign,
    ov_rh_sign_noalloc,
    ov_set_opts,
    ov_sign_apply,
    ov_solve,
    ov_strerror,
    ov_version,
    ov_wilson_apply,
    make_opts,
    lib,
    LIB_PATH,
)
