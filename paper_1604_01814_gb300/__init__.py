"""GB300 lattice-Green's-function library (Liska & Colonius, arXiv:1604.01814).

The LGF Poisson apply u = dx^2 G_L * f, the K(alpha)^{-1} apply
u = dx^2 G_K(alpha) * f and the viscous integrating factor u = E(alpha) f on
the active blocks of a block-structured lattice, computed by
hand-written CUDA kernels for sm_103a behind the C ABI of include/lgf.h.  This
package is the thin Python binding of that ABI (see _binding.py); importing it
loads liblgf.so and raises if the library has not been built.
"""
from ._binding import (EXPORTS, LGF_F32, LGF_F64, LGF_TUNE_CACHED, LGF_TUNE_OFF, LGF_TUNE_ON, lgf_autotune,
                       lgf_tune_report, LGF_OP_INTFACTOR, LGF_OP_KINV, LGF_OP_POISSON,  # noqa: F401
                       LGF_OP_POISSON_THEN_INTFACTOR, LIB_PATH, Context, LgfError, lgf_batch_apply,
                       lgf_cache_limits, lgf_ctx_create, lgf_ctx_destroy, lgf_ctx_stats, lgf_device_status, lgf_wait_selftest, lgf_curl, lgf_curl_adjoint, lgf_intfactor_apply,
                       lgf_intfactor_apply_noalloc, lgf_velocity_refresh, lgf_ib_spread, lgf_ib_interp,
                       lgf_intfactor_weights, lgf_kinv_apply, lgf_nested_projection_stage, lgf_kinv_lookup, lgf_poisson_apply, lgf_poisson_error_estimate, lgf_table_load, lgf_table_save, lgf_profile_enable,
                       lgf_profile_read, lgf_residual, lgf_status_string, lgf_table_build, lgf_table_info,
                       lgf_table_lookup, lgf_version, load)

load()
