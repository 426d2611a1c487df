"""GB300-native warm-started stochastic reconfiguration (WSSR) step.

The compute lives in libwssr.so (hand-written CUDA for sm_103a, C ABI in
include/wssr.h); ``paper_2512_05749_gb300.wssr`` is its thin ctypes binding.
"""
from .wssr import (  # noqa: F401
    WSSR, WSSRError, load, make_operator, status_string, wssr_apply_O, wssr_apply_Ot,
    wssr_create, wssr_default_options, wssr_destroy, wssr_get_status, wssr_init_subspace,
    wssr_last_launch_count, wssr_get_stats, wssr_orthonormalize, wssr_profile_begin, wssr_profile_end, wssr_step, wssr_sync, wssr_woodbury,
)
