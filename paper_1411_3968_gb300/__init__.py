"""GB300-native online muon trigger for underwater neutrino telescopes
(arXiv 1411.3968): C ABI in include/trig.h (multi-tower selection in
include/trig_array.h), sm_103a kernels in csrc/,
Python binding in _lib.  PyTorch (optional) is used only by callers for
device memory and streams; see runner.py."""
from ._lib import (  # noqa: F401
    HIT_DTYPE, STATS_DTYPE, TRIGGER_DTYPE, WINDOW_DTYPE, Detector, Result, TrigError,
    TRIG_OK, TRIG_EINVAL, TRIG_ENOMEM, TRIG_EAGAIN, TRIG_ETIMEOUT, TRIG_EDEVICE, TRIG_ECAPACITY,
    TRIG_RUN_GRAPH, TRIG_RUN_TIMED, load, trig_batch_run, trig_batch_scratch_bytes, trig_create, trig_destroy,
    trig_engine_set_mode, trig_engine_stats, trig_get_tile_config, trig_kernel_launch_count, trig_kernel_times, trig_last_error,
    trig_autotune, trig_batch_run_noalloc, trig_detector_tile_config, trig_batch_run_events,
    trig_batch_events_scratch_bytes, trig_set_events, TRIG_FLAG_EV_FULL,
    trig_poll, trig_set_tile_config, trig_slice_rows, trig_submit_slice, win_cap_for,
    Array, ASEED_DTYPE, ASTATS_DTYPE, TRIG_AFLAG_SEED_FULL, TRIG_AFLAG_WIN_FULL, TRIG_AFLAG_HIT_FULL,
    TRIG_AFLAG_TOWER_INCOMPLETE, trig_array_scratch_bytes, trig_array_select, pinned_copy,
    trig_engine_hold, trig_engine_set_staging_limit, trig_engine_fail_result_allocs, trig_set_device_wait,
    TRIG_FLAG_TIMEOUT, TRACE_DTYPE, trig_engine_trace, trig_engine_trace_read,
)
