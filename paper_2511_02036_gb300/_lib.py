"""ctypes declarations of the C ABI in include/tm.h (argument marshalling only)."""

from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
# TM_LIBRARY may name another build of the same sources (for example an instrumented one)
LIB_PATH = os.environ.get("TM_LIBRARY") or os.path.join(_HERE, "libtm.so")

c_i32, c_u64, c_i64, c_f32, c_f64, c_sz, c_p = (ctypes.c_int32, ctypes.c_uint64, ctypes.c_int64,
                                                ctypes.c_float, ctypes.c_double, ctypes.c_size_t,
                                                ctypes.c_void_p)

TM_OK = 0
TM_ERR_INVALID_ARG = 1
TM_ERR_NOT_FOUND = 2
TM_ERR_EXISTS = 3
TM_ERR_NO_MEMORY = 4
TM_ERR_CAPACITY = 5
TM_ERR_CUDA = 6
TM_ERR_TIMEOUT = 7
TM_ERR_BUSY = 8
TM_MODE_FUSED = 0
TM_MODE_PER_PAIR = 1
TM_MAX_KP_LIMIT = 8192
TM_MAX_IMAGE_SIZE = 16384
TM_PLAN_STAGES = 6
TM_BATCH_INFLIGHT = 4
TM_DEBUG_WAIT_LIMIT = 1
TM_DEBUG_STARVE_WAITS = 2
TM_DEBUG_SEARCH_THREADS = 3
TM_DEBUG_L2_PREFETCH = 4
TM_DEBUG_BRANCH_PRIORITY = 5
TM_DEBUG_QUERIES_PER_LANE = 6
TM_DEBUG_PERSISTENT = 7
TM_DEBUG_SPLIT_MIN = 8
TM_DEBUG_ENTRY_CAP = 9


class tm_camera(ctypes.Structure):
    _fields_ = [("width", c_i32), ("height", c_i32), ("fx", c_f64), ("fy", c_f64),
                ("cx", c_f64), ("cy", c_f64)]


class tm_keyframe_view(ctypes.Structure):
    _fields_ = [("n", c_i32), ("desc", c_p), ("xy", c_p), ("angle", c_p), ("level", c_p),
                ("node", c_p), ("Tcw", c_f64 * 12)]


class tm_mappoint_view(ctypes.Structure):
    _fields_ = [("n", c_i32), ("pos", c_p), ("normal", c_p), ("desc", c_p),
                ("min_dist", c_p), ("max_dist", c_p), ("skip", c_p)]


class tm_search_params(ctypes.Structure):
    _fields_ = [("hamming_max", c_i32), ("ratio_num", c_i32), ("ratio_den", c_i32),
                ("epi_chi2", c_f32), ("epipolar", c_i32), ("resolve", c_i32),
                ("rot_filter", c_i32), ("mode", c_i32), ("lanes_per_query", c_i32),
                ("dense_min", c_i32), ("epipole_px", c_f32), ("rot_mode", c_i32),
                ("baseline_min_ratio", c_f32)]


class tm_fuse_params(ctypes.Structure):
    _fields_ = [("chi2", c_f32), ("hamming_max", c_i32), ("radius_scale", c_f32)]


class tm_match(ctypes.Structure):
    _fields_ = [("q_idx", c_i32), ("t_idx", c_i32), ("dist", c_i32)]


class tm_store_stats(ctypes.Structure):
    _fields_ = [("device", c_i32), ("max_kp", c_i32), ("slots_used", c_i32),
                ("slots_free_in_budget", c_i32), ("slot_bytes", c_sz),
                ("bytes_reserved", c_sz), ("budget_bytes", c_sz)]


class tm_step(ctypes.Structure):
    _fields_ = [("kf_id", c_u64), ("nbr_ids", c_p), ("n_nbrs", c_i32),
                ("q_free_off", c_i64), ("nbr_free_off", c_i64), ("mp_begin", c_i32),
                ("mp_count", c_i32), ("fwd_mp_begin", c_i32), ("fwd_mp_count", c_i32),
                ("fwd_skip_off", c_i64), ("nbr_median_depth", c_p)]


class tm_triangulation_params(ctypes.Structure):
    _fields_ = [("cos_parallax_max", ctypes.c_double), ("chi2", ctypes.c_double),
                ("ratio_factor", ctypes.c_double)]


class tm_keyframes_packed(ctypes.Structure):
    _fields_ = [("n", c_p), ("desc", c_p), ("xy", c_p), ("angle", c_p), ("level", c_p), ("node", c_p),
                ("Tcw", c_p)]


class tm_batch_inputs(ctypes.Structure):
    _fields_ = [("masks", c_p), ("mask_bytes", c_sz), ("mps", tm_mappoint_view),
                ("n_new", c_i32), ("new_ids", c_p), ("new_kfs", c_p), ("tri", c_p), ("new_packed", c_p),
                ("mps_block", c_p), ("mps_block_bytes", c_u64)]


class tm_batch_result(ctypes.Structure):
    _fields_ = [("matches", c_p), ("match_cap", c_sz), ("n_matches", c_sz),
                ("pair_offsets", c_p), ("fuse", c_p), ("fuse_cap", c_sz), ("n_fuse", c_sz),
                ("fuse_offsets", c_p), ("n_comparisons_search", c_u64),
                ("n_comparisons_fuse", c_u64), ("fwd", c_p), ("fwd_cap", c_sz), ("n_fwd", c_sz),
                ("fwd_offsets", c_p), ("n_comparisons_fwd", c_u64), ("points", c_p),
                ("point_ok", c_p)]


class tm_server_config(ctypes.Structure):
    _fields_ = [("max_batch_requests", c_i32), ("max_inflight_batches", c_i32),
                ("queue_capacity", c_i32), ("evict_after", c_i32),
                ("search", tm_search_params), ("fuse", tm_fuse_params),
                ("triangulate", c_i32), ("tri", tm_triangulation_params)]


class tm_plan_tuning(ctypes.Structure):
    _fields_ = [("queries_per_warp", c_i32), ("persistent", c_i32), ("l2_prefetch", c_i32),
                ("branch_priority", c_i32), ("dense_min", c_i32), ("dense_split", c_i32),
                ("search_ctas", c_i32), ("tuned", c_i32), ("per_lane", c_i32), ("search_units", c_i32),
                ("entry_form", c_i32)]


class tm_fuse_apply_stats(ctypes.Structure):
    _fields_ = [("added", c_i32), ("merged_into_existing", c_i32), ("replaced_existing", c_i32),
                ("skipped_dead", c_i32), ("skipped_observed", c_i32)]


class tm_request(ctypes.Structure):
    _fields_ = [("kf_id", c_u64), ("kf", tm_keyframe_view), ("nbr_ids", c_p), ("n_nbrs", c_i32),
                ("q_free", c_p), ("nbr_free", c_p), ("mps", tm_mappoint_view),
                ("fwd_mps", tm_mappoint_view), ("fwd_skip", c_p), ("nbr_free_bytes", c_sz)]


class tm_request_info(ctypes.Structure):
    _fields_ = [("done", c_i32), ("status", c_i32), ("n_matches", c_i32), ("n_fuse", c_i32),
                ("t_submit", c_f64), ("t_admit", c_f64), ("t_done", c_f64), ("n_fwd", c_i32)]


class tm_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("admitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("failed", ctypes.c_int64), ("batches", ctypes.c_int64), ("deferrals", ctypes.c_int64),
                ("evicted", ctypes.c_int64), ("peak_pending", c_i32), ("peak_inflight", c_i32),
                ("peak_store_slots", c_i32), ("store_slot_limit", c_i32)]


P = ctypes.POINTER
# name -> (restype, argtypes)
SIGNATURES = {
    "tm_last_error": (ctypes.c_char_p, []),
    "tm_search_params_default": (None, [P(tm_search_params)]),
    "tm_fuse_params_default": (None, [P(tm_fuse_params)]),
    "tm_triangulation_params_default": (None, [P(tm_triangulation_params)]),
    "tm_ctx_create": (c_i32, [c_i32, P(tm_camera), c_i32, c_sz, P(c_p)]),
    "tm_ctx_destroy": (c_i32, [c_p]),
    "tm_store_reserve": (c_i32, [c_p, c_i32]),
    "tm_store_get_stats": (c_i32, [c_p, P(tm_store_stats)]),
    "tm_store_add_keyframe": (c_i32, [c_p, c_u64, P(tm_keyframe_view), c_p]),
    "tm_store_add_keyframes": (c_i32, [c_p, c_i32, c_p, P(tm_keyframe_view), c_p]),
    "tm_store_remove_keyframe": (c_i32, [c_p, c_u64]),
    "tm_store_remove_keyframes": (c_i32, [c_p, c_i32, c_p]),
    "tm_obs_create": (c_i32, [c_i32, P(c_p)]),
    "tm_obs_destroy": (c_i32, [c_p]),
    "tm_obs_add": (c_i32, [c_p, c_i32, c_p, c_p]),
    "tm_obs_remove": (c_i32, [c_p, c_i32, c_p, c_p]),
    "tm_obs_redundant": (c_i32, [c_p, c_i32, c_p, c_p, c_i32, c_f32, P(c_i32), P(c_i32)]),
    "tm_map_create": (c_i32, [c_i32, P(c_p)]),
    "tm_map_destroy": (c_i32, [c_p]),
    "tm_map_add_keyframe": (c_i32, [c_p, c_u64, c_i32, c_p]),
    "tm_map_remove_keyframe": (c_i32, [c_p, c_u64]),
    "tm_map_add_observations": (c_i32, [c_p, c_u64, c_i32, c_p, c_p]),
    "tm_map_fuse_apply": (c_i32, [c_p, c_u64, c_i32, c_p, c_p, c_i32, P(tm_fuse_apply_stats)]),
    "tm_map_keyframe_points": (c_i32, [c_p, c_u64, c_i32, c_p]),
    "tm_map_point_info": (c_i32, [c_p, c_i32, c_p, c_p, c_p, c_p]),
    "tm_map_redundant": (c_i32, [c_p, c_u64, c_i32, c_f32, P(c_i32), P(c_i32)]),
    "tm_store_keyframe_size": (c_i32, [c_p, c_u64, P(c_i32)]),
    "tm_search_triangulation": (c_i32, [c_p, c_u64, c_p, c_i32, P(tm_search_params), c_p, c_p,
                                        c_p, c_sz, P(c_sz), c_p, P(c_u64), c_p]),
    "tm_fuse": (c_i32, [c_p, c_u64, P(tm_mappoint_view), P(tm_fuse_params), c_p, c_sz,
                        P(c_sz), P(c_u64), c_p]),
    "tm_batch_run": (c_i32, [c_p, c_p, c_i32, P(tm_batch_inputs), P(tm_search_params),
                             P(tm_fuse_params), P(tm_batch_result), c_p]),
    "tm_batch_last_host_times": (c_i32, [c_p, c_p]),
    "tm_batch_begin": (c_i32, [c_p, c_p, c_i32, P(tm_batch_inputs), P(tm_search_params),
                               P(tm_fuse_params), P(c_u64)]),
    "tm_batch_finish": (c_i32, [c_p, c_u64, P(tm_batch_result)]),
    "tm_plan_create": (c_i32, [c_p, c_p, c_i32, P(tm_batch_inputs), P(tm_search_params),
                               P(tm_fuse_params), P(c_p)]),
    "tm_plan_run": (c_i32, [c_p, c_p]),
    "tm_debug_set": (c_i32, [c_p, c_i32, ctypes.c_int64]),
    "tm_debug_bounds": (c_i32, [c_i32, P(ctypes.c_uint32), P(c_i32)]),
    "tm_measure_int_rates": (c_i32, [c_i32, P(c_f64), P(c_f64), P(c_f64)]),
    "tm_plan_run_timed": (c_i32, [c_p, c_p]),
    "tm_plan_results": (c_i32, [c_p, P(tm_batch_result), c_p]),
    "tm_plan_info": (c_i32, [c_p, P(c_i32), P(c_i32), P(c_i32), P(c_i32)]),
    "tm_plan_stage_times": (c_i32, [c_p, c_p]),
    "tm_plan_get_tuning": (c_i32, [c_p, P(tm_plan_tuning)]),
    "tm_plan_destroy": (c_i32, [c_p]),
    "tm_server_config_default": (None, [P(tm_server_config)]),
    "tm_server_start": (c_i32, [c_p, P(tm_server_config), P(c_p)]),
    "tm_server_submit": (c_i32, [c_p, P(tm_request), P(c_u64)]),
    "tm_server_poll": (c_i32, [c_p, c_u64, c_f64, P(tm_request_info)]),
    "tm_server_take": (c_i32, [c_p, c_u64, c_p, c_p, c_p]),
    "tm_server_take_ex": (c_i32, [c_p, c_u64, c_p, c_p, c_p, c_p, c_p, c_p, c_p]),
    "tm_server_stop": (c_i32, [c_p]),
    "tm_server_get_stats": (c_i32, [c_p, P(tm_server_stats)]),
    "tm_now": (c_f64, []),
    "tm_search_pair_noalloc": (c_i32, [P(tm_camera), P(tm_keyframe_view), P(tm_keyframe_view),
                                       P(tm_search_params), c_p, c_p, c_p, c_p, c_p, c_p]),
}

_lib = None


def load():
    """Loads libtm.so from the package directory.  There is no fallback: without the CUDA
    library nothing in this package can run."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libtm.so is not built (run `python paper_2511_02036_gb300/build.py` "
                               "or __graft_entry__.build())")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib
