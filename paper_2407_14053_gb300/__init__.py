"""GB300-native DirectL light-field renderer (arXiv 2407.14053).

The renderer is the CUDA library ``libdirectl.so`` (C ABI in
``include/directl.h``).  This package holds its sources (``csrc/``), its build
script (``build.py``), a ctypes binding with the ABI's names (``_binding``)
and a torch-facing wrapper (``Renderer``, imported lazily so that building
needs no torch)."""
from ._binding import (DL_BF16, DL_DIRECTL, DL_ERR_CAPACITY, DL_ERR_CUDA, DL_ERR_DEVICE_CHECK,
                       DL_ERR_INVALID_ARG, DL_ERR_NOT_FOUND, DL_ERR_OOM, DL_ERR_TIMEOUT, DL_F16,
                       DL_F32, DL_OK, DL_REQUIRED_ONLY, DL_STANDARD, LIB_PATH, SIGNATURES,
                       DirectLError, dl_create, dl_destroy, dl_display_info, dl_display_params,
                       dl_enable_stage_timing, dl_frame_stats, dl_free_display, dl_free_scene,
                       dl_gaussians_desc, dl_get_ray_table, dl_get_subpixel_map, dl_get_view_map,
                       dl_last_error_detail, dl_last_frame_stats, dl_load_gaussians,
                       dl_query_footprint, dl_ray_table_static, dl_render_frame, dl_set_display, dl_set_option, dl_set_tile,
                       dl_stage_totals, dl_status_string, lib)


def __getattr__(name):
    if name in ("Renderer", "Batch"):
        from . import renderer
        return getattr(renderer, name)
    raise AttributeError(name)
