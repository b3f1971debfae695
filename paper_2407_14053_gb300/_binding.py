"""ctypes binding of libdirectl.so, one Python function per C ABI entry point.

Names, arguments and meanings are those of ``include/directl.h``; this module
only marshals arguments (pointers as ints, structs as ctypes structures) and
turns a negative ``dl_status`` into :class:`DirectLError`.  Every computation
happens in the CUDA library: if ``libdirectl.so`` is missing the first call
raises instead of falling back to anything else."""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdirectl.so")

DL_OK = 0
DL_ERR_INVALID_ARG = -1
DL_ERR_OOM = -2
DL_ERR_CUDA = -3
DL_ERR_NOT_FOUND = -4
DL_ERR_TIMEOUT = -5
DL_ERR_DEVICE_CHECK = -6
DL_ERR_CAPACITY = -7

DL_F32, DL_BF16, DL_F16 = 0, 1, 2
DL_DIRECTL, DL_STANDARD, DL_REQUIRED_ONLY, DL_RAYCAST, DL_STANDARD_SR = 0, 1, 2, 3, 4
DL_OPT_SORT_MODE, DL_OPT_EVAL_DIRECTL, DL_OPT_EVAL_STANDARD, DL_OPT_WARP_LIST_CAP = 1, 2, 3, 4
DL_OPT_STANDARD_VIEW_SIZE, DL_OPT_HEAP_CAPACITY, DL_OPT_KEY_EMISSION = 5, 6, 7
DL_SORT_AUTO, DL_SORT_RADIX, DL_SORT_BINNED = 0, 1, 2
DL_EVAL_DIRECT, DL_EVAL_TRANSPOSED = 0, 1

c_int32, c_int64, c_double, c_void_p = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p


class dl_gaussians_desc(ctypes.Structure):
    _fields_ = [("n", c_int64), ("sh_degree", c_int32), ("dtype", c_int32), ("mean", c_void_p),
                ("log_scale", c_void_p), ("rot_wxyz", c_void_p), ("opacity_logit", c_void_p),
                ("sh", c_void_p), ("on_device", c_int32)]


class dl_display_params(ctypes.Structure):
    _fields_ = [("width", c_int32), ("height", c_int32), ("num_views", c_int32), ("p_w", c_int32),
                ("pitch_lx", c_double), ("tan_slant", c_double), ("offset_k", c_double),
                ("view_span_deg", c_double), ("fov_x_deg", c_double), ("repurpose", c_int32),
                ("reverse_views", c_int32), ("rig", c_int32)]


class dl_frame_stats(ctypes.Structure):
    _fields_ = [("n_keys", c_int64), ("n_rays", c_int64), ("pairs_evaluated", c_int64),
                ("pairs_blended", c_int64), ("tile_w", c_int32), ("tile_h", c_int32),
                ("sort_bits", c_int32), ("n_launches", c_int32), ("lists_small", c_int64),
                ("lists_large", c_int64), ("max_list", c_int64), ("n_visible", c_int64)] + [
        (f, ctypes.c_float) for f in ("ms_project", "ms_scan", "ms_sync", "ms_emit", "ms_sort",
                                      "ms_ranges", "ms_composite", "ms_interweave", "ms_total")] + [
        ("status", c_int32), ("reemitted", c_int32)]


class dl_slot_plan(ctypes.Structure):
    _fields_ = [("scene_id", c_int32), ("display_id", c_int32), ("tile_w", c_int32),
                ("tile_h", c_int32), ("L0_c2w", c_double * 16)]


P = ctypes.POINTER
SIGNATURES = {
    "dl_create": (c_int32, [P(c_void_p), c_int32]),
    "dl_destroy": (c_int32, [c_void_p]),
    "dl_status_string": (ctypes.c_char_p, [c_int32]),
    "dl_last_error_detail": (c_int32, [c_void_p, ctypes.c_char_p, ctypes.c_size_t]),
    "dl_load_gaussians": (c_int32, [c_void_p, P(dl_gaussians_desc), c_void_p, P(c_int32)]),
    "dl_free_scene": (c_int32, [c_void_p, c_int32]),
    "dl_set_display": (c_int32, [c_void_p, P(dl_display_params), c_void_p, P(c_int32)]),
    "dl_free_display": (c_int32, [c_void_p, c_int32]),
    "dl_display_info": (c_int32, [c_void_p, c_int32, P(c_int64), P(c_double)]),
    "dl_get_view_map": (c_int32, [c_void_p, c_int32, c_void_p, c_int32, c_void_p]),
    "dl_get_subpixel_map": (c_int32, [c_void_p, c_int32, c_void_p, c_int32, c_void_p]),
    "dl_get_ray_table": (c_int32, [c_void_p, c_int32, c_void_p, c_void_p, c_int32, c_void_p]),
    "dl_render_frame": (c_int32, [c_void_p, c_int32, c_int32, P(c_double), c_int32, c_void_p,
                                  c_int32, c_void_p]),
    "dl_render_frame_async_host": (c_int32, [c_void_p, c_int32, c_int32, P(c_double), c_int32,
                                             c_void_p, c_void_p, c_void_p]),
    "dl_query_footprint": (c_int32, [c_void_p, c_int32, c_int32, c_int32, P(ctypes.c_size_t)]),
    "dl_set_tile": (c_int32, [c_void_p, c_int32, c_int32, c_int32]),
    "dl_encode_rays": (c_int32, [c_void_p, c_int32, c_void_p, c_void_p, c_void_p]),
    "dl_enable_stage_timing": (c_int32, [c_void_p, c_int32]),
    "dl_last_frame_stats": (c_int32, [c_void_p, P(dl_frame_stats)]),
    "dl_stage_totals": (c_int32, [c_void_p, P(dl_frame_stats), P(c_int32)]),
    "dl_set_option": (c_int32, [c_void_p, c_int32, c_int64]),
    "dl_ray_table_static": (c_int32, [c_int32, c_int32, c_void_p, c_void_p, c_void_p, c_void_p,
                                      P(c_int64), c_void_p]),
    "dl_batch_create": (c_int32, [c_void_p, c_int32, P(dl_slot_plan), c_double, c_void_p,
                                  P(c_void_p)]),
    "dl_batch_destroy": (c_int32, [c_void_p]),
    "dl_batch_assign": (c_int32, [c_void_p, c_int32, c_int32, c_int32, c_int32, c_int32, c_void_p]),
    "dl_batch_clear": (c_int32, [c_void_p, c_int32]),
    "dl_batch_set_pose": (c_int32, [c_void_p, c_int32, P(c_double)]),
    "dl_batch_launch": (c_int32, [c_void_p, c_void_p]),
    "dl_batch_capture": (c_int32, [c_void_p, c_void_p]),
    "dl_batch_wait": (c_int32, [c_void_p, P(ctypes.c_uint32)]),
    "dl_batch_info": (c_int32, [c_void_p, P(ctypes.c_size_t), P(c_int32)]),
    "dl_autotune_tile": (c_int32, [c_void_p, c_int32, c_int32, P(c_double), P(c_int32), c_int32,
                                   c_int32, c_void_p, P(c_int32), P(ctypes.c_float)]),
    "dl_measure_peaks": (c_int32, [c_int32, P(c_double), P(c_double), P(c_double)]),
}

_lock = threading.Lock()
_lib = None


class DirectLError(RuntimeError):
    def __init__(self, call: str, status: int, detail: str):
        super().__init__(f"{call} failed: {status_string(status)} ({status}): {detail}")
        self.status = status


def lib() -> ctypes.CDLL:
    """Load libdirectl.so (built by ``paper_2407_14053_gb300.build``)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                                   "`python -c 'import __graft_entry__ as g; g.build()'`")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def status_string(s: int) -> str:
    return lib().dl_status_string(int(s)).decode()


def _detail(ctx) -> str:
    if ctx is None:
        return ""
    buf = ctypes.create_string_buffer(512)
    lib().dl_last_error_detail(ctx, buf, len(buf))
    return buf.value.decode(errors="replace")


def _check(name: str, ctx, status: int) -> None:
    if status != DL_OK:
        raise DirectLError(name, status, _detail(ctx))


def dl_create(device: int = 0):
    h = c_void_p()
    _check("dl_create", None, lib().dl_create(ctypes.byref(h), int(device)))
    return h


def dl_destroy(ctx) -> None:
    _check("dl_destroy", None, lib().dl_destroy(ctx))


def dl_status_string(s: int) -> str:
    return status_string(s)


def dl_last_error_detail(ctx) -> str:
    return _detail(ctx)


def dl_load_gaussians(ctx, desc: dl_gaussians_desc, stream: int = 0) -> int:
    sid = c_int32()
    _check("dl_load_gaussians", ctx,
           lib().dl_load_gaussians(ctx, ctypes.byref(desc), c_void_p(stream), ctypes.byref(sid)))
    return sid.value


def dl_free_scene(ctx, scene_id: int) -> None:
    _check("dl_free_scene", ctx, lib().dl_free_scene(ctx, int(scene_id)))


def dl_set_display(ctx, params: dl_display_params, stream: int = 0) -> int:
    did = c_int32()
    _check("dl_set_display", ctx,
           lib().dl_set_display(ctx, ctypes.byref(params), c_void_p(stream), ctypes.byref(did)))
    return did.value


def dl_free_display(ctx, display_id: int) -> None:
    _check("dl_free_display", ctx, lib().dl_free_display(ctx, int(display_id)))


def dl_display_info(ctx, display_id: int):
    n = c_int64()
    b = c_double()
    _check("dl_display_info", ctx,
           lib().dl_display_info(ctx, int(display_id), ctypes.byref(n), ctypes.byref(b)))
    return n.value, b.value


def dl_get_view_map(ctx, display_id: int, out_ptr: int, out_on_device: int, stream: int = 0):
    _check("dl_get_view_map", ctx, lib().dl_get_view_map(ctx, int(display_id), c_void_p(out_ptr),
                                                          int(out_on_device), c_void_p(stream)))


def dl_get_subpixel_map(ctx, display_id: int, out_ptr: int, out_on_device: int, stream: int = 0):
    _check("dl_get_subpixel_map", ctx,
           lib().dl_get_subpixel_map(ctx, int(display_id), c_void_p(out_ptr), int(out_on_device),
                                     c_void_p(stream)))


def dl_get_ray_table(ctx, display_id: int, ray_of_ptr: int, rays_ptr: int, out_on_device: int,
                     stream: int = 0):
    _check("dl_get_ray_table", ctx,
           lib().dl_get_ray_table(ctx, int(display_id), c_void_p(ray_of_ptr), c_void_p(rays_ptr),
                                  int(out_on_device), c_void_p(stream)))


def dl_render_frame(ctx, scene_id: int, display_id: int, L0_c2w, mode: int, out_ptr: int,
                    out_on_device: int, stream: int = 0) -> None:
    L0 = (c_double * 16)(*[float(x) for x in L0_c2w])
    _check("dl_render_frame", ctx,
           lib().dl_render_frame(ctx, int(scene_id), int(display_id), L0, int(mode),
                                 c_void_p(out_ptr), int(out_on_device), c_void_p(stream)))


def dl_render_frame_async_host(ctx, scene_id: int, display_id: int, L0_c2w, mode: int,
                               out_ptr: int, stream: int, copy_stream: int) -> None:
    L0 = (c_double * 16)(*[float(x) for x in L0_c2w])
    _check("dl_render_frame_async_host", ctx,
           lib().dl_render_frame_async_host(ctx, int(scene_id), int(display_id), L0, int(mode),
                                            c_void_p(out_ptr), c_void_p(stream),
                                            c_void_p(copy_stream)))


def dl_query_footprint(ctx, scene_id: int, display_id: int, mode: int) -> int:
    b = ctypes.c_size_t()
    _check("dl_query_footprint", ctx,
           lib().dl_query_footprint(ctx, int(scene_id), int(display_id), int(mode), ctypes.byref(b)))
    return b.value


def dl_encode_rays(ctx, display_id: int, ray_rgb_ptr: int, out_ptr: int, stream: int = 0) -> None:
    _check("dl_encode_rays", ctx, lib().dl_encode_rays(ctx, int(display_id), c_void_p(ray_rgb_ptr),
                                                       c_void_p(out_ptr), c_void_p(stream)))


def dl_set_tile(ctx, mode: int, tile_w: int, tile_h: int) -> None:
    _check("dl_set_tile", ctx, lib().dl_set_tile(ctx, int(mode), int(tile_w), int(tile_h)))


def dl_set_option(ctx, option: int, value: int) -> None:
    _check("dl_set_option", ctx, lib().dl_set_option(ctx, int(option), int(value)))


def dl_enable_stage_timing(ctx, enable) -> None:
    """enable: 0 / False off, 1 / True events and pair counters, 2 events only."""
    _check("dl_enable_stage_timing", ctx, lib().dl_enable_stage_timing(ctx, int(enable)))


def dl_stage_totals(ctx):
    s = dl_frame_stats()
    n = c_int32()
    _check("dl_stage_totals", ctx, lib().dl_stage_totals(ctx, ctypes.byref(s), ctypes.byref(n)))
    return {k: getattr(s, k) for k, _ in dl_frame_stats._fields_}, n.value


def dl_last_frame_stats(ctx) -> dict:
    s = dl_frame_stats()
    _check("dl_last_frame_stats", ctx, lib().dl_last_frame_stats(ctx, ctypes.byref(s)))
    return {k: getattr(s, k) for k, _ in dl_frame_stats._fields_}


def dl_ray_table_static(width: int, height: int, V_ptr: int, src_ptr: int, ray_of_ptr: int,
                        rays_ptr: int, stream: int = 0) -> int:
    """Ray table into caller device buffers using only the library's static
    scratch (no allocation); returns N_rays."""
    n = c_int64()
    _check("dl_ray_table_static", None,
           lib().dl_ray_table_static(int(width), int(height), c_void_p(V_ptr), c_void_p(src_ptr),
                                     c_void_p(ray_of_ptr), c_void_p(rays_ptr), ctypes.byref(n),
                                     c_void_p(stream)))
    return n.value


# ---- frame batches (ctx only supplies the error detail) -----------------
def dl_batch_create(ctx, plans, margin: float = 1.25, stream: int = 0):
    """plans: sequence of (scene_id, display_id, tile_w, tile_h, L0_c2w[16])."""
    arr = (dl_slot_plan * len(plans))()
    for i, (sid, did, tw, th, L0) in enumerate(plans):
        arr[i].scene_id, arr[i].display_id, arr[i].tile_w, arr[i].tile_h = sid, did, tw, th
        arr[i].L0_c2w = (c_double * 16)(*[float(x) for x in L0])
    h = c_void_p()
    _check("dl_batch_create", ctx, lib().dl_batch_create(ctx, len(plans), arr, float(margin),
                                                         c_void_p(stream), ctypes.byref(h)))
    return h


def dl_batch_destroy(batch, ctx=None) -> None:
    _check("dl_batch_destroy", ctx, lib().dl_batch_destroy(batch))


def dl_batch_assign(batch, slot: int, scene_id: int, display_id: int, tile_w: int, tile_h: int,
                    out_ptr: int, ctx=None) -> None:
    _check("dl_batch_assign", ctx, lib().dl_batch_assign(batch, int(slot), int(scene_id),
                                                         int(display_id), int(tile_w), int(tile_h),
                                                         c_void_p(out_ptr)))


def dl_batch_clear(batch, slot: int, ctx=None) -> None:
    _check("dl_batch_clear", ctx, lib().dl_batch_clear(batch, int(slot)))


def dl_batch_set_pose(batch, slot: int, L0_c2w, ctx=None) -> None:
    L0 = (c_double * 16)(*[float(x) for x in L0_c2w])
    _check("dl_batch_set_pose", ctx, lib().dl_batch_set_pose(batch, int(slot), L0))


def dl_batch_launch(batch, stream: int = 0, ctx=None) -> None:
    _check("dl_batch_launch", ctx, lib().dl_batch_launch(batch, c_void_p(stream)))


def dl_batch_capture(batch, stream: int, ctx=None) -> None:
    _check("dl_batch_capture", ctx, lib().dl_batch_capture(batch, c_void_p(stream)))


def dl_batch_wait(batch, n_slots: int, ctx=None, raise_on_capacity: bool = True):
    """Returns the per-slot status words."""
    st = (ctypes.c_uint32 * n_slots)()
    r = lib().dl_batch_wait(batch, st)
    if r != DL_OK and (raise_on_capacity or r != DL_ERR_CAPACITY):
        _check("dl_batch_wait", ctx, r)
    return list(st)


def dl_batch_info(batch, ctx=None):
    b = ctypes.c_size_t()
    c = c_int32()
    _check("dl_batch_info", ctx, lib().dl_batch_info(batch, ctypes.byref(b), ctypes.byref(c)))
    return b.value, c.value


def dl_autotune_tile(ctx, scene_id: int, display_id: int, L0_c2w, candidates, reps: int = 3,
                     stream: int = 0):
    """Returns ((tile_w, tile_h), [median ms per candidate])."""
    L0 = (c_double * 16)(*[float(x) for x in L0_c2w])
    flat = [int(v) for c in candidates for v in c]
    cand = (c_int32 * len(flat))(*flat)
    best = (c_int32 * 2)()
    ms = (ctypes.c_float * len(candidates))()
    _check("dl_autotune_tile", ctx,
           lib().dl_autotune_tile(ctx, int(scene_id), int(display_id), L0, cand, len(candidates),
                                  int(reps), c_void_p(stream), best, ms))
    return (best[0], best[1]), list(ms)


def dl_measure_peaks(device: int = 0) -> dict:
    """Measured FP32 (scalar and packed FP32x2) TFLOP/s and ex2 results/s."""
    a, b, c = c_double(), c_double(), c_double()
    _check("dl_measure_peaks", None,
           lib().dl_measure_peaks(int(device), ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return {"fp32_tflops": a.value, "fp32x2_tflops": b.value, "ex2_per_s": c.value}
