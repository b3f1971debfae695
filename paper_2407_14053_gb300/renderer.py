"""Torch-facing wrapper of the C ABI: device tensors in, device tensors out.

Each method calls one ``dl_*`` entry point on the caller's current CUDA
stream; nothing here computes a result (see ``_binding``)."""
from __future__ import annotations

import numpy as np
import torch

from . import _binding as B

MODES = {"directl": B.DL_DIRECTL, "standard": B.DL_STANDARD, "required_only": B.DL_REQUIRED_ONLY,
         "raycast": B.DL_RAYCAST, "standard_sr": B.DL_STANDARD_SR}
DTYPES = {"f32": (B.DL_F32, torch.float32), "bf16": (B.DL_BF16, torch.bfloat16),
          "f16": (B.DL_F16, torch.float16)}


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


def display_params(d) -> B.dl_display_params:
    """dl_display_params from any object with the same field names."""
    return B.dl_display_params(int(d.width), int(d.height), int(d.num_views), int(d.p_w),
                               float(d.pitch_lx), float(d.tan_slant), float(d.offset_k),
                               float(d.view_span_deg), float(d.fov_x_deg), int(d.repurpose),
                               int(d.reverse_views), int(getattr(d, "rig", 0)))


class Renderer:
    """One ``dl_ctx`` on one CUDA device."""

    def __init__(self, device: int = 0):
        self.device = int(device)
        self.ctx = B.dl_create(self.device)
        self._displays = {}
        self._batches = []

    def close(self) -> None:
        if self.ctx is not None:
            for b in list(self._batches):
                b.close()
            B.dl_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- scenes -----------------------------------------------------------
    def load_gaussians(self, scene: dict, dtype: str = "f32") -> int:
        """Copy a scene (numpy arrays as made by ``workloads.make_scene``) to
        the library; scale, rotation, opacity and SH are stored in ``dtype``."""
        code, tdt = DTYPES[dtype]
        dev = torch.device("cuda", self.device)
        keep = {"mean": torch.as_tensor(np.ascontiguousarray(scene["mean"], np.float32)).to(dev)}
        for k in ("log_scale", "rot_wxyz", "opacity_logit", "sh"):
            keep[k] = torch.as_tensor(np.ascontiguousarray(scene[k], np.float32)).to(dev).to(tdt)
            keep[k] = keep[k].contiguous()
        desc = B.dl_gaussians_desc(int(keep["mean"].shape[0]), int(scene["sh_degree"]), code,
                                   keep["mean"].data_ptr(), keep["log_scale"].data_ptr(),
                                   keep["rot_wxyz"].data_ptr(), keep["opacity_logit"].data_ptr(),
                                   keep["sh"].data_ptr(), 1)
        sid = B.dl_load_gaussians(self.ctx, desc, _stream())
        torch.cuda.current_stream().synchronize()
        return sid

    def free_scene(self, sid: int) -> None:
        B.dl_free_scene(self.ctx, sid)

    # -- displays ---------------------------------------------------------
    def set_display(self, display) -> int:
        did = B.dl_set_display(self.ctx, display_params(display), _stream())
        self._displays[did] = (int(display.width), int(display.height), int(display.num_views))
        return did

    def free_display(self, did: int) -> None:
        B.dl_free_display(self.ctx, did)
        self._displays.pop(did, None)

    def display_info(self, did: int):
        return B.dl_display_info(self.ctx, did)

    def view_map(self, did: int) -> np.ndarray:
        w, h, _ = self._displays[did]
        out = np.empty((h, 3 * w), dtype=np.uint16)
        B.dl_get_view_map(self.ctx, did, out.ctypes.data, 0, _stream())
        return out

    def subpixel_map(self, did: int) -> np.ndarray:
        w, h, _ = self._displays[did]
        out = np.empty((h, w, 3), dtype=np.uint32)
        B.dl_get_subpixel_map(self.ctx, did, out.ctypes.data, 0, _stream())
        return out

    def ray_table(self, did: int):
        w, h, _ = self._displays[did]
        n_rays, _ = self.display_info(did)
        ray_of = np.empty((h, w, 3), dtype=np.uint32)
        rays = np.empty((n_rays, 3), dtype=np.int32)
        B.dl_get_ray_table(self.ctx, did, ray_of.ctypes.data, rays.ctypes.data, 0, _stream())
        return ray_of, rays

    def encode_rays(self, did: int, ray_rgb: torch.Tensor, out: torch.Tensor | None = None):
        """Encoded frame (h, w, 3) from per-ray RGB (N_rays, 3) on the device,
        rays numbered as ``ray_table`` reports them."""
        w, h, _ = self._displays[did]
        n_rays, _ = self.display_info(did)
        assert ray_rgb.is_cuda and ray_rgb.dtype == torch.float32 and ray_rgb.is_contiguous()
        assert ray_rgb.numel() == 3 * n_rays
        if out is None:
            out = torch.empty((h, w, 3), dtype=torch.float32, device=ray_rgb.device)
        B.dl_encode_rays(self.ctx, did, ray_rgb.data_ptr(), out.data_ptr(), _stream())
        return out

    # -- frames -----------------------------------------------------------
    def set_tile(self, mode: str, tile_w: int, tile_h: int) -> None:
        B.dl_set_tile(self.ctx, MODES[mode], tile_w, tile_h)

    def render(self, sid: int, did: int, L0, mode: str = "directl", out: torch.Tensor | None = None):
        """Encoded frame (h, w, 3) float32 on the device, enqueued on the
        current stream."""
        w, h, _ = self._displays[did]
        if out is None:
            out = torch.empty((h, w, 3), dtype=torch.float32, device=f"cuda:{self.device}")
        assert out.is_cuda and out.is_contiguous() and out.numel() == 3 * w * h
        B.dl_render_frame(self.ctx, sid, did, np.asarray(L0, np.float64).ravel(), MODES[mode],
                          out.data_ptr(), 1, _stream())
        return out

    def render_to_host(self, sid: int, did: int, L0, out: torch.Tensor, mode: str = "directl"):
        """Same frame written into a host tensor (pinned for speed); returns
        once the frame is in host memory."""
        assert not out.is_cuda and out.is_contiguous()
        B.dl_render_frame(self.ctx, sid, did, np.asarray(L0, np.float64).ravel(), MODES[mode],
                          out.data_ptr(), 0, _stream())
        return out

    def render_to_host_async(self, sid: int, did: int, L0, out: torch.Tensor,
                             copy_stream: torch.cuda.Stream, mode: str = "directl"):
        """Same frame written into a pinned host tensor by a copy on
        `copy_stream`, which overlaps the next frame rendered on the current
        stream; `out` holds the frame once `copy_stream` has reached the copy
        (e.g. copy_stream.synchronize())."""
        assert not out.is_cuda and out.is_contiguous() and out.is_pinned()
        B.dl_render_frame_async_host(self.ctx, sid, did, np.asarray(L0, np.float64).ravel(),
                                     MODES[mode], out.data_ptr(), _stream(),
                                     copy_stream.cuda_stream)
        return out

    def set_sort_mode(self, mode: str) -> None:
        """'auto', 'radix' or 'binned' (see DL_OPT_SORT_MODE)."""
        B.dl_set_option(self.ctx, B.DL_OPT_SORT_MODE,
                        {"auto": B.DL_SORT_AUTO, "radix": B.DL_SORT_RADIX, "binned": B.DL_SORT_BINNED}[mode])

    def set_eval(self, mode: str, strategy: str) -> None:
        """Evaluation strategy ('direct' or 'transposed') of 'directl' (and
        'required_only') or of 'standard'."""
        opt = B.DL_OPT_EVAL_STANDARD if mode == "standard" else B.DL_OPT_EVAL_DIRECTL
        B.dl_set_option(self.ctx, opt, {"direct": B.DL_EVAL_DIRECT,
                                        "transposed": B.DL_EVAL_TRANSPOSED}[strategy])

    def set_standard_view_size(self, view_w: int = 0, view_h: int = 0) -> None:
        """Resolution of the standard paradigm's views (0, 0: the panel's);
        below panel resolution they are upsampled while interweaving."""
        B.dl_set_option(self.ctx, B.DL_OPT_STANDARD_VIEW_SIZE, (int(view_w) << 16) | int(view_h))

    def set_heap_capacity(self, cap: int) -> None:
        """c_h of the ray-order renderer ('raycast' mode): nearest
        intersections kept per ray (1..256)."""
        B.dl_set_option(self.ctx, B.DL_OPT_HEAP_CAPACITY, int(cap))

    def set_key_emission(self, where="auto") -> None:
        """Binned DirectL frames: "projection" (or True) has the projection
        kernel emit the tile keys into slices laid out from the previous
        frame; "two_pass" (or False) uses tile metadata and a separate
        emission kernel; "auto" (default) picks the projection for scenes of
        at least 131,072 Gaussians."""
        value = {True: 1, False: 0, "projection": 1, "two_pass": 0, "auto": 2}[where]
        B.dl_set_option(self.ctx, B.DL_OPT_KEY_EMISSION, value)

    def set_warp_cap(self, cap: int) -> None:
        """Longest tile list (512 or 1024 keys; 0 = none) one warp composites."""
        B.dl_set_option(self.ctx, B.DL_OPT_WARP_LIST_CAP, int(cap))

    def enable_stage_timing(self, on: bool = True, count_pairs: bool = True) -> None:
        """CUDA events around each frame's stages; count_pairs also counts the
        compositing pairs (the kernels' counting variant)."""
        B.dl_enable_stage_timing(self.ctx, (1 if count_pairs else 2) if on else 0)

    def stats(self) -> dict:
        return B.dl_last_frame_stats(self.ctx)

    def stage_totals(self):
        """(sums over timed frames since the last call, number of frames)."""
        return B.dl_stage_totals(self.ctx)

    def footprint(self, sid: int, did: int, mode: str = "directl") -> int:
        return B.dl_query_footprint(self.ctx, sid, did, MODES[mode])

    def display_size(self, did: int):
        """(width, height, views) of a display."""
        return self._displays[did]

    # -- batches and the tile autotuner -----------------------------------
    def batch(self, plans, margin: float = 1.25) -> "Batch":
        """A frame batch; plans: [(scene_id, display_id, (tile_w, tile_h) or
        None, L0)] sizing each slot (see dl_batch_create)."""
        return Batch(self, plans, margin)

    def autotune_tile(self, sid: int, did: int, L0, candidates=((16, 16), (32, 16), (32, 32),
                                                                 (64, 32)), reps: int = 3):
        """Sets the DirectL tile to the fastest candidate; returns (best, ms)."""
        return B.dl_autotune_tile(self.ctx, sid, did, np.asarray(L0, np.float64).ravel(),
                                  candidates, reps, _stream())


class Batch:
    """A ``dl_batch``: one DirectL frame per assigned slot and launch, with
    no host synchronisation, optionally replayed from a CUDA graph."""

    def __init__(self, renderer: Renderer, plans, margin: float = 1.25):
        self.r = renderer
        self.n_slots = len(plans)
        flat = []
        for sid, did, tile, L0 in plans:
            tw, th = tile if tile else (0, 0)
            flat.append((sid, did, tw, th, np.asarray(L0, np.float64).ravel()))
        self.h = B.dl_batch_create(renderer.ctx, flat, margin, _stream())
        self.outs = [None] * self.n_slots
        renderer._batches.append(self)

    def assign(self, slot: int, sid: int, did: int, out: torch.Tensor, tile=None) -> None:
        w, h, _ = self.r._displays[did]
        assert out.is_cuda and out.dtype == torch.float32 and out.is_contiguous()
        assert out.numel() == 3 * w * h
        tw, th = tile if tile else (0, 0)
        B.dl_batch_assign(self.h, slot, sid, did, tw, th, out.data_ptr(), self.r.ctx)
        self.outs[slot] = out

    def clear(self, slot: int) -> None:
        B.dl_batch_clear(self.h, slot, self.r.ctx)
        self.outs[slot] = None

    def set_pose(self, slot: int, L0) -> None:
        B.dl_batch_set_pose(self.h, slot, np.asarray(L0, np.float64).ravel(), self.r.ctx)

    def launch(self) -> None:
        """Enqueue on the current stream."""
        B.dl_batch_launch(self.h, _stream(), self.r.ctx)

    def capture(self) -> None:
        """Capture the current assignment into a CUDA graph (current stream,
        which must not be the default stream)."""
        B.dl_batch_capture(self.h, _stream(), self.r.ctx)

    def wait(self, raise_on_capacity: bool = True):
        """Per-slot status words of the last launch (0 = ok)."""
        return B.dl_batch_wait(self.h, self.n_slots, self.r.ctx, raise_on_capacity)

    def info(self):
        """(device bytes, long-list capacity)."""
        return B.dl_batch_info(self.h, self.r.ctx)

    def close(self) -> None:
        if self.h is not None:
            B.dl_batch_destroy(self.h, self.r.ctx)
            self.h = None
            self.r._batches.remove(self)
