"""Torch-facing wrapper of the C ABI: device tensors in, device tensors out.

Each method calls one ``dl_*`` entry point on the caller's current CUDA
stream; nothing here computes a result (see ``_binding``)."""
from __future__ import annotations

import numpy as np
import torch

from . import _binding as B

MODES = {"directl": B.DL_DIRECTL, "standard": B.DL_STANDARD, "required_only": B.DL_REQUIRED_ONLY}
DTYPES = {"f32": (B.DL_F32, torch.float32), "bf16": (B.DL_BF16, torch.bfloat16),
          "f16": (B.DL_F16, torch.float16)}


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


def display_params(d) -> B.dl_display_params:
    """dl_display_params from any object with the same field names."""
    return B.dl_display_params(int(d.width), int(d.height), int(d.num_views), int(d.p_w),
                               float(d.pitch_lx), float(d.tan_slant), float(d.offset_k),
                               float(d.view_span_deg), float(d.fov_x_deg), int(d.repurpose),
                               int(d.reverse_views))


class Renderer:
    """One ``dl_ctx`` on one CUDA device."""

    def __init__(self, device: int = 0):
        self.device = int(device)
        self.ctx = B.dl_create(self.device)
        self._displays = {}

    def close(self) -> None:
        if self.ctx is not None:
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

    def set_warp_cap(self, cap: int) -> None:
        """Longest tile list (512 or 1024 keys; 0 = none) one warp composites."""
        B.dl_set_option(self.ctx, B.DL_OPT_WARP_LIST_CAP, int(cap))

    def enable_stage_timing(self, on: bool = True) -> None:
        B.dl_enable_stage_timing(self.ctx, on)

    def stats(self) -> dict:
        return B.dl_last_frame_stats(self.ctx)

    def stage_totals(self):
        """(sums over timed frames since the last call, number of frames)."""
        return B.dl_stage_totals(self.ctx)

    def footprint(self, sid: int, did: int, mode: str = "directl") -> int:
        return B.dl_query_footprint(self.ctx, sid, did, MODES[mode])
