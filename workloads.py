"""Seeded synthetic inputs for the DirectL light-field renderer.

This module only draws random numbers and lays out display descriptions. It
holds none of the method's arithmetic (no view map, no projection, no
compositing), so both the FP64 oracle (``oracle/``) and the CUDA library
(``paper_2407_14053_gb300/``) can take their inputs from it without sharing
any computation.

Distributions follow the workloads the renderer is measured on:

* ``tiny``   -- 2,000 Gaussians, means U[-1,1]^3, log-scales N(-3, 0.5),
  uniform random unit quaternions, opacity logit N(0, 1), SH degree 0 with the
  colour drawn from U[0,1]; 240x135 panel, 45 views, pitch 5.3, tan 1/6.
* ``1080p``  -- 200k Gaussians, 80 % means N(0, 0.5^2) and 20 % uniform in
  [-3,3]^3, SH degree 3 (DC from a U[0,1] colour, higher orders N(0, 0.1));
  1920x1080, 45 views, pitch 5.3, tan 1/6; FP32 storage.
* ``4k``     -- 1M Gaussians as ``1080p``; 3840x2160, 45 views, pitch 8.1,
  tan 0.18; BF16 storage of everything but the means.
* ``8k``     -- 3M Gaussians as ``1080p``; 7680x4320, 100 views, pitch 11.7,
  tan 0.2; BF16 storage.

``N(m, s)`` names a normal with mean ``m`` and standard deviation ``s``.  For
the clustered scenes the log-scale mean is ``-3 - 0.5*ln(N/2000)`` so that the
number of splat layers a pixel sees stays near the tiny scene's as N grows
(with the unscaled -3 a 1M-Gaussian scene covers each 4K tile hundreds of
times over).  The synthetic scenes stand in for the trained Blender and
Mip-NeRF360 scenes of the paper's experiments (Sec. 8.1), which are not
available here.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# Normalisation of the degree-0 real spherical harmonic, 1 / (2 sqrt(pi)).  It
# is only used to turn a drawn colour into the DC coefficient that encodes it.
_Y00 = 0.5 / math.sqrt(math.pi)


@dataclasses.dataclass(frozen=True)
class Display:
    """A lenticular panel as the renderer's ``dl_display_params`` describe it.

    ``tan_slant`` is tan(alpha) of the lens tilt, ``pitch_lx`` the line count
    L_x in subpixel widths and ``offset_k`` the lens offset K_offset (Table 1
    of the paper lists these three for each panel)."""

    width: int
    height: int
    num_views: int
    pitch_lx: float
    tan_slant: float
    offset_k: float = 0.0
    view_span_deg: float = 40.0
    fov_x_deg: float = 40.0
    p_w: int = 2
    repurpose: int = 1
    reverse_views: int = 0
    rig: int = 0  # 0: cameras on an arc; 1: off-axis cameras on a straight line

    def replace(self, **kw) -> "Display":
        return dataclasses.replace(self, **kw)


@dataclasses.dataclass(frozen=True)
class SceneSpec:
    n: int
    sh_degree: int
    layout: str  # "uniform" or "clustered"
    dtype: str  # storage dtype of scale/rotation/opacity/SH: "f32", "bf16", "f16"
    seed: int = 0

    @property
    def log_scale_mean(self) -> float:
        if self.layout == "uniform":
            return -3.0
        return -3.0 - 0.5 * math.log(self.n / 2000.0)


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    display: Display
    scene: SceneSpec
    camera_distance: float = 4.0


WORKLOADS = {
    "tiny": Workload("tiny", Display(240, 135, 45, 5.3, 1.0 / 6.0),
                     SceneSpec(2000, 0, "uniform", "f32")),
    "1080p": Workload("1080p", Display(1920, 1080, 45, 5.3, 1.0 / 6.0),
                      SceneSpec(200_000, 3, "clustered", "f32")),
    "4k": Workload("4k", Display(3840, 2160, 45, 8.1, 0.18),
                   SceneSpec(1_000_000, 3, "clustered", "bf16")),
    "8k": Workload("8k", Display(7680, 4320, 100, 11.7, 0.2),
                   SceneSpec(3_000_000, 3, "clustered", "bf16")),
}

# The three calibrated panels of Table 1 (width, height, line count, tilt in
# degrees, offset, field of view, number of views).
PAPER_PANELS = {
    "7.9in": Display(1536, 2048, 48, 6.2221, math.tan(math.radians(10.8232)), 4.2077, 40.0),
    "15.6in": Display(3840, 2160, 60, 5.3344, math.tan(math.radians(6.8526)), 1.2547, 53.0),
    "65in": Display(7680, 4320, 96, 9.3597, math.tan(math.radians(8.6517)), 23.6677, 80.0),
}


def make_scene(spec: SceneSpec) -> dict:
    """Draw a seeded Gaussian scene as float32 structure-of-arrays.

    Returns ``mean (n,3)``, ``log_scale (n,3)``, ``rot_wxyz (n,4)`` (unit
    quaternions), ``opacity_logit (n,)`` and ``sh (n,(d+1)^2,3)``."""
    rng = np.random.default_rng(spec.seed)
    n = spec.n
    if spec.layout == "uniform":
        mean = rng.uniform(-1.0, 1.0, size=(n, 3))
    elif spec.layout == "clustered":
        n_bg = n // 5
        core = rng.normal(0.0, 0.5, size=(n - n_bg, 3))
        bg = rng.uniform(-3.0, 3.0, size=(n_bg, 3))
        mean = np.concatenate([core, bg], axis=0)
        mean = mean[rng.permutation(n)]
    else:
        raise ValueError(spec.layout)
    log_scale = rng.normal(spec.log_scale_mean, 0.5, size=(n, 3))
    q = rng.normal(0.0, 1.0, size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    opacity_logit = rng.normal(0.0, 1.0, size=(n,))
    n_coef = (spec.sh_degree + 1) ** 2
    sh = np.zeros((n, n_coef, 3))
    rgb = rng.uniform(0.0, 1.0, size=(n, 3))
    sh[:, 0, :] = (rgb - 0.5) / _Y00
    if n_coef > 1:
        sh[:, 1:, :] = rng.normal(0.0, 0.1, size=(n, n_coef - 1, 3))
    return {
        "mean": np.ascontiguousarray(mean, dtype=np.float32),
        "log_scale": np.ascontiguousarray(log_scale, dtype=np.float32),
        "rot_wxyz": np.ascontiguousarray(q, dtype=np.float32),
        "opacity_logit": np.ascontiguousarray(opacity_logit, dtype=np.float32),
        "sh": np.ascontiguousarray(sh, dtype=np.float32),
        "sh_degree": spec.sh_degree,
    }


def light_field_centre(distance: float = 4.0, yaw_deg: float = 0.0) -> np.ndarray:
    """Camera-to-world pose (4x4, float64, row-major) of the light-field centre.

    The camera sits at ``distance`` on the world -z axis, turned by ``yaw_deg``
    about the world y axis, and looks at the origin.  Camera axes: x right,
    y down, z forward."""
    a = math.radians(yaw_deg)
    c, s = math.cos(a), math.sin(a)
    rot = np.array([[c, 0.0, s], [0.0, 1.0, 0.0], [-s, 0.0, c]])
    m = np.eye(4)
    m[:3, :3] = rot
    m[:3, 3] = rot @ np.array([0.0, 0.0, -distance])
    return m


def camera_path(n_frames: int, distance: float = 4.0, yaw_span_deg: float = 10.0) -> list:
    """Light-field centre poses sweeping the yaw over +-yaw_span/2 (a camera path)."""
    if n_frames <= 1:
        return [light_field_centre(distance, 0.0)]
    return [light_field_centre(distance, -0.5 * yaw_span_deg + i * yaw_span_deg / (n_frames - 1))
            for i in range(n_frames)]


def round_to_bf16(x: np.ndarray) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even), as float32."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    b = (b + 0x7FFF + lsb) >> 16 << 16
    return (b.astype(np.uint32)).view(np.float32).reshape(np.shape(x))


def round_to_f16(x: np.ndarray) -> np.ndarray:
    return np.asarray(x, dtype=np.float32).astype(np.float16).astype(np.float32)


def quantise_storage(scene: dict, dtype: str) -> dict:
    """The scene as the renderer sees it after storing scale, rotation, opacity
    and SH in ``dtype`` (means stay FP32)."""
    if dtype == "f32":
        return dict(scene)
    rnd = round_to_bf16 if dtype == "bf16" else round_to_f16
    out = dict(scene)
    for k in ("log_scale", "rot_wxyz", "opacity_logit", "sh"):
        out[k] = rnd(scene[k])
    return out


def sample_subpixels(display: Display, n_random: int, windows: int = 4, window_px: int = 32,
                     seed: int = 1) -> np.ndarray:
    """Seeded sample of subpixel linear indices ((row*w + col)*3 + k), sorted.

    ``n_random`` uniformly drawn subpixels plus every subpixel of ``windows``
    square windows of ``window_px`` pixels (one centred, the rest random)."""
    rng = np.random.default_rng(seed)
    w, h = display.width, display.height
    total = 3 * w * h
    picks = [rng.integers(0, total, size=n_random)]
    for i in range(windows):
        wp = min(window_px, w, h)
        if i == 0:
            r0, c0 = (h - wp) // 2, (w - wp) // 2
        else:
            r0 = int(rng.integers(0, h - wp + 1))
            c0 = int(rng.integers(0, w - wp + 1))
        rr, cc, kk = np.meshgrid(np.arange(r0, r0 + wp), np.arange(c0, c0 + wp), np.arange(3),
                                 indexing="ij")
        picks.append(((rr * w + cc) * 3 + kk).ravel())
    return np.unique(np.concatenate(picks).astype(np.int64))
