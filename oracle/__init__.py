"""FP64 CPU oracle for the DirectL light-field renderer -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The renderer (``paper_2407_14053_gb300``) never
does, and shares no code with it.  The arithmetic lives in ``oracle.c`` (plain
C, double precision); this module only marshals numpy arrays through ctypes
and composes the C functions into whole-frame and sampled-subpixel results:

* ``E_std[x,y,k] = C_{V(x,3y+k)}(x, y)[k]`` -- the standard paradigm
  (Alg. 1 at native resolution: render every view, then interweave);
* ``E_dl[x,y,k]  = C_v(x', y')[k]`` with ``(v, x', y', k) = M_i(x, y, k)`` --
  DirectL (Sec. 5: the ray each subpixel is given by subpixel repurposing).

Parity status per function is listed in ``oracle.h``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_HDR = os.path.join(_HERE, "oracle.h")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` with gcc (C11, -O2, OpenMP)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class OrDisplay(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("num_views", ctypes.c_int32), ("p_w", ctypes.c_int32),
                ("pitch_lx", ctypes.c_double), ("tan_slant", ctypes.c_double),
                ("offset_k", ctypes.c_double), ("view_span_deg", ctypes.c_double),
                ("fov_x_deg", ctypes.c_double), ("repurpose", ctypes.c_int32),
                ("reverse_views", ctypes.c_int32), ("rig", ctypes.c_int32)]


class OrScene(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("sh_degree", ctypes.c_int32),
                ("mean", ctypes.c_void_p), ("log_scale", ctypes.c_void_p),
                ("rot_wxyz", ctypes.c_void_p), ("opacity_logit", ctypes.c_void_p),
                ("sh", ctypes.c_void_p)]


class OrSplat(ctypes.Structure):
    _fields_ = [("u", ctypes.c_double), ("v", ctypes.c_double),
                ("conic", ctypes.c_double * 3), ("cov2d", ctypes.c_double * 3),
                ("opacity", ctypes.c_double), ("rgb", ctypes.c_double * 3),
                ("depth", ctypes.c_double), ("valid", ctypes.c_int32)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            lib.or_quantise.argtypes = [P, P, P, P]
            lib.or_view_map.argtypes = [P, P]
            lib.or_area_map.argtypes = [P, P]
            lib.or_repurpose.argtypes = [P, P, P]
            lib.or_ray_table.argtypes = [P, P, P, P, P, P, P, P]
            lib.or_cameras.argtypes = [P, P, P, P]
            lib.or_sh_basis.argtypes = [P, P]
            lib.or_sh_basis.restype = None
            lib.or_project_splat.argtypes = [P, ctypes.c_int64, P, ctypes.c_double, ctypes.c_int32,
                                             ctypes.c_int32, P]
            lib.or_project_splat.restype = None
            lib.or_project_splat_shift.argtypes = [P, ctypes.c_int64, P, ctypes.c_double,
                                                   ctypes.c_double, ctypes.c_int32, ctypes.c_int32,
                                                   P]
            lib.or_project_splat_shift.restype = None
            lib.or_render_rays.argtypes = [P, P, P, ctypes.c_int64, P, P, P, P, P, P, P, P,
                                           ctypes.c_int]
            lib.or_interweave.argtypes = [P, P, P, P]
            lib.or_raycast_rays.argtypes = [P, P, P, ctypes.c_int64, P, P, P, ctypes.c_int32, P,
                                            P, P, P, ctypes.c_int]
            lib.or_max_threads.argtypes = []
            for f in ("or_quantise", "or_view_map", "or_area_map", "or_repurpose", "or_ray_table",
                      "or_cameras", "or_render_rays", "or_interweave", "or_max_threads",
                      "or_raycast_rays"):
                getattr(lib, f).restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def _disp(d) -> OrDisplay:
    return OrDisplay(int(d.width), int(d.height), int(d.num_views), int(d.p_w), float(d.pitch_lx),
                     float(d.tan_slant), float(d.offset_k), float(d.view_span_deg),
                     float(d.fov_x_deg), int(d.repurpose), int(d.reverse_views),
                     int(getattr(d, "rig", 0)))


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def max_threads() -> int:
    return int(_load().or_max_threads())


def quantise(display):
    """(T3, Lq, Kq): the Q32 display constants."""
    lib = _load()
    out = [ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()]
    d = _disp(display)
    _check(lib.or_quantise(ctypes.byref(d), *[ctypes.byref(o) for o in out]), "quantise")
    return tuple(int(o.value) for o in out)


def view_map(display) -> np.ndarray:
    """V, uint16 of shape (h, 3w) (Eqs. (1)-(3))."""
    lib = _load()
    V = np.empty((display.height, 3 * display.width), dtype=np.uint16)
    d = _disp(display)
    _check(lib.or_view_map(ctypes.byref(d), _ptr(V)), "view_map")
    return V


def area_map(display) -> np.ndarray:
    lib = _load()
    A = np.empty((display.height, 3 * display.width), dtype=np.int64)
    d = _disp(display)
    _check(lib.or_area_map(ctypes.byref(d), _ptr(A)), "area_map")
    return A


def repurpose(display, V: np.ndarray) -> np.ndarray:
    """M_i as packed source pixels, uint32 (h, w, 3): (x' << 16) | y'."""
    lib = _load()
    V = np.ascontiguousarray(V, dtype=np.uint16)
    src = np.empty((display.height, display.width, 3), dtype=np.uint32)
    d = _disp(display)
    _check(lib.or_repurpose(ctypes.byref(d), _ptr(V), _ptr(src)), "repurpose")
    return src


def ray_table(display, V: np.ndarray, src: np.ndarray):
    """(ray_of uint32 (h,w,3), rays int32 (n_rays, 3) = (view, row, col))."""
    lib = _load()
    n = 3 * display.width * display.height
    V = np.ascontiguousarray(V, dtype=np.uint16)
    src = np.ascontiguousarray(src, dtype=np.uint32)
    ray_of = np.empty((display.height, display.width, 3), dtype=np.uint32)
    rv = np.empty(n, dtype=np.int32)
    rr = np.empty(n, dtype=np.int32)
    rc = np.empty(n, dtype=np.int32)
    nr = ctypes.c_int64()
    d = _disp(display)
    _check(lib.or_ray_table(ctypes.byref(d), _ptr(V), _ptr(src), _ptr(ray_of), _ptr(rv), _ptr(rr),
                            _ptr(rc), ctypes.byref(nr)), "ray_table")
    k = int(nr.value)
    return ray_of, np.stack([rv[:k], rr[:k], rc[:k]], axis=1)


def cameras(display, L0: np.ndarray, with_shift: bool = False):
    """Camera-to-world poses of the views (N_v, 4, 4); with_shift also
    returns each view's principal-point shift along the columns (pixels)."""
    lib = _load()
    L0 = np.ascontiguousarray(L0, dtype=np.float64)
    out = np.empty((display.num_views, 4, 4), dtype=np.float64)
    shift = np.empty(display.num_views, dtype=np.float64)
    d = _disp(display)
    _check(lib.or_cameras(ctypes.byref(d), _ptr(L0), _ptr(out), _ptr(shift)), "cameras")
    return (out, shift) if with_shift else out


def sh_basis(direction) -> np.ndarray:
    lib = _load()
    dvec = np.ascontiguousarray(direction, dtype=np.float64)
    out = np.empty(16, dtype=np.float64)
    lib.or_sh_basis(_ptr(dvec), _ptr(out))
    return out


class Scene:
    """FP64 copy of a scene dict (as made by ``workloads.make_scene``)."""

    def __init__(self, scene: dict):
        self.arrays = {k: np.ascontiguousarray(scene[k], dtype=np.float64)
                       for k in ("mean", "log_scale", "rot_wxyz", "opacity_logit", "sh")}
        self.n = int(self.arrays["mean"].shape[0])
        self.sh_degree = int(scene["sh_degree"])
        a = self.arrays
        self.c = OrScene(self.n, self.sh_degree, a["mean"].ctypes.data, a["log_scale"].ctypes.data,
                         a["rot_wxyz"].ctypes.data, a["opacity_logit"].ctypes.data,
                         a["sh"].ctypes.data)


def focal(display) -> float:
    return 0.5 * display.width / np.tan(np.radians(0.5 * display.fov_x_deg))


def project(scene: Scene, g: int, c2w: np.ndarray, display, shift: float = 0.0) -> dict:
    """Gaussian g in one camera (principal point at (w/2 + shift, h/2))."""
    lib = _load()
    c2w = np.ascontiguousarray(c2w, dtype=np.float64)
    sp = OrSplat()
    lib.or_project_splat_shift(ctypes.byref(scene.c), int(g), _ptr(c2w), float(focal(display)),
                               float(shift), int(display.width), int(display.height),
                               ctypes.byref(sp))
    return {"u": sp.u, "v": sp.v, "conic": np.array(sp.conic[:]), "cov2d": np.array(sp.cov2d[:]),
            "opacity": sp.opacity, "rgb": np.array(sp.rgb[:]), "depth": sp.depth,
            "valid": bool(sp.valid)}


def render_rays(scene: Scene, display, L0: np.ndarray, rays: np.ndarray, n_threads: int = 0):
    """Colours of rays (n,3) = (view, row, col).  Returns dict of rgb, lo, hi
    (n,3) float64, flags (n,) and n_contrib (n,)."""
    lib = _load()
    rays = np.ascontiguousarray(rays, dtype=np.int32).reshape(-1, 3)
    n = rays.shape[0]
    rv = np.ascontiguousarray(rays[:, 0])
    rr = np.ascontiguousarray(rays[:, 1])
    rc = np.ascontiguousarray(rays[:, 2])
    rgb = np.zeros((n, 3))
    lo = np.zeros((n, 3))
    hi = np.zeros((n, 3))
    flags = np.zeros(n, dtype=np.int32)
    ncon = np.zeros(n, dtype=np.int64)
    L0 = np.ascontiguousarray(L0, dtype=np.float64)
    d = _disp(display)
    _check(lib.or_render_rays(ctypes.byref(scene.c), ctypes.byref(d), _ptr(L0), n, _ptr(rv),
                              _ptr(rr), _ptr(rc), _ptr(rgb), _ptr(lo), _ptr(hi), _ptr(flags),
                              _ptr(ncon), int(n_threads)), "render_rays")
    return {"rgb": rgb, "lo": lo, "hi": hi, "flags": flags, "n_contrib": ncon}


def interweave(display, V: np.ndarray, Mm: np.ndarray) -> np.ndarray:
    lib = _load()
    V = np.ascontiguousarray(V, dtype=np.uint16)
    Mm = np.ascontiguousarray(Mm, dtype=np.float64)
    Me = np.empty((display.height, display.width, 3))
    d = _disp(display)
    _check(lib.or_interweave(ctypes.byref(d), _ptr(V), _ptr(Mm), _ptr(Me)), "interweave")
    return Me


def subpixel_rays(display, subpixels: np.ndarray, V: np.ndarray, src: np.ndarray | None):
    """The ray (view, row, col) each listed subpixel shows.  ``src`` is the
    repurposing table for DirectL, ``None`` for the standard paradigm."""
    subpixels = np.asarray(subpixels, dtype=np.int64)
    w = display.width
    pix = subpixels // 3
    k = subpixels % 3
    x = pix // w
    y = pix % w
    v = V[x, 3 * y + k].astype(np.int32)
    if src is None:
        return np.stack([v, x.astype(np.int32), y.astype(np.int32)], axis=1)
    s = src.reshape(-1)[subpixels]
    return np.stack([v, (s >> 16).astype(np.int32), (s & 0xFFFF).astype(np.int32)], axis=1)


def render_subpixels(scene: Scene, display, L0: np.ndarray, subpixels: np.ndarray, V: np.ndarray,
                     src: np.ndarray | None, n_threads: int = 0) -> dict:
    """Per-subpixel colour of the standard (``src=None``) or DirectL frame at
    the listed subpixel indices; value/lo/hi are the channel each subpixel
    shows."""
    subpixels = np.asarray(subpixels, dtype=np.int64)
    rays = subpixel_rays(display, subpixels, V, src)
    uniq, inv = np.unique(rays, axis=0, return_inverse=True)
    inv = inv.reshape(-1)
    res = render_rays(scene, display, L0, uniq, n_threads=n_threads)
    k = subpixels % 3
    return {"value": res["rgb"][inv, k], "lo": res["lo"][inv, k], "hi": res["hi"][inv, k],
            "flags": res["flags"][inv], "n_rays": int(uniq.shape[0]),
            "n_contrib": res["n_contrib"][inv]}


def raycast_rays(scene: Scene, display, L0: np.ndarray, rays: np.ndarray, heap_cap: int = 128,
                 n_threads: int = 0) -> dict:
    """Ray-order 3DGS (Sec. 7, Alg. 3) colours of rays (n,3) = (view, row,
    col) with a heap of ``heap_cap`` intersections per ray; rgb, lo, hi (n,3)
    and flags as in ``render_rays``."""
    lib = _load()
    rays = np.ascontiguousarray(rays, dtype=np.int32).reshape(-1, 3)
    n = rays.shape[0]
    rv, rr, rc = (np.ascontiguousarray(rays[:, j]) for j in range(3))
    rgb, lo, hi = np.zeros((n, 3)), np.zeros((n, 3)), np.zeros((n, 3))
    flags = np.zeros(n, dtype=np.int32)
    L0 = np.ascontiguousarray(L0, dtype=np.float64)
    d = _disp(display)
    _check(lib.or_raycast_rays(ctypes.byref(scene.c), ctypes.byref(d), _ptr(L0), n, _ptr(rv),
                               _ptr(rr), _ptr(rc), int(heap_cap), _ptr(rgb), _ptr(lo), _ptr(hi),
                               _ptr(flags), int(n_threads)), "raycast_rays")
    return {"rgb": rgb, "lo": lo, "hi": hi, "flags": flags}


def raycast_subpixels(scene: Scene, display, L0: np.ndarray, subpixels: np.ndarray, V: np.ndarray,
                      src: np.ndarray | None, heap_cap: int = 128) -> dict:
    """Per-subpixel colour of the ray-order 3DGS frame (the rays of the
    DirectL assignment when ``src`` is given, else every subpixel's own
    pixel)."""
    subpixels = np.asarray(subpixels, dtype=np.int64)
    rays = subpixel_rays(display, subpixels, V, src)
    uniq, inv = np.unique(rays, axis=0, return_inverse=True)
    inv = inv.reshape(-1)
    res = raycast_rays(scene, display, L0, uniq, heap_cap)
    k = subpixels % 3
    return {"value": res["rgb"][inv, k], "lo": res["lo"][inv, k], "hi": res["hi"][inv, k],
            "flags": res["flags"][inv], "n_rays": int(uniq.shape[0])}


def bilinear_taps(n_out: int, n_in: int, pos: np.ndarray):
    """Taps of the standard paradigm's upsampling (Alg. 1, "Resize"): output
    index i of n_out samples the input of n_in at i * n_in / n_out (the pixel
    grids share the corner: pixel (r, c) samples image point (c, r) about the
    principal point in both).  Returns (i0, i1, frac): the two input indices,
    clamped at the border, and the weight of i1."""
    pos = np.asarray(pos, dtype=np.int64)
    num = pos * n_in
    i0 = num // n_out
    frac = (num - i0 * n_out).astype(np.float64) / n_out
    return np.minimum(i0, n_in - 1), np.minimum(i0 + 1, n_in - 1), frac


def render_subpixels_lowres(scene: Scene, display, L0: np.ndarray, subpixels: np.ndarray,
                            V: np.ndarray, view_w: int, view_h: int, n_threads: int = 0) -> dict:
    """Standard paradigm with every view rendered at view_w x view_h (same
    field of view, so f scales with the width) and upsampled bilinearly while
    interweaving: subpixel (x, y, k) takes channel k of view V(x, 3y + k) at
    column y view_w / w, row x view_h / h of that view."""
    subpixels = np.asarray(subpixels, dtype=np.int64)
    w = display.width
    row = subpixels // (3 * w)
    col = (subpixels % (3 * w)) // 3
    k = subpixels % 3
    v = V.reshape(-1)[subpixels].astype(np.int64)
    x0, x1, fx = bilinear_taps(w, view_w, col)
    y0, y1, fy = bilinear_taps(display.height, view_h, row)
    taps = [(y0, x0, (1 - fy) * (1 - fx)), (y0, x1, (1 - fy) * fx),
            (y1, x0, fy * (1 - fx)), (y1, x1, fy * fx)]
    rays = np.concatenate([np.stack([v, yy, xx], axis=1) for yy, xx, _ in taps])
    uniq, inv = np.unique(rays, axis=0, return_inverse=True)
    inv = inv.reshape(4, -1)
    small = display.replace(width=int(view_w), height=int(view_h))
    res = render_rays(scene, small, L0, uniq, n_threads=n_threads)
    out = {}
    for key, name in (("value", "rgb"), ("lo", "lo"), ("hi", "hi")):
        out[key] = sum(wt * res[name][inv[t], k] for t, (_, _, wt) in enumerate(taps))
    out["flags"] = np.bitwise_or.reduce(res["flags"][inv], axis=0)
    out["n_rays"] = int(uniq.shape[0])
    return out


def render_frame(scene: Scene, display, L0: np.ndarray, mode: str = "directl",
                 n_threads: int = 0) -> dict:
    """Whole encoded image (h, w, 3) for ``mode`` in {"directl", "standard"}."""
    V = view_map(display)
    src = repurpose(display, V) if mode == "directl" else None
    sub = np.arange(3 * display.width * display.height, dtype=np.int64)
    r = render_subpixels(scene, display, L0, sub, V, src, n_threads=n_threads)
    shape = (display.height, display.width, 3)
    return {"value": r["value"].reshape(shape), "lo": r["lo"].reshape(shape),
            "hi": r["hi"].reshape(shape), "flags": r["flags"].reshape(shape), "V": V, "src": src,
            "n_rays": r["n_rays"]}
