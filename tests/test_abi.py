"""The C ABI library builds, loads without a GPU and exports every entry
point include/directl.h declares; the ctypes structures match the C layout."""
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "directl.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2407_14053_gb300 import build, _binding
    build.build()
    return _binding.lib()


def _declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:dl_status|const char\*)\s+(dl_\w+)\s*\(", text, re.M)))


def test_header_declares_expected_calls():
    names = _declared()
    for must in ("dl_create", "dl_destroy", "dl_load_gaussians", "dl_set_display", "dl_render_frame",
                 "dl_get_view_map", "dl_get_subpixel_map", "dl_get_ray_table", "dl_query_footprint"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lib._name], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT\s+(dl_\w+)$", out, re.M))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2407_14053_gb300 import _binding
    assert sorted(_binding.SIGNATURES) == _declared()


def test_struct_layouts_match_c():
    from paper_2407_14053_gb300 import _binding as B
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "directl.h"
#define P(T, f) printf(#T "." #f " %zu\n", offsetof(T, f));
int main(void) {
  printf("dl_gaussians_desc %zu\n", sizeof(dl_gaussians_desc));
  printf("dl_display_params %zu\n", sizeof(dl_display_params));
  printf("dl_frame_stats %zu\n", sizeof(dl_frame_stats));
  P(dl_gaussians_desc, sh) P(dl_gaussians_desc, on_device) P(dl_display_params, pitch_lx)
  P(dl_display_params, repurpose) P(dl_display_params, reverse_views) P(dl_display_params, rig)
  P(dl_frame_stats, ms_total)
  P(dl_frame_stats, max_list) P(dl_frame_stats, lists_small) P(dl_frame_stats, n_visible)
  P(dl_frame_stats, status) P(dl_frame_stats, reemitted)
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        lines = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    got = dict(l.split() for l in lines if l)
    assert int(got["dl_gaussians_desc"]) == ctypes_size(B.dl_gaussians_desc)
    assert int(got["dl_display_params"]) == ctypes_size(B.dl_display_params)
    assert int(got["dl_frame_stats"]) == ctypes_size(B.dl_frame_stats)
    for key, val in got.items():
        if "." in key:
            t, f = key.split(".")
            assert getattr(getattr(B, t), f).offset == int(val), key


def ctypes_size(t):
    import ctypes
    return ctypes.sizeof(t)


def test_status_strings(lib):
    from paper_2407_14053_gb300 import _binding as B
    assert B.dl_status_string(0) == "DL_OK"
    assert B.dl_status_string(-7) == "DL_ERR_CAPACITY"


def test_peaks_without_gpu_fail_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2407_14053_gb300 import _binding as B
    with pytest.raises(B.DirectLError):
        B.dl_measure_peaks(0)


def test_create_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2407_14053_gb300 import _binding as B
    with pytest.raises(B.DirectLError):
        B.dl_create(0)
