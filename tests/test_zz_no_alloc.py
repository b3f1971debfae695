"""The no-allocation ray table (dl_ray_table_static) against the ray table
dl_set_display builds.

dl_ray_table_static exists for callers that cannot call cudaMalloc (code
inside another library's memory pool, processes whose device memory is
reserved up front, real-time loops that must not synchronise the device):
it uses only a static device array of the library.  Its output must equal,
bit for bit like every integer table here, what dl_get_ray_table returns
for the same display, on consecutive calls that reuse the shared scratch."""
import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu

DISPLAYS = [
    W.WORKLOADS["tiny"].display,                                   # 240x135, 45 views
    W.Display(200, 120, 60, 5.3344, 0.1202, 1.2547, p_w=3),        # different size and params
]


def _device_tables(r, did, d):
    from paper_2407_14053_gb300 import _binding as B
    n = 3 * d.width * d.height
    stream = torch.cuda.current_stream().cuda_stream
    V = torch.empty(n, dtype=torch.int16, device="cuda")
    src = torch.empty(n, dtype=torch.int32, device="cuda")
    B.dl_get_view_map(r.ctx, did, V.data_ptr(), 1, stream)
    B.dl_get_subpixel_map(r.ctx, did, src.data_ptr(), 1, stream)
    return V, src


def _static_table(d, V, src):
    from paper_2407_14053_gb300 import _binding as B
    n = 3 * d.width * d.height
    ray_of = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    rays = torch.full((3 * n,), -7, dtype=torch.int32, device="cuda")
    nr = B.dl_ray_table_static(d.width, d.height, V.data_ptr(), src.data_ptr(), ray_of.data_ptr(),
                               rays.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    got_of = ray_of.cpu().numpy().view(np.uint32).reshape(d.height, d.width, 3)
    got_rays = rays.cpu().numpy()[:3 * nr].reshape(nr, 3)
    return got_of, got_rays


def test_static_ray_table_matches_set_display_on_consecutive_calls():
    from paper_2407_14053_gb300 import Renderer
    r = Renderer(0)
    try:
        for d in DISPLAYS + DISPLAYS[:1]:
            did = r.set_display(d)
            V, src = _device_tables(r, did, d)
            want_of, want_rays = r.ray_table(did)
            got_of, got_rays = _static_table(d, V, src)
            assert np.array_equal(got_of, want_of)
            assert np.array_equal(got_rays, want_rays)
            r.free_display(did)
    finally:
        r.close()


def test_static_ray_table_rejects_panels_over_the_limit():
    from paper_2407_14053_gb300 import DirectLError, _binding as B
    buf = torch.empty(16, dtype=torch.int32, device="cuda")
    with pytest.raises(DirectLError):
        B.dl_ray_table_static(257, 256, buf.data_ptr(), buf.data_ptr(), buf.data_ptr(),
                              buf.data_ptr(), 0)
    with pytest.raises(DirectLError):
        B.dl_ray_table_static(0, 10, buf.data_ptr(), buf.data_ptr(), buf.data_ptr(),
                              buf.data_ptr(), 0)
