"""GPU parity of the offline display tables, bit-exact against the oracle:
view-index map (Eqs. (1)-(3)), repurposed source pixels (Alg. 2) and the
R-first ray table, through the C ABI."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def renderer():
    from paper_2407_14053_gb300 import Renderer
    r = Renderer(0)
    yield r
    r.close()


def _check_tables(renderer, d):
    did = renderer.set_display(d)
    V = renderer.view_map(did)
    Vo = oracle.view_map(d)
    assert np.array_equal(V, Vo), f"view map: {int((V != Vo).sum())} subpixels differ"
    src = renderer.subpixel_map(did)
    so = oracle.repurpose(d, Vo)
    assert np.array_equal(src, so), f"repurposing: {int((src != so).sum())} subpixels differ"
    ray_of, rays = renderer.ray_table(did)
    ro, rays_o = oracle.ray_table(d, Vo, so)
    assert rays.shape == rays_o.shape
    assert np.array_equal(ray_of, ro)
    assert np.array_equal(rays, rays_o)
    n, beta = renderer.display_info(did)
    assert n == rays_o.shape[0] and abs(beta - n / (d.width * d.height)) < 1e-12
    renderer.free_display(did)


@pytest.mark.parametrize("name", ["tiny", "1080p", "4k", "8k"])
def test_workload_tables(renderer, name):
    _check_tables(renderer, W.WORKLOADS[name].display)


def test_serving_4k60_tables(renderer):
    # the serving mix's third panel: the 4K lens with 60 views
    _check_tables(renderer, W.WORKLOADS["4k"].display.replace(num_views=60))


@pytest.mark.parametrize("name", list(W.PAPER_PANELS))
def test_paper_panel_tables(renderer, name):
    _check_tables(renderer, W.PAPER_PANELS[name])


@pytest.mark.parametrize("kw", [
    dict(width=97, height=61, num_views=45, pitch_lx=5.3, tan_slant=-0.18, offset_k=2.7),
    dict(width=128, height=64, num_views=7, pitch_lx=21 / 4, tan_slant=1 / 6, offset_k=1.25, p_w=1),
    dict(width=160, height=90, num_views=60, pitch_lx=5.3344, tan_slant=0.12, offset_k=0.0, p_w=4),
    dict(width=64, height=48, num_views=1, pitch_lx=6.0, tan_slant=0.2, offset_k=0.0),
    dict(width=200, height=120, num_views=45, pitch_lx=8.1, tan_slant=0.18, offset_k=0.0, repurpose=0),
    dict(width=1, height=1, num_views=3, pitch_lx=3.0, tan_slant=0.0, offset_k=0.0),
    dict(width=333, height=7, num_views=100, pitch_lx=11.7, tan_slant=0.2, offset_k=-3.5, p_w=3),
    dict(width=96, height=64, num_views=5, pitch_lx=5.3, tan_slant=1 / 6, offset_k=0.0),
])
def test_edge_displays(renderer, kw):
    _check_tables(renderer, W.Display(**kw))


def test_encode_rays_is_the_ray_table_gather(renderer):
    # any per-ray renderer plugs in: per-ray colours -> encoded image by the
    # repurposing table (Sec. 4 step (3)), bit for bit
    import torch
    d = W.Display(160, 90, 45, 5.3, 1 / 6)
    did = renderer.set_display(d)
    ray_of, rays = renderer.ray_table(did)
    rng = np.random.default_rng(4)
    rgb = rng.uniform(-1, 2, size=(rays.shape[0], 3)).astype(np.float32)
    out = renderer.encode_rays(did, torch.as_tensor(rgb).cuda())
    torch.cuda.synchronize()
    k = np.arange(3)[None, None, :]
    assert np.array_equal(out.cpu().numpy(), rgb[ray_of, np.broadcast_to(k, ray_of.shape)])
    # a DirectL frame's subpixels regathered into ray colours re-encode to
    # the same frame
    scene = W.make_scene(W.SceneSpec(800, 1, "uniform", "f32", seed=3))
    sid = renderer.load_gaussians(scene, "f32")
    frame = renderer.render(sid, did, W.light_field_centre(4.0, 0.0), "directl")
    torch.cuda.synchronize()
    f = frame.cpu().numpy().reshape(-1)
    ray_rgb = np.zeros((rays.shape[0], 3), np.float32)
    ray_rgb[ray_of.reshape(-1), np.tile(np.arange(3), ray_of.size // 3)] = f
    again = renderer.encode_rays(did, torch.as_tensor(ray_rgb).cuda())
    torch.cuda.synchronize()
    assert np.array_equal(again.cpu().numpy().reshape(-1), f)
    renderer.free_scene(sid)
    renderer.free_display(did)
