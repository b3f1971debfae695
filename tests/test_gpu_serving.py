"""The continuous-batching server on the GPU: every served frame equals the
same frame rendered alone (bit for bit: the batch runs the same kernels),
whatever else shared its launch, including under an HBM budget that forces
scenes to be evicted and reloaded; requests that cannot fit are rejected."""
import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu


def _sources():
    scenes = {
        "uniform": (W.make_scene(W.SceneSpec(2000, 0, "uniform", "f32", seed=0)), "f32"),
        "clustered_bf16": (W.make_scene(W.SceneSpec(3000, 3, "clustered", "bf16", seed=5)), "bf16"),
        "clustered_f16": (W.make_scene(W.SceneSpec(2500, 3, "clustered", "f16", seed=6)), "f16"),
    }
    displays = {
        "tiny45": W.Display(240, 135, 45, 5.3, 1 / 6),
        "wide60": W.Display(160, 90, 60, 5.3344, 0.12, p_w=4),
    }
    return scenes, displays


def _requests(scenes, displays, n, seed, spread_s):
    from paper_2407_14053_gb300.serving import Request
    rng = np.random.default_rng(seed)
    sk, dk = sorted(scenes), sorted(displays)
    arrivals = np.sort(rng.uniform(0.0, spread_s, size=n))
    return [Request(i, sk[rng.integers(len(sk))], dk[rng.integers(len(dk))],
                    W.light_field_centre(4.0, float(rng.uniform(-5, 5))), float(arrivals[i]))
            for i in range(n)]


def _alone(r, scenes, displays, req):
    sid = r.load_gaussians(*scenes[req.scene])
    did = r.set_display(displays[req.display])
    out = r.render(sid, did, req.L0, "directl")
    torch.cuda.synchronize()
    img = out.cpu().numpy()
    r.free_scene(sid)
    r.free_display(did)
    return img


@pytest.mark.parametrize("budget_scenes", [3, 1])
def test_served_frames_equal_frames_rendered_alone(budget_scenes):
    from paper_2407_14053_gb300 import Renderer
    from paper_2407_14053_gb300.serving import Server
    scenes, displays = _sources()
    r = Renderer(0)
    try:
        plans = [("clustered_bf16", "tiny45"), ("clustered_bf16", "wide60"),
                 ("clustered_bf16", "tiny45")]
        srv = Server(r, scenes, displays, plans, W.light_field_centre(4.0, 0.0), lanes=2,
                     hbm_budget=1e12, margin=2.0, keep_outputs=True)
        if budget_scenes == 1:  # room for the lanes, both displays and one scene
            d_bytes = sum(srv.cache._size_of(("display", k)) for k in displays)
            s_max = max(srv.cache._size_of(("scene", k)) for k in scenes)
            srv.cache.budget = srv.cache.reserved + d_bytes + s_max
        reqs = _requests(scenes, displays, 18, seed=budget_scenes, spread_s=0.02)
        summary = srv.run(reqs)
        assert summary["completed"] == 18 and summary["rejected"] == 0
        assert summary["p99_ms"] >= summary["p50_ms"] > 0
        assert summary["mean_frames_per_launch"] > 1.0  # requests shared launches
        if budget_scenes == 1:
            assert srv.cache.evictions > 0
        outs = [(q, q.out.cpu().numpy()) for q in reqs]
        srv.close()
        for q, img in outs:
            assert q.status == 0
            assert np.array_equal(img, _alone(r, scenes, displays, q)), f"request {q.rid}"
    finally:
        r.close()


def test_requests_that_cannot_fit_are_rejected():
    from paper_2407_14053_gb300 import Renderer
    from paper_2407_14053_gb300.serving import REJECTED_BUDGET, REJECTED_SLOT, Request, Server
    scenes, displays = _sources()
    displays["big"] = W.Display(480, 270, 45, 5.3, 1 / 6)
    r = Renderer(0)
    try:
        srv = Server(r, scenes, displays, [("clustered_bf16", "tiny45")] * 2,
                     W.light_field_centre(4.0, 0.0), lanes=1, hbm_budget=1e12, margin=2.0)
        L0 = W.light_field_centre(4.0, 0.0)
        reqs = [Request(0, "uniform", "big", L0, 0.0),        # more rays than a slot holds
                Request(1, "uniform", "wide60", L0, 0.0),     # 60 views > the slot's 45
                Request(2, "uniform", "tiny45", L0, 0.001)]
        summary = srv.run(reqs)
        assert [q.status for q in reqs] == [REJECTED_SLOT, REJECTED_SLOT, 0]
        assert summary["completed"] == 1 and summary["rejected"] == 2
        srv.cache.budget = srv.cache.reserved + 10  # nothing fits any more
        q = Request(3, "clustered_f16", "tiny45", L0, 0.0)
        srv.run([q])
        assert q.status == REJECTED_BUDGET
        srv.close()
    finally:
        r.close()
