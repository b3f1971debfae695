"""Host logic of the frame server, without a GPU: the HBM residency cache
(least recently used eviction, pins, budget), the latency summary and the
Poisson arrival generator."""
import numpy as np
import pytest

from paper_2407_14053_gb300.serving import (REJECTED_BUDGET, Request, ResidencyCache, percentile,
                                            poisson_arrivals, summarize)


def _cache(budget, reserved, sizes):
    log = []
    c = ResidencyCache(budget, reserved, load=lambda k: log.append(("load", k)) or f"h{k}",
                       unload=lambda k, h: log.append(("unload", k)), size_of=lambda k: sizes[k])
    return c, log


def test_lru_eviction_and_pins():
    c, log = _cache(100, 10, {"a": 40, "b": 40, "c": 40, "big": 95})
    assert c.acquire("a") and c.acquire("b")
    assert c.used == 90
    assert not c.acquire("c")          # a and b pinned: nothing can go
    c.release("a")
    assert c.acquire("c")              # a (unpinned, least recent) is evicted
    assert ("unload", "a") in log and "a" not in c.items
    c.release("b")
    c.release("c")
    assert c.acquire("b")              # b resident: a hit, now most recent
    assert list(c.items) == ["c", "b"]
    assert c.acquire("a")              # evicts c (least recent unpinned), not b
    assert list(c.items) == ["b", "a"] and c.evictions == 2
    assert not c.fits("big") and not c.acquire("big")
    assert c.handle("a") == "ha"
    c.clear()
    assert c.used == 10


def test_eviction_takes_only_what_is_needed():
    c, _ = _cache(100, 0, {"a": 30, "b": 30, "c": 30, "d": 50})
    for k in "abc":
        assert c.acquire(k)
        c.release(k)
    assert c.acquire("d")              # needs 50 with 10 free: evicts a and b only
    assert list(c.items) == ["c", "d"]


def test_percentile_and_summary():
    assert percentile([], 50) != percentile([], 50)  # NaN
    assert percentile([1, 2, 3, 4], 50) == 2.5
    assert percentile(list(range(101)), 99) == pytest.approx(99.0)
    reqs = [Request(i, "s", "d", np.eye(4), arrival=0.1 * i) for i in range(10)]
    for i, r in enumerate(reqs):
        r.status, r.done = 0, r.arrival + 0.01 * (i + 1)
    reqs[-1].status = REJECTED_BUDGET
    s = summarize(reqs, launches=3, slots_used=9)
    assert s["completed"] == 9 and s["rejected"] == 1
    assert s["p50_ms"] == pytest.approx(50.0) and s["mean_frames_per_launch"] == 3.0
    assert s["frames_per_s"] == pytest.approx(9 / (0.8 + 0.09))


def test_poisson_arrivals():
    t = poisson_arrivals(20000, 250.0, seed=3)
    assert np.all(np.diff(t) > 0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() - 1 / 250.0) < 0.03 / 250.0 * 3
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.05  # exponential: CV = 1


# ---- the serving loop against a fake renderer (no GPU) -------------------
class _FakeEvent:
    def __init__(self, t):
        self.t = t

    def query(self):
        import time
        return time.perf_counter() >= self.t


class _FakeBatch:
    """Slots sized by a plan (views, Gaussians, pixels); a launch 'renders'
    each assigned slot by writing a value that identifies the frame, and
    completes 2 ms later."""

    def __init__(self, r, plans):
        self.r = r
        self.caps = [(r.displays[did][2], r.scenes[sid], r.displays[did][0] * r.displays[did][1])
                     for sid, did, _, _ in plans]
        self.slots = [None] * len(plans)
        self.poses = [None] * len(plans)
        self.launched = []

    def info(self):
        return 1000, 2048

    def assign(self, slot, sid, did, out, tile=None):
        from paper_2407_14053_gb300 import DL_ERR_CAPACITY, DirectLError
        w, h, nv = self.r.displays[did]
        cap = self.caps[slot]
        if nv > cap[0] or self.r.scenes[sid] > cap[1] or w * h > cap[2]:
            raise DirectLError("dl_batch_assign", DL_ERR_CAPACITY, "slot limits")
        self.slots[slot] = (sid, did, out)

    def clear(self, slot):
        self.slots[slot] = None

    def set_pose(self, slot, L0):
        self.poses[slot] = float(np.asarray(L0)[0, 3])

    def launch(self):
        for s, a in enumerate(self.slots):
            if a is not None:
                a[2][...] = self.r.frame_value(a[0], a[1], self.poses[s])
        self.launched.append(sum(a is not None for a in self.slots))

    def wait(self, raise_on_capacity=True):
        return [0] * len(self.slots)

    def close(self):
        pass


class _FakeRenderer:
    def __init__(self):
        self.scenes, self.displays, self.next = {}, {}, 1
        self.names = {}

    def _id(self):
        self.next += 1
        return self.next

    def load_gaussians(self, scene, dtype):
        i = self._id()
        self.scenes[i] = scene["mean"].shape[0]
        self.names[i] = scene["name"]
        return i

    def set_display(self, d):
        i = self._id()
        self.displays[i] = (d.width, d.height, d.num_views)
        self.names[i] = (d.width, d.height, d.num_views)
        return i

    def free_scene(self, i):
        del self.scenes[i]

    def free_display(self, i):
        del self.displays[i]

    def display_size(self, i):
        return self.displays[i]

    def batch(self, plans, margin):
        return _FakeBatch(self, plans)

    def frame_value(self, sid, did, pose_x):
        return hash((self.names[sid], self.names[did], round(pose_x, 9))) % 1000003

    def render(self, sid, did, L0, mode, out):
        out[...] = self.frame_value(sid, did, float(np.asarray(L0)[0, 3]))


def _fake_server(slot_plans=(("c", "d45"),) * 3, lanes=2, budget=1e12):
    import contextlib
    import time
    from paper_2407_14053_gb300.serving import Server

    class FakeServer(Server):
        def _new_stream(self):
            return None

        def _on(self, stream):
            return contextlib.nullcontext()

        def _record(self):
            return _FakeEvent(time.perf_counter() + 0.002)

        def _frame_buffer(self, w, h):
            return np.zeros((h, w, 3))

    scenes = {k: ({"mean": np.zeros((n, 3)), "sh": np.zeros((n, 16, 3)), "name": k}, "bf16")
              for k, n in (("a", 2000), ("b", 3000), ("c", 2500), ("huge", 4000))}

    class D:
        def __init__(self, w, h, v):
            self.width, self.height, self.num_views = w, h, v

    displays = {"d45": D(24, 14, 45), "d60": D(16, 9, 60), "big": D(48, 27, 45)}
    r = _FakeRenderer()
    srv = FakeServer(r, scenes, displays, list(slot_plans), np.eye(4), lanes=lanes,
                     hbm_budget=budget, keep_outputs=True)
    return srv, r, scenes, displays


def test_server_loop_serves_every_request_once():
    from paper_2407_14053_gb300.serving import REJECTED_SLOT, Request
    srv, r, scenes, displays = _fake_server()
    rng = np.random.default_rng(0)
    reqs = []
    for i in range(40):
        L0 = np.eye(4)
        L0[0, 3] = rng.uniform(-1, 1)
        reqs.append(Request(i, ["a", "b", "c", "huge"][i % 4], ["d45", "d60", "big"][i % 3], L0,
                            float(rng.uniform(0, 0.03))))
    summary = srv.run(reqs)
    ok = [q for q in reqs if q.status == 0]
    rejected = [q for q in reqs if q.status == REJECTED_SLOT]
    # scenes above c's 2500 Gaussians, 60-view and big displays exceed the
    # slots sized for (c, d45)
    expect_ok = [q for q in reqs if q.scene in ("a", "c") and q.display == "d45"]
    assert sorted(q.rid for q in ok) == sorted(q.rid for q in expect_ok)
    assert len(ok) + len(rejected) == 40
    assert summary["completed"] == len(ok) and summary["rejected"] == len(rejected)
    for q in ok:
        sid = [k for k, v in r.names.items() if v == q.scene]
        assert q.out.flat[0] == hash((q.scene, (24, 14, 45), round(float(q.L0[0, 3]), 9))) % 1000003
        assert q.launched >= q.admitted >= q.arrival and q.done >= q.launched
    assert summary["launches"] >= 1 and summary["mean_frames_per_launch"] >= 1.0


def test_server_loop_under_a_one_scene_budget():
    from paper_2407_14053_gb300.serving import Request
    srv, r, scenes, displays = _fake_server(slot_plans=(("c", "d45"),) * 2, lanes=2)
    d_bytes = srv.cache._size_of(("display", "d45"))
    s_max = max(srv.cache._size_of(("scene", k)) for k in ("a", "b", "c"))
    srv.cache.budget = srv.cache.reserved + d_bytes + s_max
    reqs = [Request(i, "ac"[i % 2], "d45", np.eye(4), 0.001 * i) for i in range(15)]
    summary = srv.run(reqs)
    assert summary["completed"] == 15 and summary["rejected"] == 0
    assert srv.cache.evictions > 0 and len(srv.cache.items) <= 2


def test_heterogeneous_slots_route_requests_by_size():
    from paper_2407_14053_gb300.serving import REJECTED_SLOT, Request
    # slot 0 holds (huge, d45); slot 1 holds 60-view frames of up to b's size
    srv, r, scenes, displays = _fake_server(slot_plans=(("huge", "d45"), ("b", "d60")), lanes=2)
    reqs = [Request(i, k, d, np.eye(4), 0.0005 * i)
            for i, (k, d) in enumerate([("huge", "d45"), ("a", "d60"), ("b", "d45"),
                                        ("huge", "d60"), ("c", "d60"), ("a", "big")] * 3)]
    summary = srv.run(reqs)
    for q in reqs:
        fits = (q.display == "d45") or (q.display == "d60" and q.scene != "huge")
        assert (q.status == 0) == fits and (q.status == REJECTED_SLOT) == (not fits), q
    assert summary["completed"] == 12 and summary["rejected"] == 6
