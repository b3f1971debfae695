"""Continuous-batching light-field frame server over the batch API.

Requests (scene, display, head pose) arrive at any time.  The server keeps
scenes and displays resident on the device, least recently used first out,
within an HBM budget, and runs two batch lanes on two CUDA streams: while
one lane's launch is on the GPU, the requests that arrived meanwhile are
assigned to the other lane's free slots and launched, so their work overlaps
on the device.  A request is admitted when a slot is free and its scene and
display are resident or can be made resident within the budget.

Every frame is rendered by the kernels of ``Renderer.render`` (the batch
runs the same per-frame stages), so a result does not depend on which other
frames shared its launch.  The paper renders one frame at a time; this
module has no counterpart there."""
from __future__ import annotations

import collections
import dataclasses
import time
from typing import Callable, Dict, Hashable, List

import numpy as np


REJECTED_BUDGET = -2  # scene or display larger than the HBM budget
REJECTED_SLOT = -3    # frame beyond a slot's hard limits


@dataclasses.dataclass
class Request:
    rid: int
    scene: Hashable
    display: Hashable
    L0: np.ndarray            # 4x4 light-field centre pose
    arrival: float            # seconds from the start of the run
    admitted: float = float("nan")
    launched: float = float("nan")
    done: float = float("nan")
    status: int = -1          # batch status word (0 = ok); -1 = not run
    out: object = None        # device frame (h, w, 3), kept when asked to
    lane: int = -1
    fallback: bool = False    # rendered alone after a capacity overflow
    too_small: set = dataclasses.field(default_factory=set)  # slot indices that cannot hold it

    @property
    def latency(self) -> float:
        return self.done - self.arrival


class ResidencyCache:
    """Device-resident items (scenes, displays) within a byte budget.

    ``acquire(key)`` makes an item resident (loading it, evicting unpinned
    items least recently used first) and pins it; ``release(key)`` unpins.
    Returns False when the item cannot fit even after evicting everything
    unpinned."""

    def __init__(self, budget: int, reserved: int, load: Callable, unload: Callable,
                 size_of: Callable):
        self.budget = int(budget)
        self.reserved = int(reserved)
        self._load, self._unload, self._size_of = load, unload, size_of
        self.items: "collections.OrderedDict[Hashable, list]" = collections.OrderedDict()
        self.loads = 0
        self.evictions = 0

    @property
    def used(self) -> int:
        return self.reserved + sum(v[1] for v in self.items.values())

    def handle(self, key):
        return self.items[key][0]

    def acquire(self, key) -> bool:
        if key in self.items:
            self.items.move_to_end(key)
            self.items[key][2] += 1
            return True
        need = int(self._size_of(key))
        if self.reserved + need > self.budget:
            return False
        victims = []
        free = self.budget - self.used
        for k, (_, size, pins) in self.items.items():
            if free >= need:
                break
            if pins == 0:
                victims.append(k)
                free += size
        if free < need:
            return False
        for k in victims:
            h, _, _ = self.items.pop(k)
            self._unload(k, h)
            self.evictions += 1
        self.items[key] = [self._load(key), need, 1]
        self.loads += 1
        return True

    def fits(self, key) -> bool:
        """Whether the item could ever be resident (alone beside the reserve)."""
        return key in self.items or self.reserved + int(self._size_of(key)) <= self.budget

    def release(self, key) -> None:
        self.items[key][2] -= 1

    def clear(self) -> None:
        for k, (h, _, _) in list(self.items.items()):
            self._unload(k, h)
        self.items.clear()


def percentile(x, q: float) -> float:
    """Linear-interpolated percentile (numpy's default), NaN for no data."""
    x = np.asarray(x, dtype=np.float64)
    return float(np.percentile(x, q)) if x.size else float("nan")


def summarize(reqs: List[Request], launches: int, slots_used: int) -> dict:
    done = [r for r in reqs if r.status >= 0]
    rejected = sum(1 for r in reqs if r.status < -1)
    lat = [r.latency for r in done]
    t_first = min((r.arrival for r in reqs), default=0.0)
    t_last = max((r.done for r in done), default=0.0)
    span = max(t_last - t_first, 1e-9)
    classes = {}
    for key in sorted({r.display for r in done}, key=str):
        cl = [r for r in done if r.display == key]
        classes[str(key)] = {
            "frames": len(cl), "p50_ms": 1e3 * percentile([r.latency for r in cl], 50),
            "p99_ms": 1e3 * percentile([r.latency for r in cl], 99),
            "service_ms_mean": 1e3 * float(np.mean([r.done - r.launched for r in cl])),
            "fallbacks": sum(1 for r in cl if r.fallback)}
    return {"requests": len(reqs), "completed": len(done), "rejected": rejected,
            "per_display": classes,
            "failed": sum(1 for r in done if r.status != 0 and not r.fallback),
            "fallbacks": sum(1 for r in done if r.fallback),
            "p50_ms": 1e3 * percentile(lat, 50), "p99_ms": 1e3 * percentile(lat, 99),
            "mean_ms": 1e3 * float(np.mean(lat)) if lat else float("nan"),
            "frames_per_s": len(done) / span, "makespan_s": span, "launches": launches,
            "mean_frames_per_launch": slots_used / max(launches, 1)}


class Server:
    """Continuous batching over ``lanes`` batches with one slot per entry of
    ``slot_plans``.

    scenes: key -> (scene arrays as from ``workloads.make_scene``, storage
    dtype); displays: key -> display (fields of ``dl_display_params``).
    slot_plans: [(scene key, display key)], the frame that sizes each slot
    (the same in every lane; rendered at plan_pose, a 4x4 light-field centre),
    so slots of different sizes serve different request classes.  A request takes the first free slot that holds it;
    requests no slot can hold, or whose scene or display alone exceed the
    budget, are rejected (status REJECTED_SLOT / REJECTED_BUDGET).
    keep_outputs: True keeps every request's device frame in ``Request.out``;
    a set of request ids keeps those only."""

    def __init__(self, renderer, scenes: Dict, displays: Dict, slot_plans, plan_pose,
                 lanes: int = 2, hbm_budget: float = 150e9, margin: float = 1.3, tile=None,
                 keep_outputs=False):
        self.r = renderer
        self.scene_src, self.display_src = scenes, displays
        self.tile = tile
        self.keep_outputs = keep_outputs
        self.n_slots = len(slot_plans)
        # the plan frames' scenes and displays are resident while lanes are made
        sids = {k: renderer.load_gaussians(*scenes[k]) for k in {p[0] for p in slot_plans}}
        dids = {k: renderer.set_display(displays[k]) for k in {p[1] for p in slot_plans}}
        plans = [(sids[sk], dids[dk], tile, plan_pose) for sk, dk in slot_plans]
        self.lanes = []
        for li in range(lanes):
            b = renderer.batch(plans, margin)
            self.lanes.append({"batch": b, "stream": self._new_stream(), "event": None,
                               "slot_req": [None] * self.n_slots, "busy": False})
        reserved = sum(l["batch"].info()[0] for l in self.lanes)
        for sid in sids.values():
            renderer.free_scene(sid)
        for did in dids.values():
            renderer.free_display(did)

        def size_of(key):
            kind, k = key
            if kind == "scene":
                s, dt = scenes[k]
                per = 4 if dt == "f32" else 2
                n = s["mean"].shape[0]
                return n * (12 + per * (3 + 4 + 1 + s["sh"].shape[1] * 3))
            d = displays[k]
            px = d.width * d.height
            return px * (3 * 2 + 3 * 4 * 3 + 8 * 3)  # view map, ray tables, grouped rays

        def load(key):
            kind, k = key
            if kind == "scene":
                return renderer.load_gaussians(*scenes[k])
            return renderer.set_display(displays[k])

        def unload(key, h):
            (renderer.free_scene if key[0] == "scene" else renderer.free_display)(h)

        self.cache = ResidencyCache(int(hbm_budget), reserved, load, unload, size_of)
        self.launches = 0
        self.slots_used = 0
        self.rejected: List[Request] = []

    # -- device plumbing (torch streams, events and frame buffers) ---------
    def _new_stream(self):
        import torch
        return torch.cuda.Stream()

    def _on(self, stream):
        import torch
        return torch.cuda.stream(stream)

    def _record(self):
        import torch
        ev = torch.cuda.Event()
        ev.record()
        return ev

    def _frame_buffer(self, w: int, h: int):
        import torch
        return torch.empty((h, w, 3), dtype=torch.float32, device="cuda")

    # -- one lane ---------------------------------------------------------
    def _harvest(self, lane, now: float) -> None:
        b = lane["batch"]
        status = b.wait(raise_on_capacity=False)
        for s, req in enumerate(lane["slot_req"]):
            if req is None:
                continue
            req.status = int(status[s])
            if req.status != 0:  # over the slot's key or list capacity: render it alone
                with self._on(lane["stream"]):
                    self.r.render(self.cache.handle(("scene", req.scene)),
                                  self.cache.handle(("display", req.display)), req.L0, "directl",
                                  req.out)
                lane["stream"].synchronize()
                req.fallback = True
                now = self.clock()
            req.done = now
            b.clear(s)
            self.cache.release(("scene", req.scene))
            self.cache.release(("display", req.display))
            if not (self.keep_outputs is True or
                    (isinstance(self.keep_outputs, (set, frozenset)) and req.rid in self.keep_outputs)):
                req.out = None
            lane["slot_req"][s] = None
        lane["busy"] = False

    def _reject(self, req: Request, code: int, now: float) -> None:
        req.status = code
        req.done = now
        self.rejected.append(req)

    def _fill(self, lane, queue: "collections.deque", now: float, li: int) -> None:
        from ._binding import DL_ERR_CAPACITY, DirectLError
        b = lane["batch"]
        free = [s for s, q in enumerate(lane["slot_req"]) if q is None]
        skipped = collections.deque()
        while free and queue:
            req = queue.popleft()
            ks, kd = ("scene", req.scene), ("display", req.display)
            if not (self.cache.fits(ks) and self.cache.fits(kd)):
                self._reject(req, REJECTED_BUDGET, now)
                continue
            if not self.cache.acquire(ks):
                skipped.append(req)
                continue
            if not self.cache.acquire(kd):
                self.cache.release(ks)
                skipped.append(req)
                continue
            sid = self.cache.handle(ks)
            did = self.cache.handle(kd)
            w, h, _ = self.r.display_size(did)
            with self._on(lane["stream"]):
                req.out = self._frame_buffer(w, h)
            s = None
            for cand in free:  # the first free slot large enough
                if cand in req.too_small:
                    continue
                try:
                    b.assign(cand, sid, did, req.out, tile=self.tile)
                    s = cand
                    break
                except DirectLError as e:
                    if e.status != DL_ERR_CAPACITY:
                        raise
                    req.too_small.add(cand)
            if s is None:
                self.cache.release(ks)
                self.cache.release(kd)
                req.out = None
                if len(req.too_small) == self.n_slots:
                    self._reject(req, REJECTED_SLOT, now)
                else:
                    skipped.append(req)  # a larger slot is busy
                continue
            free.remove(s)
            b.set_pose(s, req.L0)
            req.admitted = now
            req.lane = li
            lane["slot_req"][s] = req
        queue.extendleft(reversed(skipped))
        n = sum(q is not None for q in lane["slot_req"])
        if n:
            with self._on(lane["stream"]):
                b.launch()
                lane["event"] = self._record()
            lane["busy"] = True
            t = self.clock()
            for q in lane["slot_req"]:
                if q is not None:
                    q.launched = t
            self.launches += 1
            self.slots_used += n

    # -- the loop ---------------------------------------------------------
    def run(self, requests: List[Request], poll_s: float = 50e-6) -> dict:
        """Serves the requests at their arrival times (seconds from now);
        returns the summary (p50/p99 latency, frames/s, ...)."""
        reqs = sorted(requests, key=lambda q: q.arrival)
        t0 = time.perf_counter()
        self.clock = lambda: time.perf_counter() - t0
        queue: "collections.deque" = collections.deque()
        i, n_done = 0, 0
        self.rejected = []
        while n_done + len(self.rejected) < len(reqs):
            now = self.clock()
            while i < len(reqs) and reqs[i].arrival <= now:
                queue.append(reqs[i])
                i += 1
            progressed = False
            for li, lane in enumerate(self.lanes):
                if lane["busy"] and lane["event"].query():
                    k = sum(q is not None for q in lane["slot_req"])
                    self._harvest(lane, self.clock())
                    n_done += k
                    progressed = True
                if not lane["busy"] and queue:
                    self._fill(lane, queue, self.clock(), li)
                    progressed = progressed or lane["busy"]
            if not progressed:
                if i < len(reqs) and not queue and not any(l["busy"] for l in self.lanes):
                    time.sleep(max(0.0, min(reqs[i].arrival - self.clock(), 0.005)))
                else:
                    time.sleep(poll_s)
        return summarize(reqs, self.launches, self.slots_used)

    def close(self) -> None:
        for lane in self.lanes:
            lane["batch"].close()
        self.cache.clear()


def poisson_arrivals(n: int, rate_per_s: float, seed: int = 0) -> np.ndarray:
    """Arrival times (s) of a Poisson process: cumulative exponential gaps."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=n))
