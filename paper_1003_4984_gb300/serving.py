"""Continuous-batching lensing server on one GPU.

Requests (a contiguous RING target range of a resident map, with its spin,
stencil size K and deflections) are admitted while their device buffers fit
in an HBM budget that also counts the resident maps and plans (a request that
alone exceeds what is left runs when nothing else is admitted), then advanced
chunk by chunk: every scheduling round builds
a batch of chunks taken round-robin from all admitted requests (new arrivals
join the next round while earlier requests are still running) and runs it as
one persistent batched launch.  Two batch objects on two streams keep one
batch executing while the next is staged, so work from different requests
overlaps on the device.  Maps and plans (xi tables) stay resident between
requests.  Admission work (deflections produced by a callable, output
buffers) is queued on the caller's current stream, and each launch stream
waits for it before reading them.  Completion is detected on the host with
CUDA events; there is no device-side waiting.  A request can be cancelled
while pending or running: no further chunks of it are scheduled and its
memory returns once its chunks in flight have finished.

Results do not depend on how requests are mixed: each target is computed by
the same per-point code from the same inputs whatever batch carries it.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

from .api import Batch, LaunchCfg, Plan


@dataclass
class Request:
    rid: int
    map_key: tuple            # (nside, spin) of a registered map
    K: int
    first: int
    count: int
    defl: object              # device tensor (count, 2), or a callable producing it at admission
    arrival: float = 0.0      # seconds from the start of the run
    precision: str = "mixed"
    # filled in by the server
    out: object = None
    var: object = None
    done_points: int = 0
    next_point: int = 0
    admitted_at: float | None = None
    finished_at: float | None = None
    nbytes: int = 0
    cancelled: bool = False
    scheduled_points: int = 0

    @property
    def latency(self) -> float | None:
        return None if self.finished_at is None else self.finished_at - self.arrival


@dataclass
class _InFlight:
    event: object
    chunks: list = field(default_factory=list)  # (request, n_points)


class LensServer:
    def __init__(self, hbm_budget: float = 150e9, batch_points: int = 1 << 22, chunk_points: int = 1 << 21,
                 max_jobs: int = 64, cfg: LaunchCfg | None = None, device: int = 0):
        import torch

        if int(batch_points) < 2 or int(chunk_points) < 2 or int(max_jobs) < 1:
            raise ValueError("batch_points and chunk_points must be at least 2, max_jobs at least 1")
        self.torch = torch
        self.dev = torch.device("cuda", device)
        self.budget = float(hbm_budget)
        self.batch_points = int(batch_points)
        self.chunk_points = int(chunk_points)
        self.max_jobs = int(max_jobs)
        self.cfg = cfg
        self.maps: dict = {}
        self.spectra: dict = {}
        self.plans: dict = {}
        self.in_use = 0          # device bytes of the admitted requests' buffers
        self.resident = 0        # device bytes of the resident maps and plans
        self.pending: collections.deque = collections.deque()
        self.active: list = []
        self.finished: list = []
        self.cancelled: list = []
        self.streams = [torch.cuda.Stream(self.dev), torch.cuda.Stream(self.dev)]
        self.batches = [Batch(max_jobs), Batch(max_jobs)]
        self.inflight: list = [None, None]
        self.turn = 0
        self.launches = 0

    # ------------------------------------------------------------ residency
    def register_map(self, nside: int, spin: int, tensor, cl, cl_bb=None):
        """Keep an unlensed map and its spectrum resident on the device (counted
        against the HBM budget).  The batched launch serves spin-0 and spin-2 maps."""
        if spin not in (0, 2):
            raise ValueError(f"map ({nside}, {spin}): the server lenses spin-0 and spin-2 maps")
        key = (nside, spin)
        if key in self.maps:
            self.resident -= self.maps[key].numel() * self.maps[key].element_size()
        self.maps[key] = tensor
        self.spectra[key] = (cl, cl_bb)
        self.resident += tensor.numel() * tensor.element_size()

    def plan_for(self, req: Request) -> Plan:
        key = (*req.map_key, req.K, req.precision)
        if key not in self.plans:
            cl, bb = self.spectra[req.map_key]
            nside, spin = req.map_key
            self.plans[key] = Plan(nside, cl, bb, spin=spin, K=req.K, precision=req.precision)
            self.resident += self.plans[key].device_bytes()
            if self.cfg is not None:
                self.plans[key].set_launch(self.cfg)
        return self.plans[key]

    def used_bytes(self) -> int:
        """Device bytes counted against the budget: resident maps and plans plus the
        buffers of the admitted requests."""
        return self.resident + self.in_use

    @staticmethod
    def request_bytes(req: Request) -> int:
        spin = req.map_key[1]
        return req.count * (16 + (8 if spin == 0 else 16) + 8)

    # ------------------------------------------------------------ admission
    def check(self, req: Request):
        """Raise ValueError unless the request's map is registered, its range lies inside
        it, its stencil size and precision are ones the library plans, and its
        deflections (unless a callable makes them at admission) have one row per target."""
        if req.map_key not in self.maps:
            raise ValueError(f"request {req.rid}: no map registered for {req.map_key}")
        npix = 12 * req.map_key[0] * req.map_key[0]
        if req.count < 0 or req.first < 0 or req.first + req.count > npix:
            raise ValueError(f"request {req.rid}: target range [{req.first}, {req.first + req.count}) "
                             f"outside the map's {npix} pixels")
        if req.K not in (16, 24, 32, 48):
            raise ValueError(f"request {req.rid}: K must be 16, 24, 32 or 48 (got {req.K})")
        if req.precision not in ("fp64", "mixed"):
            raise ValueError(f"request {req.rid}: precision must be 'fp64' or 'mixed'")
        if req.defl is None:
            raise ValueError(f"request {req.rid}: no deflections")
        if not callable(req.defl) and tuple(req.defl.shape) != (req.count, 2):
            raise ValueError(f"request {req.rid}: deflections of shape {tuple(req.defl.shape)}, "
                             f"expected ({req.count}, 2)")

    def submit(self, req: Request):
        """Queue a request (checked first)."""
        self.check(req)
        self.pending.append(req)

    def cancel(self, rid: int) -> bool:
        """Cancel request ``rid``: a pending one is dropped, an admitted one gets no
        further chunks and returns its memory when its chunks in flight finish.
        Returns False if the request is unknown or already finished."""
        for req in list(self.pending):
            if req.rid == rid:
                self.pending.remove(req)
                req.cancelled = True
                self.cancelled.append(req)
                return True
        for req in self.active:
            if req.rid == rid and not req.cancelled:
                req.cancelled = True
                req.next_point = req.count  # nothing more is scheduled
                if req.done_points == req.scheduled_points:
                    self._release(req)
                return True
        return False

    def _release(self, req: Request):
        self.active.remove(req)
        self.in_use -= req.nbytes
        (self.cancelled if req.cancelled else self.finished).append(req)

    def _admit(self, now: float):
        torch = self.torch
        while self.pending:
            req = self.pending[0]
            nb = self.request_bytes(req)
            self.plan_for(req)  # its tables stay resident and count against the budget
            if self.used_bytes() + nb > self.budget and self.active:
                break  # wait for memory to free up (an oversized request runs alone)
            self.pending.popleft()
            spin = req.map_key[1]
            if callable(req.defl):
                req.defl = req.defl()
            req.out = torch.empty((req.count,) if spin == 0 else (req.count, 2), dtype=torch.float64,
                                  device=self.dev)
            req.var = torch.empty(req.count, dtype=torch.float64, device=self.dev)
            req.nbytes = nb
            req.admitted_at = now
            self.in_use += nb
            self.active.append(req)
            if req.count == 0:  # nothing to lens: done at admission
                req.finished_at = now
                self._release(req)

    # ------------------------------------------------------------ scheduling
    def _build_jobs(self):
        jobs, chunks, budget = [], [], self.batch_points
        progressed = True
        while budget > 0 and len(jobs) < self.max_jobs and progressed:
            progressed = False
            for req in self.active:
                if budget <= 0 or len(jobs) >= self.max_jobs:
                    break
                left = req.count - req.next_point
                if left <= 0:
                    continue
                n = min(left, self.chunk_points, budget)
                if n < left:
                    n &= ~1  # keep the next chunk's outputs on 16-byte boundaries
                    if n == 0:
                        # one point of room left in a batch that already holds work (the
                        # sizes are at least 2): the next batch takes an even chunk
                        continue
                a = req.next_point
                req.scheduled_points = a + n
                jobs.append((self.plan_for(req), req.first + a, n, self.maps[req.map_key], req.defl[a:a + n],
                             req.out[a:a + n], req.var[a:a + n], None))
                chunks.append((req, n))
                req.next_point += n
                budget -= n
                progressed = True
        return jobs, chunks

    def _launch(self, slot: int):
        jobs, chunks = self._build_jobs()
        if not jobs:
            return False
        b, s = self.batches[slot], self.streams[slot]
        # the admission work (deflections from a callable, output buffers) was queued on the
        # current stream: the launch stream waits for it, and the caching allocator is told
        # that these buffers are in use on the launch stream
        s.wait_stream(self.torch.cuda.current_stream(self.dev))
        for req, _ in chunks:
            for t in (req.defl, req.out, req.var):
                t.record_stream(s)
        b.stage(jobs, self.cfg.tile_points if self.cfg else 0)
        b.launch(self.cfg, stream=s)
        ev = self.torch.cuda.Event()
        ev.record(s)
        self.inflight[slot] = _InFlight(ev, chunks)
        self.launches += 1
        return True

    def _retire(self, slot: int, now_fn):
        f = self.inflight[slot]
        if f is None or not f.event.query():
            return False
        now = now_fn()
        for req, n in f.chunks:
            req.done_points += n
            if req.done_points == req.count:
                req.finished_at = now
                self._release(req)
            elif req.cancelled and req.done_points == req.scheduled_points:
                req.finished_at = now
                self._release(req)
        self.inflight[slot] = None
        return True

    # ------------------------------------------------------------ main loop
    def run(self, requests, time_scale: float = 1.0, idle_sleep: float = 2e-4, on_tick=None):
        """Serve ``requests`` (sorted by arrival time, seconds) in real time.

        ``on_tick(server, now)``, if given, is called once per scheduling round (a
        caller can cancel requests from it).  Returns the finished requests (the
        cancelled ones are in ``self.cancelled``); latency = completion - arrival."""
        t0 = time.perf_counter()

        def now():
            return (time.perf_counter() - t0) / time_scale

        for r in requests:  # every request is checked before anything runs
            self.check(r)
        todo = collections.deque(sorted(requests, key=lambda r: r.arrival))
        while todo or self.pending or self.active or any(self.inflight):
            t = now()
            while todo and todo[0].arrival <= t:
                self.submit(todo.popleft())
            if on_tick is not None:
                on_tick(self, t)
            self._admit(t)
            busy = False
            for slot in (0, 1):
                busy |= self._retire(slot, now)
            for _ in range(2):
                slot = self.turn
                if self.inflight[slot] is None:
                    if self._launch(slot):
                        busy = True
                    self.turn ^= 1
            if not busy:
                time.sleep(idle_sleep)
        return self.finished

    def close(self):
        for b in self.batches:
            b.close()
        for p in self.plans.values():
            p.close()


def latency_stats(finished) -> dict:
    """p50/p99/mean/max latency (ms) and served points per second of finished requests
    (latency = completion - arrival; rate over the span from the first arrival to the
    last completion).  With no finished request the statistics are None."""
    import numpy as np

    if not finished:
        return {"requests": 0, "p50_ms": None, "p99_ms": None, "mean_ms": None, "max_ms": None, "points": 0,
                "points_per_s": None, "span_s": None}
    lat = np.array([r.latency for r in finished]) * 1e3
    pts = sum(r.count for r in finished)
    span = max(r.finished_at for r in finished) - min(r.arrival for r in finished)
    return {"requests": len(finished), "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()), "max_ms": float(lat.max()),
            "points": int(pts), "points_per_s": pts / span, "span_s": span}
