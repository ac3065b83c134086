"""Host logic of the continuous-batching server (paper_1003_4984_gb300.serving) on
the CPU: the server runs unchanged, with stand-ins for the CUDA pieces it
touches (streams, events, the batched launch, plans, device buffers).  The
stand-in launch "lenses" a target by a fixed function of its map value and
deflection and counts how often each output is written, so the tests see
which targets each launch received.  An event reports completion on its
second or fourth poll, so every launch stays in flight for at least one
scheduling round and the two batch slots do not finish together.

Covered: every target of every request lensed exactly once with the right
map, deflection and output slices, in launches shared by several requests;
admission that waits on the HBM budget (resident maps and plans counted);
a request larger than the remaining budget served alone; cancellation of
pending and running requests and the return of their memory; empty and
invalid requests; stream ordering (each launch stream waits for the
admission stream, buffers recorded on it); deflections produced at
admission."""
import numpy as np
import pytest

from paper_1003_4984_gb300 import serving
from paper_1003_4984_gb300.serving import LensServer, Request, latency_stats

pytestmark = pytest.mark.timeout(30)  # a scheduling loop that never ends fails here

PLAN_BYTES = 4096


class FakeTensor(np.ndarray):
    """numpy array with the few tensor methods the server calls."""

    def record_stream(self, s):
        s.recorded += 1

    def numel(self):
        return self.size

    def element_size(self):
        return self.itemsize


def fake(a):
    return np.asarray(a, dtype=np.float64).view(FakeTensor)


class FakeStream:
    def __init__(self, *args):
        self.waits = 0
        self.recorded = 0

    def wait_stream(self, other):
        assert isinstance(other, FakeStream)
        self.waits += 1


class FakeEvent:
    """Completes on its second or, for every other event, its fourth poll, so that the
    two batch slots fall out of step and one relaunches while the other is busy."""
    made = 0

    def __init__(self):
        FakeEvent.made += 1
        self.need = 2 if FakeEvent.made % 2 else 4
        self.polls = 0
        self.stream = None

    def record(self, s):
        self.stream = s

    def query(self):
        self.polls += 1
        return self.polls >= self.need


class FakeCuda:
    Event = FakeEvent

    def __init__(self):
        self.stream = FakeStream()

    def current_stream(self, dev=None):
        return self.stream


class FakeTorch:
    float64 = np.float64

    def __init__(self):
        self.cuda = FakeCuda()
        self.allocated = 0

    def empty(self, shape, dtype=None, device=None):
        self.allocated += 1
        return fake(np.full(shape, np.nan))


class FakePlan:
    made = []

    def __init__(self, nside, cl, cl_bb=None, spin=0, K=32, precision="mixed"):
        self.key = (nside, spin, K, precision)
        self.closed = False
        FakePlan.made.append(self)

    def device_bytes(self):
        return PLAN_BYTES

    def set_launch(self, cfg):
        self.cfg = cfg

    def close(self):
        self.closed = True


class FakeBatch:
    """Runs the staged jobs at launch: out = map[target] + deflection (spin 0: its
    first component), var counts the writes of each target."""
    launches = []

    def __init__(self, max_jobs):
        self.max_jobs = max_jobs
        self.jobs = None

    def stage(self, jobs, tile_points=0):
        assert 0 < len(jobs) <= self.max_jobs
        self.jobs = list(jobs)

    def launch(self, cfg=None, stream=None):
        assert isinstance(stream, FakeStream)
        rec = []
        for plan, first, n, m, d, o, v, s in self.jobs:
            assert d.shape == (n, 2) and o.shape[0] == n and v.shape == (n,)
            idx = first + np.arange(n)
            o[...] = (m[idx] + d[:, 0]) if o.ndim == 1 else (m[idx] + d)
            v[...] = np.where(np.isnan(v), 0.0, v) + 1.0
            rec.append((plan.key, first, n))
        FakeBatch.launches.append(rec)

    def close(self):
        pass


@pytest.fixture
def server_factory(monkeypatch):
    import torch

    monkeypatch.setattr(torch.cuda, "Stream", FakeStream)
    monkeypatch.setattr(serving, "Batch", FakeBatch)
    monkeypatch.setattr(serving, "Plan", FakePlan)
    FakeBatch.launches = []
    FakePlan.made = []
    FakeEvent.made = 0

    def make(budget=1e12, batch_points=5000, chunk_points=1500, max_jobs=8):
        srv = LensServer(hbm_budget=budget, batch_points=batch_points, chunk_points=chunk_points,
                         max_jobs=max_jobs)
        srv.torch = FakeTorch()
        rng = np.random.default_rng(11)
        for nside, spin in ((16, 0), (16, 2), (32, 0)):
            npix = 12 * nside * nside
            m = fake(rng.standard_normal((npix,) if spin == 0 else (npix, 2)))
            srv.register_map(nside, spin, m, cl=np.ones(3 * nside))
        return srv

    return make


def _defl(count, seed):
    return fake(np.random.default_rng(seed).standard_normal((count, 2)))


def _expected(srv, r):
    m = srv.maps[r.map_key]
    idx = r.first + np.arange(r.count)
    return (m[idx] + r.defl[:, 0]) if r.map_key[1] == 0 else (m[idx] + r.defl)


def test_every_target_lensed_once_in_shared_launches(server_factory):
    srv = server_factory()
    rng = np.random.default_rng(3)
    reqs, chunks_alone = [], 0
    for rid in range(20):
        key = [(16, 0), (16, 2), (32, 0)][rid % 3]
        npix = 12 * key[0] ** 2
        count = int(rng.integers(1, 3000))
        first = int(rng.integers(0, npix - count + 1))
        reqs.append(Request(rid, key, int(rng.choice([16, 32])), first, count, _defl(count, 100 + rid),
                            arrival=0.0))
        chunks_alone += -(-count // 1500)
    done = srv.run(reqs)
    assert sorted(r.rid for r in done) == list(range(20))
    assert srv.in_use == 0 and not srv.active and not srv.pending
    for r in done:
        np.testing.assert_array_equal(np.asarray(r.out), _expected(srv, r))
        np.testing.assert_array_equal(np.asarray(r.var), np.ones(r.count))  # written exactly once
        assert r.done_points == r.count and r.latency is not None and r.latency >= 0
    # launches carry chunks of several requests, within the batch limits
    assert len(FakeBatch.launches) == srv.launches < chunks_alone
    assert any(len({k for k, _, _ in rec}) > 1 for rec in FakeBatch.launches)
    for rec in FakeBatch.launches:
        assert len(rec) <= 8 and sum(n for _, _, n in rec) <= 5000
    st = latency_stats(done)
    assert st["requests"] == 20 and st["points"] == sum(r.count for r in reqs)
    assert st["p99_ms"] >= st["p50_ms"] >= 0


def test_chunks_start_on_even_offsets(server_factory):
    srv = server_factory(batch_points=1001, chunk_points=777, max_jobs=3)
    r = Request(0, (32, 0), 16, 5, 5000, _defl(5000, 7), arrival=0.0)
    srv.run([r])
    offs = [f - r.first for rec in FakeBatch.launches for _, f, _ in rec]
    sizes = [n for rec in FakeBatch.launches for _, _, n in rec]
    assert sum(sizes) == 5000 and all(o % 2 == 0 for o in offs)
    assert offs == sorted(offs) and offs[0] == 0
    np.testing.assert_array_equal(np.asarray(r.var), np.ones(5000))


def test_smallest_chunks_still_progress(server_factory):
    # two-point chunks and batches: every batch holds one even chunk, the last point alone
    srv = server_factory(batch_points=2, chunk_points=2, max_jobs=2)
    reqs = [Request(0, (16, 0), 16, 3, 7, _defl(7, 1), arrival=0.0),
            Request(1, (16, 2), 16, 0, 5, _defl(5, 2), arrival=0.0)]
    done = srv.run(reqs)
    assert sorted(r.rid for r in done) == [0, 1]
    sizes = [n for rec in FakeBatch.launches for _, _, n in rec]
    assert sum(sizes) == 12 and all(n in (1, 2) for n in sizes) and sizes.count(1) == 2
    for r in done:
        np.testing.assert_array_equal(np.asarray(r.var), np.ones(r.count))
    for bad in (dict(batch_points=1), dict(chunk_points=1), dict(max_jobs=0)):
        with pytest.raises(ValueError, match="at least"):
            server_factory(**bad)


def test_resident_maps_and_plans_count_against_the_budget(server_factory):
    srv = server_factory()
    maps = sum(m.numel() * m.element_size() for m in srv.maps.values())
    assert srv.resident == maps and srv.used_bytes() == maps
    srv.plan_for(Request(0, (16, 2), 32, 0, 1, None))
    srv.plan_for(Request(1, (16, 2), 32, 0, 1, None))  # the same plan: counted once
    assert srv.resident == maps + PLAN_BYTES and len(FakePlan.made) == 1
    # re-registering a map replaces its bytes
    srv.register_map(16, 0, fake(np.zeros(12 * 16 * 16 * 2)), cl=np.ones(48))
    assert srv.resident == maps + 12 * 16 * 16 * 8 + PLAN_BYTES
    srv.close()
    assert all(p.closed for p in FakePlan.made)


def test_budget_admission_waits_and_oversized_request_runs_alone(server_factory):
    srv = server_factory(budget=1.0)
    count = 2000
    keys = ((32, 0), (16, 2))
    nb = max(LensServer.request_bytes(Request(0, k, 16, 0, count, None)) for k in keys)
    for key in keys:
        srv.plan_for(Request(0, key, 16, 0, 1, None))
    srv.budget = srv.used_bytes() + 1.5 * nb  # room for one request of this size
    reqs = [Request(rid, keys[rid % 2], 16, 100 * rid, count, _defl(count, rid), arrival=0.0)
            for rid in range(5)]
    big = Request(5, (32, 0), 16, 7, 3 * count, _defl(3 * count, 50), arrival=0.0)
    assert srv.used_bytes() + LensServer.request_bytes(big) > srv.budget
    reqs.append(big)
    seen = []

    def tick(s, now):
        seen.append((len(s.active), s.used_bytes()))

    done = srv.run(reqs, on_tick=tick)
    assert len(done) == 6 and srv.in_use == 0
    assert max(a for a, _ in seen) == 1  # never two requests admitted at once
    assert all(u <= srv.budget or a == 1 for a, u in seen)
    assert any(u > srv.budget for _, u in seen)  # the oversized one ran, alone
    spans = sorted((r.admitted_at, r.finished_at) for r in done)
    assert all(a1 >= f0 for (_, f0), (a1, _) in zip(spans, spans[1:]))
    for r in done:
        np.testing.assert_array_equal(np.asarray(r.out), _expected(srv, r))


def test_cancel_pending_and_running_requests(server_factory):
    srv = server_factory(batch_points=1000, chunk_points=500)
    reqs = [Request(rid, (32, 0), 32, 3000 * rid, 3000, _defl(3000, 200 + rid), arrival=0.0) for rid in range(4)]
    state = {"running": None, "pending": False, "held": None}

    def tick(s, now):
        if state["running"] is None:
            # cancelled as soon as it has chunks in flight: one batch slot then retires and
            # relaunches while the other still holds a chunk of it
            r1 = next((r for r in s.active if r.rid == 1 and r.scheduled_points > r.done_points), None)
            if r1 is not None:
                state["running"] = s.cancel(1)
                # its chunks in flight still hold its memory
                state["held"] = r1 in s.active and s.in_use >= r1.nbytes
                state["scheduled"] = r1.scheduled_points
                state["launches"] = len(FakeBatch.launches)
        if not state["pending"] and any(r.rid == 9 for r in s.pending):
            state["pending"] = s.cancel(9)

    late = Request(9, (16, 0), 16, 0, 1000, _defl(1000, 9), arrival=0.0)
    srv.pending.append(late)  # queued before the run starts, cancelled while pending
    done = srv.run(reqs, on_tick=tick)
    assert state["running"] and state["pending"] and state["held"]
    assert sorted(r.rid for r in done) == [0, 2, 3]
    assert sorted(r.rid for r in srv.cancelled) == [1, 9]
    c1 = next(r for r in srv.cancelled if r.rid == 1)
    assert 0 < c1.done_points < c1.count and c1.done_points == c1.scheduled_points
    # no chunk of it was scheduled after the cancellation
    assert c1.scheduled_points == state["scheduled"]
    assert not any(k == (32, 0, 32, "mixed") and c1.first <= f < c1.first + c1.count
                   for rec in FakeBatch.launches[state["launches"]:] for k, f, _ in rec)
    assert srv.in_use == 0 and not srv.active
    assert late.out is None  # never admitted, no buffers
    assert srv.cancel(1) is False and srv.cancel(12345) is False
    # the cancelled request's scheduled prefix was lensed once, nothing after it
    v = np.asarray(c1.var)
    assert np.all(v[:c1.done_points] == 1.0) and np.all(np.isnan(v[c1.done_points:]))
    for r in done:
        np.testing.assert_array_equal(np.asarray(r.out), _expected(srv, r))


def test_empty_and_invalid_requests(server_factory):
    srv = server_factory()
    empty = Request(1, (16, 2), 32, 5, 0, fake(np.zeros((0, 2))), arrival=0.0)
    full = Request(0, (16, 0), 16, 10, 300, _defl(300, 1), arrival=0.0)
    done = srv.run([full, empty])
    assert sorted(r.rid for r in done) == [0, 1] and srv.in_use == 0 and not srv.active
    assert empty.latency is not None and empty.done_points == 0
    assert all(n > 0 for rec in FakeBatch.launches for _, _, n in rec)  # the empty one never launched
    n_launch = srv.launches
    with pytest.raises(ValueError, match="outside the map"):
        srv.run([Request(2, (16, 0), 16, 12 * 16 * 16 - 5, 10, _defl(10, 2))])
    with pytest.raises(ValueError, match="outside the map"):
        srv.run([Request(3, (16, 0), 16, -1, 10, _defl(10, 3))])
    with pytest.raises(ValueError, match="no map registered"):
        srv.run([Request(4, (64, 0), 16, 0, 10, _defl(10, 4))])
    # a bad request among good ones: nothing runs
    with pytest.raises(ValueError, match="outside the map"):
        srv.run([Request(5, (16, 0), 16, 0, 10, _defl(10, 5)),
                 Request(6, (16, 2), 16, 0, 12 * 16 * 16 + 1, _defl(12 * 16 * 16 + 1, 6))])
    # stencil sizes and precisions the library does not plan, missing or mis-shaped
    # deflections, a spin-1 map (the batched launch serves spin 0 and 2)
    for bad, msg in [(Request(7, (16, 0), 20, 0, 10, _defl(10, 7)), "K must be"),
                     (Request(8, (16, 0), 16, 0, 10, _defl(10, 8), precision="fp32"), "precision"),
                     (Request(9, (16, 0), 16, 0, 10, None), "no deflections"),
                     (Request(10, (16, 2), 16, 0, 10, _defl(9, 10)), r"expected \(10, 2\)")]:
        with pytest.raises(ValueError, match=msg):
            srv.run([Request(11, (16, 0), 16, 0, 10, _defl(10, 11)), bad])
    with pytest.raises(ValueError, match="spin-0 and spin-2"):
        srv.register_map(16, 1, fake(np.zeros((12 * 16 * 16, 2))), cl=np.ones(48))
    assert srv.launches == n_launch and not srv.pending and not srv.active


def test_launch_streams_wait_for_admission_and_record_buffers(server_factory):
    srv = server_factory(batch_points=2000, chunk_points=700)
    reqs = [Request(rid, (32, 0), 16, 1000 * rid, 1800, _defl(1800, rid), arrival=0.0) for rid in range(3)]
    srv.run(reqs)
    waits = sum(s.waits for s in srv.streams)
    recorded = sum(s.recorded for s in srv.streams)
    chunks = sum(len(rec) for rec in FakeBatch.launches)
    assert waits == srv.launches  # every launch waits for the admission stream
    assert recorded == 3 * chunks  # deflections, outputs and variances of every chunk
    assert all(s.waits > 0 for s in srv.streams)  # both batch slots were used


def test_deflections_are_produced_at_admission(server_factory):
    srv = server_factory(budget=1.0)
    calls = []

    def maker(rid, count):
        def make():
            calls.append((rid, len(srv.finished)))  # made when its turn for memory came
            return _defl(count, 300 + rid)
        return make

    srv.budget = srv.used_bytes() + 1.2 * LensServer.request_bytes(Request(0, (16, 0), 16, 0, 1500, None)) \
        + 2 * PLAN_BYTES
    reqs = [Request(rid, (16, 0), 16, 10 * rid, 1500, maker(rid, 1500), arrival=0.0) for rid in range(3)]
    done = srv.run(reqs)
    assert calls == [(0, 0), (1, 1), (2, 2)] and len(done) == 3
    for r in done:
        np.testing.assert_array_equal(np.asarray(r.defl), np.asarray(_defl(1500, 300 + r.rid)))
        np.testing.assert_array_equal(np.asarray(r.out), _expected(srv, r))


def test_latency_statistics():
    reqs = [Request(i, (16, 0), 16, 0, 10 * (i + 1), None, arrival=0.1 * i) for i in range(100)]
    for i, r in enumerate(reqs):
        r.finished_at = r.arrival + 0.001 * (i + 1)  # latencies 1 .. 100 ms
    st = latency_stats(reqs)
    assert st["requests"] == 100 and st["max_ms"] == pytest.approx(100.0) and st["mean_ms"] == pytest.approx(50.5)
    assert st["p50_ms"] == pytest.approx(50.5) and st["p99_ms"] == pytest.approx(99.01)
    assert st["points"] == sum(10 * (i + 1) for i in range(100))
    assert st["span_s"] == pytest.approx(9.9 + 0.1) and st["points_per_s"] == pytest.approx(st["points"] / 10.0)
    assert latency_stats([])["requests"] == 0 and latency_stats([])["p99_ms"] is None
