"""Host logic of the serving loop (admission, continuous batching, faults) with a fake GPU.

The loop in paper_1811_01566_gb300.serve drives an executor; here the
executor is a fake with a manual clock, so admission order, HBM-budget
eviction, rejection, cancellation and failure isolation are checked on the
CPU.  Faults are injected on the host only (a launch that raises, a request
that does not fit); nothing here touches a GPU.
"""
from types import SimpleNamespace

import numpy as np
import pytest

from paper_1811_01566_gb300.serve import Request, Server, latency_stats


class Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t


class FakeExecutor:
    """Each launch takes `duration` seconds of the fake clock; images are filled with the rid."""

    def __init__(self, clock, duration=1.0, fail_rids=()):
        self.clock, self.duration, self.fail = clock, duration, set(fail_rids)
        self.created, self.released, self.launches, self.batches = 0, 0, [], []
        self.eager = []

    def footprint(self, req, batch=None):
        if req.grid.nx <= 0:
            raise ValueError("invalid grid")
        return req.rf_host.nbytes

    def launch_eager(self, req):
        h = {"done_at": None, "reqs": []}
        self.eager.append(req.rid)
        self.launch(h, [req])
        return h

    def create(self, req):
        if req.grid.nz <= 0:
            raise ValueError("invalid grid")
        self.created += 1
        return {"done_at": None, "reqs": []}

    def launch(self, h, reqs):
        if any(r.rid in self.fail for r in reqs):
            raise RuntimeError("injected launch failure")
        h["done_at"] = self.clock() + self.duration
        h["reqs"] = list(reqs)
        for r in reqs:
            self.launches.append((r.rid, self.clock()))
        self.batches.append([r.rid for r in reqs])

    def done(self, h):
        return h["done_at"] is not None and self.clock() >= h["done_at"]

    def result(self, h):
        return [np.full((2, 2), float(r.rid)) for r in h["reqs"]]

    def release(self, h):
        self.released += 1


def req(rid, shape=0, nbytes=10, arrival=0.0, nz=4):
    probe = SimpleNamespace(n_elements=8 + shape, pitch=3e-4, fs=5e7, c=1540.0, f_number=1.5, apod=0)
    grid = SimpleNamespace(nz=nz, nx=4, x_min=0.0, x_max=1e-3, z_min=1e-3, z_max=2e-3)
    rf = np.zeros(nbytes // 2, dtype=np.int16).reshape(1, 1, 1, -1)
    return Request(rid, "stai", probe, grid, rf, arrival=arrival)


def drive(server, clock, until, dt=0.5):
    while clock.t <= until:
        server.step()
        clock.t += dt


def test_continuous_admission_fifo_within_shape():
    clock = Clock()
    ex = FakeExecutor(clock, duration=1.0)
    s = Server(ex, hbm_budget=1000, max_slots_per_shape=2, clock=clock)
    for i in range(3):
        s.submit(req(i))
    s.step()
    assert [r for r, _ in ex.launches] == [0, 1]          # two slots of the shape
    clock.t = 1.0
    s.step()                                             # 0 and 1 retire, 2 is admitted
    assert [r for r, _ in ex.launches] == [0, 1, 2]
    assert ex.launches[2][1] == 1.0
    clock.t = 2.0
    s.step()
    assert sorted(s.results) == [0, 1, 2]
    assert s.results[2].latency == pytest.approx(2.0)
    assert ex.created == 2


def test_other_shapes_are_not_blocked_behind_a_busy_shape():
    clock = Clock()
    ex = FakeExecutor(clock, duration=5.0)
    s = Server(ex, hbm_budget=1000, max_slots_per_shape=1, clock=clock)
    s.submit(req(0, shape=0))
    s.submit(req(1, shape=0))   # waits for shape 0's only slot
    s.submit(req(2, shape=1))   # must not wait behind request 1
    s.step()
    assert [r for r, _ in ex.launches] == [0, 2]


def test_hbm_budget_evicts_idle_slots_of_other_shapes():
    clock = Clock()
    ex = FakeExecutor(clock, duration=1.0)
    s = Server(ex, hbm_budget=100, max_slots_per_shape=4, clock=clock)
    s.submit(req(0, shape=0, nbytes=60))
    s.submit(req(1, shape=1, nbytes=60))   # does not fit while shape 0 holds 60
    s.step()
    assert [r for r, _ in ex.launches] == [0]
    clock.t = 1.0
    s.step()                               # 0 retires, its idle slot is evicted, 1 runs
    assert [r for r, _ in ex.launches] == [0, 1]
    assert ex.released == 1
    assert s.used <= 100


def test_request_larger_than_budget_is_rejected_and_others_proceed():
    clock = Clock()
    ex = FakeExecutor(clock)
    s = Server(ex, hbm_budget=50, clock=clock)
    s.submit(req(0, nbytes=400))
    s.submit(req(1, shape=1, nbytes=20))
    s.step()
    assert s.results[0].error.startswith("rejected")
    assert [r for r, _ in ex.launches] == [1]


def test_cancel_before_launch_and_failures_stay_isolated():
    clock = Clock()
    ex = FakeExecutor(clock, duration=1.0, fail_rids={3})
    s = Server(ex, hbm_budget=1000, max_slots_per_shape=1, clock=clock)
    for i in range(4):
        s.submit(req(i))
    s.submit(req(9, shape=2, nz=0))        # invalid geometry: create() raises
    bad = req(8, shape=3)
    bad.grid.nx = 0
    s.submit(bad)                          # invalid geometry: footprint() raises
    assert s.cancel(2)
    s.step()
    assert s.results[9].error.startswith("rejected")
    assert s.results[8].error.startswith("rejected")
    drive(s, clock, until=5.0)
    assert s.results[2].error == "cancelled"
    assert s.results[3].error.startswith("launch failed")
    assert s.results[0].error is None and s.results[1].error is None
    assert s.results[1].db[0, 0] == 1.0
    assert not s.cancel(0)                  # already answered


def test_run_feeds_arrivals_in_time_order_and_reports_percentiles():
    clock = Clock()
    ex = FakeExecutor(clock, duration=0.25)

    class Ticking(Server):
        def step(self):
            n = super().step()
            clock.t += 0.05
            return n

    s = Ticking(ex, hbm_budget=1000, max_slots_per_shape=2, clock=clock)
    reqs = [req(i, arrival=0.1 * i) for i in range(20)]
    res = s.run(reqs)
    assert sorted(res) == list(range(20))
    st = latency_stats(res)
    assert st["n"] == 20 and 0.2 <= st["p50_ms"] / 1e3 <= st["p99_ms"] / 1e3 < 1.0


def test_queued_requests_of_a_shape_run_as_one_batch():
    clock = Clock()
    ex = FakeExecutor(clock, duration=1.0)
    s = Server(ex, hbm_budget=1000, max_slots_per_shape=1, clock=clock, max_batch=3)
    for i in range(5):
        s.submit(req(i))
    s.submit(req(9, shape=1))
    s.step()
    assert ex.batches == [[0, 1, 2], [9]]            # FIFO within the shape, up to 3 at once
    clock.t = 1.0
    s.step()
    assert ex.batches[-1] == [3, 4]
    clock.t = 2.0
    s.step()
    assert sorted(s.results) == [0, 1, 2, 3, 4, 9]
    assert all(s.results[i].db[0, 0] == float(i) for i in (0, 1, 2, 3, 4, 9))
    # every request arrived before its shape had a slot: all cold; a later one is warm
    assert all(s.results[i].cold for i in (0, 1, 2, 3, 4))
    s.submit(req(5))
    s.step()
    clock.t = 3.0
    s.step()
    assert not s.results[5].cold


def _wait(pred, timeout=5.0):
    import time as _t
    t_end = _t.time() + timeout
    while not pred() and _t.time() < t_end:
        _t.sleep(0.001)
    assert pred()


def test_slot_creation_off_the_admission_path():
    """While a new shape's slot is being built on the creator thread, requests of other
    shapes keep being admitted and retired; the new shape's requests wait in order."""
    import threading

    clock = Clock()
    gate = threading.Event()

    class SlowCreate(FakeExecutor):
        def create(self, req):
            if req.probe.n_elements == 9:       # shape 1 takes long to build
                assert gate.wait(5.0)
            return super().create(req)

    ex = SlowCreate(clock, duration=1.0)
    s = Server(ex, hbm_budget=1000, max_slots_per_shape=1, clock=clock, async_create=True)
    s.submit(req(0, shape=0))
    _wait(lambda: (s.step(), len(ex.launches) == 1)[1])
    s.submit(req(1, shape=1))
    s.submit(req(2, shape=0))
    s.submit(req(3, shape=1))
    s.step()                                 # shape 1 creation starts; shape 0's slot is busy
    clock.t = 1.0
    _wait(lambda: (s.step(), 2 in [r for r, _ in ex.launches])[1])
    assert [r for r, _ in ex.launches] == [0, 2]     # shape 0 kept running
    clock.t = 2.0
    s.step()
    assert 2 in s.results and 1 not in s.results
    gate.set()
    _wait(lambda: (s.step(), 1 in [r for r, _ in ex.launches])[1])
    clock.t = 3.0
    s.step()
    clock.t = 4.0
    s.step()
    assert [r for r, _ in ex.launches] == [0, 2, 1, 3]
    # 1 and 3 arrived before their shape's slot existed (cold); 2 found shape 0's slot built
    assert s.results[1].cold and s.results[3].cold and not s.results[2].cold
    s.close()


def test_failed_slot_creation_rejects_that_shape_only():
    clock = Clock()

    class FailCreate(FakeExecutor):
        def create(self, req):
            if req.probe.n_elements == 9:
                raise ValueError("geometry refused")
            return super().create(req)

    ex = FailCreate(clock, duration=1.0)
    s = Server(ex, hbm_budget=1000, clock=clock, async_create=True)
    s.submit(req(1, shape=1))
    s.submit(req(0, shape=0))
    s.submit(req(2, shape=1))
    _wait(lambda: (s.step(), 1 in s.results and 2 in s.results)[1])
    assert s.results[1].error.startswith("rejected") and s.results[2].error.startswith("rejected")
    clock.t = 1.0
    s.step()
    assert s.results[0].error is None
    s.close()


def test_cold_requests_run_eagerly_while_their_slot_is_built():
    import threading

    clock = Clock()
    gate = threading.Event()

    class SlowCreate(FakeExecutor):
        def create(self, req):
            assert gate.wait(5.0)
            return super().create(req)

    ex = SlowCreate(clock, duration=1.0)
    s = Server(ex, hbm_budget=1000, max_slots_per_shape=1, clock=clock, async_create=True,
               eager_cold=True)
    s.submit(req(0, shape=0))
    s.submit(req(1, shape=0))
    s.step()                                     # slot creation starts; both run eagerly
    assert ex.eager == [0, 1] and ex.created == 0
    clock.t = 1.0
    s.step()
    assert s.results[0].cold and s.results[1].cold and s.results[0].error is None
    assert s.used == 10                          # eager memory returned; the slot being built keeps its share
    gate.set()
    _wait(lambda: (s.step(), ex.created == 1 and not s._creating(req(2).key()))[1])
    s.submit(req(2, shape=0))
    s.step()
    assert ex.eager == [0, 1] and [r for r, _ in ex.launches][-1] == 2   # on the built slot
    clock.t = 2.0
    s.step()
    assert not s.results[2].cold
    s.close()


def test_cuda_executor_reuses_streams_and_never_destroys_them():
    """A released slot's stream goes to the next slot; none is destroyed, so pinned buffers that
    outlive a slot never record events on a dead stream (host logic, fake library)."""
    import torch
    from paper_1811_01566_gb300.serve import CudaExecutor

    class _Stream:
        def __init__(self):
            self.syncs = 0

        def synchronize(self):
            self.syncs += 1

    class _Wf:
        created = 0

        def stream_create(self, device=None):
            _Wf.created += 1
            return _Stream()

        def stream_destroy(self, stream):
            raise AssertionError("a slot stream was destroyed")

    ex = CudaExecutor(device=torch.device("cpu"))
    ex.wf = _Wf()
    s1, s2 = ex._take_stream(), ex._take_stream()
    assert s1 is not s2 and _Wf.created == 2
    h = {"stream": s1, "own_stream": True, "rf": object()}
    ex.release(h)
    assert h == {} and s1.syncs == 1
    assert ex._take_stream() is s1 and _Wf.created == 2      # reused, not created anew
    ex.release({"stream": s2, "own_stream": False})          # eager handle: pool stream, not kept
    assert ex._take_stream() is not s2 and _Wf.created == 3
