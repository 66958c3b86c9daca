"""Host logic of the continuous-batching server, with a stand-in backend and a virtual clock."""
import numpy as np
import pytest

from paper_2412_14671_gb300.serve import Job, MusterServer, poisson_arrivals, summary


class Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        assert dt >= 0
        self.t += dt


class FakeBackend:
    """A job needs `total steps` quanta of work; each advance of one job costs `dt` seconds."""

    def __init__(self, clock, bytes_per_voxel=100, dt=0.01, lag=1):
        self.clock = clock
        self.bpv = bytes_per_voxel
        self.dt = dt
        self.lag = lag  # pumps between the last launch and the stream being drained
        self.live = {}
        self.created = self.destroyed = 0
        self.log = []

    def footprint(self, job):
        return int(np.prod(job.images.shape)) * self.bpv

    def create(self, job):
        self.created += 1
        c = {"id": self.created, "key": job.key()}
        self.live[c["id"]] = c
        return c

    def destroy(self, ctx):
        self.destroyed += 1
        del self.live[ctx["id"]]

    def start(self, ctx, job):
        assert ctx["key"] == job.key()
        total = sum(job.params["steps_per_level"][: job.params["n_levels"]])
        self.log.append(("start", job.id))
        return {"ctx": ctx, "job": job, "left": total, "drain": self.lag}

    def advance(self, h, steps):
        if h["left"] > 0:
            h["left"] = max(0, h["left"] - steps)
            self.clock.t += self.dt
            return True
        if h["drain"] > 0:
            h["drain"] -= 1
        return False

    def ready(self, h):
        return h["left"] == 0 and h["drain"] == 0

    def collect(self, h):
        self.log.append(("done", h["job"].id))
        return h["job"].images.sum(axis=(1, 2, 3)), float(h["job"].id)

    def drained(self, h):
        # a cancelled job gets no more launches; its stream drains over `lag` pumps
        if h["drain"] > 0:
            h["drain"] -= 1
        return h["drain"] == 0

    def release(self, h):
        self.log.append(("released", h["job"].id))


def make_job(i, shape=(8, 8, 8), n=3, steps=(10,), arrival=0.0):
    imgs = np.full((n,) + shape, float(i), dtype=np.float32)
    return Job(i, imgs, dict(n_levels=len(steps), steps_per_level=list(steps)), arrival=arrival)


def test_all_jobs_served_and_results_by_id():
    clk = Clock()
    be = FakeBackend(clk)
    srv = MusterServer(be, hbm_budget=10**9, max_active=4, quantum=3, clock=clk, sleep=clk.sleep)
    jobs = [make_job(i, arrival=0.0) for i in range(10)]
    res = srv.run(jobs)
    assert [r.id for r in res] == list(range(10))
    for r in res:
        assert r.final_loss == float(r.id)
        np.testing.assert_array_equal(r.velocities, np.full(3, r.id * 512.0, dtype=np.float32))
        assert r.finished >= r.admitted >= r.arrival
    assert srv.peak_active == 4
    assert not srv.active and not srv.queue


def test_budget_is_never_exceeded_and_fcfs():
    clk = Clock()
    be = FakeBackend(clk)
    small = 3 * 512 * 100
    srv = MusterServer(be, hbm_budget=2 * small + small // 2, max_active=8, quantum=5, clock=clk, sleep=clk.sleep)
    jobs = [make_job(i) for i in range(7)]
    srv.run(jobs)
    assert srv.peak_in_use <= srv.budget
    assert srv.peak_active == 2  # only two contexts fit
    starts = [j for e, j in be.log if e == "start"]
    assert starts == sorted(starts)  # first come, first served


def test_context_reuse_by_key_and_eviction():
    clk = Clock()
    be = FakeBackend(clk)
    a = 3 * 512 * 100  # shape (8,8,8), 3 sessions
    b = 3 * 16 ** 3 * 100
    srv = MusterServer(be, hbm_budget=b + a, max_active=1, quantum=100, clock=clk, sleep=clk.sleep)
    jobs = [make_job(0), make_job(1), make_job(2, shape=(16, 16, 16)), make_job(3, shape=(16, 16, 16)), make_job(4)]
    for k, j in enumerate(jobs):
        j.arrival = float(k)  # serial, in order
    srv.run(jobs)
    # job 1 reuses job 0's context; job 3 reuses job 2's; job 4 finds its idle context still there
    assert be.created == 2 and srv.reused == 3 and srv.evicted == 0
    srv2 = MusterServer(FakeBackend(clk), hbm_budget=b, max_active=1, quantum=100, clock=clk, sleep=clk.sleep)
    srv2.run([make_job(0, arrival=0.0), make_job(1, shape=(16, 16, 16), arrival=1.0)])
    assert srv2.evicted == 1 and srv2.backend.destroyed == 1  # the small idle context made room
    assert srv2.in_use == b
    srv2.close()
    assert srv2.in_use == 0 and not srv2.backend.live


def test_head_of_line_waits_for_memory():
    clk = Clock()
    be = FakeBackend(clk)
    small = 3 * 512 * 100
    big = 3 * 16 ** 3 * 100
    srv = MusterServer(be, hbm_budget=big + small, max_active=8, quantum=2, clock=clk, sleep=clk.sleep)
    jobs = [make_job(0, steps=(50,)), make_job(1, shape=(16, 16, 16)), make_job(2, shape=(16, 16, 16)), make_job(3)]
    srv.run(jobs)
    starts = [j for e, j in be.log if e == "start"]
    assert starts == [0, 1, 2, 3]
    assert srv.peak_in_use <= srv.budget


def test_job_larger_than_budget_is_rejected():
    clk = Clock()
    srv = MusterServer(FakeBackend(clk), hbm_budget=1000, clock=clk, sleep=clk.sleep)
    with pytest.raises(ValueError):
        srv.submit(make_job(0))


def test_arrivals_and_latency_with_virtual_clock():
    clk = Clock()
    be = FakeBackend(clk, dt=0.5)

    srv = MusterServer(be, hbm_budget=10**9, max_active=2, quantum=10, clock=clk, sleep=clk.sleep)
    jobs = [make_job(0, arrival=0.0), make_job(1, arrival=0.0), make_job(2, arrival=0.0)]
    res = srv.run(jobs)
    # one quantum finishes a job; two slots: jobs 0 and 1 share the first pumps, job 2 follows
    lat = {r.id: r.latency for r in res}
    assert lat[2] > lat[0] and lat[2] > lat[1]
    s = summary(res, makespan=clk.t)
    assert s["subjects"] == 3 and s["p99_latency_s"] >= s["p50_latency_s"] > 0
    assert s["subjects_per_hour"] == pytest.approx(3 * 3600 / clk.t)


def test_waits_for_future_arrivals():
    clk = Clock()
    be = FakeBackend(clk)
    srv = MusterServer(be, hbm_budget=10**9, clock=clk, sleep=clk.sleep)
    res = srv.run([make_job(0, arrival=2.0), make_job(1, arrival=5.0)])
    assert [r.id for r in res] == [0, 1]
    assert res[0].admitted == pytest.approx(2.0) and res[1].admitted == pytest.approx(5.0)
    assert all(r.latency < 0.1 for r in res)


def test_poisson_arrivals():
    t = poisson_arrivals(20000, rate=2.0, seed=3)
    assert np.all(np.diff(t) > 0)
    assert np.mean(np.diff(t)) == pytest.approx(0.5, rel=0.03)
    np.testing.assert_array_equal(t, poisson_arrivals(20000, rate=2.0, seed=3))


def test_bad_server_arguments():
    with pytest.raises(ValueError):
        MusterServer(FakeBackend(Clock()), hbm_budget=1, max_active=0)


class DeviceOOM(RuntimeError):
    pass


class SmallDeviceBackend(FakeBackend):
    """A device with less memory than the server's budget assumes (another process holds the
    rest): creating a context beyond `capacity` bytes raises an out-of-memory error."""

    def __init__(self, clock, capacity, **kw):
        super().__init__(clock, **kw)
        self.capacity = capacity
        self.held = 0
        self.peak_held = 0

    def create(self, job):
        need = self.footprint(job)
        if self.held + need > self.capacity:
            raise DeviceOOM("out of memory")
        c = super().create(job)
        c["bytes"] = need
        self.held += need
        self.peak_held = max(self.peak_held, self.held)
        return c

    def destroy(self, ctx):
        self.held -= ctx["bytes"]
        super().destroy(ctx)

    @staticmethod
    def is_out_of_memory(e):
        return isinstance(e, DeviceOOM)


def test_device_out_of_memory_waits_for_a_retirement_and_frees_idle_contexts():
    clk = Clock()
    small = 3 * 512 * 100  # (8,8,8) x 3 sessions; job 2's (10,10,10) context needs about twice that
    be = SmallDeviceBackend(clk, capacity=2 * small + 10)
    srv = MusterServer(be, hbm_budget=10 * small, max_active=3, quantum=5, clock=clk, sleep=clk.sleep)
    jobs = [make_job(0, steps=(20,)), make_job(1, steps=(40,)), make_job(2, shape=(10, 10, 10), steps=(10,)),
            make_job(3, steps=(10,))]
    res = srv.run(jobs)
    assert [r.id for r in res] == [0, 1, 2, 3]
    assert srv.oom_events >= 1 and srv.evicted >= 1  # job 2 waited, then job 0's idle context was freed
    assert be.peak_held <= be.capacity
    starts = [j for e, j in be.log if e == "start"]
    assert starts == [0, 1, 2, 3]  # first come, first served across the wait
    srv.close()
    assert be.held == 0


def test_a_job_the_device_can_never_hold_raises():
    clk = Clock()
    be = SmallDeviceBackend(clk, capacity=100)
    srv = MusterServer(be, hbm_budget=10**9, max_active=2, quantum=5, clock=clk, sleep=clk.sleep)
    with pytest.raises(DeviceOOM):
        srv.run([make_job(0)])


def test_other_errors_of_context_creation_are_not_swallowed():
    clk = Clock()

    class Broken(FakeBackend):
        def create(self, job):
            raise ValueError("bad parameters")

        @staticmethod
        def is_out_of_memory(e):
            return False

    srv = MusterServer(Broken(clk), hbm_budget=10**9, max_active=2, quantum=5, clock=clk, sleep=clk.sleep)
    with pytest.raises(ValueError, match="bad parameters"):
        srv.run([make_job(0)])


def _drive(srv, max_pumps=10000):
    for _ in range(max_pumps):
        if not srv.queue and not srv.active:
            return
        srv.pump()
    raise AssertionError("server did not finish")


def test_cancel_a_queued_job():
    clk = Clock()
    be = FakeBackend(clk)
    srv = MusterServer(be, hbm_budget=10**9, max_active=1, quantum=5, clock=clk, sleep=clk.sleep)
    for i in range(3):
        srv.submit(make_job(i, steps=(20,)))
    srv.pump()  # job 0 admitted, 1 and 2 queued
    assert srv.cancel(1) and not srv.cancel(1) and not srv.cancel(99)
    _drive(srv)
    assert [r.id for r in srv.results] == [0, 2] and srv.cancelled == [1]
    assert [j for e, j in be.log if e == "start"] == [0, 2]
    assert not srv.cancel(0)  # already finished


def test_cancel_a_running_job_drains_then_frees_its_slot_and_context():
    clk = Clock()
    be = FakeBackend(clk, lag=3)
    srv = MusterServer(be, hbm_budget=10**9, max_active=1, quantum=5, clock=clk, sleep=clk.sleep)
    srv.submit(make_job(0, steps=(200,)))
    srv.submit(make_job(1, steps=(200,)))
    for _ in range(4):
        srv.pump()
    assert [a["job"].id for a in srv.active] == [0]
    assert srv.cancel(0)
    srv.pump()  # no further launches for job 0; its stream is still draining
    assert [a["job"].id for a in srv.active] == [0]
    _drive(srv)
    assert [r.id for r in srv.results] == [1] and srv.cancelled == [0]
    assert ("released", 0) in be.log and ("done", 0) not in be.log
    # job 1 has the same problem key, so it ran in job 0's released context
    assert be.created == 1 and srv.reused == 1
    assert srv.in_use == sum(n for _, _, n in srv.idle.values())


def test_engine_backend_cancellation_hooks_without_a_device():
    """EngineBackend.drained / release with stand-ins for the events, the context and torch."""
    from types import SimpleNamespace

    from paper_2412_14671_gb300.serve import EngineBackend

    class Event:
        def __init__(self, done):
            self.done = done

        def query(self):
            return self.done

    class Reg:
        stream = "unset"

        def set_stream(self, handle):
            self.stream = handle

    fake_torch = SimpleNamespace(cuda=SimpleNamespace(default_stream=lambda dev: SimpleNamespace(cuda_stream=0)))
    st, reg = object(), Reg()
    be = SimpleNamespace(torch=fake_torch, device=0, used={id(st)})
    h = {"events": [Event(True), Event(False)], "ctx": {"reg": reg}, "stream": st}
    assert not EngineBackend.drained(be, h)
    h["events"][1].done = True
    assert EngineBackend.drained(be, h)
    EngineBackend.release(be, h)
    assert reg.stream == 0 and not be.used
