"""Continuous batching of registration jobs on one GPU.

Jobs (an N-session series each, with its own shape and parameters) arrive over
time. The server admits the job at the head of the queue when a slot is free and
its device footprint (``muster_footprint``) fits the HBM budget; each admitted
job runs in its own registration context on its own CUDA stream, with its images
resident on the device. Every pump of the loop advances each active job by a
quantum of gradient steps (``muster_advance``: CUDA-graph replays, no host
wait), so jobs at different pyramid levels and steps run concurrently and their
kernels overlap on the GPU; the oldest job's stream has the higher priority. A job whose schedule is done and whose stream has
drained is read back and its context goes to an idle pool keyed by (shape,
sessions, parameters): the next job with the same key reuses the buffers and the
captured graphs, and idle contexts are destroyed (oldest first) only when an
admission needs their memory, because freeing device memory synchronises the
whole device. Latency is measured from arrival to result.

The loop talks to a backend object, so the admission and accounting logic is
the same with the GPU engine (``EngineBackend``) and with the stand-in the
host-side tests use.
"""
from __future__ import annotations

import collections
import dataclasses
import time
from typing import Any, Callable, Deque, Dict, List, Optional, Sequence, Tuple

import numpy as np


@dataclasses.dataclass
class Job:
    id: int
    images: np.ndarray  # (N, D, H, W) float32, host
    params: Dict[str, Any]
    arrival: float = 0.0  # seconds after the server starts
    times: Optional[Sequence[float]] = None

    def key(self) -> Tuple:
        items = []
        for k, v in sorted(self.params.items()):
            items.append((k, tuple(v) if isinstance(v, (list, tuple)) else v))
        return (tuple(self.images.shape), tuple(items))


@dataclasses.dataclass
class Result:
    id: int
    velocities: Any
    final_loss: float
    arrival: float
    admitted: float
    finished: float

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


class EngineBackend:
    """Subjects on the CUDA engine.

    Contexts take their memory from torch's caching allocator (destroying one does not
    synchronise the device). Each active subject runs on a stream of its own: the oldest
    subject (by arrival) on a high-priority stream, the others on low-priority streams,
    so the GPU finishes subjects in arrival order and the others use the SMs that the
    oldest leaves idle (small kernels, coarse levels, kernel tails). Each subject keeps at
    most `depth` quanta of steps queued on the device (an event per quantum), so a change
    of priority takes effect within a few quanta.

    Jobs whose parameters do not choose the adjoint mode run with the deterministic
    (exact-sum) adjoint, so a subject's result is bit for bit the same alone and in any
    mix; deterministic=False makes the floating-point reductions the default instead."""

    def __init__(self, device: int = 0, max_active: int = 16, depth: int = 2, deterministic: bool = True):
        import torch

        self.torch = torch
        self.device = device
        self.depth = int(depth)
        self.deterministic = int(bool(deterministic))
        with torch.cuda.device(device):
            self.high = [torch.cuda.Stream(device=device, priority=-1) for _ in range(max_active)]
            self.low = [torch.cuda.Stream(device=device, priority=0) for _ in range(max_active)]
        self.used = set()

    def _params(self, job: Job) -> Dict[str, Any]:
        return dict({"deterministic": self.deterministic}, **job.params)

    def footprint(self, job: Job) -> int:
        from .api import footprint

        return footprint(job.images.shape[1:], job.images.shape[0], **self._params(job))

    def create(self, job: Job):
        from .api import Muster

        with self.torch.cuda.device(self.device):
            reg = Muster(job.images.shape[1:], job.images.shape[0], allocator="torch", **self._params(job))
        return {"reg": reg}

    def destroy(self, ctx) -> None:
        ctx["reg"].close()

    @staticmethod
    def is_out_of_memory(e: Exception) -> bool:
        from ._native import EOOM, MusterError

        return isinstance(e, MusterError) and e.code == EOOM

    def _take(self, pool):
        for st in pool:
            if id(st) not in self.used:
                self.used.add(id(st))
                return st
        raise RuntimeError("no free stream")

    def start(self, ctx, job: Job):
        st = self._take(self.low)
        ctx["reg"].set_stream(st.cuda_stream)
        ctx["reg"].set_images(job.images, times=job.times)
        return {"ctx": ctx, "stream": st, "high": False, "events": [], "done": False}

    def prioritize(self, handles) -> None:
        """handles: the active subjects, oldest first."""
        for rank, h in enumerate(handles):
            want_high = rank == 0
            if h["high"] != want_high:
                st = self._take(self.high if want_high else self.low)
                h["ctx"]["reg"].set_stream(st.cuda_stream)  # ordered after the old stream's work
                self.used.discard(id(h["stream"]))
                h["stream"], h["high"] = st, want_high

    def advance(self, h, steps: int) -> bool:
        ev = h["events"]
        while ev and ev[0].query():
            ev.pop(0)
        if h["done"] or len(ev) >= self.depth:
            return False
        h["done"] = h["ctx"]["reg"].advance(steps)
        e = self.torch.cuda.Event()
        e.record(h["stream"])
        ev.append(e)
        return True

    def ready(self, h) -> bool:
        return h["done"] and all(e.query() for e in h["events"])

    def drained(self, h) -> bool:
        """Every quantum issued for this subject has finished on the GPU."""
        return all(e.query() for e in h["events"])

    def release(self, h) -> None:
        """Hands a cancelled subject's stream back; its context (mid-schedule) is reusable,
        as the next subject's set_images resets the optimisation state."""
        h["ctx"]["reg"].set_stream(self.torch.cuda.default_stream(self.device).cuda_stream)
        self.used.discard(id(h["stream"]))

    def collect(self, h):
        reg = h["ctx"]["reg"]
        vel = reg.velocities(reg.params.n_levels - 1, device=False)
        loss = reg.loss_split()["total"]
        # park the idle context on the (unused) default stream, so that its next subject
        # does not wait on whatever the released stream runs next
        reg.set_stream(self.torch.cuda.default_stream(self.device).cuda_stream)
        self.used.discard(id(h["stream"]))
        return vel, loss


def serve_plain(jobs: Sequence[Job], clock: Callable[[], float] = time.perf_counter,
                sleep: Callable[[float], None] = time.sleep, **muster_kwargs) -> List[Result]:
    """The plain one-subject-at-a-time path through the public API: in arrival order,
    each subject gets a new context (device memory from cudaMalloc), its images, the
    whole schedule, its velocities read back, and the context destroyed."""
    from .api import Muster

    t0 = clock()
    out = []
    for job in sorted(jobs, key=lambda j: (j.arrival, j.id)):
        now = clock() - t0
        if job.arrival > now:
            sleep(job.arrival - now)
        admitted = clock() - t0
        with Muster(job.images.shape[1:], job.images.shape[0], **dict(job.params, **muster_kwargs)) as reg:
            reg.set_images(job.images, times=job.times)
            reg.run()
            vel = reg.velocities(reg.params.n_levels - 1, device=False)
            loss = reg.loss_split()["total"]
        out.append(Result(job.id, vel, float(loss), job.arrival, admitted, clock() - t0))
    return sorted(out, key=lambda r: r.id)


class MusterServer:
    """FCFS admission by memory budget and slots, round-robin step quanta, a pool of idle contexts."""

    def __init__(self, backend, hbm_budget: int, max_active: int = 16, quantum: int = 20,
                 clock: Callable[[], float] = time.perf_counter, sleep: Callable[[float], None] = time.sleep,
                 poll: float = 2e-4):
        if max_active < 1 or quantum < 1:
            raise ValueError("max_active and quantum must be >= 1")
        self.backend = backend
        self.budget = int(hbm_budget)
        self.max_active = int(max_active)
        self.quantum = int(quantum)
        self.clock = clock
        self.sleep = sleep
        self.poll = poll  # host back-off while every active job is issued and none has drained
        self.queue: Deque[Tuple[Job, int]] = collections.deque()
        self.active: List[dict] = []
        self.idle: "collections.OrderedDict[int, Tuple[Tuple, Any, int]]" = collections.OrderedDict()
        self._idle_seq = 0
        self.results: List[Result] = []
        self.in_use = 0  # bytes of every live context, active or idle
        self.peak_in_use = 0
        self.peak_active = 0
        self.created = 0
        self.reused = 0
        self.evicted = 0
        self.oom_events = 0  # context creations the device refused although the budget allowed them
        self.cancelled: List[int] = []  # ids of jobs cancelled before their result
        self.t0 = clock()

    def now(self) -> float:
        return self.clock() - self.t0

    def submit(self, job: Job) -> None:
        need = int(self.backend.footprint(job))
        if need > self.budget:
            raise ValueError("job %d needs %d bytes, more than the whole budget" % (job.id, need))
        self.queue.append((job, need))

    def cancel(self, job_id: int) -> bool:
        """Cancels a queued or running job; False if it is unknown or already finished. A
        queued job leaves the queue. A running job gets no further steps; once the work
        already issued for it has drained, its context goes to the idle pool. Neither
        produces a result."""
        for k, (job, _) in enumerate(self.queue):
            if job.id == job_id:
                del self.queue[k]
                self.cancelled.append(job_id)
                return True
        for a in self.active:
            if a["job"].id == job_id and not a.get("cancel"):
                a["cancel"] = True
                return True
        return False

    def _take_idle(self, key) -> Optional[Any]:
        for seq, (k, ctx, _) in self.idle.items():
            if k == key:
                del self.idle[seq]
                return ctx
        return None

    def _evict_for(self, need: int) -> bool:
        while self.in_use + need > self.budget and self.idle:
            _, (_, ctx, nbytes) = self.idle.popitem(last=False)
            self.backend.destroy(ctx)
            self.in_use -= nbytes
            self.evicted += 1
        return self.in_use + need <= self.budget

    def _create(self, job: Job) -> Optional[Any]:
        """backend.create, for when the device has less free memory than the budget assumed
        (memory held by other processes or by fragmentation): on an out-of-memory error the
        idle contexts are freed and the creation is tried once more; if that fails too while
        other jobs run, the job stays at the head of the queue until one of them retires
        (returns None). With no job running it can never fit, and the error is raised."""
        is_oom = getattr(self.backend, "is_out_of_memory", None)
        try:
            return self.backend.create(job)
        except Exception as e:
            if is_oom is None or not is_oom(e):
                raise
            self.oom_events += 1
        while self.idle:
            _, (_, ctx, nbytes) = self.idle.popitem(last=False)
            self.backend.destroy(ctx)
            self.in_use -= nbytes
            self.evicted += 1
        try:
            return self.backend.create(job)
        except Exception as e:
            if not is_oom(e) or not self.active:
                raise
            self.oom_events += 1
            return None

    def _admit(self) -> None:
        # first come, first served: a job at the head that does not fit blocks the rest
        while self.queue and len(self.active) < self.max_active:
            job, need = self.queue[0]
            ctx = self._take_idle(job.key())
            if ctx is not None:
                self.reused += 1
            else:
                if not self._evict_for(need):
                    break
                ctx = self._create(job)
                if ctx is None:
                    break  # the device is short of what the budget counted on: wait for a retirement
                self.in_use += need
                self.created += 1
            self.queue.popleft()
            self.peak_in_use = max(self.peak_in_use, self.in_use)
            h = self.backend.start(ctx, job)
            self.active.append({"job": job, "need": need, "ctx": ctx, "h": h, "admitted": self.now()})
            self.peak_active = max(self.peak_active, len(self.active))

    def pump(self) -> int:
        """One pass: admit, advance every active job by a quantum, retire the finished ones."""
        self._admit()
        if hasattr(self.backend, "prioritize"):
            self.backend.prioritize([a["h"] for a in sorted(self.active, key=lambda a: (a["job"].arrival, a["job"].id))])
        issued = False
        for a in self.active:
            if not a.get("cancel"):
                issued = bool(self.backend.advance(a["h"], self.quantum)) or issued
        keep = []
        for a in self.active:
            if a.get("cancel"):
                if self.backend.drained(a["h"]):
                    self.backend.release(a["h"])
                    self.cancelled.append(a["job"].id)
                    self.idle[self._idle_seq] = (a["job"].key(), a["ctx"], a["need"])
                    self._idle_seq += 1
                else:
                    keep.append(a)
            elif self.backend.ready(a["h"]):
                vel, loss = self.backend.collect(a["h"])
                job = a["job"]
                self.results.append(Result(job.id, vel, float(loss), job.arrival, a["admitted"], self.now()))
                self.idle[self._idle_seq] = (job.key(), a["ctx"], a["need"])
                self._idle_seq += 1
            else:
                keep.append(a)
        retired = len(self.active) - len(keep)
        self.active = keep
        if not issued and not retired:
            self.sleep(self.poll)
        return retired

    def run(self, jobs: Sequence[Job]) -> List[Result]:
        """Serve jobs that arrive job.arrival seconds after this call; returns results by job id."""
        pending = sorted(jobs, key=lambda j: j.arrival)
        self.t0 = self.clock()
        i = 0
        while i < len(pending) or self.queue or self.active:
            t = self.now()
            while i < len(pending) and pending[i].arrival <= t:
                self.submit(pending[i])
                i += 1
            if not self.queue and not self.active:
                self.sleep(max(0.0, pending[i].arrival - t))  # idle until the next arrival
                continue
            self.pump()
        return sorted(self.results, key=lambda r: r.id)

    def close(self) -> None:
        while self.idle:
            _, (_, ctx, nbytes) = self.idle.popitem(last=False)
            self.backend.destroy(ctx)
            self.in_use -= nbytes


def summary(results: Sequence[Result], makespan: float) -> Dict[str, float]:
    """Served subjects per hour and arrival-to-result latency percentiles."""
    lat = np.array([r.latency for r in results]) if results else np.zeros(1)
    return {
        "subjects": len(results),
        "makespan_s": makespan,
        "subjects_per_hour": 3600.0 * len(results) / makespan if makespan > 0 else 0.0,
        "p50_latency_s": float(np.percentile(lat, 50)),
        "p99_latency_s": float(np.percentile(lat, 99)),
        "mean_latency_s": float(lat.mean()),
    }


def poisson_arrivals(n: int, rate: float, seed: int = 0) -> np.ndarray:
    """Arrival times (s) of a Poisson stream of `rate` jobs per second."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=n))
