"""Continuous-batching waveform service on one GPU.

Requests (one (a, s, m) evolution each) queue up; the service admits them
while their device footprint fits in a memory budget, keeps every admitted
job's state resident on the device, advances admitted jobs in slices of time
steps, streams each job's waveform samples to the host after every slice, and
retires finished jobs so that their memory and slot admit the next requests.
Requests that arrive while others are running join without waiting for them.
The scheduling policies are described on WaveformService; the default
("async") gives every job its own CUDA stream with a priority by age.
Results do not depend on the mix: a job's arithmetic is the same alone and
in any batch (bit-identical).

All device work runs in libteuk (teuk_create / teuk_batch_* / teuk_extract);
this module only schedules.
"""
from __future__ import annotations

import concurrent.futures as cf
import dataclasses
import heapq
import time
from typing import Callable, Optional

import numpy as np

from . import teuk as T


@dataclasses.dataclass
class Request:
    """One waveform job.  Grid r* in [rstar_min, rstar_max], nr x nth points;
    a circular equatorial orbit at r0 with Gaussian width sigma; waveform at
    rstar_ext every `every` steps.  The time step follows teuk_stable_dt with
    c_r, c_theta (unless dt is given) and eps is the strength of the angular
    dissipation (teuk_set_dissipation); c_theta = 0.8 needs eps = 1, the bare
    scheme (eps = 0) c_theta = 0.1."""
    a: float
    s: int
    m: int
    nr: int
    nth: int
    steps: int
    r0: float = 10.0
    sigma: float = 0.05
    rstar_min: float = -100.0
    rstar_max: float = 600.0
    rstar_ext: float = 500.0
    every: int = 10
    c_r: float = 0.5
    c_theta: float = 0.8
    eps: float = 1.0
    dt: Optional[float] = None  # None: teuk_stable_dt with c_r, c_theta
    arrival: float = 0.0        # seconds (service clock) at which it may be admitted
    keep_state: bool = False    # read the final Phi, Pi back into Result.state before retiring


def footprint_bytes(req: Request, slice_steps: int) -> int:
    """Device memory of one admitted job: two state copies (64 B/point),
    coefficient planes (168 B/point), b at nodes (8 B/point), half step
    (32 B/point), waveform ring for one slice, source window (small)."""
    pts = req.nr * req.nth
    ring = (slice_steps // req.every + 2) * req.nth * 16
    return pts * (64 + 168 + 8 + 32) + ring + (1 << 20)


@dataclasses.dataclass
class Result:
    rid: int
    request: Request
    t: np.ndarray            # sample times (M)
    phi: np.ndarray          # [samples, nth] complex waveform
    submitted: float         # service-clock seconds
    admitted: float
    finished: float
    state: Optional[tuple] = None  # (Phi, Pi) at the last step when the request asked for it

    @property
    def latency(self) -> float:
        return self.finished - self.submitted


class WaveformService:
    """Continuous batching with admission by device memory.

    policy="share": every admitted job advances in every slice (processor
    sharing: short jobs finish early, long ones stretch).
    policy="fill": each slice runs admitted jobs in arrival order until they
    hold `fill_points` grid points (enough to keep the GPU busy); the others
    stay resident but paused, so the oldest jobs run at nearly full speed and
    small jobs still share launches.
    policy="priority": every admitted job advances in every slice, but the
    jobs that "fill" would run (the oldest, up to `fill_points`) run on
    high-priority CUDA streams and the others on low-priority ones, so the
    younger jobs take only what the older ones leave of the GPU (the batch's
    per-job launches run each job on its own stream).
    policy="async" (default): no common slices.  Every admitted job runs on its own
    CUDA stream; the oldest jobs (up to `fill_points`) each get their next
    slice as soon as their previous one has finished (polled with CUDA
    events, never waited for), so a small job's samples are streamed and the
    job retired as soon as it is done, not when the largest job's slice ends.
    With `age_priority` (default) the streams carry CUDA priorities by age
    rank among the running jobs (the oldest highest, promoted as older jobs
    retire): a younger job's kernels then take only the SMs an older job's
    kernels leave free, as in first-come first-served order, instead of
    slowing a small older job down to the pace of a large younger one.
    With order="remaining" the async policy ranks the running jobs by the
    work they have left (remaining steps x grid points) instead of by age:
    every running job gets its next slice, and the stream priorities follow
    that rank (the least work highest; a job moves down when a smaller one
    arrives), so short requests pass a long job that is already running
    (shortest remaining work first) while the long job takes the SMs they
    leave free.
    batch_mode (the common-slice policies "share", "fill", "priority"): the
    batch's launch form, TEUK_OPT_BATCH_MODE; 0 steps every running job with
    one multi-job launch per kernel and time step, which serves many small
    grids far faster than a launch per job (default: per-job launches)."""

    def __init__(self, memory_budget: int, slice_steps: int = 640, max_jobs: int = 4096,
                 stream=None, clock: Callable[[], float] = time.perf_counter, policy: str = "async",
                 fill_points: int = 2_000_000, age_priority: bool = True, order: str = "age",
                 batch_mode: Optional[int] = None):
        if slice_steps < 2 or slice_steps % 2:
            raise ValueError("slice_steps must be even and >= 2")
        if policy not in ("share", "fill", "priority", "async"):
            raise ValueError("policy is 'share', 'fill', 'priority' or 'async'")
        if order not in ("age", "remaining") or (order == "remaining" and policy != "async"):
            raise ValueError("order is 'age' or, with the async policy, 'remaining'")
        self.order = order
        self.policy = policy
        self.fill_points = int(fill_points)
        self.budget = int(memory_budget)
        self.slice = int(slice_steps)
        self.max_jobs = int(max_jobs)
        self.stream = stream
        self._clock = clock
        self._t0 = clock()
        self.batch = T.Batch(stream=stream)
        self.batch.set_option(T.TEUK_OPT_GRAPH_CHUNK, 64 if self.slice % 64 == 0 else 2)
        if batch_mode is not None:   # the common-slice policies' launch form (teuk_batch)
            self.batch.set_option(T.TEUK_OPT_BATCH_MODE, int(batch_mode))
        self._queue: list = []      # heap of (arrival, rid)
        self._requests: dict = {}
        self._submitted: dict = {}
        self._running: dict = {}    # rid -> dict(solver, job, admitted, t, phi)
        self._used = 0
        self._next = 0
        self.results: dict = {}
        self._dt_cache: dict = {}
        # time steps are prepared on host threads while the GPU runs slices
        # (teuk_stable_dt scans the whole grid; the ctypes call releases the GIL)
        self._pool = cf.ThreadPoolExecutor(max_workers=4)
        self.slices = 0
        self.age_priority = bool(age_priority) and policy == "async"
        self._prio = None           # (least, greatest) CUDA stream priority, read at the first admission

    # -- clock -------------------------------------------------------------
    def now(self) -> float:
        return self._clock() - self._t0

    # -- requests ------------------------------------------------------------
    def submit(self, req: Request) -> int:
        if footprint_bytes(req, self.slice) > self.budget:
            raise ValueError("request needs more device memory than the whole budget")
        rid = self._next
        self._next += 1
        self._requests[rid] = req
        self._submitted[rid] = max(req.arrival, 0.0)
        self._dt_future(req)
        heapq.heappush(self._queue, (req.arrival, rid))
        return rid

    def pending(self) -> int:
        return len(self._queue)

    def running(self) -> int:
        return len(self._running)

    def memory_in_use(self) -> int:
        return self._used

    def _dt_future(self, r: Request):
        key = (r.nr, r.nth, r.rstar_min, r.rstar_max, r.a, r.s, r.m, r.c_r, r.c_theta)
        if r.dt is None and key not in self._dt_cache:
            self._dt_cache[key] = self._pool.submit(T.stable_dt, r.nr, r.nth, r.rstar_min, r.rstar_max,
                                                    r.a, r.s, r.m, r.c_r, r.c_theta)
        return key

    def _dt(self, r: Request) -> float:
        if r.dt is not None:
            return float(r.dt)
        return self._dt_cache[self._dt_future(r)].result()

    def _admit(self):
        now = self.now()
        while self._queue and self._queue[0][0] <= now and len(self._running) < self.max_jobs:
            arrival, rid = self._queue[0]
            r = self._requests[rid]
            need = footprint_bytes(r, self.slice)
            if self._used + need > self.budget:
                break                      # first-come first-served: wait for memory to free up
            if r.dt is None and not self._dt_cache[self._dt_future(r)].done() and self._running:
                break                      # its time step is still being prepared; others keep running
            heapq.heappop(self._queue)
            if self._prio is None and (self.policy == "priority" or self.age_priority):
                import torch
                self._prio = torch.cuda.Stream.priority_range()  # least and greatest priority
            # each handle sets up on its own stream, concurrently with the running slice
            low_stream = None
            if self._prio is not None:
                import torch
                low_stream = torch.cuda.Stream(priority=self._prio[0])
            elif self.policy == "async":
                import torch
                low_stream = torch.cuda.Stream()  # the job's own stream
            g = T.Solver(r.nr, r.nth, r.rstar_min, r.rstar_max, self._dt(r), r.a, r.s, r.m, stream=low_stream)
            g.set_dissipation(r.eps)
            g.set_source(r0=r.r0, sigma=r.sigma)
            g.set_extraction(r.rstar_ext, r.every, capacity=self.slice // r.every + 2)
            self._used += need
            self._running[rid] = dict(solver=g, job=None, remaining=r.steps, admitted=self.now(), t=[], phi=[],
                                      need=need, high=False, stream=low_stream, event=None, inflight=0,
                                      level=None if self._prio is None else self._prio[0])

    def _schedule(self):
        """Choose the jobs that advance in the next slice and make the batch
        hold exactly them (paused jobs keep their state on the device)."""
        order = sorted(self._running, key=lambda rid: (self._submitted[rid], rid))
        want, pts = set(), 0
        for rid in order:
            st = self._running[rid]
            if st["remaining"] == 0:
                continue
            if self.policy != "share" and want and pts >= self.fill_points:
                if self.policy == "fill":
                    break
                want.add(rid)  # priority: runs, at low priority
                continue
            want.add(rid)
            if self.policy == "priority" and not st["high"]:
                import torch
                st["solver"].set_stream(torch.cuda.Stream(priority=self._prio[1]))  # promoted for good
                st["high"] = True
            r = self._requests[rid]
            pts += r.nr * r.nth
        for rid in order:
            st = self._running[rid]
            if st["job"] is not None and rid not in want:
                st["remaining"] = self.batch.remaining(st["job"])
                self.batch.remove(st["job"])
                st["job"] = None
            elif st["job"] is None and rid in want:
                st["job"] = self.batch.add(st["solver"], st["remaining"])

    def _retire(self, rid, fin):
        st = self._running.pop(rid)
        if st["job"] is not None:
            self.batch.remove(st["job"])
        state = st["solver"].state() if self._requests[rid].keep_state else None
        st["solver"].close()
        self._used -= st["need"]
        r = self._requests[rid]
        t = np.concatenate(st["t"]) if st["t"] else np.zeros(0)
        phi = np.concatenate(st["phi"]) if st["phi"] else np.zeros((0, r.nth), complex)
        self.results[rid] = Result(rid, r, t, phi, self._submitted[rid], st["admitted"], fin, state)

    def _drain(self):
        """Stream every running job's new samples; retire finished jobs."""
        self.batch.sync()
        done = []
        for rid, st in self._running.items():
            if st["job"] is None:
                if st["remaining"] == 0:
                    done.append(rid)          # nothing to step (steps = 0)
                continue
            t, w = st["solver"].extract(cap=self.slice // self._requests[rid].every + 2)
            if len(t):
                st["t"].append(t)
                st["phi"].append(w)
            st["remaining"] = self.batch.remaining(st["job"])
            if st["remaining"] == 0:
                done.append(rid)
        fin = self.now()
        for rid in done:
            self._retire(rid, fin)

    def _step_async(self) -> bool:
        """One iteration of the event-driven loop: harvest the jobs whose
        slice has finished, admit arrivals, give idle jobs of the running set
        their next slice.  Never blocks on the GPU."""
        import torch
        progressed = False
        for rid in list(self._running):
            st = self._running[rid]
            ev = st["event"]
            if ev is not None and ev.query():
                t, w = st["solver"].extract(cap=self.slice // self._requests[rid].every + 2)
                if len(t):
                    st["t"].append(t)
                    st["phi"].append(w)
                st["remaining"] -= st["inflight"]
                st["inflight"], st["event"] = 0, None
                progressed = True
            if st["event"] is None and st["remaining"] == 0:
                self._retire(rid, self.now())
                progressed = True
        self._admit()
        pts = 0
        by_work = self.order == "remaining"
        if by_work:
            def rank_key(q):
                r = self._requests[q]
                return (self._running[q]["remaining"] * r.nr * r.nth, self._submitted[q], q)
        else:
            def rank_key(q):
                return (self._submitted[q], q)
        for rank, rid in enumerate(sorted(self._running, key=rank_key)):
            st = self._running[rid]
            if pts and pts >= self.fill_points and not by_work:
                break
            r = self._requests[rid]
            pts += r.nr * r.nth
            if st["event"] is None and st["remaining"] > 0:
                if self.age_priority:
                    # CUDA priorities: smaller numbers are higher, from high (greatest)
                    # up to low (least); the first in rank gets the greatest.  By age a
                    # job is only promoted; by remaining work it also moves down when a
                    # job with less work arrives
                    want = min(self._prio[1] + rank, self._prio[0])
                    if want < st["level"] or (by_work and want != st["level"]):
                        st["stream"] = torch.cuda.Stream(priority=want)
                        st["solver"].set_stream(st["stream"])
                        st["level"] = want
                n = min(self.slice, st["remaining"])
                st["solver"].step(n)
                ev = torch.cuda.Event()
                ev.record(st["stream"])
                st["event"], st["inflight"] = ev, n
                self.slices += 1
                progressed = True
        if not progressed:
            if not self._running and not self._queue:
                return False
            wait = self._queue[0][0] - self.now() if (self._queue and not self._running) else 0.0
            time.sleep(min(max(wait, 0.0005), 0.01))
        return True

    def step(self) -> bool:
        """One service iteration: launch a slice for the admitted jobs, admit
        arrivals (their set-up overlaps the slice), then stream samples and
        retire finished jobs.  New jobs join the batch at the next slice.
        Returns False when nothing is queued or running."""
        if self.policy == "async":
            return self._step_async()
        had_jobs = bool(self._running)
        if had_jobs:
            self._schedule()
            self.batch.step(self.slice)
            self.slices += 1
        self._admit()
        if had_jobs:
            self._drain()
        elif not self._running:
            if not self._queue:
                return False
            wait = self._queue[0][0] - self.now()   # idle until the next arrival
            if wait > 0:
                time.sleep(min(wait, 0.01))
        return True

    def run(self, until_empty: bool = True, max_seconds: float = float("inf")):
        t_end = self.now() + max_seconds
        while self.now() < t_end:
            if not self.step() and until_empty:
                break
        return self.results

    def close(self):
        """Release every job still admitted and the service's batch; safe to
        call more than once."""
        self._pool.shutdown(wait=True)
        self.batch.close()          # releases the handles, which are then destroyed
        for st in self._running.values():
            st["solver"].close()
        self._running.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def latency_stats(results) -> dict:
    lat = np.array([r.latency for r in results.values()])
    if lat.size == 0:
        return dict(p50=None, p99=None, mean=None, n=0)
    return dict(p50=float(np.percentile(lat, 50)), p99=float(np.percentile(lat, 99)),
                mean=float(lat.mean()), n=int(lat.size))
