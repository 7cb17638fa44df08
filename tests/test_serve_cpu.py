"""Host logic of the waveform service (paper_1206_0270_gb300/serve.py) on the
CPU: admission by device-memory footprint in arrival order, arrivals not
admitted early, the "fill" and "share" scheduling policies, the default
"async" policy (per-job streams, completion events, priorities by age rank
and their promotion), waveform assembly across slices, retirement and the
argument checks.  The library's Solver and Batch are replaced by fakes that
count time steps and produce samples exactly where the real extraction
would (every `every` steps), CUDA events and streams by fakes whose work
completes when recorded, and the service runs on a fake clock; nothing here
touches a GPU."""
import numpy as np
import pytest

from paper_1206_0270_gb300 import serve as S

# a scheduling mistake can leave the service loop waiting for work that never
# finishes; each test ends within seconds when the logic is right
pytestmark = pytest.mark.timeout(120)


class FakeSolver:
    def __init__(self, nr, nth, rstar_min, rstar_max, dt, a, s, m, stream=None):
        self.nr, self.nth, self.dt = nr, nth, dt
        self.n = 0
        self.every = None
        self.pending = []
        self.closed = False
        self.advanced_at = []      # batch slice index of every advance
        self.priorities = [getattr(stream, "priority", None)]
        self.ticks = None          # shared step log of the async loop

    def set_stream(self, stream=None):
        self.priorities.append(stream.priority)

    def step(self, n):             # the async policy steps handles directly
        self.advance(n, None)
        if self.ticks is not None:
            self.ticks.append(self)

    def set_source(self, **kw):
        pass

    def set_dissipation(self, eps):
        self.eps = eps

    def set_extraction(self, rstar_ext, every, capacity):
        self.every, self.capacity = every, capacity

    def advance(self, n, tick):
        for _ in range(n):
            self.n += 1
            if self.n % self.every == 0:
                self.pending.append(self.n)
        assert len(self.pending) <= self.capacity, "ring buffer would have overflowed"
        if n:
            self.advanced_at.append(tick)

    def extract(self, cap):
        k, self.pending = self.pending[:cap], self.pending[cap:]
        t = np.array(k, dtype=float) * self.dt
        return t, np.outer(t, np.arange(1, self.nth + 1)).astype(complex)

    def close(self):
        self.closed = True


class FakeBatch:
    made = []

    def __init__(self, stream=None):
        self.jobs, self.next, self.ticks = {}, 0, 0
        self.options = {}
        FakeBatch.made.append(self)

    def set_option(self, option, value):
        self.options[option] = value

    def add(self, solver, steps):
        jid = self.next
        self.next += 1
        self.jobs[jid] = [solver, int(steps)]
        return jid

    def remove(self, jid):
        del self.jobs[jid]

    def step(self, max_steps):
        # each job advances min(max_steps, its remaining steps)
        for job in self.jobs.values():
            n = min(max_steps, job[1])
            job[0].advance(n, self.ticks)
            job[1] -= n
        self.ticks += 1

    def remaining(self, jid):
        return self.jobs[jid][1]

    def sync(self):
        pass

    def close(self):
        pass


class FakeLib:
    TEUK_OPT_GRAPH_CHUNK = 4
    TEUK_OPT_BATCH_MODE = 6
    Solver = FakeSolver
    Batch = FakeBatch
    made = []

    @staticmethod
    def stable_dt(nr, nth, rmin, rmax, a, s, m, c_r=0.5, c_theta=0.1):
        return 0.25


class Clock:
    """Advances by `tick` seconds per reading: the loop always makes progress."""
    def __init__(self, tick=1e-3):
        self.t, self.tick = 0.0, tick

    def __call__(self):
        self.t += self.tick
        return self.t


@pytest.fixture
def fake(monkeypatch):
    made = []

    class Tracking(FakeSolver):
        def __init__(self, *args, **kw):
            super().__init__(*args, **kw)
            made.append(self)
    lib = type("Lib", (FakeLib,), {"Solver": Tracking})
    monkeypatch.setattr(S, "T", lib)
    monkeypatch.setattr(S.time, "sleep", lambda s: None)
    return made


def request(nr=64, nth=8, steps=100, arrival=0.0, every=10):
    return S.Request(a=0.5, s=-2, m=2, nr=nr, nth=nth, steps=steps, arrival=arrival, every=every)


def run(svc, watch=None):
    while svc.step():
        assert svc.memory_in_use() <= svc.budget
        if watch is not None:
            watch(svc)
    return svc.results


def test_admission_by_footprint_in_arrival_order(fake):
    slice_steps = 20
    need = S.footprint_bytes(request(), slice_steps)
    svc = S.WaveformService(memory_budget=2 * need + need // 2, slice_steps=slice_steps,
                            clock=Clock(), policy="share")
    rids = [svc.submit(request(steps=40 + 20 * k)) for k in range(5)]
    seen = []
    res = run(svc, lambda s: seen.append(s.running()))
    assert max(seen) == 2                       # two fit the budget, never three
    assert sorted(res) == rids
    adm = [res[r].admitted for r in rids]
    assert adm == sorted(adm)                   # first come, first served
    assert all(s.closed for s in fake) and svc.memory_in_use() == 0
    svc.close()


def test_waveform_samples_are_complete_and_ordered(fake):
    svc = S.WaveformService(memory_budget=1 << 34, slice_steps=20, clock=Clock(), policy="share")
    steps = [0, 7, 20, 55, 130]
    rids = [svc.submit(request(steps=n, every=5)) for n in steps]
    res = run(svc)
    for rid, n in zip(rids, steps):
        r = res[rid]
        expect = np.arange(5, n + 1, 5) * 0.25
        np.testing.assert_array_equal(r.t, expect)
        np.testing.assert_array_equal(r.phi, np.outer(expect, np.arange(1, 9)).astype(complex))
        assert r.finished >= r.admitted >= r.submitted
    svc.close()


def test_arrivals_are_not_admitted_early(fake):
    clock = Clock(tick=1e-3)
    svc = S.WaveformService(memory_budget=1 << 34, slice_steps=20, clock=clock, policy="share")
    early = svc.submit(request(steps=20, arrival=0.0))
    late = svc.submit(request(steps=20, arrival=0.5))
    res = run(svc)
    assert res[late].admitted >= 0.5 and res[late].submitted == 0.5
    assert res[early].admitted < 0.5
    svc.close()


def test_fill_runs_the_oldest_jobs_first(fake):
    # fill_points = one job's grid: the jobs run one after another, in arrival order
    svc = S.WaveformService(memory_budget=1 << 34, slice_steps=20, clock=Clock(), policy="fill",
                            fill_points=64 * 8)
    for _ in range(3):
        svc.submit(request(steps=60))
    run(svc)
    spans = [(min(s.advanced_at), max(s.advanced_at)) for s in fake]
    assert spans[0][1] < spans[1][0] and spans[1][1] < spans[2][0], spans
    svc.close()


def test_share_advances_every_admitted_job(fake):
    svc = S.WaveformService(memory_budget=1 << 34, slice_steps=20, clock=Clock(), policy="share")
    for _ in range(3):
        svc.submit(request(steps=60))
    run(svc)
    ticks = [s.advanced_at for s in fake]
    assert ticks[0] == ticks[1] == ticks[2] and len(ticks[0]) == 3
    svc.close()


def test_argument_checks(fake):
    with pytest.raises(ValueError):
        S.WaveformService(memory_budget=1 << 30, slice_steps=7)
    with pytest.raises(ValueError):
        S.WaveformService(memory_budget=1 << 30, policy="lifo")
    svc = S.WaveformService(memory_budget=1 << 20, slice_steps=20, clock=Clock())
    with pytest.raises(ValueError):
        svc.submit(request(nr=4096, nth=256))   # larger than the whole budget
    svc.close()


def test_latency_stats():
    assert S.latency_stats({})["n"] == 0
    res = {i: S.Result(i, request(), np.zeros(0), np.zeros((0, 8)), 0.0, 0.0, float(i + 1)) for i in range(100)}
    st = S.latency_stats(res)
    assert st["p50"] == pytest.approx(50.5) and st["mean"] == pytest.approx(50.5)


# ---------------------------------------------------------------------------
# The async policy (default): per-job streams, events, priorities by age
# ---------------------------------------------------------------------------

class FakeEvent:
    """Work on the fake streams completes as soon as it is recorded."""
    def __init__(self):
        self.recorded = False

    def record(self, stream):
        self.recorded = True

    def query(self):
        return self.recorded


class FakeStream:
    def __init__(self, priority=0):
        self.priority = priority

    @staticmethod
    def priority_range():
        return (0, -5)             # least, greatest


@pytest.fixture
def fake_cuda(monkeypatch, fake):
    import sys
    import types
    torch = types.SimpleNamespace(cuda=types.SimpleNamespace(Event=FakeEvent, Stream=FakeStream,
                                                             synchronize=lambda: None))
    monkeypatch.setitem(sys.modules, "torch", torch)
    return fake


def test_async_policy_completes_every_job(fake_cuda):
    svc = S.WaveformService(memory_budget=1 << 34, slice_steps=20, clock=Clock())
    assert svc.policy == "async"
    steps = [0, 7, 45, 130]
    rids = [svc.submit(request(steps=n, every=5)) for n in steps]
    res = run(svc)
    for rid, n in zip(rids, steps):
        np.testing.assert_array_equal(res[rid].t, np.arange(5, n + 1, 5) * 0.25)
    assert all(s.closed for s in fake_cuda) and svc.memory_in_use() == 0
    svc.close()


def test_async_priorities_follow_age_and_promote(fake_cuda):
    # four equal jobs admitted at once: the oldest runs at the greatest
    # priority (-5), the next at -4, ...; as older jobs retire the younger are
    # promoted, never demoted
    svc = S.WaveformService(memory_budget=1 << 34, slice_steps=20, clock=Clock())
    for k in range(4):
        svc.submit(request(steps=40 + 20 * k))
    run(svc)
    first = [s.priorities[1] for s in fake_cuda]
    assert first == [-5, -4, -3, -2], first
    for s in fake_cuda:
        assert s.priorities[0] == 0                                  # admitted at the least priority
        assert all(b < a for a, b in zip(s.priorities[1:], s.priorities[2:]))  # only promotions
    assert fake_cuda[3].priorities[-1] == -5                          # the last job ends up oldest
    svc.close()


def test_async_runs_oldest_jobs_up_to_fill_points(fake_cuda):
    log = []
    svc = S.WaveformService(memory_budget=1 << 34, slice_steps=20, clock=Clock(), fill_points=64 * 8)
    for _ in range(3):
        svc.submit(request(steps=60))
    svc._admit()
    for s in fake_cuda:
        s.ticks = log
    run(svc)
    order = [fake_cuda.index(s) for s in log]
    assert order == sorted(order), order      # one job at a time, in arrival order
    svc.close()


def test_age_priority_can_be_switched_off(fake_cuda):
    svc = S.WaveformService(memory_budget=1 << 34, slice_steps=20, clock=Clock(), age_priority=False)
    for _ in range(2):
        svc.submit(request(steps=40))
    run(svc)
    assert all(s.priorities == [0] for s in fake_cuda)   # default-priority streams, never moved
    svc.close()


def test_async_by_remaining_work_runs_every_job_and_ranks_by_work(fake_cuda):
    # a long job admitted first, then short ones: every job advances in every
    # round (no fill cutoff), the shortest remaining work gets the greatest
    # priority, and the long job moves down when shorter ones arrive
    log = []
    svc = S.WaveformService(memory_budget=1 << 34, slice_steps=20, clock=Clock(), fill_points=64 * 8,
                            order="remaining")
    svc.submit(request(steps=400))
    svc._admit()
    fake_cuda[0].ticks = log
    svc.step()                                   # the long job alone: greatest priority
    assert fake_cuda[0].priorities[-1] == -5
    for n in (40, 80):
        svc.submit(request(steps=n))
    svc._admit()
    for s in fake_cuda:
        s.ticks = log
    svc.step()
    assert [s.priorities[-1] for s in fake_cuda] == [-3, -5, -4]
    res = run(svc)
    assert len(res) == 3 and all(s.closed for s in fake_cuda)
    # the short jobs finish before the long one although it came first
    assert max(res[1].finished, res[2].finished) <= res[0].finished
    with pytest.raises(ValueError):
        S.WaveformService(memory_budget=1 << 30, policy="fill", order="remaining")
    svc.close()


def test_batch_mode_option_reaches_the_batch(fake):
    # the common-slice policies can step their jobs with multi-job launches
    svc = S.WaveformService(memory_budget=1 << 34, slice_steps=20, clock=Clock(), policy="share", batch_mode=0)
    assert FakeBatch.made[-1].options == {FakeLib.TEUK_OPT_GRAPH_CHUNK: 2, FakeLib.TEUK_OPT_BATCH_MODE: 0}
    for n in (30, 50):
        svc.submit(request(steps=n))
    res = run(svc)
    assert sorted(len(r.t) for r in res.values()) == [3, 5]
    svc.close()
    svc = S.WaveformService(memory_budget=1 << 34, slice_steps=20, clock=Clock(), policy="share")
    assert FakeLib.TEUK_OPT_BATCH_MODE not in FakeBatch.made[-1].options
    svc.close()


def test_service_as_context_manager_releases_jobs(fake):
    # leaving the block early (here after one step) closes every admitted job
    with S.WaveformService(memory_budget=1 << 40, slice_steps=20, clock=Clock(), policy="share") as svc:
        for k in range(3):
            svc.submit(request(steps=200))
        svc.step()
        assert svc.running() == 3
    assert svc.running() == 0 and all(s.closed for s in fake)
    svc.close()                                  # a second close is harmless
