"""Continuous-batching service: admission by device memory, jobs joining and
leaving between slices, streamed waveforms; each result is the same alone and
in the mix, and a job served in the mix matches the FP64 oracle."""
import numpy as np
import pytest

from oracle import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def serve():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1206_0270_gb300 import build
    build.build()
    from paper_1206_0270_gb300 import serve as S
    return S


def reqs(S):
    R = S.Request
    return [
        R(a=0.9, s=-2, m=2, nr=600, nth=64, steps=900, r0=10.0, sigma=1.0, rstar_ext=40.0, every=10),
        R(a=0.3, s=-2, m=1, nr=300, nth=32, steps=320, r0=8.0, sigma=2.0, rstar_ext=30.0, every=8, arrival=0.0),
        R(a=0.7, s=0, m=3, nr=1000, nth=128, steps=1500, r0=12.0, sigma=1.0, rstar_ext=50.0, every=5),
        R(a=0.0, s=-2, m=2, nr=200, nth=16, steps=2, r0=6.0, sigma=3.0, rstar_ext=20.0, every=1),
        R(a=0.5, s=2, m=-1, nr=400, nth=48, steps=700, r0=9.0, sigma=1.5, rstar_ext=30.0, every=7),
    ]


def run_alone(S, r):
    svc = S.WaveformService(memory_budget=1 << 34, slice_steps=64)
    rid = svc.submit(r)
    res = svc.run()
    svc.close()
    return res[rid]


@pytest.mark.parametrize("policy,fill,mode", [("share", 0, None), ("fill", 60000, None), ("fill", 1, None),
                                              ("priority", 60000, None), ("async", 60000, None),
                                              ("async", 1, None), ("share", 0, 0), ("fill", 60000, 0)])
def test_results_same_alone_and_in_the_mix(serve, policy, fill, mode):
    # mode 0: the common slices step the jobs with multi-job launches
    S = serve
    rs = reqs(S) + [S.Request(a=0.2, s=-2, m=2, nr=100, nth=8, steps=0, sigma=3.0, rstar_ext=10.0)]
    alone = [run_alone(S, r) for r in rs]
    # the mix: a budget that fits about two jobs at a time, staggered arrivals
    budget = 2 * S.footprint_bytes(rs[2], 64)
    svc = S.WaveformService(memory_budget=budget, slice_steps=64, policy=policy, fill_points=fill,
                            batch_mode=mode)
    ids = []
    for k, r in enumerate(rs):
        r2 = S.Request(**{**r.__dict__, "arrival": 0.002 * k})
        ids.append(svc.submit(r2))
    peak = 0
    while svc.step():
        peak = max(peak, svc.memory_in_use())
        assert svc.memory_in_use() <= budget
    assert peak > S.footprint_bytes(rs[2], 64)   # jobs really overlapped on the device
    assert svc.slices > 0
    for rid, a in zip(ids, alone):
        r = svc.results[rid]
        assert len(r.t) == r.request.steps // r.request.every
        np.testing.assert_array_equal(r.t, a.t)
        np.testing.assert_array_equal(r.phi, a.phi)
        assert r.finished >= r.admitted >= r.submitted - 1e-9
    st = S.latency_stats(svc.results)
    assert st["n"] == len(rs) and st["p99"] >= st["p50"] > 0
    svc.close()


def test_admission_respects_budget_and_rejects_oversize(serve):
    S = serve
    r = S.Request(a=0.5, s=-2, m=2, nr=400, nth=64, steps=200, sigma=1.0, rstar_ext=30.0)
    one = S.footprint_bytes(r, 64)
    svc = S.WaveformService(memory_budget=int(1.5 * one), slice_steps=64)
    for _ in range(3):
        svc.submit(r)
    svc.step()
    assert svc.running() == 1 and svc.pending() == 2    # only one fits
    svc.run()
    assert len(svc.results) == 3 and svc.memory_in_use() == 0
    with pytest.raises(ValueError):
        svc.submit(S.Request(a=0.5, s=-2, m=2, nr=40000, nth=512, steps=10))
    svc.close()


@pytest.mark.parametrize("policy", ["async", "fill", "share"])
def test_served_job_matches_oracle(serve, policy):
    # A Kerr job with source, extraction and the angular dissipation arrives
    # mid-stream, waits for memory behind older jobs, runs beside them and
    # leaves; its streamed waveform and final state equal the oracle's run of
    # the same evolution within the parity tolerance.
    S = serve
    nr, nth, rmin, rmax, a, s, m = 300, 32, -20.0, 60.0, 0.9, -2, 2
    dt = O.stable_dt(nr, nth, rmin, rmax, a, s, m, 0.5, 0.8)
    target = S.Request(a=a, s=s, m=m, nr=nr, nth=nth, steps=700, r0=8.0, sigma=1.0, rstar_min=rmin, rstar_max=rmax,
                       rstar_ext=20.0, every=7, dt=dt, eps=1.0, keep_state=True, arrival=0.006)
    rs = [S.Request(**{**r.__dict__, "arrival": 0.002 * k}) for k, r in enumerate(reqs(S))]
    budget = 2 * S.footprint_bytes(rs[2], 64)
    svc = S.WaveformService(memory_budget=budget, slice_steps=64, policy=policy, fill_points=60000)
    for r in rs[:3]:
        svc.submit(r)
    tid = svc.submit(target)
    for r in rs[3:]:
        svc.submit(r)
    svc.run()
    res = svc.results[tid]
    assert res.admitted > min(svc.results[q].admitted for q in svc.results)   # it did not start first
    ora = O.Solver(nr, nth, rmin, rmax, dt, a, s, m)
    ora.set_dissipation(1.0)
    ora.set_initial(np.zeros((nr, nth), complex), np.zeros((nr, nth), complex))
    ora.set_source(r0=8.0, sigma=1.0)
    ora.set_extraction(20.0, 7)
    ora.step(700)
    to, wo = ora.samples()
    po, qo = ora.state()
    np.testing.assert_array_equal(res.t, to)
    rel = lambda x, y: abs(x - y).max() / abs(y).max()
    assert rel(res.phi, wo) <= 1e-10
    assert rel(res.state[0], po) <= 1e-10 and rel(res.state[1], qo) <= 1e-10
    svc.close()
