"""Batched stepping (teuk_batch_*): many independent evolutions advanced by
shared launches give the same bits as stepping each handle alone, and match
the oracle."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1206_0270_gb300 import inputs

pytestmark = pytest.mark.gpu

# uneven grids, spins, modes, sources and step counts; some with the angular
# dissipation (eps > 0, with the larger time step it allows) and some without
JOBS = [
    dict(nr=300, nth=64, a=0.9, s=-2, m=2, steps=131, src=dict(r0=8.0, sigma=0.5), ext=(10.0, 7), eps=1.0),
    dict(nr=120, nth=32, a=0.0, s=-2, m=2, steps=64, src=None, ext=(5.0, 4), eps=0.0),
    dict(nr=77, nth=96, a=0.5, s=0, m=1, steps=200, src=dict(r0=6.0, sigma=1.0), ext=None, eps=0.0),
    dict(nr=40, nth=256, a=0.7, s=2, m=-3, steps=37, src=dict(r0=5.0, sigma=1.0), ext=(0.0, 5), eps=1.0),
    dict(nr=64, nth=20, a=0.3, s=-2, m=0, steps=0, src=None, ext=None, eps=0.0),
    dict(nr=500, nth=128, a=0.95, s=-2, m=4, steps=129, src=dict(r0=12.0, sigma=0.3), ext=(30.0, 10), eps=0.5),
]
RMIN, RMAX = -20.0, 40.0


@pytest.fixture(scope="module")
def teuk():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1206_0270_gb300 import build
    build.build()
    from paper_1206_0270_gb300 import teuk as T
    return T


def make(T, j, seed):
    dt = O.stable_dt(j["nr"], j["nth"], RMIN, RMAX, j["a"], j["s"], j["m"], 0.5, 0.8 if j["eps"] else 0.1)
    g = T.Solver(j["nr"], j["nth"], RMIN, RMAX, dt, j["a"], j["s"], j["m"])
    g.set_dissipation(j["eps"])
    g.set_initial(*inputs.random_fields(j["nr"], j["nth"], seed=seed))
    if j["src"]:
        g.set_source(**j["src"])
    if j["ext"]:
        g.set_extraction(j["ext"][0], j["ext"][1], capacity=64)
    return g, dt


def collect(g, j):
    out = list(g.state())
    if j["ext"]:
        out.append(g.extract()[1])
    return out


def run_alone(T):
    res = []
    for q, j in enumerate(JOBS):
        g, _ = make(T, j, q)
        g.step(j["steps"])
        res.append(collect(g, j))
        g.close()
    return res


@pytest.mark.parametrize("pdl,chunk,block,ctas,mode", [
    (1, 64, 0, 0, 0), (0, 64, 0, 0, 0), (1, 8, 512, 0, 0), (1, 2, 256, 0, 0), (1, 64, 64, 0, 0), (1, 64, 96, 0, 0),
    (1, 64, 0, 1, 0), (0, 6, 0, 2, 0), (1, 64, 64, 64, 0),
    (1, 64, 0, 0, 1), (0, 2, 0, 0, 1), (1, 6, 0, 0, 1)])
def test_batch_equals_individual_runs(teuk, pdl, chunk, block, ctas, mode):
    # mode 0: one launch per kernel for all jobs (one CTA per tile, or a
    # persistent grid of `ctas` CTAs per SM looping over the tiles); mode 1:
    # per-job launches
    alone = run_alone(teuk)
    B = teuk.Batch()
    B.set_option(teuk.TEUK_OPT_PDL, pdl)
    B.set_option(teuk.TEUK_OPT_GRAPH_CHUNK, chunk)
    B.set_option(teuk.TEUK_OPT_BLOCK_THREADS, block)
    B.set_option(teuk.TEUK_OPT_BATCH_CTAS, ctas)
    B.set_option(teuk.TEUK_OPT_BATCH_MODE, mode)
    solvers = []
    for q, j in enumerate(JOBS):
        g, _ = make(teuk, j, q)
        solvers.append(g)
        B.add(g, j["steps"])
    done = B.step(10 ** 6)
    assert done == max(j["steps"] for j in JOBS)
    B.sync()
    for q, (g, j) in enumerate(zip(solvers, JOBS)):
        assert B.remaining(q) == 0
        assert g.step_count == j["steps"]
        for x, y in zip(collect(g, j), alone[q]):
            np.testing.assert_array_equal(x, y)
    B.close()


def test_batch_in_slices_remove_and_autotune(teuk):
    alone = run_alone(teuk)
    B = teuk.Batch()
    solvers = []
    for q, j in enumerate(JOBS):
        g, _ = make(teuk, j, q)
        solvers.append(g)
        B.add(g, j["steps"])
    best = B.autotune()          # timed steps count as progress
    assert best in (0, 1, 2, 3)
    B.step(5)
    B.set_option(teuk.TEUK_OPT_BATCH_MODE, 0)  # switch modes mid-run, odd slices
    B.step(33)
    B.set_option(teuk.TEUK_OPT_BATCH_MODE, 1)
    B.step(7)
    B.set_option(teuk.TEUK_OPT_BATCH_MODE, 0)
    B.step(3)
    B.sync()
    # take job 1 out, finish it alone, the others in the batch
    r1 = B.remaining(1)
    B.remove(1)
    solvers[1].step(r1)
    while B.step(17):
        pass
    B.sync()
    for q, (g, j) in enumerate(zip(solvers, JOBS)):
        assert g.step_count == j["steps"]
        for x, y in zip(collect(g, j), alone[q]):
            np.testing.assert_array_equal(x, y)
    B.close()


@pytest.mark.parametrize("mode,ctas", [(0, 0), (0, 4), (1, 0)])
def test_batch_matches_oracle(teuk, mode, ctas):
    # the multi-job launches (mode 0; one CTA per tile, or persistent) and
    # per-job launches (mode 1)
    j = JOBS[0]
    g, dt = make(teuk, j, 0)
    other, _ = make(teuk, JOBS[3], 3)
    B = teuk.Batch()
    B.set_option(teuk.TEUK_OPT_BATCH_CTAS, ctas)
    B.set_option(teuk.TEUK_OPT_BATCH_MODE, mode)
    B.add(g, j["steps"])
    B.add(other, JOBS[3]["steps"])
    B.step(j["steps"])
    B.sync()
    ora = O.Solver(j["nr"], j["nth"], RMIN, RMAX, dt, j["a"], j["s"], j["m"])
    ora.set_dissipation(j["eps"])
    ora.set_initial(*inputs.random_fields(j["nr"], j["nth"], seed=0))
    ora.set_source(**j["src"])
    ora.set_extraction(*j["ext"])
    ora.step(j["steps"])
    po, qo = ora.state()
    pg, qg = g.state()
    assert abs(pg - po).max() / abs(po).max() <= 1e-10
    assert abs(qg - qo).max() / abs(qo).max() <= 1e-10
    to, wo = ora.samples()
    tg, wg = g.extract()
    np.testing.assert_array_equal(tg, to)
    assert abs(wg - wo).max() / abs(wo).max() <= 1e-10
    B.close()


def test_batch_bad_arguments(teuk):
    B = teuk.Batch()
    g = teuk.Solver(40, 2048, RMIN, RMAX, 1e-3, 0.5, -2, 2)
    with pytest.raises(teuk.TeukError):
        B.add(g, 10)              # nth > 512
    h = teuk.Solver(40, 32, RMIN, RMAX, 1e-3, 0.5, -2, 2)
    B.add(h, 10)
    with pytest.raises(teuk.TeukError):
        B.add(h, 10)              # twice
    with pytest.raises(teuk.TeukError):
        B.remove(7)
    # a handle in a batch is driven by the batch only
    for call in (lambda: h.step(1), lambda: h.set_source(r0=8.0, sigma=1.0),
                 lambda: h.set_extraction(0.0, 2)):
        with pytest.raises(teuk.TeukError) as e:
            call()
        assert e.value.code == -5
    assert teuk.teuk_destroy(h.h) == -5
    B.remove(0)
    h.step(1)                    # usable again after removal
    with pytest.raises(teuk.TeukError):
        B.set_option(teuk.TEUK_OPT_BLOCK_THREADS, 100)
    for bad in (-1, 65):
        with pytest.raises(teuk.TeukError):
            B.set_option(teuk.TEUK_OPT_BATCH_CTAS, bad)
    assert B.step(0) == 0
    B.close()


@pytest.mark.parametrize("mode", [0, 1])
def test_batch_mixes_fixed_point_and_fp64_jobs(teuk, mode):
    # jobs with the fixed-point and with the FP64 Pi rows in one batch: each
    # equals the same job stepped alone with its own setting
    picks = [0, 2, 3, 5]
    def build(q):
        j = JOBS[q]
        g, _ = make(teuk, j, q)
        if q % 2 == 0:
            g.set_option(teuk.TEUK_OPT_FIXED_POINT, 0)
        return g, j
    alone = []
    for q in picks:
        g, j = build(q)
        g.step(j["steps"])
        alone.append(collect(g, j))
        g.close()
    B = teuk.Batch()
    B.set_option(teuk.TEUK_OPT_BATCH_MODE, mode)
    solvers = []
    for q in picks:
        g, j = build(q)
        solvers.append((g, j))
        B.add(g, j["steps"])
    B.step(10 ** 6)
    B.sync()
    for (g, j), ref in zip(solvers, alone):
        for x, y in zip(collect(g, j), ref):
            np.testing.assert_array_equal(x, y)
    B.close()


@pytest.mark.parametrize("mode", ["auto", 0, "persistent"])
def test_mode_batch_at_full_size_equals_individual_runs(teuk, mode):
    """The batched-modes workload at its own sizes: a = 0.7, r0 = 8, m = 1..8
    on 4096 x {32, 32, 64, 64, 128, 128, 256, 256}, r* in [-100, 600], with
    the source and waveform extraction, in the benchmark's launch
    configuration (autotuned) and in the multi-job launches (one CTA per tile,
    and persistent).  Uneven
    step counts (640 .. 1200) must give each job the same bits as stepping
    its handle alone; the single-job path is held to the oracle by the
    parity tests."""
    w = inputs.MODE_BATCH
    rmin, rmax = w["rstar_min"], w["rstar_max"]
    jobs = []
    for q, (m, nth) in enumerate(w["modes"]):
        jobs.append(dict(m=m, nth=nth, steps=640 + 80 * q))

    def make_job(q, j):
        dt = O.stable_dt(w["nr"], j["nth"], rmin, rmax, w["a"], w["s"], j["m"], w["c_r"], w["c_theta"])
        g = teuk.Solver(w["nr"], j["nth"], rmin, rmax, dt, w["a"], w["s"], j["m"])
        g.set_dissipation(w["eps"])
        g.set_initial(*inputs.random_fields(w["nr"], j["nth"], seed=100 + q))
        g.set_source(r0=w["r0"], sigma=w["sigma"])
        g.set_extraction(w["extraction"]["rstar"], w["extraction"]["every"], capacity=j["steps"] // 10 + 2)
        return g

    alone = []
    for q, j in enumerate(jobs):
        g = make_job(q, j)
        g.step(j["steps"])
        alone.append(list(g.state()) + [g.extract()[1]])
        g.close()
    B = teuk.Batch()
    solvers = [make_job(q, j) for q, j in enumerate(jobs)]
    for g, j in zip(solvers, jobs):
        B.add(g, j["steps"])
    if mode == "auto":
        B.autotune()
    elif mode == "persistent":
        B.set_option(teuk.TEUK_OPT_BATCH_CTAS, 8)
        B.set_option(teuk.TEUK_OPT_BATCH_MODE, 0)
    else:
        B.set_option(teuk.TEUK_OPT_BATCH_MODE, mode)
    while B.step(10 ** 6):
        pass
    B.sync()
    for q, (g, j) in enumerate(zip(solvers, jobs)):
        assert g.step_count == j["steps"]
        for x, y in zip(list(g.state()) + [g.extract()[1]], alone[q]):
            np.testing.assert_array_equal(x, y)
    B.close()
    for g in solvers:
        g.close()


@pytest.mark.parametrize("ctas", [0, 3])
def test_multi_job_groups_beyond_64_jobs(teuk, ctas):
    """80 small jobs in mode 0: 65 complex fixed-point jobs with the
    dissipation (two launch groups: 64 + 1) and five each with real planes,
    with FP64 Pi rows and without the dissipation (a group each), with one
    CTA per tile or a persistent grid; every job equals the same job
    stepped alone, bit for bit."""
    rng = np.random.default_rng(70)
    specs = []
    for q in range(80):
        a = 0.0 if q % 16 == 0 else float(rng.uniform(0.1, 0.9))   # a = 0: real planes
        specs.append(dict(nr=int(rng.integers(24, 90)), nth=int(rng.choice([8, 20, 32, 48, 64, 100])), a=a,
                          s=-2, m=int(rng.integers(1, 4)), steps=int(rng.integers(3, 40)),
                          src=dict(r0=6.0, sigma=1.0) if q % 2 else None, ext=(5.0, 3) if q % 4 == 1 else None,
                          eps=0.0 if q % 16 == 4 else 1.0, fx=0 if q % 16 == 8 else 1))

    def build(q):
        j = specs[q]
        g, _ = make(teuk, j, 1000 + q)
        if not j["fx"]:
            g.set_option(teuk.TEUK_OPT_FIXED_POINT, 0)
        return g, j

    alone = []
    for q in range(len(specs)):
        g, j = build(q)
        g.step(j["steps"])
        alone.append(collect(g, j))
        g.close()
    B = teuk.Batch()
    B.set_option(teuk.TEUK_OPT_BATCH_CTAS, ctas)
    B.set_option(teuk.TEUK_OPT_BATCH_MODE, 0)
    solvers = []
    for q in range(len(specs)):
        g, j = build(q)
        solvers.append((g, j))
        B.add(g, j["steps"])
    # 2 launches per group per time step plus one counter update per slice:
    # five groups
    assert B.launches_for(2) == 2 * 2 * 5 + 1
    while B.step(10 ** 6):
        pass
    B.sync()
    for (g, j), ref in zip(solvers, alone):
        assert g.step_count == j["steps"]
        for x, y in zip(collect(g, j), ref):
            np.testing.assert_array_equal(x, y)
    B.close()
    for g, _ in solvers:
        g.close()


def test_template_bank_at_full_size_every_launch_form(teuk):
    """The template-bank workload at its full grid sizes: 256 seeded jobs, a
    in [0, 0.95], r0 in [6, 20], m = 1..4, 2048..16384 x 64..256 (304 M grid
    points, 83 GB resident), with the source, waveform extraction and the
    workload's dissipation; uneven short step counts (6..12) so that jobs
    leave at slice boundaries after odd slices.  Per-job launches, multi-job
    launches (one CTA per tile: four launch groups of 64) and the persistent
    multi-job launches each give every job the same final state, bit for bit
    (compared by digest), as the job stepped alone."""
    import hashlib
    T = teuk
    rule = inputs.STEP_RULE
    rmin, rmax = -100.0, 600.0
    jobs = inputs.template_bank(256)
    for q, j in enumerate(jobs):
        j["sigma"] = max(0.05, 2.0 * 700.0 / (j["nr"] - 1))
        j["steps"] = 6 + q % 7
        j["dt"] = T.stable_dt(j["nr"], j["nth"], rmin, rmax, j["a"], j["s"], j["m"], rule["c_r"], rule["c_theta"])

    def make_job(j):
        g = T.Solver(j["nr"], j["nth"], rmin, rmax, j["dt"], j["a"], j["s"], j["m"])
        g.set_dissipation(rule["eps"])
        g.set_source(r0=j["r0"], sigma=j["sigma"])
        g.set_extraction(500.0, 3, capacity=8)
        return g

    def digest(g):
        phi, pi = g.state()
        return hashlib.sha256(phi.tobytes() + pi.tobytes() + g.extract()[1].tobytes()).hexdigest()

    alone = []
    for j in jobs:
        g = make_job(j)
        g.step(j["steps"])
        alone.append(digest(g))
        g.close()
    for mode, ctas in ((1, 0), (0, 0), (0, 8)):
        B = T.Batch()
        B.set_option(T.TEUK_OPT_BATCH_CTAS, ctas)
        B.set_option(T.TEUK_OPT_BATCH_MODE, mode)
        solvers = [make_job(j) for j in jobs]
        for g, j in zip(solvers, jobs):
            B.add(g, j["steps"])
        while B.step(10 ** 6):
            pass
        B.sync()
        got = [digest(g) for g in solvers]
        B.close()
        for g in solvers:
            g.close()
        bad = [q for q in range(len(jobs)) if got[q] != alone[q]]
        assert not bad, (mode, ctas, bad[:10])


def test_persistent_multi_job_fp64_rows_of_16_columns(teuk):
    # FP64 jobs on rows of at most 16 columns in the persistent multi-job
    # form: 16-column tiles of 16 rows, two sets of shared rows (54 KB per
    # CTA, above the 48 KB default); every job equals itself stepped alone
    specs = [dict(nr=n, nth=t, a=0.6, s=-2, m=2, steps=k, src=dict(r0=8.0, sigma=1.0), ext=(5.0, 3), eps=1.0)
             for n, t, k in ((90, 16, 23), (140, 8, 31), (60, 12, 17))]

    def build(q):
        g, _ = make(teuk, specs[q], 500 + q)
        g.set_option(teuk.TEUK_OPT_FIXED_POINT, 0)
        return g, specs[q]
    alone = []
    for q in range(len(specs)):
        g, j = build(q)
        g.step(j["steps"])
        alone.append(collect(g, j))
        g.close()
    for ctas in (0, 2):
        B = teuk.Batch()
        B.set_option(teuk.TEUK_OPT_BATCH_CTAS, ctas)
        B.set_option(teuk.TEUK_OPT_BATCH_MODE, 0)
        solvers = [build(q) for q in range(len(specs))]
        for g, j in solvers:
            B.add(g, j["steps"])
        while B.step(10 ** 6):
            pass
        B.sync()
        for (g, j), ref in zip(solvers, alone):
            for x, y in zip(collect(g, j), ref):
                np.testing.assert_array_equal(x, y)
        B.close()
        for g, _ in solvers:
            g.close()
