"""teuk_step_noalloc: one time step with the half step in the library's static
device scratch, for callers that cannot call cudaMalloc while they step (a
real-time loop that must not block in the allocator, or a process whose device
memory belongs to another framework's pool).

Checked through the C ABI against the allocating entry point (teuk_step on a
handle), on two calls in a row.  This file is collected last so that a run
stopping at its first failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

from oracle import oracle as O
from paper_1206_0270_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1206_0270_gb300 import build
    build.build()
    from paper_1206_0270_gb300 import teuk as T
    return torch, T


def rel(a, b):
    return abs(a - b).max() / max(abs(b).max(), 1e-300)


@pytest.mark.parametrize("nr,nth", [(300, 64), (8192, 128)])
def test_noalloc_step_matches_allocating_step_twice(env, nr, nth):
    torch, T = env
    rmin, rmax, a, s, m = -100.0, 600.0, 0.9, -2, 2
    dt = O.stable_dt(nr, nth, rmin, rmax, a, s, m)
    phi0, pi0 = inputs.random_fields(nr, nth, seed=nr)
    stream = torch.cuda.current_stream()
    src = dict(r0=10.0, sigma=0.05 if nr == 8192 else 2.0)

    # allocating entry point: two steps of the handle's own state
    ref = T.Solver(nr, nth, rmin, rmax, dt, a, s, m, stream=stream)
    ref.set_initial(phi0, pi0)
    ref.set_source(**src)
    ref.step(1)
    p1_ref, q1_ref = ref.state()
    ref.step(1)
    p2_ref, q2_ref = ref.state()

    # no-allocation entry point: caller-owned device buffers, steps 0 and 1
    h = T.Solver(nr, nth, rmin, rmax, dt, a, s, m, stream=stream)
    h.set_source(**src)
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to("cuda")
    phi_a, pi_a = dev(phi0), dev(pi0)
    phi_a[0] = 0
    phi_a[-1] = 0
    pi_a[0] = 0
    pi_a[-1] = 0
    phi_b, pi_b = torch.empty_like(phi_a), torch.empty_like(pi_a)
    ptr = lambda t: C.c_void_p(t.data_ptr())
    T._check(T.teuk_step_noalloc(h.h, ptr(phi_a), ptr(pi_a), ptr(phi_b), ptr(pi_b), 0), h.h, "noalloc 1")
    torch.cuda.synchronize()
    p1, q1 = phi_b.cpu().numpy(), pi_b.cpu().numpy()
    T._check(T.teuk_step_noalloc(h.h, ptr(phi_b), ptr(pi_b), ptr(phi_a), ptr(pi_a), 1), h.h, "noalloc 2")
    torch.cuda.synchronize()
    p2, q2 = phi_a.cpu().numpy(), pi_a.cpu().numpy()

    assert rel(p1, p1_ref) <= TOL and rel(q1, q1_ref) <= TOL
    assert rel(p2, p2_ref) <= TOL and rel(q2, q2_ref) <= TOL
    # the handle's own state was not touched
    assert h.step_count == 0
    ref.close()
    h.close()


def test_noalloc_rejects_grids_beyond_the_scratch(env):
    torch, T = env
    nr, nth = 8194, 128          # (nr - 1) * nth = 1,048,704 > 1,048,576
    h = T.Solver(nr, nth, -100.0, 600.0, 1e-3, 0.9, -2, 2)
    x = torch.zeros((nr, nth), dtype=torch.complex128, device="cuda")
    y = torch.zeros_like(x)
    p = lambda t: C.c_void_p(t.data_ptr())
    rc = T.teuk_step_noalloc(h.h, p(x), p(x), p(y), p(y), 0)
    assert rc == -1
    assert "static scratch" in T.teuk_last_error(h.h).decode()
    h.close()


def test_noalloc_rejects_overlapping_buffers(env):
    # outputs that share bytes with an input (here shifted by one row) or with
    # each other are refused before any device work
    torch, T = env
    nr, nth = 64, 32
    h = T.Solver(nr, nth, -20.0, 40.0, 1e-3, 0.5, -2, 2)
    x = torch.zeros((4 * nr, nth), dtype=torch.complex128, device="cuda")  # every range below lies inside
    base = x.data_ptr()
    row = nth * 16
    p = lambda off: C.c_void_p(base + off)
    span = nr * row
    cases = [
        (0, span, span + row, 2 * span + row),          # phi_out starts inside pi_in
        (0, span, 2 * span, 2 * span + row),            # the two outputs overlap
        (0, span, row, 2 * span + 2 * row),             # phi_out overlaps phi_in
    ]
    for a_in, b_in, a_out, b_out in cases:
        rc = T.teuk_step_noalloc(h.h, p(a_in), p(b_in), p(a_out), p(b_out), 0)
        assert rc == -1, (a_in, b_in, a_out, b_out)
        assert "overlaps" in T.teuk_last_error(h.h).decode()
    torch.cuda.synchronize()
    h.close()
