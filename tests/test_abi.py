"""The C-ABI library builds, loads and exports every function include/teuk.h
declares; host-only entry points behave.  No GPU needed."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "teuk.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(teuk_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1206_0270_gb300 import build
    build.build()
    from paper_1206_0270_gb300 import teuk
    return teuk


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ["teuk_create", "teuk_set_source", "teuk_step", "teuk_extract", "teuk_destroy",
              "teuk_set_initial", "teuk_set_extraction", "teuk_stable_dt"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    import ctypes
    so = ctypes.CDLL(lib.LIB_PATH)
    for name in declared_functions():
        assert hasattr(so, name), name
    # the binding covers exactly the declared functions
    assert sorted(lib.EXPORTED) == declared_functions()


def test_stable_dt_matches_oracle_rule(lib):
    from oracle import oracle as O
    for (nr, nth, rmin, rmax, a, s, m, cr, ct) in [
            (1024, 64, -100.0, 300.0, 0.0, -2, 2, 0.5, 0.1),
            (513, 32, -50.0, 100.0, 0.9, -2, 2, 0.5, 0.1),
            (200, 8, -20.0, 40.0, 0.7, 0, 3, 0.5, 10.0),   # radial limit binds
            (300, 17, -30.0, 60.0, 0.3, 2, -1, 0.25, 0.05)]:
        d_lib = lib.stable_dt(nr, nth, rmin, rmax, a, s, m, cr, ct)
        d_ora = O.stable_dt(nr, nth, rmin, rmax, a, s, m, cr, ct)
        assert d_lib == pytest.approx(d_ora, rel=1e-12)


def test_bad_arguments_are_rejected_without_gpu(lib):
    assert lib.teuk_strerror(-1).decode() == "bad argument"
    with pytest.raises(lib.TeukError) as e:
        lib.stable_dt(3, 8, -10.0, 10.0, 0.0, -2, 2)      # nr < 4
    assert e.value.code == -1
    with pytest.raises(lib.TeukError):
        lib.stable_dt(64, 8, -10.0, 10.0, 1.0, -2, 2)     # |a| >= 1
    with pytest.raises(lib.TeukError):
        lib.stable_dt(64, 8, -10.0, 10.0, 0.5, 1, 2)      # s not in {-2, 0, 2}
    with pytest.raises(lib.TeukError):
        lib.stable_dt(64, 8, 10.0, -10.0, 0.5, -2, 2)     # empty range
    # create rejects a bad grid before touching the device
    g = lib.teuk_grid(64, 8, -10.0, 10.0, -1.0)
    import ctypes
    h = ctypes.c_void_p()
    assert lib.teuk_create(ctypes.byref(g), 0.5, -2, 2, None, ctypes.byref(h)) == -1
    assert not h.value


def test_launch_count_null_handle(lib):
    assert lib.teuk_launches_for(None, 10) == -1
    assert lib.teuk_step_count(None) == -1


def test_every_entry_point_rejects_null_objects_without_gpu(lib):
    # Each call given a NULL handle, batch or output pointer reports
    # TEUK_ERR_BAD_ARG (-1 for the counting calls, an empty message for the
    # error-text calls) before it touches the device or dereferences anything.
    import ctypes as C
    zero = {C.c_int: 0, C.c_long: 0, C.c_double: 0.0, C.c_uint: 0}
    special = {
        "teuk_strerror": None,              # takes a code, not an object
        "teuk_fixed_dot": ((0, 0, 1, None, None, None, None, None), -1),   # nterms 0
        "teuk_fixed_d6": ((0, -1, None, None), -1),                        # count < 0
    }
    seen = []
    for name in lib.EXPORTED:
        f = getattr(lib, name)
        if name in special:
            if special[name] is None:
                continue
            args, want = special[name]
        else:
            args = tuple(zero.get(t) for t in f.argtypes)   # None for every pointer
            want = b"" if f.restype is C.c_char_p else -1
        assert f(*args) == want, name
        seen.append(name)
    assert len(seen) == len(lib.EXPORTED) - 1
    assert lib.teuk_strerror(0).decode() == "ok"


def test_no_cpu_fallback(lib, tmp_path):
    # The binding refuses to load without libteuk.so, and without a GPU the
    # product calls fail with an error instead of computing on the host.
    import importlib.util
    import shutil
    pkg = tmp_path / "nolib"
    pkg.mkdir()
    shutil.copy(os.path.join(ROOT, "paper_1206_0270_gb300", "teuk.py"), pkg / "teuk.py")
    spec = importlib.util.spec_from_file_location("teuk_without_library", str(pkg / "teuk.py"))
    with pytest.raises(ImportError, match="no CPU fallback"):
        spec.loader.exec_module(importlib.util.module_from_spec(spec))
    try:
        g = lib.Solver(64, 8, -10.0, 10.0, 0.01, 0.5, -2, 2)
    except lib.TeukError as e:
        assert e.code == -3                                   # TEUK_ERR_CUDA: no device here
    else:
        g.close()
        pytest.skip("a GPU is present: the device path ran")
    with pytest.raises(lib.TeukError) as e:
        lib.fixed_d6(np.ones((2, 7)), device=True)            # never served by the host build
    assert e.value.code == -3
