"""Host-only checks of the C ABI: the library loads, exports every function that
include/lrspike.h declares, and rejects bad options before touching the GPU."""
import ctypes
import os
import re

import pytest

from paper_2504_11167_gb300 import solver

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "lrspike.h")).read()
    return sorted(set(re.findall(r"\b(lrspike_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2504_11167_gb300 import _build
    _build.build()
    return solver.load_library()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "lrspike_create" in names and "lrspike_solve_transpose" in names
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(solver.EXPORTS)


def _opts(lib, n=1000, k=8, p=4, r=2):
    o = solver.Options()
    assert lib.lrspike_options_default(ctypes.byref(o), n, k, p, r) == 0
    return o


def test_defaults(lib):
    o = _opts(lib)
    assert (o.n, o.k, o.p, o.r) == (1000, 8, 4, 2)
    assert o.precision == 0 and o.compress == 0 and o.reduced == 0 and o.outer == 0
    assert o.tol == 1e-12 and o.max_iter == 50 and o.max_nrhs == 16
    assert lib.lrspike_options_default(None, 1, 1, 1, 1) == 1
    assert (o.oversample, o.power_iters, o.seed) == (2, 2, 0x4C52535049)
    assert (o.otf_tol, o.otf_max_iter) == (1e-8, 100)


@pytest.mark.parametrize("changes", [
    dict(n=20000, k=100, r=8, pivoting=1),                 # wide bands: no pivoting
    dict(n=20000, k=100, r=8, compress=1),                 # wide bands: SPIKE compression only
    dict(n=20000, k=100, r=8, oversample=60),              # more than 64 sketch columns
    dict(n=20000, k=100, r=33),                            # r > 32 with the FULL reduced system
    dict(n=20000, k=100, r=65, reduced=1, precision=2),    # r > 64
    dict(n=20000, k=200, r=16, oversample=120, precision=2),  # more than 128 sketch columns (mixed)
    dict(precision=3),                                     # BF16 operands: wide bands only
    dict(reduced=2, pivoting=1),                           # OTF: no pivoting
    dict(reduced=2, outer=1),                              # OTF: outer IR or NONE
    dict(reduced=2, graph_safe=1),                         # OTF: not graph_safe
])
def test_create_reports_unbuilt_combinations(lib, changes):
    o = _opts(lib, n=changes.pop("n", 1000), k=changes.pop("k", 8), p=4, r=changes.pop("r", 2))
    for f, v in changes.items():
        setattr(o, f, v)
    h = ctypes.c_void_p()
    assert lib.lrspike_create(ctypes.byref(o), None, ctypes.byref(h)) == 7
    assert not h.value


@pytest.mark.parametrize("field,value", [("k", 1025), ("k", -1), ("r", 9), ("r", -1), ("p", 0),
                                         ("n", 0), ("max_nrhs", 0), ("max_nrhs", 17),
                                         ("precision", 7), ("outer", 5), ("compress", 2), ("reduced", 3),
                                         ("otf_tol", 0.0), ("otf_max_iter", 0)])
def test_create_rejects_bad_options(lib, field, value):
    o = _opts(lib)
    setattr(o, field, value)
    h = ctypes.c_void_p()
    st = lib.lrspike_create(ctypes.byref(o), None, ctypes.byref(h))
    assert st == 1, (field, value, st)
    assert not h.value
    assert len(lib.lrspike_last_error(None)) > 0


def test_otf_needs_partitions_and_rank(lib):
    for p, r in ((1, 2), (4, 0)):
        o = _opts(lib, p=p, r=r)
        o.reduced = 2
        h = ctypes.c_void_p()
        assert lib.lrspike_create(ctypes.byref(o), None, ctypes.byref(h)) == 1
        assert b"OTF" in lib.lrspike_last_error(None)


def test_create_rejects_partitions_not_wider_than_k(lib):
    o = _opts(lib, n=40, k=8, p=5, r=2)      # n_i = 8 = k
    h = ctypes.c_void_p()
    assert lib.lrspike_create(ctypes.byref(o), None, ctypes.byref(h)) == 1
    assert b"n_i > k" in lib.lrspike_last_error(None)


def test_null_handle_calls(lib):
    assert lib.lrspike_destroy(None) == 0
    assert lib.lrspike_factor(None, None, 0) == 1
    assert lib.lrspike_solve(None, None, None, 1, 1, None) == 1
    assert lib.lrspike_launch_count(None) == 0


def test_missing_library_raises(tmp_path, monkeypatch):
    monkeypatch.setattr(solver, "_lib", None)
    with pytest.raises(solver.LRSpikeError):
        solver.load_library(str(tmp_path / "nope.so"))


def test_fp64_probe_rejects_bad_arguments(lib):
    out = ctypes.c_double(0.0)
    assert lib.lrspike_fp64_fma_probe(0, ctypes.byref(out), None) == 1
    assert lib.lrspike_fp64_fma_probe(100, None, None) == 1
