"""CPU checks of the C ABI: the library loads, exports every symbol that
include/spid.h declares, rejects invalid arguments before touching a GPU, and
its host-side compression factor matches the paper's worked values."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from paper_2103_01380_gb300 import spid

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2103_01380_gb300 import build
    build.build()
    return spid.load_library()


def _declared_symbols():
    text = open(os.path.join(ROOT, "include", "spid.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(spid_[a-z_0-9]+)\s*\(", text)))


def test_header_and_binding_agree():
    assert _declared_symbols() == sorted(spid.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_symbols():
        assert hasattr(lib, name), name


def test_status_strings(lib):
    for code, name in spid.STATUS_NAMES.items():
        assert lib.spid_status_string(code).decode() == name


def _create(**kw):
    base = dict(m=[64], n=[16], off=[0], ld=[64], k_max=4, p=4, tol=0.0, precision="fp32")
    base.update(kw)
    return spid.Plan(**base)


@pytest.mark.parametrize("kw", [
    dict(m=[0]), dict(n=[0]), dict(ld=[32]), dict(off=[2]), dict(ld=[66]),
    dict(k_max=0), dict(p=-1), dict(k_max=60, p=10), dict(tol=-1.0), dict(precision="fp64", off=[1]),
])
def test_invalid_descriptors_are_rejected_without_a_gpu(lib, kw):
    with pytest.raises(spid.SpidError) as e:
        _create(**kw)
    assert e.value.status == 1, str(e.value)


def test_null_plan_is_rejected(lib):
    assert lib.spid_graph_launch_host(None, None, None, None, None) == 1
    assert lib.spid_finalize(None, None) == 1
    assert lib.spid_sketch(None, None, 0, 1, None) == 1


def test_compression_factor_matches_oracle_and_paper(lib):
    cases = [([400], [100], [1], 80.0),
             ([20] * 5, [100] * 5, [6, 12, 6, 12, 12], 1.7361111111111112),
             ([50, 50], [100, 100], [24, 30], 1.2345679012345678)]
    for m, n, k, val in cases:
        assert spid.compression_factor(m, n, k) == pytest.approx(val, rel=1e-14)
        assert spid.compression_factor(m, n, k) == pytest.approx(oracle.compression_factor(m, n, k),
                                                                 rel=1e-15)
    assert spid.compression_factor([10], [10], [0]) == float("inf")


def test_invalid_point_sets_are_rejected(lib):
    # argument checks run before any device call
    from paper_2103_01380_gb300 import inputs
    win = inputs.pack_blocks([np.ones((20, 5))])
    ok = dict(crows=[np.arange(5)], idxs=[np.zeros((20, 2), np.int32)], ws=[np.ones((20, 2))])
    for bad in (dict(crows=[np.array([0, 1, 99])]),                       # row out of range
                dict(idxs=[np.full((20, 2), 7, np.int32)]),               # coarse index out of range
                dict(ws=[np.full((20, 2), np.nan)])):                    # non-finite weight
        a = dict(ok, **bad)
        with pytest.raises(spid.SpidError) as ei:
            spid.SubPlan.from_points(win.m, win.n, win.off, win.ld, a["crows"], a["idxs"],
                                     a["ws"], 3)
        assert ei.value.status == 1


def test_producer_rejects_bad_arguments(lib):
    import ctypes
    buf = ctypes.create_string_buffer(64)
    p = ctypes.addressof(buf)
    be = 5 * 8 ** 3
    for args in ((p, be, p, be, 16, 8, 5, 0.01, 0.01),          # in == out
                 (p, be, p + 16, be, 16, 5, 5, 0.01, 0.01),     # grid % edge != 0
                 (p, be, p + 16, be, 16, 8, 3, 0.01, 0.01),     # nq < 4
                 (p, be, p + 16, be, 16, 8, 5, 0.0, 0.01),      # dt <= 0
                 (p, be - 1, p + 16, be, 16, 8, 5, 0.01, 0.01)):   # box stride too small
        assert lib.spid_producer_step(*args, None) == 1


def test_host_buffer_marshalling_checks():
    # the binding's host-pointer checks for spid_graph_launch_host run on the CPU
    import torch
    a = np.zeros(16, dtype=np.float32)
    assert spid._host_ptr(a, np.float32, 64) == a.ctypes.data
    t = torch.zeros(16, dtype=torch.float32)
    assert spid._host_ptr(t, np.float32, 64) == t.data_ptr()
    with pytest.raises(ValueError):
        spid._host_ptr(a, np.float32, 65)            # shorter than needed
    with pytest.raises(ValueError):
        spid._host_ptr(a, np.float64, 8)             # wrong element type
    with pytest.raises(ValueError):
        spid._host_ptr(a[::2], np.float32, 8)        # not contiguous
    with pytest.raises(ValueError):
        spid._host_ptr(t[::2], np.float32, 8)
