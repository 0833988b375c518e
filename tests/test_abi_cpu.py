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
    assert lib.spid_graph_launch_host(None, None, None, None, None, None, None, None) == 1
    assert lib.spid_finalize(None, None) == 1
    assert lib.spid_sketch_accumulate(None, None, 0, 1, None) == 1


def _box_plan(precision="fp32", nq=5, XYZ=(64, 24, 20), org=((0, 0, 0),), ext=((32, 8, 8),),
              split=False, snap_stride=None, n=None, **kw):
    lay = spid.BoxLayout(nq, *XYZ, org, ext, split_qoi=split, snap_stride=snap_stride)
    return spid.Plan(None, n if n is not None else [16] * lay.num_sub, None, None, k_max=4, p=4,
                     precision=precision, boxes=lay, **kw)


@pytest.mark.parametrize("kw,status", [
    (dict(org=((2, 0, 0),)), 1),                     # x origin not 16-byte aligned
    (dict(ext=((30, 8, 8),)), 1),                    # x extent not 16-byte aligned
    (dict(org=((48, 0, 0),)), 1),                    # box leaves the field along x
    (dict(org=((0, 20, 0),)), 1),                    # ... along y
    (dict(ext=((32, 8, 0),)), 1),                    # empty box
    (dict(XYZ=(66, 24, 20)), 1),                     # X not a multiple of 4
    (dict(snap_stride=5 * 64 * 24 * 20 - 4), 1),     # snapshots overlap
    (dict(split=True, num_qoi=3), 1),                # num_qoi neither 0 nor nq
    (dict(qoi=[7], num_qoi=5), 1),                   # QoI label out of range
    (dict(num_qoi=2), 1),                            # per-QoI totals without labels
    (dict(precision="tf32", ext=((16, 8, 8),)), 7),  # tensor cores: x runs of 32 only
])
def test_invalid_box_layouts_are_rejected_without_a_gpu(lib, kw, status):
    with pytest.raises(spid.SpidError) as e:
        _box_plan(**kw)
    assert e.value.status == status, str(e.value)


@pytest.mark.parametrize("split,num_sub", [(0, 2), (1, 1), (1, 6)])
def test_box_count_must_match_num_sub(lib, split, num_sub):
    # the C check itself (the binding derives num_sub from the layout)
    import ctypes
    org = np.array([0, 0, 0], dtype=np.int32)
    ext = np.array([32, 8, 8], dtype=np.int32)
    n = np.full(num_sub, 16, dtype=np.int32)
    b = spid._BoxLayout()
    b.nq, b.X, b.Y, b.Z, b.snap_stride, b.num_box = 5, 64, 24, 20, 5 * 64 * 24 * 20, 1
    b.org3 = org.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    b.ext3 = ext.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    b.split_qoi = split
    d = spid._Desc()
    d.num_sub = num_sub
    d.n = n.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    d.k_max, d.p, d.precision, d.seed = 4, 4, 1, 1
    d.boxes = ctypes.pointer(b)
    h = ctypes.c_void_p()
    assert lib.spid_plan_create(ctypes.byref(d), None, ctypes.byref(h)) == 1


def test_box_layout_rows_and_qoi_labels():
    lay = spid.BoxLayout(5, 64, 24, 20, [(0, 0, 0), (32, 4, 2)], [(32, 8, 4), (32, 16, 16)],
                         split_qoi=True)
    assert lay.num_sub == 10
    assert list(lay.m) == [32 * 8 * 4] * 5 + [32 * 16 * 16] * 5
    stacked = spid.BoxLayout(5, 64, 24, 20, [(0, 0, 0)], [(32, 8, 4)])
    assert list(stacked.m) == [5 * 32 * 8 * 4]


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
