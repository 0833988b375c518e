"""GPU parity on the shapes of the paper-derived workloads, at full
per-subdomain size, the oracle run on sampled subdomains:
  * prescribed spectrum sigma_i = 10^{-i/4} (m = 16384, n = 256), adaptive
    rank to tolerance 1e-3 with k_max = 32, p = 10;
  * uneven cubic boxes (edges 8..32, x 5 QoIs; windows 64..1024 snapshots,
    so some subdomains span two 512-column groups), adaptive 1e-3;
  * 32^3 x 5 boxes (m = 163840) of a 256^3 field, n = 256, snapshot-major
    window sketched in micro-batches of 64 columns as snapshots arrive,
    k = 30, p = 10.
Tolerances as in test_gpu_parity (derived there)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2103_01380_gb300 import inputs, spid
from _helpers import STATUS_OK, adaptive_margin, rel_fro, separated_prefix, U_MODE
from test_gpu_parity import GAP, Y_TOL, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2103_01380_gb300 import build
    build.build()


def check_sampled(win, g, precision, k_max, p, tol, samples, seed=0x5EED0001, err_target=None):
    u = U_MODE[precision]
    for s in samples:
        A = win.block(s).astype(np.float64)
        o = oracle.spid(A, k_max + p, k_max, tol, u, seed, want_y=True)
        dy = rel_fro(g["Y"][s], o["Y"])
        assert dy <= Y_TOL[precision], ("Y", s, dy)
        kg, ko = int(g["k"][s]), int(o["k"])
        if tol > 0 and kg != ko:
            margin = adaptive_margin(o["Y"], k_max, tol, ko)
            assert abs(kg - ko) <= (1 if precision == "fp32" else 2), ("k", s, kg, ko)
            if precision == "fp32":
                assert margin <= 64 * Y_TOL[precision], ("k margin", s, margin)
        pre = min(separated_prefix(o["Y"], max(ko, 1), GAP[precision], u), ko, kg)
        assert list(g["J"][s][:pre]) == list(o["J"][:pre]), ("J", s, g["J"][s][:kg], o["J"][:ko])
        eg = np.sqrt(g["err"][s, 0] / g["err"][s, 1])
        eo = np.sqrt(o["e2"] / o["a2"])
        assert eg <= max(err_target or 0.0, 2.0 * eo, 1e-6), ("err", s, eg, eo)


_SPECTRUM_WINDOW = {}


def _spectrum_window():
    if "w" not in _SPECTRUM_WINDOW:
        sig = 10.0 ** (-np.arange(1, 257) / 4.0)
        blocks = [inputs.spectrum_matrix(16384, 256, sig, seed=3 + s) for s in range(4)]
        _SPECTRUM_WINDOW["w"] = inputs.pack_blocks(blocks)
    return _SPECTRUM_WINDOW["w"]


@pytest.mark.parametrize("precision", ["fp32", "tf32", "bf16x3"])
def test_geometric_spectrum_adaptive_full_size(precision):
    win = _spectrum_window()
    g = run_gpu(win, precision, 32, p=10, tol=1e-3, reconstruct=False)
    assert g["status"] in STATUS_OK
    check_sampled(win, g, precision, 32, 10, 1e-3, samples=(0, 3), err_target=3e-3)
    # the best rank-12 error sits at 1e-3: adaptive ranks land just above it
    assert 10 <= int(np.median(g["k"])) <= 18
    assert np.sqrt(g["total"][0] / g["total"][1]) <= 3e-3


def test_geometric_spectrum_bf16_hits_its_noise_floor():
    # single-pass BF16 rounds A and Omega to 8 significand bits: the sketch's
    # noise (~1e-3 of ||Y||) sits at the tolerance, the rank guard (2^-8 |R_00|)
    # stops near sigma_10, and the error lands above 1e-3 -- reported, not hidden
    win = _spectrum_window()
    g = run_gpu(win, "bf16", 32, p=10, tol=1e-3, reconstruct=False)
    assert g["status"] in STATUS_OK
    check_sampled(win, g, "bf16", 32, 10, 1e-3, samples=(1,), err_target=3e-2)
    rel = np.sqrt(g["total"][0] / g["total"][1])
    assert rel <= 3e-2


@pytest.mark.parametrize("precision", ["fp32", "tf32"])
def test_uneven_boxes_adaptive(precision):
    boxes = inputs.uneven_boxes(8, seed=4)
    win = inputs.uneven_window(boxes)
    assert int(win.n.max()) > 512                       # two column groups somewhere
    g = run_gpu(win, precision, 32, p=10, tol=1e-3, reconstruct=False)
    assert g["status"] in STATUS_OK
    order = [int(i) for i in np.argsort(win.m * win.n)]
    wide = [i for i in order if win.n[i] > 512][0]      # smallest box with two column groups
    check_sampled(win, g, precision, 32, 10, 1e-3, samples=sorted({order[0], order[1], wide}),
                  err_target=1e-3)
    assert np.sqrt(g["total"][0] / g["total"][1]) <= 1e-3


def test_insitu_boxes_streamed_snapshot_major():
    # 4 boxes of 32^3 x 5 QoIs of the 256^3 field, n = 256, snapshot-major
    win = inputs.tgv3d_window(grid=256, box=32, n=256, boxes=4, layout="snapshot")
    assert int(win.m[0]) == 163840
    g = run_gpu(win, "tf32", 30, p=10, batches=64, reconstruct=False)
    assert g["status"] in STATUS_OK
    one = run_gpu(win, "tf32", 30, p=10, reconstruct=False)
    # the two schedules cut the 5120 row chunks into different partial sums:
    # the sketches agree up to FP32 re-association, about u sqrt(chunks)
    chunks = -(-int(win.m[0]) // 32)
    for s in range(4):
        assert rel_fro(g["Y"][s], one["Y"][s]) <= 2 * 2.0**-24 * np.sqrt(chunks)
    check_sampled(win, g, "tf32", 30, 10, 0.0, samples=(2,), err_target=1e-3)
    assert np.sqrt(g["total"][0] / g["total"][1]) <= 1e-3
