"""GPU parity of the error pass itself: A_hat = A(:,J) C and the Section 5.1
error sums, computed by the library from ITS OWN factors (k, J, C read back),
against the FP64 oracle's reconstruct_error on the same factors.  This
isolates the reconstruction from the sketch precision.

Bounds (element-wise, from the arithmetic):
  * tensor-core form (three-term TF32 split, FP32 accumulation):
      |A_hat - A_hat_o| <= 2 [(2.5 2^-21 + 3 (k + 1) 2^-24) (|A_J| |C|) + 2^-24 |A_hat_o|]
    (hi = tf32(x) leaves |lo| <= 2^-11 |x|; the lo operands lose at most
    2^-10 of themselves; the dropped lo x lo term is <= 2^-22; 3k products are
    summed in FP32; the result is stored in FP32; factor 2 for the unknown
    internal accumulation order of the tensor core);
  * CUDA-core form: (k + 1) 2^-24 (|A_J| |C|) + 2^-24 |A_hat_o|, doubled likewise;
  * sqrt(e2): |gpu - oracle| <= ||A_hat - A_hat_o||_F (triangle inequality)
    plus FP32 rounding of the squares; a2 to 1e-6 relative.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from _helpers import STATUS_OK
from paper_2103_01380_gb300 import inputs, spid
from test_gpu_parity import _lowrank_window, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2103_01380_gb300 import build
    build.build()
    spid.load_library()
    torch.cuda.init()


def _window():
    # ragged rows (not multiples of 128), column counts across the 256-column
    # blocks and not multiples of 16, one tall block spanning many CTAs
    m = [33, 200, 1000, 4099, 70001]
    n = [40, 300, 130, 600, 257]
    return _lowrank_window(5, m, n, 6, seed=50, noise=1e-3)


def _check_error_pass(win, g, tensor_core):
    for s in range(win.num_sub):
        A = win.block(s).astype(np.float64)
        k = int(g["k"][s])
        J = np.asarray(g["J"][s][:k], dtype=np.int64)
        C = np.asarray(g["C"][s][:k], dtype=np.float64)
        Ah_o, e2, a2 = oracle.reconstruct_error(A, J, C)
        B = np.abs(A[:, J]) @ np.abs(C) if k else np.zeros_like(A)
        if tensor_core:
            bound = 2 * ((2.5 * 2.0**-21 + 3 * (k + 1) * 2.0**-24) * B + 2.0**-24 * np.abs(Ah_o))
        else:
            bound = 2 * ((k + 1) * 2.0**-24 * B + 2.0**-24 * np.abs(Ah_o))
        diff = np.abs(g["Ahat"][s].astype(np.float64) - Ah_o)
        worst = np.max(diff - bound) if diff.size else 0.0
        assert worst <= 0.0, ("Ahat", s, k, float(np.max(diff)), float(worst))
        dF = np.sqrt(np.sum(diff ** 2))
        eg, eo = np.sqrt(g["err"][s, 0]), np.sqrt(e2)
        # FP32 differences and Kahan-summed squares: a few u of e itself
        assert abs(eg - eo) <= 1.01 * dF + 8 * 2.0**-24 * eo + 1e-30, ("e", s, eg, eo, dF)
        assert g["err"][s, 1] == pytest.approx(a2, rel=1e-6)


@pytest.mark.parametrize("precision", ["tf32", "bf16", "bf16x3"])
@pytest.mark.parametrize("k_max", [5, 20, 32])
def test_tensor_core_error_pass_on_own_factors(precision, k_max):
    win = _window()
    g = run_gpu(win, precision, k_max, p=8, flags=spid.FLAG_TC_ERROR)
    assert g["status"] in STATUS_OK
    assert int(g["k"].max()) > 0
    _check_error_pass(win, g, tensor_core=True)
    # window totals are the subdomain sums, and the CF sums are exact
    assert g["total"][0] == pytest.approx(g["err"][:, 0].sum(), rel=1e-12)
    assert g["total"][1] == pytest.approx(g["err"][:, 1].sum(), rel=1e-12)
    mn = float(np.sum(win.m.astype(np.float64) * win.n))
    kd = float(np.sum(g["k"] * (win.m.astype(np.float64) + win.n)))
    assert g["total"][2] == mn and g["total"][3] == kd


def test_tensor_core_and_cuda_core_error_passes_agree():
    win = _window()
    g_tc = run_gpu(win, "tf32", 20, p=8, flags=spid.FLAG_TC_ERROR)
    g_cc = run_gpu(win, "tf32", 20, p=8)
    # the sketch, QR and factors do not depend on the error-pass form
    assert np.array_equal(g_tc["k"], g_cc["k"]) and np.array_equal(g_tc["J"], g_cc["J"])
    assert all(np.array_equal(a, b) for a, b in zip(g_tc["C"], g_cc["C"]))   # ragged list
    _check_error_pass(win, g_cc, tensor_core=False)
    for s in range(win.num_sub):
        a2 = g_cc["err"][s, 1]
        assert g_tc["err"][s, 1] == pytest.approx(a2, rel=1e-6)
        d = np.sqrt(np.sum((g_tc["Ahat"][s].astype(np.float64) -
                                   g_cc["Ahat"][s].astype(np.float64)) ** 2) / a2)
        assert abs(np.sqrt(g_tc["err"][s, 0] / a2) - np.sqrt(g_cc["err"][s, 0] / a2)) <= 1.01 * d + 1e-6


def test_tensor_core_error_pass_repeats_bit_identically():
    # fixed schedule, fixed-order folds: the same call gives the same bits
    win = _window()
    plan = spid.Plan.for_window(win, k_max=12, p=8, precision="tf32", flags=spid.FLAG_TC_ERROR)
    w = torch.from_numpy(win.data).cuda()
    plan.sketch(w)
    plan.finalize()
    outs = []
    for _ in range(3):
        err = torch.zeros(2 * win.num_sub, dtype=torch.float64, device="cuda")
        tot = torch.zeros(4, dtype=torch.float64, device="cuda")
        plan.error(w, err, tot)
        torch.cuda.synchronize()
        outs.append((err.cpu().numpy(), tot.cpu().numpy()))
    for e, t in outs[1:]:
        assert np.array_equal(e, outs[0][0]) and np.array_equal(t, outs[0][1])
    assert plan.device_status() in STATUS_OK


def test_tensor_core_error_pass_rank_zero_blocks():
    # zero blocks get k = 0: A_hat = 0 and e2 = a2 = 0, next to a block of rank > 0
    blocks = [np.zeros((300, 40)), inputs.separated_lowrank(500, 70, 4, 7), np.zeros((129, 17))]
    win = inputs.pack_blocks(blocks)
    g = run_gpu(win, "tf32", 8, p=4, flags=spid.FLAG_TC_ERROR)
    assert g["status"] in STATUS_OK
    assert g["k"][0] == 0 and g["k"][2] == 0 and g["k"][1] > 0
    assert np.all(g["err"][[0, 2]] == 0.0)
    assert np.all(g["Ahat"][0] == 0.0) and np.all(g["Ahat"][2] == 0.0)
    _check_error_pass(win, g, tensor_core=True)
