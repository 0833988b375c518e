"""GPU parity of the coarse-grid column ID (Section 2 SubID / SPID,
Algorithms 2-3, Section 5.2) through the C ABI against the FP64 oracle on the
same seeded inputs.

Tolerances:
  * the coarse matrix B = A(J, :) is a gather of FP32 values: bit-exact;
  * pivots J: identical over the oracle's separated prefix of B (gap 1e-3 and
    the FP32 rounding floor, as for the FP32 sketch path); the coarse skeleton
    B(:, I_B) is then bit-exact too;
  * C_B: rel. Frobenius <= max(1e-5, 8 cond(R11) u), u = 2^-24;
  * SPID A_hat = M B(:,I_B) C_B: rel. Frobenius <= 2e-5 (FP32 trilinear weights
    and sums on top of the C_B tolerance);
  * error sums: sqrt(e2) within the A_hat difference (triangle inequality) and
    FP32 rounding; ||A||^2 to 1e-6 relative; CF sums exact.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2103_01380_gb300 import inputs, spid
from _helpers import r11_condition, rel_fro, separated_prefix

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2103_01380_gb300 import build
    build.build()
    spid.load_library()
    torch.cuda.init()


def run_sub(win, stride, k_max, tol=0.0, batches=None, reconstruct=True):
    plan = spid.SubPlan.for_window(win, stride, k_max=k_max, tol=tol)
    w = torch.from_numpy(win.data).cuda()
    if batches is None:
        plan.sample(w)
    else:
        for c0 in range(0, int(win.n.max()), batches):
            plan.sample(w, c0, batches)
    plan.finalize()
    S = win.num_sub
    res = {"plan": plan, "B": plan.coarse()}
    for form, tag in ((spid.FORM_SPID, "spid"), (spid.FORM_SUBID, "subid")):
        err = torch.zeros(2 * S, dtype=torch.float64, device="cuda")
        tot = torch.zeros(4, dtype=torch.float64, device="cuda")
        plan.error(w, form, err, tot)
        torch.cuda.synchronize()
        res["err_" + tag] = err.cpu().numpy().reshape(-1, 2)
        res["total_" + tag] = tot.cpu().numpy()
    if reconstruct:
        out = torch.zeros_like(w)
        plan.reconstruct(None, out, spid.FORM_SPID)
        torch.cuda.synchronize()
        ow = inputs.Window(out.cpu().numpy(), win.m, win.n, win.off, win.ld)
        res["Ahat_spid"] = [ow.block(s).copy() for s in range(S)]
    res["k"], res["J"], res["C"], res["Bskel"] = plan.factors()
    res["status"] = plan.device_status()
    return res


def check_sub_parity(win, stride, k_max, tol=0.0, **kw):
    g = run_sub(win, stride, k_max, tol, **kw)
    assert g["status"] == 0
    boxes = win.meta["boxes"]
    for s in range(win.num_sub):
        A = win.block(s).astype(np.float64)
        box = boxes[s]
        o = oracle.subid(A, box, stride, k_max, tol, U32, want_ahat=True)
        Bo = oracle.subsample(A, box, stride)
        assert np.array_equal(g["B"][s].astype(np.float64), Bo), ("B", s)
        kg, ko = int(g["k"][s]), o["k"]
        pre = min(separated_prefix(Bo, max(ko, 1), 1e-3, U32), ko, kg)
        assert list(g["J"][s][:pre]) == list(o["J"][:pre]), ("J", s, g["J"][s], o["J"], pre)
        if tol == 0.0:
            assert kg == ko, ("k", s, kg, ko)
        if kg == ko and list(g["J"][s][:kg]) == list(o["J"]):
            # C(:, J) = I exactly; the skeleton is the gathered columns
            assert np.array_equal(g["C"][s][:kg][:, o["J"]], np.eye(kg, dtype=np.float32))
            assert np.array_equal(g["Bskel"][s][:, :kg].astype(np.float64), o["Bskel"])
            ct = max(1e-5, 8.0 * r11_condition(Bo, ko) * U32)
            assert rel_fro(g["C"][s][:kg], o["C"]) <= ct, ("C", s)
            d = rel_fro(g["Ahat_spid"][s], o["Ahat_spid"])
            assert d <= 2e-5 + ct, ("Ahat", s, d)
            for tag, e2o in (("spid", o["e2_spid"]), ("subid", o["e2_subid"])):
                eg = np.sqrt(g["err_" + tag][s, 0])
                # ||A_hat_gpu - A_hat_oracle||_F: measured for SPID; for SubID
                # ||A(:,J)|| ||C_gpu - C_oracle|| plus the FP32 error pass
                if tag == "spid":
                    dA = d * np.linalg.norm(o["Ahat_spid"])
                else:
                    dA = (ct + 8 * kg * U32) * np.linalg.norm(o["C"]) * np.sqrt(o["a2"])
                assert abs(eg - np.sqrt(e2o)) <= 1.01 * dA + 8 * U32 * np.sqrt(o["a2"]), \
                    (tag, s, eg, np.sqrt(e2o))
        for tag in ("spid", "subid"):
            assert g["err_" + tag][s, 1] == pytest.approx(o["a2"], rel=1e-6)
    m = win.m.astype(np.float64)
    n = win.n.astype(np.float64)
    mc = g["plan"].mc.astype(np.float64)
    k = g["k"].astype(np.float64)
    assert g["total_spid"][2] == np.sum(m * n) and g["total_spid"][3] == np.sum(k * (mc + n))
    assert g["total_subid"][3] == np.sum(k * (m + n))
    return g


def test_subsample_parity_and_fixed_rank():
    boxes = [(5, 16, 16, 16), (1, 9, 10, 11), (3, 7, 5, 13), (2, 1, 4, 6)]
    win = inputs.box_window(boxes, [60, 33, 80, 17], seed=11, noise=1e-4)
    check_sub_parity(win, (3, 3, 3), 6)


@pytest.mark.parametrize("stride", [(1, 1, 1), (2, 3, 4), (5, 5, 5)])
def test_strides_including_plain_column_id(stride):
    boxes = [(2, 12, 10, 9), (1, 16, 16, 16), (4, 5, 6, 7)]
    win = inputs.box_window(boxes, 48, seed=21, noise=1e-4)
    check_sub_parity(win, stride, 5)


def test_adaptive_rank_and_streamed_columns():
    boxes = [(5, 16, 16, 16)] * 3 + [(1, 20, 8, 12)]
    win = inputs.box_window(boxes, 256, seed=31, noise=1e-5)
    g = check_sub_parity(win, (3, 3, 3), 16, tol=1e-2, batches=64)
    assert np.all(g["k"] >= 1) and np.all(g["k"] <= 16)


def test_large_coarse_grid_reads_columns_twice_and_rewrites_w():
    # m_c = 8000 and 2400: too many rows for the per-warp shared column buffers, so
    # each MGS pass reads the column from memory; a fixed rank of 5 makes the QR
    # rewrite its working copy once the pending-update slots are full
    boxes = [(1, 40, 40, 40), (1, 30, 20, 16)]
    win = inputs.box_window(boxes, 40, seed=45, noise=1e-4)
    g = check_sub_parity(win, (2, 2, 2), 5)
    assert list(g["k"]) == [5, 5]


def test_edge_cases_rank_capped_by_coarse_rows_and_columns():
    # k_max above n and above m_c; a single-point box; a one-column window
    boxes = [(1, 3, 3, 3), (1, 1, 1, 1), (2, 4, 4, 4)]
    win = inputs.box_window(boxes, [5, 7, 1], seed=41, noise=1e-2)
    g = check_sub_parity(win, (2, 2, 2), 12)
    assert g["k"][0] <= 5 and g["k"][1] <= 1 and g["k"][2] <= 1


def test_e3_rank_one_tgv_compression_factor():
    # Section 5.2: 64^3 points, u1 of the TGV, 100 snapshots, interval 3: rank 1
    # and CF = m n / (k (m_c + n)) ~ 2400 with an interpolation error of ~ 1-2 %
    t = np.linspace(0.0, 10.0, 100)
    u1 = inputs.tgv3d_u1(64, t)
    win = inputs.pack_blocks([u1])
    win.meta["boxes"] = np.array([[1, 64, 64, 64]], dtype=np.int32)
    g = run_sub(win, (3, 3, 3), 4, tol=1e-3, reconstruct=False)
    assert g["status"] == 0 and int(g["k"][0]) == 1
    cf = g["total_spid"][2] / g["total_spid"][3]
    assert cf == pytest.approx(64 ** 3 * 100 / (22 ** 3 + 100))
    assert 2400 <= cf <= 2450
    rel = np.sqrt(g["total_spid"][0] / g["total_spid"][1])
    o = oracle.subid(u1.astype(np.float64), (1, 64, 64, 64), (3, 3, 3), 4, 1e-3, U32)
    assert o["k"] == 1
    assert rel == pytest.approx(np.sqrt(o["e2_spid"] / o["a2"]), rel=1e-3)
    assert 1e-3 < rel < 3e-2
    # the SubID form keeps the fine skeleton column: CF = m n / (m + n) ~ 100
    assert round(g["total_subid"][2] / g["total_subid"][3]) == 100


def test_nonfinite_coarse_matrix_is_reported():
    boxes = [(1, 6, 6, 6), (1, 6, 6, 6)]
    win = inputs.box_window(boxes, 10, seed=51)
    win.block(0)[0, 3] = np.nan          # row 0 is a coarse point
    g = run_sub(win, (2, 2, 2), 3, reconstruct=False)
    assert g["status"] == 6             # SPID_ERR_NONFINITE
    assert g["k"][0] == 0 and g["k"][1] > 0


def test_nonfinite_in_a_later_gather_part_is_reported():
    # two boxes x 10 snapshots are too few columns to fill the GPU, so the gather
    # splits each 12^3-row coarse column into parts; the inf sits in the last one
    boxes = [(1, 24, 24, 24), (1, 24, 24, 24)]
    win = inputs.box_window(boxes, 10, seed=53)
    win.block(1)[(22 * 24 + 22) * 24 + 22, 7] = np.inf   # coarse point (11, 11, 11)
    g = run_sub(win, (2, 2, 2), 3, reconstruct=False)
    assert g["status"] == 6
    assert g["k"][1] == 0 and g["k"][0] > 0


def test_sample_then_repeat_is_bit_identical():
    boxes = [(5, 16, 16, 16)] * 4
    win = inputs.box_window(boxes, 128, seed=61, noise=1e-4)
    a = run_sub(win, (3, 3, 3), 8, reconstruct=False)
    b = run_sub(win, (3, 3, 3), 8, reconstruct=False)
    assert np.array_equal(a["J"], b["J"])
    assert all(np.array_equal(x, y) for x, y in zip(a["C"], b["C"]))
    assert np.array_equal(a["err_spid"], b["err_spid"])
    assert np.array_equal(a["total_spid"], b["total_spid"])


def test_fine_skeleton_and_staged_spid_passes_agree():
    # With the window, the SPID error pass and reconstruction interpolate the k
    # skeleton columns once (F = M B(:, I_B), m x k) and form A_hat = F C_B in
    # the rank-k error kernel; without it, the reconstruction forms G = B(:,
    # I_B) C_B on the coarse grid first and then M G.  Both are exact
    # rearrangements of M B(:, I_B) C_B (M is linear), so they differ by FP32
    # rounding only: per element at most (k + 4) ulps of
    # sum_p max|B(:, I_B)(:, p)| |C_B(p, j)| (trilinear weights are convex),
    # x8 for the unknown contraction order.  The error sums follow from the
    # A_hat difference (triangle inequality) and the compensated FP32 sums.
    boxes = [(5, 16, 16, 16), (2, 20, 8, 12), (3, 32, 32, 32), (1, 8, 8, 8), (4, 9, 4, 4),
             (2, 6, 2, 6), (1, 7, 5, 3)]
    n = [70, 33, 40, 129, 64, 20, 31]
    win = inputs.box_window(boxes, n, seed=71, noise=1e-4)
    check_sub_parity(win, (3, 3, 3), 6)
    plan = spid.SubPlan.for_window(win, (3, 3, 3), k_max=6)
    w = torch.from_numpy(win.data).cuda()
    plan.sample(w)
    plan.finalize()
    S = win.num_sub
    err = torch.zeros(2 * S, dtype=torch.float64, device="cuda")
    tot = torch.zeros(4, dtype=torch.float64, device="cuda")
    plan.error(w, spid.FORM_SPID, err, tot)
    fine = torch.zeros_like(w)
    staged = torch.zeros_like(w)
    plan.reconstruct(w, fine, spid.FORM_SPID)
    plan.reconstruct(None, staged, spid.FORM_SPID)
    torch.cuda.synchronize()
    assert plan.device_status() == 0
    k, _, C, Bsk = plan.factors()
    e = err.cpu().numpy().reshape(-1, 2)
    wf = inputs.Window(fine.cpu().numpy(), win.m, win.n, win.off, win.ld)
    wt = inputs.Window(staged.cpu().numpy(), win.m, win.n, win.off, win.ld)
    for s in range(S):
        kk = int(k[s])
        a_f, a_t = wf.block(s).astype(np.float64), wt.block(s).astype(np.float64)
        bmax = np.abs(Bsk[s][:, :kk].astype(np.float64)).max(axis=0) if kk else np.zeros(0)
        scale = (np.abs(C[s][:kk].astype(np.float64)) * bmax[:, None]).sum(axis=0)   # per column
        assert np.all(np.abs(a_f - a_t) <= 8 * (kk + 4) * U32 * scale[None, :] + 1e-30), s
        A = win.block(s).astype(np.float64)
        e2 = float(((A - a_t) ** 2).sum())
        a2 = float((A ** 2).sum())
        d = np.linalg.norm(a_f - a_t)
        assert abs(e[s, 0] - e2) <= 2 * np.sqrt(e2) * d + d * d + 1e-5 * e2, s
        assert e[s, 1] == pytest.approx(a2, rel=1e-6)
    plan.close()
