"""GPU parity of the coarse-grid ID on arbitrary point sets (unstructured
grids: Section 2 allows the rows of A in any order; Section 5.1 compresses the
2D TGV on randomly generated points) through the C ABI against the FP64
oracle on the same seeded inputs.

Tolerances (as for boxes):
  * B = A(coarse rows, :) is a gather of FP32 values: bit-exact;
  * J over the oracle's separated prefix of B (gap 1e-3 and the FP32 rounding
    floor); the skeleton B(:, I_B) then bit-exact;
  * C_B: rel. Frobenius <= max(1e-5, 8 cond(R11) u), u = 2^-24;
  * SPID A_hat = M B(:, I_B) C_B: rel. Frobenius <= 2e-5 + the C tolerance
    (FP32 stencil sums and the rank-k product on top of C);
  * error sums: within the A_hat difference (triangle inequality) and FP32
    rounding; ||A||^2 to 1e-6; CF sums exact.
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


def point_window(npts, n, nbx, nby, frac, t, method, seed, qois=("u1", "u2"), modes=4,
                 noise=1e-4):
    """Random points of the 2D TGV field partitioned into nbx x nby blocks; per
    block a random coarse subset (frac of its points) and its stencil."""
    pts, A = inputs.unstructured_tgv2d(npts, n, seed=seed, qois=qois, smooth_modes=modes,
                                       noise=noise)
    nq = len(qois)
    blocks, crows, idxs, ws = [], [], [], []
    for b, part in enumerate(inputs.point_partitions(pts, nbx, nby)):
        rows = np.concatenate([q * npts + part for q in range(nq)])
        blocks.append(A[rows])
        mc = max(4, int(round(frac * len(part))))
        cr, ix, w = inputs.coarse_stencil(pts[part], mc, t, seed=seed + 100 + b, nq=nq,
                                          method=method)
        crows.append(cr)
        idxs.append(ix)
        ws.append(w)
    win = inputs.pack_blocks(blocks)
    return win, crows, idxs, ws


def run_points(win, crows, idxs, ws, k_max, tol=0.0, batches=None):
    plan = spid.SubPlan.from_points(win.m, win.n, win.off, win.ld, crows, idxs, ws, k_max, tol)
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
    out = torch.zeros_like(w)
    plan.reconstruct(None, out, spid.FORM_SPID)          # F C_B, no window
    out2 = torch.zeros_like(w)
    plan.reconstruct(w, out2, spid.FORM_SPID)            # the error kernel's A_hat
    torch.cuda.synchronize()
    o1 = inputs.Window(out.cpu().numpy(), win.m, win.n, win.off, win.ld)
    o2 = inputs.Window(out2.cpu().numpy(), win.m, win.n, win.off, win.ld)
    res["Ahat"] = [o1.block(s).copy() for s in range(S)]
    res["Ahat_w"] = [o2.block(s).copy() for s in range(S)]
    res["k"], res["J"], res["C"], res["Bskel"] = plan.factors()
    res["status"] = plan.device_status()
    return res


def check_points_parity(win, crows, idxs, ws, k_max, tol=0.0, **kw):
    g = run_points(win, crows, idxs, ws, k_max, tol, **kw)
    assert g["status"] == 0
    for s in range(win.num_sub):
        A = win.block(s).astype(np.float64)
        o = oracle.subid_points(A, crows[s], idxs[s], ws[s], k_max, tol, U32, want_ahat=True)
        Bo = A[np.asarray(crows[s])]
        assert np.array_equal(g["B"][s].astype(np.float64), Bo), ("B", s)
        kg, ko = int(g["k"][s]), o["k"]
        pre = min(separated_prefix(Bo, max(ko, 1), 1e-3, U32), ko, kg)
        assert list(g["J"][s][:pre]) == list(o["J"][:pre]), ("J", s)
        if tol == 0.0:
            assert kg == ko, ("k", s, kg, ko)
        # the two GPU reconstructions are the same rank-k product in two kernels
        scale = np.abs(g["Ahat"][s]).max() + 1e-30
        assert np.max(np.abs(g["Ahat_w"][s] - g["Ahat"][s])) <= 64 * U32 * scale, ("Ahat_w", s)
        if kg == ko and list(g["J"][s][:kg]) == list(o["J"]):
            assert np.array_equal(g["C"][s][:kg][:, o["J"]], np.eye(kg, dtype=np.float32))
            assert np.array_equal(g["Bskel"][s][:, :kg].astype(np.float64), o["Bskel"])
            ct = max(1e-5, 8.0 * r11_condition(Bo, ko) * U32)
            assert rel_fro(g["C"][s][:kg], o["C"]) <= ct, ("C", s)
            d = rel_fro(g["Ahat"][s], o["Ahat_spid"])
            assert d <= 2e-5 + ct, ("Ahat", s, d)
            eg = np.sqrt(g["err_spid"][s, 0])
            dA = d * np.linalg.norm(o["Ahat_spid"])
            assert abs(eg - np.sqrt(o["e2_spid"])) <= 1.01 * dA + 8 * U32 * np.sqrt(o["a2"]) + \
                64 * U32 * np.sqrt(A.size) * scale, ("e_spid", s)
        for tag in ("spid", "subid"):
            assert g["err_" + tag][s, 1] == pytest.approx(o["a2"], rel=1e-6)
    m = win.m.astype(np.float64)
    n = win.n.astype(np.float64)
    mc = np.array([len(c) for c in crows], dtype=np.float64)
    k = g["k"].astype(np.float64)
    assert g["total_spid"][2] == np.sum(m * n) and g["total_spid"][3] == np.sum(k * (mc + n))
    assert g["total_subid"][3] == np.sum(k * (m + n))
    return g


@pytest.mark.parametrize("method,t", [("linear", 3), ("idw", 4), ("idw", 1)])
def test_unstructured_tgv_parity(method, t):
    win, crows, idxs, ws = point_window(1200, 90, 2, 2, 0.25, t, method, seed=21)
    check_points_parity(win, crows, idxs, ws, 6)


def test_unstructured_adaptive_streamed_columns_ragged():
    # uneven blocks (random points), window crossing 256-column blocks, columns
    # gathered in micro-batches of 64 as snapshots arrive
    win, crows, idxs, ws = point_window(2500, 300, 3, 2, 0.2, 3, "linear", seed=31)
    g = check_points_parity(win, crows, idxs, ws, 12, tol=1e-3, batches=64)
    assert np.all(g["k"] >= 1)


def test_box_as_point_set_matches_the_box_plan():
    # the same box through both plan kinds: identical B, J, C (same gather, same
    # QR kernel); A_hat from the 8-point stencil vs the trilinear kernel agree to
    # FP32 rounding
    box, stride = (3, 10, 8, 12), (3, 3, 4)
    win = inputs.box_window([box, box], [50, 70], seed=41, noise=1e-4)
    bp = spid.SubPlan.for_window(win, stride, k_max=5)
    from test_oracle_points import _box_as_points
    crow, idx, w = _box_as_points(box, stride)
    pp = spid.SubPlan.from_points(win.m, win.n, win.off, win.ld, [crow, crow], [idx, idx], [w, w], 5)
    dev = torch.from_numpy(win.data).cuda()
    outs = []
    for plan in (bp, pp):
        plan.sample(dev)
        plan.finalize()
        out = torch.zeros_like(dev)
        plan.reconstruct(None, out, spid.FORM_SPID)
        torch.cuda.synchronize()
        outs.append((plan.coarse(), plan.factors(), out.cpu().numpy()))
        assert plan.device_status() == 0
    (Bb, fb, ob), (Bp, fp, op) = outs
    for s in range(2):
        assert np.array_equal(Bb[s], Bp[s])
    assert np.array_equal(fb[0], fp[0]) and np.array_equal(fb[1], fp[1])
    for s in range(2):
        assert np.array_equal(fb[2][s], fp[2][s])
    assert np.max(np.abs(ob - op)) <= 64 * U32 * np.abs(ob).max()
    bp.close()
    pp.close()
