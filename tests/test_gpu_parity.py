"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle on
the same seeded inputs.

Tolerances (element-wise relative Frobenius norms unless stated):
  * Philox words: bit-exact.  Omega: FP64 <= 1e-13 abs, FP32 <= 2e-5 abs.
  * Sketch Y: FP64 <= 1e-13, FP32 <= 2e-6, TF32 <= 3e-3 (FP32 data truncated
    to TF32's 10-bit mantissa, two roundings of ~2^-11 each, random signs).
  * J: identical over the oracle's separated pivot prefix (gap 1e-6 FP64,
    1e-3 FP32, 2e-2 TF32); past it several pivots are valid and only the
    reconstruction is compared.
  * C and A_hat: <= 1e-10 in FP64 mode, <= 1e-5 in FP32 mode (on inputs whose
    R11 is well conditioned for C; A_hat always).
  * Relative error sqrt(e2/a2): |gpu - oracle| <= the A_hat difference bound.
  * TF32: final relative error <= max(1e-3, 2 x oracle) on the workloads here.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2103_01380_gb300 import inputs, spid
from _helpers import (GAP, Y_TOL, ahat_matches_factors, compare_with_oracle, oracle_window, rel_fro,
                      separated_prefix, U_MODE)

pytestmark = pytest.mark.gpu

# GAP / Y_TOL (tests/_helpers.py): BF16 keeps 8 significand bits of A and
# Omega (two roundings of up to 2^-9); 3xBF16 drops only the lo x lo product and
# the 16-bit tails (~2^-16)
# final relative error the low-precision sketches must reach on the separated
# low-rank inputs here (data noise 1e-3 sets the oracle's own error)
ERR_CAP = {"tf32": 1e-3, "bf16x3": 1e-3, "bf16": 1e-2}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2103_01380_gb300 import build
    build.build()
    spid.load_library()
    torch.cuda.init()


def _dev(win):
    return torch.from_numpy(win.data).cuda()


def run_gpu(win, precision, k_max, p=10, tol=0.0, seed=0x5EED0001, flags=0, window=None,
            batches=None, reconstruct=True, qoi=None, num_qoi=0):
    plan = spid.Plan.for_window(win, k_max=k_max, p=p, tol=tol, precision=precision, seed=seed,
                                flags=flags, qoi=qoi, num_qoi=num_qoi)
    w = _dev(win) if window is None else window
    if batches is None:
        plan.sketch(w)
    else:
        for c0 in range(0, int(win.n.max()), batches):
            plan.sketch(w, c0, batches)
    plan.finalize()
    err = torch.zeros(2 * win.num_sub, dtype=torch.float64, device="cuda")
    tot = torch.zeros(plan.total_len, dtype=torch.float64, device="cuda")
    plan.error(w, err, tot)
    out = torch.zeros_like(w) if reconstruct else None
    if reconstruct:
        plan.reconstruct(w, out)
    torch.cuda.synchronize()
    k, J, C = plan.factors()
    Y = plan.sketches()
    res = {"k": k, "J": J, "C": C, "Y": Y, "err": err.cpu().numpy().reshape(-1, 2),
           "total": tot.cpu().numpy(), "status": plan.device_status(), "plan": plan}
    if reconstruct:
        ow = inputs.Window(out.cpu().numpy(), win.m, win.n, win.off, win.ld)
        res["Ahat"] = [ow.block(s).copy() for s in range(win.num_sub)]
    return res


def check_parity(win, precision, k_max, p=10, tol=0.0, seed=0x5EED0001, c_tol=None,
                 ahat_tol=None, min_prefix=0, **kw):
    g = run_gpu(win, precision, k_max, p, tol, seed, **kw)
    o = oracle_window(win, k_max + p, k_max, tol, precision, seed)
    compare_with_oracle([win.block(s) for s in range(win.num_sub)], g, o, precision, k_max, tol,
                        c_tol=c_tol, ahat_tol=ahat_tol, min_prefix=min_prefix)
    return g, o


# ---------------------------------------------------------------- RNG
def test_philox_bitexact():
    rng = np.random.default_rng(3)
    ctr = rng.integers(0, 2 ** 32, size=(20000, 4), dtype=np.uint64).astype(np.uint32)
    ctr[:3] = [[0, 0, 0, 0], [0xffffffff] * 4, [0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344]]
    for key in [(0, 0), (0xffffffff, 0xffffffff), (0xa4093822, 0x299f31d0), (12345, 678)]:
        out = torch.zeros(ctr.size, dtype=torch.int32, device="cuda")
        spid.philox(torch.from_numpy(ctr.view(np.int32)).cuda(), key[0], key[1], out)
        torch.cuda.synchronize()
        got = out.cpu().numpy().view(np.uint32).reshape(-1, 4)
        want = oracle.philox4x32_10(ctr, key)
        assert np.array_equal(got, want)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-13), ("fp32", 2e-5)])
def test_omega_matches_oracle(precision, tol):
    seed, r0, nrows, l = 0x5EED0002, 12345, 4000, 42
    dt = torch.float64 if precision == "fp64" else torch.float32
    out = torch.zeros(nrows * l, dtype=dt, device="cuda")
    spid.omega(seed, r0, nrows, l, precision, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64).reshape(nrows, l).T
    want = oracle.omega(seed, r0, nrows, l)
    assert np.max(np.abs(got - want)) <= tol


# ---------------------------------------------------------------- whole path
def _lowrank_window(S, m, n, r, seed, noise=1e-4, dtype=np.float32, layout="subdomain", decay=0.5):
    blocks = [inputs.separated_lowrank(m[s] if np.ndim(m) else m, n[s] if np.ndim(n) else n, r,
                                       seed + s, decay=decay, noise=noise) for s in range(S)]
    return inputs.pack_blocks(blocks, dtype=dtype, layout=layout)


def test_fp64_parity_tgv2d_full_config():
    # 2D analytic TGV + 1e-6 noise, m = 8192, n = 128, k = 10, p = 10 (Section 5.1 case)
    A = inputs.tgv2d(nx=64, n=128, noise=1e-6, seed=1)
    win = inputs.pack_blocks([A], dtype=np.float64)
    g, o = check_parity(win, "fp64", 10, c_tol=1e-10, ahat_tol=1e-10, seed=0x5EED0001)
    assert g["k"][0] == 10
    rel = np.sqrt(g["total"][0] / g["total"][1])
    assert rel < 1e-5
    assert g["total"][2] / g["total"][3] == pytest.approx(8192 * 128 / (10 * (8192 + 128)))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_parity_ragged_multi_subdomain(precision):
    # several subdomains with ragged rows (not a multiple of 32) and columns
    # crossing 128-column tiles and column groups
    m = [33, 200, 1000, 517]
    n = [40, 300, 130, 600] if precision == "fp32" else [40, 300, 130, 257]
    dt = np.float64 if precision == "fp64" else np.float32
    win = _lowrank_window(4, m, n, 6, seed=10, dtype=dt)
    tol = 1e-10 if precision == "fp64" else 1e-5
    check_parity(win, precision, 5, p=8, c_tol=tol, ahat_tol=tol, min_prefix=5)


@pytest.mark.parametrize("precision", ["tf32", "bf16x3", "bf16"])
def test_tensor_core_sketch_accuracy_and_parity(precision):
    m = [33, 200, 1000, 4099]
    n = [40, 300, 130, 600]
    win = _lowrank_window(4, m, n, 6, seed=20, noise=1e-3)
    g, o = check_parity(win, precision, 5, p=8,
                        ahat_tol=1e-4 if precision == "bf16x3" else None)
    for s in range(4):
        eg = np.sqrt(g["err"][s, 0] / g["err"][s, 1])
        eo = np.sqrt(o["e2"][s] / o["a2"][s])
        assert eg <= max(ERR_CAP[precision], 2.0 * eo), (s, eg, eo)


@pytest.mark.parametrize("precision,prefix", [("tf32", 5), ("bf16x3", 5), ("bf16", 3)])
def test_tensor_core_separated_pivots(precision, prefix):
    # leading columns decided with a wide margin (each residual ~2x the next):
    # the tensor-core sketches must pick the oracle's pivots over the whole
    # separated prefix and the same rank; C within 8 cond(R11) u of the oracle's
    m = [33, 200, 1000, 4099]
    n = [40, 300, 130, 600]
    blocks = [inputs.separated_columns(m[s], n[s], 5, 20 + s, ratio=0.5, noise=1e-4)
              for s in range(4)]
    win = inputs.pack_blocks(blocks)
    g, o = check_parity(win, precision, 5, p=8, c_tol=1e-5, min_prefix=prefix)
    assert list(g["k"]) == [5, 5, 5, 5]


def test_snapshot_major_layout():
    # [j][s][r] window: every snapshot contiguous, ld = sum of padded rows
    win = _lowrank_window(3, [100, 64, 257], [90, 90, 90], 5, seed=30, layout="snapshot")
    for prec in ("fp32", "tf32", "bf16x3"):
        check_parity(win, prec, 4, p=6, ahat_tol={"fp32": 1e-5, "bf16x3": 1e-4}.get(prec),
                     min_prefix=0 if prec == "tf32" else 4)


@pytest.mark.parametrize("slice_cols", [64, 32, 16])
def test_strided_blocks_with_ragged_windows(slice_cols):
    # subdomains of whole 32-row chunks side by side in every snapshot row
    # (one tensor map of whole rows serves them all), window lengths that end
    # inside a slice (those slices read through the subdomain's own map, which
    # zero-fills past its last column), micro-batches of 48 columns, and NaN in
    # every element no subdomain owns: a box read past a subdomain's columns
    # into a kept result would turn it to NaN
    m, n = [64, 96, 32, 128, 64], [100, 64, 37, 130, 81]
    S, L, N = len(m), sum(m), max(n)
    blocks = [inputs.separated_lowrank(m[s], n[s], 4, 60 + s, decay=0.5, noise=1e-4)
              for s in range(S)]
    data = np.full(L * N, np.nan, dtype=np.float32)
    off = np.concatenate([[0], np.cumsum(m)[:-1]]).astype(np.int64)
    win = inputs.Window(data, np.array(m), np.array(n), off, np.full(S, L, dtype=np.int64))
    for s in range(S):
        win.block(s)[...] = blocks[s]
    plan = spid.Plan.for_window(win, k_max=4, p=6, precision="tf32", seed=0x5EED0001)
    if slice_cols != 64:
        plan.set_tuning(dict(plan.tuning(), sketch_slice_cols=slice_cols))
    w = _dev(win)
    for c0 in range(0, N, 48):
        plan.sketch(w, c0, 48)
    plan.finalize()
    torch.cuda.synchronize()
    Y = plan.sketches()
    assert plan.device_status() in (0, spid.SPID_ERR_RANK)
    ref = inputs.pack_blocks(blocks)            # the same blocks, contiguous
    bp = spid.Plan.for_window(ref, k_max=4, p=6, precision="tf32", seed=0x5EED0001)
    bp.sketch(_dev(ref))
    torch.cuda.synchronize()
    Yb = bp.sketches()
    o = oracle_window(ref, 10, 4, 0.0, "tf32", 0x5EED0001)
    # one launch per subdomain reads through the same shared map
    ps = spid.Plan.for_window(win, k_max=4, p=6, precision="tf32", seed=0x5EED0001,
                              flags=spid.FLAG_PER_SUBDOMAIN)
    if slice_cols != 64:
        ps.set_tuning(dict(ps.tuning(), sketch_slice_cols=slice_cols))
    ps.sketch(w)
    torch.cuda.synchronize()
    Yp = ps.sketches()
    for s in range(S):
        assert np.all(np.isfinite(Y[s])), s
        assert rel_fro(Y[s], Yb[s]) <= 1e-5, s     # the same TF32 products, other FP32 order
        assert rel_fro(Yp[s], Yb[s]) <= 1e-5, s
        assert rel_fro(Y[s], o["Y"][s]) <= Y_TOL["tf32"], s
    plan.close()
    bp.close()
    ps.close()


@pytest.mark.parametrize("precision", ["fp32", "tf32", "bf16", "bf16x3"])
def test_edge_cases(precision):
    # n < k_max, n = 1, m < 32, k_max = 1
    blocks = [inputs.separated_lowrank(20, 3, 2, 1), inputs.separated_lowrank(5, 1, 1, 2),
              inputs.separated_lowrank(70, 50, 4, 3)]
    win = inputs.pack_blocks(blocks)
    g, o = check_parity(win, precision, 6, p=4)
    assert g["k"][0] <= 3 and g["k"][1] == 1
    g1, o1 = check_parity(win, precision, 1, p=4)
    assert list(g1["k"]) == [1, 1, 1]


def test_zero_window_gives_rank_zero():
    win = inputs.pack_blocks([np.zeros((64, 20)), np.zeros((40, 10))])
    g = run_gpu(win, "fp32", 4, p=4)
    assert list(g["k"]) == [0, 0]
    assert np.all(g["J"] == -1)
    assert np.all(g["err"] == 0.0)
    assert g["status"] == 0


def test_nonfinite_input_is_reported():
    A = inputs.separated_lowrank(64, 20, 3, 1)
    A[5, 7] = np.nan
    win = inputs.pack_blocks([A, inputs.separated_lowrank(64, 20, 3, 2)])
    g = run_gpu(win, "fp32", 4, p=4, reconstruct=False)
    assert g["status"] == 6            # SPID_ERR_NONFINITE
    assert g["k"][0] == 0 and g["k"][1] > 0


def test_adaptive_rank_geometric_spectrum():
    # sigma_i = 10^{-i/4}: adaptive tolerance 1e-3 (Remark 2.1 reading)
    sig = 10.0 ** (-np.arange(1, 129) / 4.0)
    blocks = [inputs.spectrum_matrix(2048, 128, sig, seed=3 + s) for s in range(3)]
    win = inputs.pack_blocks(blocks)
    for prec in ("fp32", "tf32", "bf16x3"):
        g, o = check_parity(win, prec, 32, p=10, tol=1e-3,
                            ahat_tol={"fp32": 1e-5, "bf16x3": 1e-4}.get(prec))
        for s in range(3):
            if prec != "fp32":
                assert abs(int(g["k"][s]) - int(o["k"][s])) <= 2
            assert np.sqrt(g["err"][s, 0] / g["err"][s, 1]) <= 3e-3


def test_per_subdomain_launches_match_batched():
    win = _lowrank_window(5, [300, 129, 640, 64, 1000], [200, 64, 100, 513, 77], 5, seed=40)
    for prec in ("fp32", "tf32", "bf16x3"):
        a = run_gpu(win, prec, 5, p=6)
        b = run_gpu(win, prec, 5, p=6, flags=spid.FLAG_PER_SUBDOMAIN)
        for s in range(5):
            assert rel_fro(a["Y"][s], b["Y"][s]) <= 1e-6
            assert list(a["J"][s]) == list(b["J"][s])
            assert rel_fro(a["Ahat"][s], b["Ahat"][s]) <= 1e-5


def test_streamed_micro_batches_match_one_shot():
    win = _lowrank_window(3, [500, 777, 256], [256, 200, 130], 5, seed=50)
    for prec in ("fp32", "tf32", "bf16", "bf16x3"):
        a = run_gpu(win, prec, 5, p=6)
        b = run_gpu(win, prec, 5, p=6, batches=64)
        c = run_gpu(win, prec, 5, p=6, batches=1)
        for s in range(3):
            assert rel_fro(b["Y"][s], a["Y"][s]) <= 1e-6
            assert rel_fro(c["Y"][s], a["Y"][s]) <= 1e-6
            assert list(b["J"][s]) == list(a["J"][s])


def test_sketch_is_scale_equivariant_fp64():
    # Omega fixed, so Y(2^7 A) = 2^7 Y(A) exactly and J, C are unchanged
    A = inputs.separated_lowrank(300, 40, 5, 9, noise=1e-3)
    w1 = inputs.pack_blocks([A], dtype=np.float64)
    w2 = inputs.pack_blocks([A * 2.0 ** 7], dtype=np.float64)
    a = run_gpu(w1, "fp64", 4, p=6)
    b = run_gpu(w2, "fp64", 4, p=6)
    assert np.array_equal(b["Y"][0], a["Y"][0] * 2.0 ** 7)
    assert list(a["J"][0]) == list(b["J"][0])
    assert np.array_equal(a["C"][0], b["C"][0])


def _split_qoi(win, nq=5):
    """The same window with every (box, QoI) block as its own subdomain
    (Section 5.3: each QoI of each sub-domain compressed on its own)."""
    mq = win.m // nq
    off = (win.off[:, None] + mq[:, None] * np.arange(nq)[None, :]).reshape(-1)
    return inputs.Window(win.data, np.repeat(mq, nq), np.repeat(win.n, nq), off,
                         np.repeat(win.ld, nq), dict(win.meta))


@pytest.mark.parametrize("precision", ["tf32", "fp32"])
def test_tgv3d_full_size_per_qoi(precision):
    # 64 boxes of 16^3 x 5 QoIs (n = 512) as 320 (box, QoI) subdomains, adaptive
    # tol 1e-3, k <= 20, p = 10: every QoI within 1e-3 over the domain (Section
    # 5.1 reports each QoI); the oracle on every QoI of three sampled boxes
    win = _split_qoi(inputs.tgv3d_window(grid=64, box=16, n=512))
    qoi = np.tile(np.arange(5), 64)
    g = run_gpu(win, precision, 20, p=10, tol=1e-3, qoi=qoi, num_qoi=5)
    per_q = g["plan"].per_qoi_rel_err(g["total"])
    assert np.all(per_q <= 1e-3), per_q
    # the per-QoI fold equals the per-subdomain sums, summed per QoI
    ge, ga = oracle.qoi_totals(qoi, g["err"][:, 0], g["err"][:, 1], 5)
    t = g["total"]
    assert np.allclose(t[4::2], ge, rtol=1e-12) and np.allclose(t[5::2], ga, rtol=1e-12)
    for b in (0, 27, 63):
        subs = list(range(5 * b, 5 * b + 5))
        sw = inputs.pack_blocks([win.block(s) for s in subs])
        o = oracle_window(sw, 30, 20, 1e-3, precision, 0x5EED0001)
        gs = {"k": g["k"][subs], "J": g["J"][subs], "C": [g["C"][s] for s in subs],
              "Y": [g["Y"][s] for s in subs], "err": g["err"][subs], "status": g["status"]}
        compare_with_oracle([win.block(s) for s in subs], gs, o, precision, 20, 1e-3, sample=True)
        for i, s in enumerate(subs):
            A = win.block(s).astype(np.float64)
            eg = np.sqrt(g["err"][s, 0] / g["err"][s, 1])
            eo = np.sqrt(o["e2"][i] / o["a2"][i])
            assert eg <= max(1e-3, 2 * eo), (s, eg, eo)
            assert ahat_matches_factors(A, g["J"][s], g["C"][s], g["Ahat"][s], int(g["k"][s])), s


def test_insitu_full_size_per_qoi_sampled():
    # the in-situ workload as it is timed: 512 boxes of 32^3 x 5 QoIs of a 256^3
    # field (2560 (box, QoI) subdomains, m = 32768), n = 256 sketched in
    # micro-batches of 64, TF32, adaptive tol 1e-3, k <= 30, p = 10; the oracle
    # on every QoI of two sampled boxes
    S, edge, grid, n = 512, 32, 256, 256
    origins = [(bx * edge, by * edge, bz * edge) for bz in range(8) for by in range(8)
               for bx in range(8)]
    field = inputs.DeviceField(origins, edge, grid, inputs.fourier_modes(seed=2))
    m, mq = 5 * edge ** 3, edge ** 3
    window = torch.empty(n * S * m, device="cuda", dtype=torch.float32)
    t_all = 10.0 * np.arange(n) / (n - 1)
    for j0 in range(0, n, 64):
        field.fill_subdomain_major(window, t_all[j0:j0 + 64], j0, n)
    del field
    off = (np.arange(S)[:, None] * n * m + mq * np.arange(5)[None, :]).reshape(-1)
    plan = spid.Plan([mq] * (5 * S), [n] * (5 * S), off, [m] * (5 * S), k_max=30, p=10,
                     tol=1e-3, precision="tf32", seed=0x5EED0005,
                     qoi=np.tile(np.arange(5), S), num_qoi=5)
    for j0 in range(0, n, 64):
        plan.sketch(window, j0, 64)
    plan.finalize()
    err = torch.zeros(2 * 5 * S, dtype=torch.float64, device="cuda")
    tot = torch.zeros(plan.total_len, dtype=torch.float64, device="cuda")
    plan.error(window, err, tot)
    torch.cuda.synchronize()
    status = plan.device_status()
    assert status in (0, spid.SPID_ERR_RANK)
    per_q = plan.per_qoi_rel_err(tot)
    assert np.all(per_q <= 1e-3), per_q
    k, J, C = plan.factors()
    Y = plan.sketches()
    e = err.cpu().numpy().reshape(-1, 2)
    for b in (0, 301):
        subs = list(range(5 * b, 5 * b + 5))
        host = window[b * n * m:(b + 1) * n * m].view(n, m).cpu().numpy()
        blocks = [host[:, q * mq:(q + 1) * mq].T.astype(np.float64) for q in range(5)]
        sw = inputs.pack_blocks(blocks, dtype=np.float64)
        o = oracle_window(sw, 40, 30, 1e-3, "tf32", 0x5EED0005)
        gs = {"k": k[subs], "J": J[subs], "C": [C[s] for s in subs], "Y": [Y[s] for s in subs],
              "err": e[subs], "status": status}
        compare_with_oracle(blocks, gs, o, "tf32", 30, 1e-3, sample=True)
        for i, s in enumerate(subs):
            eg = np.sqrt(e[s, 0] / e[s, 1])
            eo = np.sqrt(o["e2"][i] / o["a2"][i])
            assert eg <= max(1e-3, 2 * eo), (s, eg, eo)
    plan.close()
