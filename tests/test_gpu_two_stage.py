"""GPU parity of the modified (two-stage) SPID (Section 3.3.2, Algorithm 6)
through the C ABI against the FP64 oracle on the same seeded inputs.

  * stage 1, per time block: J_b identical over the separated prefix of the
    block's sketch (the rule of tests/test_gpu_parity.py), k_b equal;
  * when every block agrees, A0' is the same on both sides and the final J
    (= I_U(J2)) is identical over the separated prefix of A0''s sketch;
  * then A_hat = A(:, J) C1' within 1e-9 (FP64) / 1e-4 (FP32: two solves of
    cond(R11) u each, composed) and the error within the A_hat difference;
  * always: C1'(:, J) = I exactly, J are window columns, the CF sums exact, and
    the final error within max(cap, 2 x the oracle's) for TF32.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2103_01380_gb300 import inputs, spid
from _helpers import STATUS_OK, rel_fro, separated_prefix, U_MODE
from test_gpu_parity import GAP

pytestmark = pytest.mark.gpu

SEED = 0x5EED0001


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2103_01380_gb300 import build
    build.build()
    spid.load_library()
    torch.cuda.init()


def _window(m, n, r, seed, noise, dtype):
    blocks = [inputs.separated_lowrank(m[s], n, r, seed + s, noise=noise) for s in range(len(m))]
    return inputs.pack_blocks(blocks, dtype=dtype)


def run_ts(win, precision, N, k, k2_max, tol2, p=6):
    plan = spid.TsPlan.for_window(win, blocks=N, k=k, k2_max=k2_max, tol2=tol2, p=p,
                                  precision=precision, seed=SEED)
    w = torch.from_numpy(win.data).cuda()
    for b in range(N):           # blocks may arrive in any order
        plan.block(w, (b * 3) % N if N % 3 else b)
    plan.finalize(w)
    err = torch.zeros(2 * win.num_sub, dtype=torch.float64, device="cuda")
    tot = torch.zeros(4, dtype=torch.float64, device="cuda")
    plan.error(w, err, tot)
    out = torch.zeros_like(w)
    plan.reconstruct(w, out)
    torch.cuda.synchronize()
    k2, J, C = plan.factors()
    blocks = [plan.block_factors(b) for b in range(N)]
    ow = inputs.Window(out.cpu().numpy(), win.m, win.n, win.off, win.ld)
    return {"k": k2, "J": J, "C": C, "blocks": blocks, "err": err.cpu().numpy().reshape(-1, 2),
            "total": tot.cpu().numpy(), "Ahat": [ow.block(s).copy() for s in range(win.num_sub)],
            "status": plan.device_status()}


def check_ts(win, precision, N, k, k2_max, tol2, p=6):
    g = run_ts(win, precision, N, k, k2_max, tol2, p)
    assert g["status"] in STATUS_OK
    u = U_MODE[precision]
    full = 0
    for s in range(win.num_sub):
        A = win.block(s).astype(np.float64)
        m, n = A.shape
        nb = n // N
        o = oracle.two_stage(A, N, k, p, k2_max, tol2, u, SEED)
        kg = int(g["k"][s])
        Jg = g["J"][s][:kg]
        # always: an interpolative decomposition of A on window columns
        assert np.all((Jg >= 0) & (Jg < n)) and len(set(Jg.tolist())) == kg
        assert np.array_equal(g["C"][s][:kg][:, Jg], np.eye(kg, dtype=g["C"][s].dtype))
        # stage 1 per block
        same = True
        for b in range(N):
            kb_g, Jb_g, _ = g["blocks"][b]
            Ab = A[:, b * nb:(b + 1) * nb]
            Yb = oracle.sketch(Ab, k + p, SEED)
            pre = min(separated_prefix(Yb, k, GAP[precision], u), int(o["kb"][b]), int(kb_g[s]))
            assert list(Jb_g[s][:pre]) == list(o["Jb"][b][:pre]), ("Jb", s, b)
            same &= (int(kb_g[s]) == int(o["kb"][b]) and
                     list(Jb_g[s][:kb_g[s]]) == list(o["Jb"][b][:o["kb"][b]]))
        if not same:
            continue
        # stage 2 on the same A0'
        A0 = np.zeros((m, N * k))
        for b in range(N):
            for q in range(o["kb"][b]):
                A0[:, b * k + q] = A[:, b * nb + o["Jb"][b, q]]
        Y2 = oracle.sketch(A0, k2_max + p, SEED)
        pre2 = min(separated_prefix(Y2, max(o["k"], 1), GAP[precision], u), o["k"], kg)
        assert list(Jg[:pre2]) == list(o["J"][:pre2]), ("J", s, Jg, o["J"])
        if kg == o["k"] and list(Jg) == list(o["J"]) and precision in ("fp64", "fp32"):
            full += 1
            Ah_o = A[:, o["J"]] @ o["C"]
            tol = 1e-9 if precision == "fp64" else 1e-4
            d = rel_fro(g["Ahat"][s], Ah_o)
            assert d <= tol, ("Ahat", s, d)
            eg, eo = np.sqrt(g["err"][s, 0]), np.sqrt(o["e2"])
            assert abs(eg - eo) <= 1.01 * d * np.linalg.norm(Ah_o) + 8 * u * np.sqrt(o["a2"]), \
                ("err", s, eg, eo)
        if precision == "tf32":
            rg = np.sqrt(g["err"][s, 0] / g["err"][s, 1])
            assert rg <= max(1e-3, 2.0 * np.sqrt(o["e2"] / o["a2"])), ("tf32 err", s, rg)
    mm, nn, kk = win.m.astype(np.float64), win.n.astype(np.float64), g["k"].astype(np.float64)
    assert g["total"][2] == np.sum(mm * nn) and g["total"][3] == np.sum(kk * (mm + nn))
    return g, full


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_two_stage_parity(precision):
    dt = np.float64 if precision == "fp64" else np.float32
    win = _window([300, 1000, 777, 2048], 128, 6, seed=70, noise=1e-6, dtype=dt)
    g, full = check_ts(win, precision, 4, 4, 12, 1e-3)
    assert full >= 2          # the comparison reached the final factors


def test_two_stage_tensor_core_accuracy():
    win = _window([1000, 2048, 4099], 256, 6, seed=80, noise=1e-4, dtype=np.float32)
    check_ts(win, "tf32", 8, 8, 24, 1e-3)


def test_two_stage_one_block_and_many_blocks():
    win = _window([512, 640], 96, 5, seed=90, noise=1e-6, dtype=np.float32)
    check_ts(win, "fp32", 1, 6, 6, 1e-3)
    check_ts(win, "fp32", 12, 3, 16, 1e-3)


def test_two_stage_deduplicates_a_low_rank_window():
    # exact rank 3: each block keeps up to k = 5 columns (pivots past 3 are FP32
    # rounding noise), and stage 2's tolerance keeps 3 of the 5 N
    blocks = [inputs.lowrank(400, 64, 3, seed=100 + s) for s in range(3)]
    win = inputs.pack_blocks(blocks, dtype=np.float32)
    g = run_ts(win, "fp32", 4, 5, 12, 1e-5)
    assert g["status"] in STATUS_OK
    for b in range(4):
        assert all(3 <= int(v) <= 5 for v in g["blocks"][b][0])
    assert list(g["k"]) == [3, 3, 3]
    rel = np.sqrt(g["total"][0] / g["total"][1])
    assert rel < 1e-5


def test_reused_plan_clears_slots_a_lower_rank_leaves():
    # the plan first sees a window whose blocks keep k columns each, then one
    # where subdomain 0 is zero (its blocks keep none): stage 2 must see zero
    # slots there, as a fresh plan does
    N, k = 4, 4
    wa = _window([300, 257], 64, 6, seed=150, noise=1e-3, dtype=np.float32)
    wb = _window([300, 257], 64, 6, seed=150, noise=1e-3, dtype=np.float32)
    wb.block(0)[:] = 0.0

    def run(plan, win):
        w = torch.from_numpy(win.data).cuda()
        for b in range(N):
            plan.block(w, b)
        plan.finalize(w)
        err = torch.zeros(2 * win.num_sub, dtype=torch.float64, device="cuda")
        tot = torch.zeros(4, dtype=torch.float64, device="cuda")
        plan.error(w, err, tot)
        torch.cuda.synchronize()
        k2, J, C = plan.factors()
        return k2, J, C, err.cpu().numpy(), [plan.block_factors(b)[0] for b in range(N)]

    mk = lambda: spid.TsPlan.for_window(wa, blocks=N, k=k, k2_max=8, tol2=1e-3, p=6,
                                        precision="fp32", seed=SEED)
    reused = mk()
    ga = run(reused, wa)
    assert all(int(v[0]) == k for v in ga[4])
    gb = run(reused, wb)
    fresh = mk()
    gf = run(fresh, wb)
    assert all(int(v[0]) == 0 for v in gb[4])
    assert np.array_equal(gb[0], gf[0]) and np.array_equal(gb[1], gf[1])
    for x, y in zip(gb[2], gf[2]):
        assert np.array_equal(x, y)
    assert np.array_equal(gb[3], gf[3])
    reused.close()
    fresh.close()
