"""The parity checker itself (tests/_helpers.compare_with_oracle), on the CPU:
fed the oracle's own result it passes; fed that result with one thing made
wrong -- a rank, a pivot inside the separated prefix, a coefficient, the
identity block, the rank-cut status, the sketch -- it fails.  This is what
guards the GPU parity tests against checks that pass vacuously."""
import copy

import numpy as np
import pytest

import oracle
from paper_2103_01380_gb300 import inputs
from _helpers import SPID_ERR_RANK, U_MODE, compare_with_oracle, oracle_window, separated_prefix


def _perfect(win, precision, k_max, p, tol=0.0, seed=7):
    """The oracle's result dressed as a result of the CUDA path."""
    o = oracle_window(win, k_max + p, k_max, tol, precision, seed)
    dt = np.float64 if precision == "fp64" else np.float32
    g = {"k": o["k"].copy(), "J": o["J"].copy(), "Y": [y.copy() for y in o["Y"]],
         "C": [c.astype(dt) for c in o["C"]], "err": np.stack([o["e2"], o["a2"]], axis=1),
         "status": SPID_ERR_RANK if np.any(o["k"] < o["k_qr"]) else 0, "Ahat": []}
    for s in range(win.num_sub):
        k = int(o["k"][s])
        Ah, _, _ = oracle.reconstruct_error(win.block(s).astype(np.float64), o["J"][s][:k],
                                            o["C"][s][:k])
        g["Ahat"].append(Ah)
    return g, o


def _win():
    blocks = [inputs.separated_lowrank(m, n, 6, seed=3 + i, noise=1e-4)
              for i, (m, n) in enumerate([(300, 40), (129, 70), (500, 33)])]
    return inputs.pack_blocks(blocks, dtype=np.float64)


def _check(win, g, o, **kw):
    compare_with_oracle([win.block(s) for s in range(win.num_sub)], g, o, "fp64", 5,
                        c_tol=1e-10, ahat_tol=1e-10, **kw)


def test_the_oracle_passes_its_own_checker():
    win = _win()
    g, o = _perfect(win, "fp64", 5, 5)
    _check(win, g, o, min_prefix=5)


@pytest.mark.parametrize("edit", ["k_minus", "k_plus", "pivot", "coef", "identity", "status",
                                  "sketch", "J_tail", "ahat"])
def test_a_planted_mistake_fails_the_checker(edit):
    win = _win()
    g0, o = _perfect(win, "fp64", 5, 5)
    g = copy.deepcopy(g0)
    s = 1
    k = int(g["k"][s])
    assert k == 5
    if edit == "k_minus":          # a GPU that kept one pivot fewer than the oracle
        g["k"][s] = k - 1
        g["J"][s][k - 1] = -1
    elif edit == "k_plus":
        g["k"][s] = k + 1
    elif edit == "pivot":          # a different pivot inside the separated prefix
        g["J"][s][1], g["J"][s][2] = g["J"][s][2], g["J"][s][1]
    elif edit == "coef":
        j = [c for c in range(70) if c not in set(g["J"][s][:k])][0]
        g["C"][s][0, j] += 1e-6
    elif edit == "identity":
        g["C"][s][0, g["J"][s][0]] = 1.0 + 2.0 ** -40
    elif edit == "status":
        g["status"] = SPID_ERR_RANK if g0["status"] == 0 else 0
    elif edit == "sketch":
        g["Y"][s] = g["Y"][s] * (1.0 + 1e-9)
    elif edit == "J_tail":         # an index left past k
        g["J"][s][k - 1] = g["J"][s][k - 1]
        g["k"][s] = k - 1
    elif edit == "ahat":
        g["Ahat"][s] = g["Ahat"][s] + 1e-6 * np.abs(g["Ahat"][s]).max()
    with pytest.raises(AssertionError):
        _check(win, g, o)


def test_separated_prefix_is_not_vacuous():
    # the inputs built to be separated (decay 0.5 between singular values) give
    # a full prefix, so J is compared over every kept pivot
    win = _win()
    o = oracle_window(win, 10, 5, 0.0, "fp64", 7)
    for s in range(win.num_sub):
        assert separated_prefix(o["Y"][s], 5, 1e-6, U_MODE["fp64"]) == 5
    g, _ = _perfect(win, "fp64", 5, 5)
    with pytest.raises(AssertionError):
        # demanding more than the data allows fails (the prefix check is live)
        flat = inputs.pack_blocks([np.ones((50, 20)) + 1e-9 * np.random.default_rng(0).standard_normal((50, 20))],
                                  dtype=np.float64)
        gf, of = _perfect(flat, "fp64", 5, 5)
        compare_with_oracle([flat.block(0)], gf, of, "fp64", 5, min_prefix=3)


def test_rank_cut_status_follows_the_oracle_guard():
    # rank 2 plus a 1e-6 component: a guard at TF32's roundoff (2 * 2^-11 of
    # |R_00|) cuts the third pivot with a wide margin, so the status is checked
    rng = np.random.default_rng(5)
    blocks = []
    for s in range(2):
        U = np.linalg.qr(rng.standard_normal((200, 3)))[0]
        V = np.linalg.qr(rng.standard_normal((40, 3)))[0]
        blocks.append(U @ np.diag([1.0, 0.3, 1e-6]) @ V.T)
    win = inputs.pack_blocks(blocks, dtype=np.float32)
    o = oracle_window(win, 9, 5, 0.0, "tf32", 7)
    assert np.all(o["k"] == 2) and np.all(o["k_qr"] == 5)
    g, _ = _perfect(win, "tf32", 5, 4)
    assert g["status"] == SPID_ERR_RANK
    compare_with_oracle([win.block(s) for s in range(2)], g, o, "tf32", 5)
    g["status"] = 0
    with pytest.raises(AssertionError):
        compare_with_oracle([win.block(s) for s in range(2)], g, o, "tf32", 5)
    # and a generic matrix (no cut) must not report one
    G = inputs.pack_blocks([rng.standard_normal((200, 40))], dtype=np.float32)
    og = oracle_window(G, 9, 5, 0.0, "tf32", 7)
    gg, _ = _perfect(G, "tf32", 5, 4)
    assert gg["status"] == 0
    compare_with_oracle([G.block(0)], gg, og, "tf32", 5)
    gg["status"] = SPID_ERR_RANK
    with pytest.raises(AssertionError):
        compare_with_oracle([G.block(0)], gg, og, "tf32", 5)
