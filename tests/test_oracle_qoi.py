"""Pins for the oracle's per-QoI errors and its rank-guard outcome.

Section 5.1 reports the relative Frobenius error of each quantity of interest
on its own, and Section 5.3 compresses each QoI of each sub-domain as its own
ID.  The oracle gives per-QoI sums for a box whose rows stack the QoIs
(``error_per_qoi``) and per-QoI totals over subdomains that each hold one QoI
(``qoi_totals``).  The pins below are exact invariants of those definitions:
scaling a QoI block by a power of two scales its error terms exactly, a zero
block contributes nothing, exact low-rank data leaves no error in any block,
and the blocks partition the whole-box sums.  A wrong block boundary, an
interleaved row split or a dropped block fails at least one of them.

CPU only (no GPU marker)."""
import numpy as np
import pytest

import oracle
from paper_2103_01380_gb300 import inputs


def _spid(A, k=4, l=10, tol=0.0, seed=7):
    o = oracle.spid(A, l, k, tol, 2.0 ** -53, seed)
    return o["J"][:o["k"]], o["C"][:o["k"]], o


def test_blocks_partition_the_box_sums():
    A = np.random.default_rng(1).standard_normal((5 * 24, 40))
    J, C, o = _spid(A)
    e2, a2 = oracle.error_per_qoi(A, J, C, 5)
    assert abs(e2.sum() - o["e2"]) <= 1e-13 * o["e2"]
    assert abs(a2.sum() - o["a2"]) <= 1e-13 * o["a2"]
    # each block's a2 is the squared norm of its own rows (QoI slowest)
    for q in range(5):
        ref = float((A[q * 24:(q + 1) * 24] ** 2).sum())
        assert abs(a2[q] - ref) <= 1e-13 * ref


def test_power_of_two_scaled_blocks_scale_exactly():
    # A = [X; 2X; 4X; X/2]: every term of block q is 4^s times block 0's, so
    # the sums scale bitwise and the relative errors are bitwise equal.
    X = np.random.default_rng(2).standard_normal((30, 25))
    sc = [1.0, 2.0, 4.0, 0.5]
    A = np.vstack([c * X for c in sc])
    J, C, _ = _spid(A, k=3)
    e2, a2 = oracle.error_per_qoi(A, J, C, 4)
    assert e2[0] > 0.0
    for q, c in enumerate(sc):
        assert e2[q] == c * c * e2[0]
        assert a2[q] == c * c * a2[0]
        assert np.sqrt(e2[q] / a2[q]) == np.sqrt(e2[0] / a2[0])


def test_interleaved_split_is_not_the_block_split():
    # the same data with rows interleaved across QoIs gives other sums, so the
    # scaled-copy pin above distinguishes the two readings of "QoI rows"
    X = np.random.default_rng(3).standard_normal((30, 25))
    A = np.vstack([X, 2.0 * X])
    J, C, _ = _spid(A, k=3)
    e2, _ = oracle.error_per_qoi(A, J, C, 2)
    Ahat = A[:, J] @ C
    inter = [float(((A[q::2] - Ahat[q::2]) ** 2).sum()) for q in range(2)]
    assert not np.allclose(inter, e2, rtol=1e-6)
    assert abs(e2[1] / e2[0] - 4.0) == 0.0


def test_zero_block_contributes_nothing():
    X = np.random.default_rng(4).standard_normal((20, 30))
    A = np.vstack([X, np.zeros_like(X), X])
    J, C, _ = _spid(A, k=4)
    e2, a2 = oracle.error_per_qoi(A, J, C, 3)
    assert e2[1] == 0.0 and a2[1] == 0.0
    assert e2[0] > 0.0 and e2[0] == e2[2]


def test_exact_low_rank_has_no_error_in_any_block():
    A = inputs.lowrank(5 * 40, 60, 3, seed=5)
    J, C, _ = _spid(A, k=3)
    e2, a2 = oracle.error_per_qoi(A, J, C, 5)
    assert np.all(e2 <= 1e-26 * a2.sum())


def test_stacked_tgv_box_pressure_dominates():
    # the 3D TGV box of Section 5.2 stacks (rho, u, v, w, p) with p ~ 100:
    # a rank-1 ID of the stack fits p and rho to ~1e-3 but not the velocity,
    # which is what per-QoI reporting exposes
    t = 10.0 * np.arange(64) / 63.0
    A = inputs.tgv3d_box((0, 0, 0), (8, 8, 8), 64, t, inputs.fourier_modes(seed=2),
                         dtype=np.float64)
    J, C, _ = _spid(A, k=1, l=11)
    e2, a2 = oracle.error_per_qoi(A, J, C, 5)
    rel = np.sqrt(e2 / a2)
    whole = np.sqrt(e2.sum() / a2.sum())
    assert whole < 1e-2
    assert rel[4] < 1e-2 and rel[0] < 1e-2
    assert max(rel[1], rel[2], rel[3]) > 10 * whole


def test_qoi_totals_scale_and_partition():
    rng = np.random.default_rng(6)
    B, nq = 4, 3
    e0 = rng.uniform(0.1, 1.0, B)
    a0 = rng.uniform(1.0, 2.0, B)
    # subdomain s = b nq + q holds QoI q of box b, scaled by 2^q
    qoi = np.tile(np.arange(nq), B)
    e2 = np.concatenate([[e0[b] * 4.0 ** q for q in range(nq)] for b in range(B)])
    a2 = np.concatenate([[a0[b] * 4.0 ** q for q in range(nq)] for b in range(B)])
    ge, ga = oracle.qoi_totals(qoi, e2, a2, nq)
    for q in range(nq):
        assert ge[q] == 4.0 ** q * ge[0] and ga[q] == 4.0 ** q * ga[0]
    assert abs(ge.sum() - e2.sum()) <= 1e-15 * e2.sum()
    # an empty QoI index gives zero totals
    ge4, ga4 = oracle.qoi_totals(qoi, e2, a2, nq + 1)
    assert ge4[nq] == 0.0 and ga4[nq] == 0.0
    with pytest.raises(ValueError):
        oracle.qoi_totals(qoi, e2, a2, nq - 1)


def test_guard_cut_is_reported_by_kqr():
    # exactly rank 2: the QR keeps producing rounding-level pivots up to k = 5;
    # a guard at FP32 roundoff keeps 2 (a cut), one at FP64 roundoff keeps all;
    # a generic Gaussian matrix is never cut
    A = inputs.lowrank(200, 40, 2, seed=8)
    _, _, o = _spid(A, k=5, l=15)
    assert o["k"] == 5 and o["k_qr"] == 5      # FP64 roundoff pivots sit above 2^-52 |R_00|
    f = oracle.spid(A, 15, 5, 0.0, 2.0 ** -24, 7)
    assert f["k"] == 2 and f["k_qr"] == 5      # an FP32-roundoff guard cuts them
    G = np.random.default_rng(9).standard_normal((200, 40))
    _, _, g = _spid(G, k=5, l=15)
    assert g["k"] == g["k_qr"] == 5
    # the guard in TF32's roundoff cuts a geometric spectrum whose pivots fall
    # below 2 * 2^-11 of the first one
    S = inputs.spectrum_matrix(300, 60, 10.0 ** (-np.arange(1, 61) / 2.0), seed=10)
    o2 = oracle.spid(S, 20, 10, 0.0, 2.0 ** -11, 11)
    assert o2["k"] < o2["k_qr"] == 10
