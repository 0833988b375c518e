"""Pins of the oracle's subsampled ID / single-pass ID (Section 2, SubID and SPID
paragraphs, Algorithms 2 and 3; Section 5.2 subsampling study; appendix
Theorems A.2 and A.3) against what the paper and the mathematics fix:

  * the coarse grids of the paper's 64-point runs (intervals 3, 7, 9 keep both
    ends) and its printed compression factors (about 100 without subsampling,
    about 2400 at interval 3, rank 1, 100 snapshots);
  * subsampling = an index gather written independently with numpy;
  * trilinear interpolation reproduces every trilinear field exactly and every
    coarse node value, and does not reproduce a quadratic;
  * interval 1 reduces SubID and SPID to the plain column ID of A;
  * Theorem A.3 (SPID) and Theorem A.2 (SubID, read with the n x n Gram
    matrices A^T A and B^T B so that the dimensions agree) hold with a dense M.
"""
import numpy as np
import pytest

import oracle
from paper_2103_01380_gb300 import inputs


def _axis(e, s):
    # independent restatement: every s-th point, plus the last point
    idx = list(range(0, e, s))
    if idx[-1] != e - 1:
        idx.append(e - 1)
    return np.array(idx)


@pytest.mark.parametrize("e,s,count", [(64, 3, 22), (64, 7, 10), (64, 9, 8), (64, 1, 64),
                                       (16, 3, 6), (16, 5, 4), (1, 3, 1), (2, 5, 2)])
def test_coarse_axis_counts_and_ends(e, s, count):
    idx = oracle.coarse_axis(e, s)
    assert len(idx) == count
    assert idx[0] == 0 and idx[-1] == e - 1
    assert np.array_equal(idx, _axis(e, s))


def test_coarse_axis_appends_a_short_last_interval():
    # reading for (e - 1) % s != 0: the end point is kept as a last, shorter interval
    assert list(oracle.coarse_axis(10, 4)) == [0, 4, 8, 9]
    assert list(oracle.coarse_axis(7, 4)) == [0, 4, 6]


def test_e3_compression_factors():
    # Section 5.2: 64^3 points (u1), 100 snapshots, rank 1: CF ~ 100 without
    # subsampling and ~ 2400 with interval 3 (the skeleton keeps coarse rows only)
    box, n = (1, 64, 64, 64), 100
    m = 64 ** 3
    mc = oracle.coarse_rows(box, (3, 3, 3))
    assert mc == 22 ** 3
    cf_full = oracle.compression_factor([m], [n], [1])
    cf_sub = oracle.compression_factor([m], [n], [1], stored_rows=[mc])
    assert cf_full == pytest.approx(m * n / (m + n))
    assert round(cf_full) == 100
    assert cf_sub == pytest.approx(m * n / (mc + n))
    assert 2400 <= cf_sub <= 2450


@pytest.mark.parametrize("box,stride", [((2, 5, 7, 10), (2, 3, 4)), ((3, 4, 4, 4), (1, 1, 1)),
                                        ((1, 1, 6, 9), (3, 2, 4))])
def test_subsample_is_the_coarse_index_gather(box, stride):
    rng = np.random.default_rng(1)
    n = 7
    A = rng.standard_normal((int(np.prod(box)), n))
    B = oracle.subsample(A, box, stride)
    nq, ez, ey, ex = box
    A5 = A.reshape(nq, ez, ey, ex, n)
    want = A5[:, _axis(ez, stride[0])][:, :, _axis(ey, stride[1])][:, :, :, _axis(ex, stride[2])]
    assert np.array_equal(B, want.reshape(-1, n))
    assert B.shape[0] == oracle.coarse_rows(box, stride)


def _trilinear_field(box, n, seed):
    nq, ez, ey, ex = box
    rng = np.random.default_rng(seed)
    z, y, x = np.meshgrid(np.arange(ez), np.arange(ey), np.arange(ex), indexing="ij")
    mono = [np.ones_like(x), x, y, z, x * y, x * z, y * z, x * y * z]
    F = np.zeros((nq, ez, ey, ex, n))
    for q in range(nq):
        for j in range(n):
            c = rng.standard_normal(8)
            F[q, ..., j] = sum(ci * mi for ci, mi in zip(c, mono))
    return F.reshape(-1, n)


@pytest.mark.parametrize("box,stride", [((2, 7, 9, 10), (3, 4, 4)), ((1, 5, 6, 13), (2, 5, 3)),
                                        ((2, 4, 3, 5), (1, 1, 1)), ((1, 1, 1, 9), (1, 1, 4))])
def test_trilinear_reproduces_trilinear_fields(box, stride):
    A = _trilinear_field(box, 4, seed=3)
    F = oracle.trilinear(oracle.subsample(A, box, stride), box, stride)
    assert np.max(np.abs(F - A)) <= 1e-12 * np.max(np.abs(A))


def test_trilinear_keeps_nodes_and_misses_a_quadratic():
    box, stride = (2, 7, 9, 10), (3, 4, 4)
    mc = oracle.coarse_rows(box, stride)
    G = np.random.default_rng(4).standard_normal((mc, 3))
    F = oracle.trilinear(G, box, stride)
    assert np.array_equal(oracle.subsample(F, box, stride), G)
    nq, ez, ey, ex = box
    x = np.broadcast_to(np.arange(ex, dtype=np.float64), (nq, ez, ey, ex)).reshape(-1, 1)
    Q = x ** 2
    Fq = oracle.trilinear(oracle.subsample(Q, box, stride), box, stride)
    assert np.max(np.abs(Fq - Q)) > 0.5   # between nodes a parabola is not linear


def test_interval_one_is_the_plain_column_id():
    box = (2, 6, 5, 7)
    A = inputs.smooth_box_field(box, 30, seed=8, noise=1e-4)
    o = oracle.subid(A, box, (1, 1, 1), 5, 0.0, 2.0 ** -53, want_ahat=True)
    assert o["mc"] == A.shape[0]
    Jq, R, k, _ = oracle.qrcp_mgs(A, 5)
    assert list(o["J"]) == list(Jq[:k])
    C = oracle.coefficients(R, Jq, k)
    assert np.allclose(o["C"], C, rtol=0, atol=1e-12 * np.max(np.abs(C)))
    Ah, e2, a2 = oracle.reconstruct_error(A, o["J"], o["C"])
    assert o["e2_subid"] == pytest.approx(e2, rel=1e-12)
    assert o["e2_spid"] == pytest.approx(e2, rel=1e-12)   # M = I
    assert np.allclose(o["Ahat_spid"], Ah, rtol=0, atol=1e-12 * np.max(np.abs(A)))


@pytest.mark.parametrize("box,stride,k", [((1, 9, 9, 9), (2, 2, 2), 3),
                                          ((2, 8, 10, 12), (3, 3, 4), 4),
                                          ((1, 17, 13, 11), (4, 3, 5), 2)])
def test_theorems_a2_a3_with_dense_interpolation(box, stride, k):
    A = inputs.smooth_box_field(box, 40, seed=7, noise=1e-3)
    o = oracle.subid(A, box, stride, k, 0.0, 2.0 ** -53, want_ahat=True)
    B = oracle.subsample(A, box, stride)
    mc = B.shape[0]
    M = oracle.trilinear(np.eye(mc), box, stride)          # dense operator, column by column
    J, C = o["J"], o["C"]
    assert np.array_equal(o["Bskel"], B[:, J])
    Bh = B[:, J] @ C
    # the SPID reconstruction is M B(:, I_B) C_B, and the squared errors match it
    assert np.max(np.abs(o["Ahat_spid"] - M @ Bh)) <= 1e-12 * np.max(np.abs(A))
    assert o["e2_spid"] == pytest.approx(np.sum((A - M @ Bh) ** 2), rel=1e-10)
    assert o["e2_subid"] == pytest.approx(np.sum((A - A[:, J] @ C) ** 2), rel=1e-10)
    # Theorem A.3: ||A - M B_hat||_2 <= ||A - M B||_2 + ||M||_2 ||B - B_hat||_2
    lhs = np.linalg.norm(A - M @ Bh, 2)
    rhs = np.linalg.norm(A - M @ B, 2) + np.linalg.norm(M, 2) * np.linalg.norm(B - Bh, 2)
    assert lhs <= rhs * (1 + 1e-12)
    # Theorem A.2 for every tau of a grid (each tau gives an upper bound)
    sv = np.linalg.svd(B, compute_uv=False)
    lhs2 = np.linalg.norm(A - A[:, J] @ C, 2)
    nC, nBB = np.linalg.norm(C, 2), np.linalg.norm(B - Bh, 2)
    AtA, BtB = A.T @ A, B.T @ B
    checked = 0
    for tau in np.logspace(-3, 4, 40):
        eps = np.linalg.eigvalsh(AtA - tau * BtB).max()
        a1, a2 = tau * sv[k] ** 2 + eps, tau + eps / sv[k - 1] ** 2
        if a1 < 0 or a2 < 0:
            continue
        assert lhs2 <= ((1 + nC) * np.sqrt(a1) + nBB * np.sqrt(a2)) * (1 + 1e-12), tau
        checked += 1
    assert checked >= 20
