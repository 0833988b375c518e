"""Pins of the oracle's modified (two-stage) SPID (Section 3.3.2, Algorithm 6)
against what the algebra of the method fixes:

  * the composition is the product it claims: C1' = C1 blockdiag(C_b), written
    out independently with numpy from the stage factors, and J = b n/N + I_b(p)
    for every stage-2 pick q = b k + p;
  * C1'(:, J) = I exactly (an interpolative decomposition of A);
  * the final error obeys the triangle inequality through the stages:
    ||A - A(:,J) C1'|| <= ||A - A0' C0'|| + ||A0' - A0'(:,J2) C1|| ||C0'||_2;
  * exact low rank r <= k: every stage is exact and stage 2 keeps r columns;
  * one block (N = 1): stage 1 is the plain sketched ID of A, whose skeleton
    stage 2 re-selects from.
"""
import numpy as np
import pytest

import oracle
from paper_2103_01380_gb300 import inputs

U64 = 2.0 ** -53
SEED = 0x5EED0001


def _blockdiag(Cb, kb, nb):
    N, k = Cb.shape[0], Cb.shape[1]
    M = np.zeros((N * k, N * nb))
    for b in range(N):
        M[b * k:b * k + kb[b], b * nb:(b + 1) * nb] = Cb[b, :kb[b]]
    return M


def _stage_matrices(A, o, N):
    m, n = A.shape
    nb = n // N
    k = o["Jb"].shape[1]
    A0 = np.zeros((m, N * k))
    for b in range(N):
        for p in range(o["kb"][b]):
            A0[:, b * k + p] = A[:, b * nb + o["Jb"][b, p]]
    return A0, _blockdiag(o["Cb"], o["kb"], nb)


@pytest.mark.parametrize("N,k,k2max,tol2", [(4, 8, 16, 1e-4), (2, 6, 12, 1e-3), (8, 4, 32, 1e-6)])
def test_composition_is_the_product_and_an_id(N, k, k2max, tol2):
    A = inputs.separated_lowrank(300, 64, 5, 3, noise=1e-6)
    o = oracle.two_stage(A, N, k, 6, k2max, tol2, U64, SEED)
    n = A.shape[1]
    nb = n // N
    A0, C0 = _stage_matrices(A, o, N)
    assert np.allclose(o["C"], o["C1"] @ C0, rtol=0, atol=1e-13 * max(1.0, np.abs(o["C"]).max()))
    for i, q in enumerate(o["J2"]):
        b, p = divmod(int(q), k)
        assert o["J"][i] == b * nb + o["Jb"][b, p]
    assert np.array_equal(o["C"][:, o["J"]], np.eye(o["k"]))
    # the stages' own skeletons: A_b(:, I_b) are columns of A, A0'(:, J2) = A(:, J)
    assert np.array_equal(A0[:, o["J2"]], A[:, o["J"]])


@pytest.mark.parametrize("N", [2, 4, 8])
def test_error_through_the_stages(N):
    A = inputs.separated_lowrank(400, 128, 10, 5, noise=1e-4)
    o = oracle.two_stage(A, N, 8, 6, 24, 1e-3, U64, SEED)
    A0, C0 = _stage_matrices(A, o, N)
    e_final = np.linalg.norm(A - A[:, o["J"]] @ o["C"])
    assert o["e2"] == pytest.approx(e_final ** 2, rel=1e-10)
    e1 = np.linalg.norm(A - A0 @ C0)
    e2 = np.linalg.norm(A0 - A0[:, o["J2"]] @ o["C1"])
    assert e_final <= e1 + e2 * np.linalg.norm(C0, 2) + 1e-12 * np.linalg.norm(A)


def test_exact_low_rank_is_reproduced_and_deduplicated():
    # every block of a rank-3 matrix has rank 3: stage 1 keeps 3 per block
    # (the rank guard with the FP32 unit roundoff drops the FP64 rounding-noise
    # pivots), stage 2 keeps 3 of the 3 N
    A = inputs.lowrank(250, 96, 3, seed=9)
    o = oracle.two_stage(A, 4, 6, 6, 12, 1e-8, 2.0 ** -24, SEED)
    assert list(o["kb"]) == [3, 3, 3, 3]
    assert o["k"] == 3
    assert np.sqrt(o["e2"] / o["a2"]) < 1e-12


def test_one_block_reselects_from_the_plain_sketched_id():
    A = inputs.separated_lowrank(200, 40, 6, 11, noise=1e-5)
    o = oracle.two_stage(A, 1, 10, 6, 10, 1e-3, U64, SEED)
    s1 = oracle.spid(A, 16, 10, 0.0, U64, SEED)
    assert list(o["Jb"][0][:o["kb"][0]]) == list(s1["J"][:s1["k"]])
    assert set(o["J"].tolist()) <= set(s1["J"][:s1["k"]].tolist())
    assert o["k"] <= s1["k"]
