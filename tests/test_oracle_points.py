"""Pins of the oracle's coarse-grid ID on arbitrary point sets (Section 2: the
rows of A may follow a flattened unstructured grid "possibly without specific
ordering"; Section 5.1 compresses the TGV on randomly generated points), where
the coarse rows are an explicit list and M a fixed-width stencil:

  * a structured box written as a point set (its coarse rows and the trilinear
    weights, restated here with numpy as an 8-point stencil) gives the box
    oracle's J, C and errors -- the stencil path equals the pinned box path;
  * M = I (every row coarse, one-point stencils) is the plain column ID of A;
  * a field in the range of M (A = M G0, G0 of rank r, coarse rows mapped to
    themselves) is reproduced exactly once k >= r;
  * relabelling the points (a permutation of the rows, with the coarse list
    and the stencils relabelled alike) changes nothing but the order of sums;
  * Theorem A.3 holds for a random (non-geometric) stencil operator;
  * the paper's Section 5.1 case: the 2D TGV u1 on random points is rank one
    and its SubID error is at the FP64 rounding level.
"""
import numpy as np
import pytest

import oracle
from paper_2103_01380_gb300 import inputs


def _axis(e, s):
    idx = list(range(0, e, s))
    if idx[-1] != e - 1:
        idx.append(e - 1)
    return np.array(idx)


def _box_as_points(box, stride):
    """Coarse rows and the 8-point trilinear stencil of a box, restated with numpy."""
    nq, ez, ey, ex = box
    ax = [_axis(e, s) for e, s in zip((ez, ey, ex), stride)]
    cz, cy, cx = (len(a) for a in ax)
    crow = [((q * ez + z) * ey + y) * ex + x for q in range(nq) for z in ax[0] for y in ax[1]
            for x in ax[2]]

    def cell(a, x):
        if len(a) == 1:
            return 0, 0.0
        lo = min(np.searchsorted(a, x, side="right") - 1, len(a) - 2)
        return lo, (x - a[lo]) / (a[lo + 1] - a[lo])

    idx, w = [], []
    for q in range(nq):
        for z in range(ez):
            a, wz = cell(ax[0], z)
            for y in range(ey):
                b, wy = cell(ax[1], y)
                for x in range(ex):
                    c, wx = cell(ax[2], x)
                    ii, ww = [], []
                    for dz in (0, 1):
                        for dy in (0, 1):
                            for dx in (0, 1):
                                wt = ((wz if dz else 1 - wz) * (wy if dy else 1 - wy) *
                                      (wx if dx else 1 - wx))
                                zz, yy, xx = min(a + dz, cz - 1), min(b + dy, cy - 1), min(c + dx, cx - 1)
                                ii.append(((q * cz + zz) * cy + yy) * cx + xx)
                                ww.append(wt)
                    idx.append(ii)
                    w.append(ww)
    return np.array(crow), np.array(idx), np.array(w)


@pytest.mark.parametrize("box,stride,k", [((1, 9, 9, 9), (2, 2, 2), 3),
                                          ((2, 8, 10, 12), (3, 3, 4), 4),
                                          ((1, 7, 5, 11), (4, 3, 5), 2)])
def test_box_written_as_points_matches_the_box_oracle(box, stride, k):
    A = inputs.smooth_box_field(box, 30, seed=3, noise=1e-4)
    crow, idx, w = _box_as_points(box, stride)
    p = oracle.subid_points(A, crow, idx, w, k, 0.0, 2.0 ** -53, want_ahat=True)
    b = oracle.subid(A, box, stride, k, 0.0, 2.0 ** -53, want_ahat=True)
    assert p["mc"] == b["mc"] and p["k"] == b["k"]
    assert list(p["J"]) == list(b["J"])
    assert np.allclose(p["C"], b["C"], rtol=0, atol=1e-12 * max(1.0, np.abs(b["C"]).max()))
    assert np.array_equal(p["Bskel"], b["Bskel"])
    assert p["e2_subid"] == pytest.approx(b["e2_subid"], rel=1e-12)
    assert p["e2_spid"] == pytest.approx(b["e2_spid"], rel=1e-10)
    assert np.max(np.abs(p["Ahat_spid"] - b["Ahat_spid"])) <= 1e-12 * np.abs(A).max()


def test_identity_operator_is_the_plain_column_id():
    pts, A = inputs.unstructured_tgv2d(60, 24, seed=4, smooth_modes=4, noise=1e-5)
    m = A.shape[0]
    p = oracle.subid_points(A, np.arange(m), np.arange(m).reshape(m, 1), np.ones((m, 1)), 5,
                            want_ahat=True)
    Jq, R, k, _ = oracle.qrcp_mgs(A, 5)
    assert p["mc"] == m and list(p["J"]) == list(Jq[:k])
    # library special case: LAPACK's pivoted QR picks the same leading columns
    import scipy.linalg
    _, _, piv = scipy.linalg.qr(A, pivoting=True, mode="economic")
    assert list(p["J"][:3]) == list(piv[:3])
    _, e2, _ = oracle.reconstruct_error(A, p["J"], p["C"])
    assert p["e2_subid"] == pytest.approx(e2, rel=1e-12)
    assert p["e2_spid"] == pytest.approx(e2, rel=1e-12)


@pytest.mark.parametrize("method,t", [("linear", 3), ("idw", 4)])
def test_fields_in_the_range_of_m_are_reproduced(method, t):
    rng = np.random.default_rng(5)
    pts = rng.uniform(0, 2 * np.pi, size=(300, 2))
    crow, idx, w = inputs.coarse_stencil(pts, 40, t, seed=6, method=method)
    M = np.zeros((300, 40))
    for r in range(300):
        for q in range(t):
            M[r, idx[r, q]] += w[r, q]
    assert np.allclose(M[crow], np.eye(40))                 # coarse points map to themselves
    G0 = rng.standard_normal((40, 3)) @ rng.standard_normal((3, 50))   # rank 3
    A = M @ G0
    p = oracle.subid_points(A, crow, idx, w, 6, 0.0, 2.0 ** -53)
    assert p["k"] >= 3                 # rounding noise past rank 3 may pass the FP64 guard
    assert np.sqrt(p["e2_spid"] / p["a2"]) <= 1e-13
    assert np.sqrt(p["e2_subid"] / p["a2"]) <= 1e-13


def test_relabelling_the_points_changes_nothing():
    pts, A = inputs.unstructured_tgv2d(200, 40, seed=7, smooth_modes=3, noise=1e-4)
    crow, idx, w = inputs.coarse_stencil(pts, 50, 3, seed=8, nq=2)
    p0 = oracle.subid_points(A, crow, idx, w, 5, 1e-3, 2.0 ** -53)
    perm = np.random.default_rng(9).permutation(A.shape[0])  # new row r holds old row perm[r]
    inv = np.argsort(perm)
    A1 = A[perm]
    p1 = oracle.subid_points(A1, inv[crow], idx[perm], w[perm], 5, 1e-3, 2.0 ** -53)
    assert p1["k"] == p0["k"] and list(p1["J"]) == list(p0["J"])
    assert np.array_equal(p1["C"], p0["C"])                  # B and its QR are the same
    assert p1["e2_spid"] == pytest.approx(p0["e2_spid"], rel=1e-12)
    assert p1["e2_subid"] == pytest.approx(p0["e2_subid"], rel=1e-12)


def test_theorem_a3_with_a_random_stencil():
    rng = np.random.default_rng(10)
    pts, A = inputs.unstructured_tgv2d(150, 30, seed=11, smooth_modes=5, noise=1e-3)
    m = A.shape[0]
    crow = np.sort(rng.choice(m, size=40, replace=False))
    t = 5
    idx = rng.integers(0, 40, size=(m, t))
    w = rng.standard_normal((m, t))
    o = oracle.subid_points(A, crow, idx, w, 4, 0.0, 2.0 ** -53, want_ahat=True)
    M = np.zeros((m, 40))
    for r in range(m):
        for q in range(t):
            M[r, idx[r, q]] += w[r, q]
    B = A[crow]
    Bh = B[:, o["J"]] @ o["C"]
    assert np.max(np.abs(o["Ahat_spid"] - M @ Bh)) <= 1e-12 * np.abs(M @ Bh).max()
    lhs = np.linalg.norm(A - M @ Bh, 2)
    rhs = np.linalg.norm(A - M @ B, 2) + np.linalg.norm(M, 2) * np.linalg.norm(B - Bh, 2)
    assert lhs <= rhs * (1 + 1e-12)


def test_section_5_1_random_points_rank_one():
    # u1 of the 2D TGV on 20^2 random points, 100 snapshots to t = 10: rank one
    # and an error at the FP64 rounding level for the column ID (Section 5.1)
    pts, A = inputs.unstructured_tgv2d(400, 100, seed=12, qois=("u1",))
    m = A.shape[0]
    o = oracle.subid_points(A, np.arange(m), np.arange(m).reshape(m, 1), np.ones((m, 1)), 4,
                            1e-12, 2.0 ** -53)
    assert o["k"] == 1
    assert np.sqrt(o["e2_subid"] / o["a2"]) <= 1e-14
    # CF = m n / (k (m + n)) = 400 * 100 / 500 = 80, the paper's "approx 80"
    assert m * 100 / (o["k"] * (m + 100)) == pytest.approx(80.0)
