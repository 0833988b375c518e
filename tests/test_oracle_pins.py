"""Pins for the FP64 CPU oracle: each test checks the oracle against something
other than itself -- published known-answer vectors, closed forms, exact
special cases, LAPACK's pivoted QR, scipy's deterministic ID, brute force on
tiny inputs and the compression factors printed in arXiv 2103.01380.

CPU only (no GPU marker)."""
import itertools
import os

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.stats as st

import oracle
from paper_2103_01380_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- Philox / Omega
def _kat_rows():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            v = [int(x, 16) for x in line.split()]
            rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,expect", _kat_rows())
def test_philox_known_answer_vectors(ctr, key, expect):
    out = oracle.philox4x32_10(ctr, key)[0]
    assert [int(x) for x in out] == expect


def test_omega_is_standard_gaussian():
    # 40 x 25000 = 1e6 draws: moments within 5 sigma of N(0,1), KS test.
    om = oracle.omega(seed=0x5EED0002, r0=0, nrows=25000, l=40).reshape(-1)
    N = om.size
    assert abs(om.mean()) < 5.0 / np.sqrt(N)
    assert abs(om.var() - 1.0) < 5.0 * np.sqrt(2.0 / N)
    assert abs(st.skew(om)) < 5.0 * np.sqrt(6.0 / N)
    assert abs(st.kurtosis(om, fisher=False) - 3.0) < 5.0 * np.sqrt(24.0 / N)
    assert st.kstest(om, "norm").pvalue > 1e-4
    # rows of Omega are uncorrelated
    om2 = oracle.omega(seed=7, r0=0, nrows=20000, l=8)
    cc = np.corrcoef(om2)
    assert np.max(np.abs(cc - np.eye(8))) < 5.0 / np.sqrt(20000)


def test_omega_counter_layout():
    # Omega(i, r) depends only on (seed, i, r): any window of rows agrees.
    a = oracle.omega(11, 0, 300, 13)
    b = oracle.omega(11, 100, 150, 13)
    assert np.array_equal(a[:, 100:250], b)
    # group g = i // 4 of row r comes from one Philox call with counter (r, g, 0, 0)
    x = oracle.philox4x32_10([[5, 2, 0, 0]], [11, 0])[0].astype(np.float64)
    u = (x + 0.5) * 2.0 ** -32
    g = [np.sqrt(-2 * np.log(u[0])) * np.cos(2 * np.pi * u[1]),
         np.sqrt(-2 * np.log(u[0])) * np.sin(2 * np.pi * u[1]),
         np.sqrt(-2 * np.log(u[2])) * np.cos(2 * np.pi * u[3]),
         np.sqrt(-2 * np.log(u[2])) * np.sin(2 * np.pi * u[3])]
    np.testing.assert_allclose(a[8:12, 5], g, rtol=1e-15, atol=0)


# ---------------------------------------------------------------- sketch
def test_sketch_of_unit_matrix_is_omega_column():
    m, n, l = 57, 9, 11
    Om = oracle.omega(3, 0, m, l)
    for (i, j) in [(0, 0), (56, 8), (20, 4)]:
        A = np.zeros((m, n))
        A[i, j] = 1.0
        Y = oracle.sketch(A, l, 3)
        assert np.array_equal(Y[:, j], Om[:, i])
        Y[:, j] = 0.0
        assert not Y.any()


def test_sketch_matches_dense_product_and_is_linear():
    rng = np.random.default_rng(5)
    m, n, l = 300, 17, 12
    A, B = rng.standard_normal((m, n)), rng.standard_normal((m, n))
    Om = oracle.omega(99, 0, m, l)
    YA = oracle.sketch(A, l, 99)
    np.testing.assert_allclose(YA, Om @ A, rtol=0, atol=1e-12 * np.abs(Om).sum(1).max())
    YC = oracle.sketch(2.0 * A - 3.0 * B, l, 99)
    np.testing.assert_allclose(YC, 2.0 * YA - 3.0 * oracle.sketch(B, l, 99), atol=1e-11)
    # columns are sketched independently: any split of the window gives the same Y bitwise
    assert np.array_equal(np.concatenate([oracle.sketch(A[:, :5], l, 99),
                                          oracle.sketch(A[:, 5:], l, 99)], axis=1), YA)


# ---------------------------------------------------------------- pivoted QR
def _separated_sketch(seed=1, m=200, n=30, l=12, r=8):
    A = inputs.separated_lowrank(m, n, r, seed=seed, decay=0.6, noise=1e-3)
    return oracle.sketch(A, l, seed)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_qrcp_matches_lapack_geqp3(seed):
    Y = _separated_sketch(seed)
    k = 6
    J, R, kk, _ = oracle.qrcp_mgs(Y, k)
    assert kk == k
    _, Rs, P = sla.qr(Y, pivoting=True)
    assert list(J) == list(P[:k])
    # |R| agrees (rows may differ in sign between MGS and Householder)
    np.testing.assert_allclose(np.abs(R[:, P]), np.abs(Rs[:k, :]), rtol=0,
                               atol=1e-12 * np.abs(Rs).max())


def test_qrcp_mgs_equals_householder():
    for seed in range(4):
        Y = _separated_sketch(seed + 10, n=40, l=16, r=12)
        J1, R1, k1, _ = oracle.qrcp_mgs(Y, 10)
        J2, R2, k2, _ = oracle.qrcp_householder(Y, 10)
        assert k1 == k2 == 10 and list(J1) == list(J2)
        np.testing.assert_allclose(np.abs(R1), np.abs(R2), atol=1e-12 * np.abs(R1).max())


def test_qrcp_greedy_choice_by_brute_force():
    # At each step the pivot maximises the residual norm after projecting out
    # the span of the columns already chosen (computed here by least squares).
    rng = np.random.default_rng(4)
    for trial in range(5):
        Y = rng.standard_normal((6, 10)) * (0.5 ** np.arange(10))[None, rng.permutation(10)]
        J, R, k, _ = oracle.qrcp_mgs(Y, 5)
        chosen = []
        for j in range(k):
            best, arg = -1.0, -1
            for c in range(10):
                if c in chosen:
                    continue
                if chosen:
                    S = Y[:, chosen]
                    res = Y[:, c] - S @ np.linalg.lstsq(S, Y[:, c], rcond=None)[0]
                else:
                    res = Y[:, c]
                if res @ res > best * (1 + 1e-12):
                    best, arg = res @ res, c
            assert J[j] == arg
            assert abs(R[j, arg] - np.sqrt(best)) <= 1e-10 * np.sqrt(best)
            chosen.append(arg)


def test_qrcp_ties_go_to_lowest_index():
    Y = np.zeros((4, 6))
    Y[0, 3] = Y[1, 1] = Y[2, 5] = 2.0    # three columns of equal norm
    Y[3, 0] = 1.0
    J, R, k, _ = oracle.qrcp_mgs(Y, 4)
    assert list(J[:4]) == [1, 3, 5, 0]
    J2, _, _, _ = oracle.qrcp_householder(Y, 4)
    assert list(J2[:4]) == [1, 3, 5, 0]


def test_adaptive_stop_matches_trailing_norms():
    # Remark 2.1 reading: smallest k with ||R22^(k)||_F <= tol ||Y||_F.
    A = inputs.spectrum_matrix(400, 60, 10.0 ** (-np.arange(1, 41) / 4.0), seed=3)
    Y = oracle.sketch(A, 42, 3)
    _, Rs, P = sla.qr(Y, pivoting=True)
    ny = np.linalg.norm(Y)
    for tol in [1e-1, 1e-2, 1e-3, 1e-4]:
        J, R, k, _ = oracle.qrcp_mgs(Y, 32, tol)
        trail = [np.linalg.norm(Rs[kk:, kk:]) / ny for kk in range(33)]
        expect = next(kk for kk in range(33) if trail[kk] <= tol or kk == 32)
        assert k == expect, (tol, k, expect)


# ---------------------------------------------------------------- coefficients
def test_coefficients_identity_and_triangular_solve():
    Y = _separated_sketch(7, n=25, l=10, r=9)
    k = 5
    J, R, kk, _ = oracle.qrcp_mgs(Y, k)
    C = oracle.coefficients(R, J, k)
    assert np.array_equal(C[:, J], np.eye(k))              # Lemma A.1 item 1, exact
    rest = [c for c in range(25) if c not in set(J)]
    T = sla.solve_triangular(R[:, J], R[:, rest], lower=False)
    np.testing.assert_allclose(C[:, rest], T, rtol=1e-12, atol=1e-12)


def test_coefficients_match_scipy_interp_decomp():
    import scipy.linalg.interpolative as sli
    Y = _separated_sketch(9, n=30, l=14, r=10)
    k = 6
    J, R, kk, _ = oracle.qrcp_mgs(Y, k)
    C = oracle.coefficients(R, J, k)
    idx, proj = sli.interp_decomp(Y.copy(order="F"), k, rand=False)
    assert set(idx[:k].tolist()) == set(J.tolist())
    # scipy's projection is expressed in its own skeleton order
    Cs = np.zeros((k, 30))
    Cs[:, idx[:k]] = np.eye(k)
    Cs[:, idx[k:]] = proj
    order = [list(idx[:k]).index(j) for j in J]
    np.testing.assert_allclose(C, Cs[order], rtol=0, atol=1e-10 * max(1, np.abs(Cs).max()))


# ---------------------------------------------------------------- whole SPID
@pytest.mark.parametrize("r,k", [(3, 3), (3, 5), (1, 1)])
def test_exact_low_rank_is_reproduced(r, k):
    A = inputs.lowrank(500, 40, r, seed=r + k)
    res = oracle.spid(A, k + 10, k, 0.0, oracle.U_MODE["fp64"], 0x5EED)
    rel = np.sqrt(res["e2"] / res["a2"])
    assert rel <= 1e-13, rel
    assert np.array_equal(res["C"][:res["k"], res["J"][:res["k"]]], np.eye(res["k"]))


def test_analytic_tgv_is_rank_one():
    # Section 5.1: the analytic TGV velocity is rank one in time; error ~ machine precision.
    A = inputs.tgv2d(nx=20, n=100, noise=0.0)[:400]        # u1 on the 20^2 grid
    res = oracle.spid(A, 11, 1, 0.0, oracle.U_MODE["fp64"], 1)
    assert res["k"] == 1
    assert np.sqrt(res["e2"] / res["a2"]) <= 1e-14
    assert oracle.compression_factor([400], [100], [1]) == pytest.approx(80.0, rel=1e-12)
    both = inputs.tgv2d(nx=64, n=128, noise=0.0)           # u1 and u2 stacked: still rank one
    res = oracle.spid(both, 11, 1, 0.0, oracle.U_MODE["fp64"], 1)
    assert np.sqrt(res["e2"] / res["a2"]) <= 1e-14


def test_error_is_between_svd_floor_and_best_subset():
    # Brute force over all size-k column subsets with least-squares coefficients.
    rng = np.random.default_rng(12)
    for trial in range(3):
        A = inputs.spectrum_matrix(30, 10, 0.4 ** np.arange(10), seed=trial) \
            + 1e-3 * rng.standard_normal((30, 10))
        sv = np.linalg.svd(A, compute_uv=False)
        for k in (1, 2, 3):
            best = np.inf
            for sub in itertools.combinations(range(10), k):
                S = A[:, sub]
                E = A - S @ np.linalg.lstsq(S, A, rcond=None)[0]
                best = min(best, np.linalg.norm(E))
            res = oracle.spid(A, k + 6, k, 0.0, oracle.U_MODE["fp64"], 100 + trial)
            e = np.sqrt(res["e2"])
            floor = np.sqrt((sv[k:] ** 2).sum())
            assert floor <= best * (1 + 1e-12)
            assert best <= e * (1 + 1e-12)
            # Lemma A.1 item 6 bound (existence ID) with sigma_{k+1}, as a loose statistic
            assert e <= 10.0 * np.sqrt(k * (10 - k) + 1) * sv[k] * np.sqrt(10)


def test_geometric_spectrum_error_tracks_closed_form():
    # sigma_i = 10^{-i/4}: the best rank-k relative error is
    # sqrt(sum_{i>k} s_i^2 / sum s_i^2) (Eckart-Young).  The sketched ID must sit
    # above that floor and, with p = 10 oversampling, within a small factor of
    # the direct column ID of A (Algorithm 1, here scipy's deterministic ID).
    import scipy.linalg.interpolative as sli
    sig = 10.0 ** (-np.arange(1, 257) / 4.0)
    A = inputs.spectrum_matrix(2048, 256, sig, seed=3)
    for k in (4, 8, 12, 16):
        floor = np.sqrt((sig[k:] ** 2).sum() / (sig ** 2).sum())
        res = oracle.spid(A, k + 10, k, 0.0, oracle.U_MODE["fp64"], 77)
        rel = np.sqrt(res["e2"] / res["a2"])
        idx, proj = sli.interp_decomp(A.copy(order="F"), k, rand=False)
        direct = np.linalg.norm(A - sli.reconstruct_matrix_from_id(A[:, idx[:k]], idx, proj)) \
            / np.linalg.norm(A)
        assert floor <= direct * (1 + 1e-12) and floor <= rel
        assert rel <= 4.0 * direct and rel <= 5.0 * floor, (k, rel, direct, floor)


def test_relative_error_definition_and_scale_invariance():
    rng = np.random.default_rng(1)
    A = rng.standard_normal((64, 12))
    J = np.arange(12, dtype=np.int32)
    _, e2, a2 = oracle.reconstruct_error(A, J, np.eye(12))
    assert e2 == 0.0 and a2 == pytest.approx((A ** 2).sum(), rel=1e-15)
    B = inputs.separated_lowrank(200, 20, 6, seed=2, noise=1e-4)
    r1 = oracle.spid(B, 14, 4, 0.0, oracle.U_MODE["fp64"], 5)
    r2 = oracle.spid(B * 2.0 ** 7, 14, 4, 0.0, oracle.U_MODE["fp64"], 5)
    assert list(r1["J"]) == list(r2["J"])
    assert np.array_equal(r1["C"], r2["C"])
    assert r1["e2"] / r1["a2"] == r2["e2"] / r2["a2"]


def test_rank_guard_drops_exactly_dependent_pivots():
    # integer rank-2 matrix: the third pivot has R_33 at rounding level
    A = np.zeros((40, 8))
    A[:, 0] = 1.0
    A[:, 1] = np.arange(40)
    for c in range(2, 8):
        A[:, c] = (c - 1) * A[:, 0] + (3 - c) * A[:, 1]
    res = oracle.spid(A, 9, 5, 0.0, oracle.U_MODE["fp64"] * 1e3, 3)
    assert res["k"] == 2
    assert np.sqrt(res["e2"] / res["a2"]) < 1e-12


# ---------------------------------------------------------------- compression factor
def _cf_rows():
    rows = []
    with open(os.path.join(GOLDEN, "compression_factors.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            p = [x.strip() for x in line.split("|")]
            ints = lambda s: [int(x) for x in s.split(",")]
            rows.append((p[0], ints(p[1]), ints(p[2]), int(p[3]), ints(p[4]), float(p[5]),
                         float(p[6])))
    return rows


@pytest.mark.parametrize("label,m,s,n,k,value,rtol", _cf_rows())
def test_compression_factor_printed_values(label, m, s, n, k, value, rtol):
    cf = oracle.compression_factor(m, [n] * len(m), k, stored_rows=s)
    assert cf == pytest.approx(value, rel=rtol), (label, cf)


def test_partitioning_gain_table2():
    # Section 3.2: 5 partitions give a CF "almost 70% larger" than 1 partition.
    one = oracle.compression_factor([100], [100], [48])
    five = oracle.compression_factor([20] * 5, [100] * 5, [6, 12, 6, 12, 12])
    assert 1.6 < five / one < 1.7
