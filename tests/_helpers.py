"""Shared test helpers: oracle runs, separation of pivots, relative errors, and
the parity checker that compares a result of the CUDA path with the oracle's
(a CPU function, so that its own tests can feed it deliberately wrong results)."""
import numpy as np

import oracle

U_MODE = {"fp64": 2.0 ** -53, "fp32": 2.0 ** -24, "tf32": 2.0 ** -11, "bf16": 2.0 ** -9,
          "bf16x3": 2.0 ** -16}


def rel_fro(a, b) -> float:
    """||a - b||_F / ||b||_F (0 when both are zero)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    if nb == 0.0:
        return float(np.linalg.norm(a))
    return float(np.linalg.norm(a - b) / nb)


def separated_prefix(Y: np.ndarray, k: int, gap: float, u: float = 0.0, tau: float = 8.0) -> int:
    """Number of leading pivot steps of the oracle's pivoted QR of Y that are
    decided with a margin: the best residual norm^2 beats the runner-up by a
    relative gap >= `gap`, AND the residual norms differ by more than the
    rounding floor tau * u * ||Y||_F * sqrt(j + 1) that a backward-stable QR in
    unit roundoff u can move them by.  J must agree bit-exactly over this
    prefix; past it several pivots are valid and only reconstructions compare."""
    Y = np.asarray(Y, dtype=np.float64)
    l, n = Y.shape
    J, R, kk, _ = oracle.qrcp_mgs(Y, k)
    col2 = (Y * Y).sum(0)
    ny = np.linalg.norm(Y)
    for j in range(kk):
        nu = col2 - (R[:j] ** 2).sum(0) if j > 0 else col2.copy()
        nu[J[:j]] = -np.inf
        order = np.sort(nu)[::-1]
        best = order[0]
        second = order[1] if n - j > 1 else -np.inf
        if not (best > 0) or (best - second) / best < gap:
            return j
        if np.sqrt(best) - np.sqrt(max(second, 0.0)) <= tau * u * ny * np.sqrt(j + 1):
            return j
    return kk


def r11_condition(Y: np.ndarray, k: int) -> float:
    """2-norm condition number of the oracle's R11 (k leading pivots of Y)."""
    if k <= 0:
        return 1.0
    J, R, kk, _ = oracle.qrcp_mgs(np.asarray(Y, dtype=np.float64), k)
    return float(np.linalg.cond(R[:kk][:, J[:kk]]))


def adaptive_margin(Y: np.ndarray, kmax: int, tol: float, k: int) -> float:
    """Relative distance of the adaptive stopping test from its threshold at the
    oracle's decision k (min over the two trailing norms that bracket it)."""
    J, R, kk, nY2 = oracle.qrcp_mgs(np.asarray(Y, dtype=np.float64), kmax)
    col2 = (np.asarray(Y, dtype=np.float64) ** 2).sum(0)
    def trail(j):
        nu = col2 - (R[:j] ** 2).sum(0) if j > 0 else col2.copy()
        nu[J[:j]] = 0.0
        return nu.clip(min=0).sum()
    thr = tol * tol * nY2
    ms = []
    for j in (k - 1, k):
        if 0 <= j <= kk:
            ms.append(abs(trail(j) - thr) / thr)
    return min(ms) if ms else np.inf


def oracle_window(win, l, kmax, tol, precision, seed):
    """Oracle SPID over every subdomain of a window (values taken exactly into FP64)."""
    return oracle.spid_batch(win.data, win.m, win.n, win.off, win.ld, l, kmax, tol,
                             U_MODE[precision], seed, want_y=True)


def oracle_reconstruction(A: np.ndarray, J, C, k: int) -> np.ndarray:
    Ahat, _, _ = oracle.reconstruct_error(A, np.asarray(J[:k], dtype=np.int32), C[:k])
    return Ahat


def guard_margin(Y: np.ndarray, kmax: int, u: float, k: int, tol: float = 0.0) -> float:
    """Distance of the pivots that bracket the oracle's rank-guard decision k
    (the last kept, k - 1, and the first dropped, k) from the guard threshold
    2 u |R_00|, relative to ||Y||_F.  A sketch that differs from the oracle's
    by rounding moves every |R_jj| by about its relative difference times
    ||Y||_F, so a k that differs by one is valid only when this is that small."""
    Y = np.asarray(Y, dtype=np.float64)
    J, R, kk, _ = oracle.qrcp_mgs(Y, kmax, tol)
    if kk == 0:
        return np.inf
    thr = 2.0 * u * abs(R[0, J[0]])
    ny = np.linalg.norm(Y)
    ms = [abs(abs(R[j, J[j]]) - thr) / ny for j in (k - 1, k) if 0 <= j < kk]
    return min(ms) if ms else np.inf


Y_TOL = {"fp64": 1e-13, "fp32": 2e-6, "tf32": 3e-3, "bf16": 1.5e-2, "bf16x3": 1e-4}
GAP = {"fp64": 1e-6, "fp32": 1e-3, "tf32": 2e-2, "bf16": 1e-1, "bf16x3": 1e-3}
SPID_ERR_RANK = 8
# statuses of a run whose purpose is not the rank decision: SPID_OK, or the
# informational rank-guard cut (its factors are valid)
STATUS_OK = (0, SPID_ERR_RANK)


def compare_with_oracle(blocks, g: dict, o: dict, precision: str, k_max: int, tol: float = 0.0,
                        c_tol=None, ahat_tol=None, min_prefix: int = 0, sample: bool = False):
    """Assert that the CUDA path's result g matches the oracle's o.

    blocks: the subdomains' data matrices (m_s x n_s).  g: k [S], J [S, k_max],
    C (list of k_max x n_s), Y (list of l x n_s), err [S, 2], status, and
    optionally Ahat (list).  o: oracle.spid_batch(..., want_y=True).
    Tolerances, from the arithmetic: Y by Y_TOL; J bit-exact over the oracle's
    separated prefix (at least min_prefix pivots on inputs built to be
    separated); k equal unless the adaptive test or the rank guard sits within
    rounding of its threshold (then +-1); the rank-cut status set exactly when
    the oracle's guard cut some subdomain (unless such a subdomain is within
    rounding); C(:, J) = I exactly; C within max(c_tol, 8 cond(R11) u); A_hat
    within ahat_tol; each error within the triangle-inequality bound.
    sample=True: the blocks are a sample of the plan's subdomains, so the
    window-wide status must show a cut the sample has, but may show others."""
    u = U_MODE[precision]
    # the QR's own rounding of |R_jj| (FP32 reflectors in every FP32-window mode)
    u_qr = 2.0 ** -53 if precision == "fp64" else 2.0 ** -24
    ambiguous_cut = False
    expect_cut = False
    for s, A in enumerate(blocks):
        A = np.asarray(A, dtype=np.float64)
        Yo = o["Y"][s]
        dy = rel_fro(g["Y"][s], Yo)
        assert dy <= Y_TOL[precision], ("Y", s, dy)
        ko, kg = int(o["k"][s]), int(g["k"][s])
        kqr = int(o["k_qr"][s])
        # a pivot moves by about the sketches' difference plus the QR's rounding
        band = 2.0 * dy + 16 * u_qr * np.sqrt(k_max + 16)
        gm = guard_margin(Yo, k_max, u, ko, tol)
        near_guard = gm <= band
        if kg != ko:
            if tol > 0 and adaptive_margin(Yo, k_max, tol, ko) <= 64 * Y_TOL[precision]:
                pass   # adaptive stop taken from sketches that differ by rounding
            else:
                assert abs(kg - ko) <= 1 and near_guard, ("k", s, kg, ko, gm)
        if ko < kqr:
            expect_cut = True
        if near_guard:
            ambiguous_cut = True
        sep = separated_prefix(Yo, max(ko, 1), GAP[precision], u)
        assert min(sep, ko) >= min(min_prefix, ko), ("separated prefix too short", s, sep, ko)
        pre = min(sep, ko, kg)
        assert list(g["J"][s][:pre]) == list(o["J"][s][:pre]), ("J", s, g["J"][s], o["J"][s], pre)
        Jg = g["J"][s][:kg]
        assert np.all(np.asarray(g["J"][s][kg:]) == -1), ("J past k", s)
        if kg:
            # C(:, J) = I exactly (Lemma A.1 item 1)
            assert np.array_equal(g["C"][s][:kg][:, Jg], np.eye(kg, dtype=g["C"][s].dtype)), ("C(:,J)", s)
        if kg == ko and list(Jg) == list(o["J"][s][:ko]):
            if c_tol is not None:
                # C = R11^-1 R12 moves by about cond(R11) times the relative
                # perturbation of the sketch: its rounding u, or the measured
                # difference of the two sketches (summation order) if larger
                ct = max(c_tol, 8.0 * r11_condition(Yo, ko) * max(u, dy))
                dc = rel_fro(g["C"][s][:kg], o["C"][s][:ko])
                assert dc <= ct, ("C", s, dc, ct)
            if ahat_tol is not None and "Ahat" in g:
                Ahat_o, e2, a2 = oracle.reconstruct_error(A, o["J"][s][:ko], o["C"][s][:ko])
                d = rel_fro(g["Ahat"][s], Ahat_o)
                assert d <= ahat_tol, ("Ahat", s, d)
                eg = np.sqrt(g["err"][s][0] / g["err"][s][1]) if g["err"][s][1] > 0 else 0.0
                eo = np.sqrt(e2 / a2) if a2 > 0 else 0.0
                # |e_gpu - e_oracle| <= ||Ahat_gpu - Ahat_oracle|| / ||A|| (triangle inequality)
                assert abs(eg - eo) <= d * 1.01 + 4 * u * np.sqrt(A.size), ("err", s, eg, eo)
                rel = 1e-6 if precision != "fp64" else 1e-12
                assert abs(g["err"][s][1] - a2) <= rel * a2, ("a2", s)
    status = int(g["status"])
    assert status in (0, SPID_ERR_RANK), ("status", status)
    if sample:
        if expect_cut and not ambiguous_cut:
            assert status == SPID_ERR_RANK, ("rank-cut status", status, expect_cut)
    elif not ambiguous_cut:
        assert (status == SPID_ERR_RANK) == expect_cut, ("rank-cut status", status, expect_cut)


def ahat_matches_factors(A, J, C, Ahat, k: int, fp64: bool = False) -> bool:
    """The CUDA path's reconstruction of its OWN factors (J, C) against the
    oracle's reconstruction of the same factors, element-wise: products and
    sums of k terms in the working precision u,
    |d| <= 2 [(k + 1) u (|A_J| |C|) + u |A_hat|].  Unlike a comparison with
    the oracle's factors, this holds however ill-conditioned R11 is."""
    A = np.asarray(A, dtype=np.float64)
    if k == 0:
        return bool(np.all(np.asarray(Ahat) == 0))
    u = 2.0 ** -53 if fp64 else 2.0 ** -24
    Cf = np.asarray(C[:k], dtype=np.float64)
    Ao, _, _ = oracle.reconstruct_error(A, np.asarray(J[:k], dtype=np.int32), Cf)
    bound = 2.0 * ((k + 1) * u * (np.abs(A[:, J[:k]]) @ np.abs(Cf)) + u * np.abs(Ao))
    return bool(np.all(np.abs(np.asarray(Ahat, dtype=np.float64) - Ao) <= bound + 1e-300))
