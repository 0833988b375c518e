"""Shared test helpers: oracle runs, separation of pivots, relative errors."""
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
