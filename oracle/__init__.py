"""Plain FP64 CPU oracle for the sketched column interpolative decomposition.

TEST INFRASTRUCTURE ONLY.  This package is the oracle the CUDA path is checked
against.  Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU
baseline leg (and its ``--impl reference`` arm) may import it.  It shares no
code with ``paper_2103_01380_gb300`` and never imports it.

The arithmetic lives in ``spid_oracle.c`` (plain C, FP64, one loop nest per
definition, each function citing the passage of arXiv 2103.01380 it follows);
this module only compiles it with gcc and marshals numpy arrays through ctypes.

Pins: every function here is checked in ``tests/test_oracle_*.py`` against
what the paper and the mathematics fix (published Philox known-answer vectors,
closed forms, exact special cases, LAPACK's pivoted QR, brute force on tiny
inputs, the paper's printed compression factors).  No function is
"parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "spid_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_u32p = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile spid_oracle.c into oracle/_build/liboracle.so with gcc."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        c = ctypes
        lib.orc_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
        lib.orc_philox4x32_10.restype = None
        lib.orc_omega_entry.argtypes = [c.c_uint64, c.c_int64, c.c_int64]
        lib.orc_omega_entry.restype = c.c_double
        lib.orc_omega.argtypes = [c.c_uint64, c.c_int64, c.c_int64, c.c_int32, _f64p]
        lib.orc_omega.restype = None
        lib.orc_sketch.argtypes = [_f64p, c.c_int64, c.c_int64, c.c_int64, c.c_int32,
                                   c.c_uint64, _f64p]
        lib.orc_sketch.restype = None
        for name in ("orc_qrcp_mgs", "orc_qrcp_householder"):
            fn = getattr(lib, name)
            fn.argtypes = [_f64p, c.c_int32, c.c_int64, c.c_int32, c.c_double, _i32p, _f64p,
                           c.POINTER(c.c_double)]
            fn.restype = c.c_int
        lib.orc_rank_guard.argtypes = [_f64p, c.c_int64, _i32p, c.c_int32, c.c_double]
        lib.orc_rank_guard.restype = c.c_int
        lib.orc_coefficients.argtypes = [_f64p, c.c_int64, _i32p, c.c_int32, _f64p]
        lib.orc_coefficients.restype = None
        lib.orc_reconstruct_error.argtypes = [_f64p, c.c_int64, c.c_int64, c.c_int64, _i32p,
                                              c.c_int32, _f64p, c.c_void_p, c.c_int64,
                                              c.POINTER(c.c_double), c.POINTER(c.c_double)]
        lib.orc_reconstruct_error.restype = None
        lib.orc_compression_factor.argtypes = [c.c_int32, _i64p, c.c_void_p, _i64p, _i32p]
        lib.orc_compression_factor.restype = c.c_double
        lib.orc_spid_batch.argtypes = [_f64p, c.c_int32, _i64p, _i64p, _i64p, _i64p,
                                       c.c_int32, c.c_int32, c.c_double, c.c_double, c.c_uint64,
                                       c.c_void_p, _i32p, _i32p, _i32p, _f64p, _f64p, _f64p]
        lib.orc_error_per_qoi.argtypes = [_f64p, c.c_int64, c.c_int64, c.c_int64, _i32p,
                                          c.c_int32, _f64p, c.c_int32, _f64p, _f64p]
        lib.orc_error_per_qoi.restype = None
        lib.orc_qoi_totals.argtypes = [c.c_int32, _i32p, _f64p, _f64p, c.c_int32, _f64p, _f64p]
        lib.orc_qoi_totals.restype = None
        lib.orc_spid_batch.restype = c.c_int
        lib.orc_coarse_axis.argtypes = [c.c_int32, c.c_int32, c.c_void_p]
        lib.orc_coarse_axis.restype = c.c_int
        lib.orc_coarse_rows.argtypes = [_i32p, _i32p]
        lib.orc_coarse_rows.restype = c.c_int64
        lib.orc_subsample.argtypes = [_f64p, c.c_int64, c.c_int64, _i32p, _i32p, _f64p]
        lib.orc_subsample.restype = None
        lib.orc_trilinear.argtypes = [_f64p, c.c_int64, _i32p, _i32p, _f64p, c.c_int64]
        lib.orc_trilinear.restype = None
        lib.orc_subid.argtypes = [_f64p, c.c_int64, c.c_int64, _i32p, _i32p, c.c_int32,
                                  c.c_double, c.c_double, _i32p, _f64p, c.c_void_p, _f64p,
                                  c.c_void_p]
        lib.orc_subid.restype = c.c_int
        lib.orc_subid_points.argtypes = [_f64p, c.c_int64, c.c_int64, c.c_int64, _i32p,
                                         c.c_int64, c.c_int32, _i32p, _f64p, c.c_int32,
                                         c.c_double, c.c_double, _i32p, _f64p, c.c_void_p,
                                         _f64p, c.c_void_p]
        lib.orc_subid_points.restype = c.c_int
        lib.orc_two_stage.argtypes = [_f64p, c.c_int64, c.c_int64, c.c_int64, c.c_int32,
                                      c.c_int32, c.c_int32, c.c_int32, c.c_double, c.c_double,
                                      c.c_uint64, _i32p, _f64p, _i32p, _i32p, _f64p, _i32p,
                                      _f64p, _f64p]
        lib.orc_two_stage.restype = c.c_int
        lib.orc_num_threads.argtypes = []
        lib.orc_num_threads.restype = c.c_int
        _lib = lib
        return lib


# Unit roundoff per arithmetic mode, used by the rank guard (|R_jj| > 2 u |R_00|).
U_MODE = {
    "fp64": 2.0 ** -53,
    "fp32": 2.0 ** -24,
    "tf32": 2.0 ** -11,
}


def num_threads() -> int:
    return int(_load().orc_num_threads())


def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 of each 4-word counter row under a 2-word key."""
    lib = _load()
    ctr = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32).reshape(-1, 4))
    key = np.ascontiguousarray(np.asarray(key, dtype=np.uint32).reshape(2))
    out = np.empty_like(ctr)
    one = np.empty(4, dtype=np.uint32)
    for t in range(ctr.shape[0]):
        lib.orc_philox4x32_10(np.ascontiguousarray(ctr[t]), key, one)
        out[t] = one
    return out


def omega(seed: int, r0: int, nrows: int, l: int) -> np.ndarray:
    """Omega(:, r0:r0+nrows) as an l x nrows FP64 array."""
    out = np.empty((nrows, l), dtype=np.float64)  # column-major l x nrows
    _load().orc_omega(seed, r0, nrows, l, out.reshape(-1))
    return out.T.copy()


def sketch(A: np.ndarray, l: int, seed: int) -> np.ndarray:
    """Y = Omega A for an m x n matrix A (any layout; copied column-major)."""
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    Af = np.ascontiguousarray(A.T)  # row j of Af = column j of A
    Y = np.empty((n, l), dtype=np.float64)
    _load().orc_sketch(Af.reshape(-1), m, n, m, l, seed, Y.reshape(-1))
    return Y.T.copy()


def _qrcp(name: str, Y: np.ndarray, kmax: int, tol: float):
    Y = np.asarray(Y, dtype=np.float64)
    l, n = Y.shape
    W = np.ascontiguousarray(Y.T).reshape(-1).copy()
    J = np.full(kmax, -1, dtype=np.int32)
    R = np.zeros(kmax * n, dtype=np.float64)
    nY2 = ctypes.c_double(0.0)
    k = getattr(_load(), name)(W, l, n, kmax, tol, J, R, ctypes.byref(nY2))
    return J, R.reshape(kmax, n), int(k), float(nY2.value)


def qrcp_mgs(Y, kmax: int, tol: float = 0.0):
    """Pivoted modified Gram-Schmidt QR of Y (l x n).

    Returns (J, R, k, ||Y||_F^2); R is kmax x n in ORIGINAL column numbering."""
    return _qrcp("orc_qrcp_mgs", Y, kmax, tol)


def qrcp_householder(Y, kmax: int, tol: float = 0.0):
    """Householder QR with column pivoting; same conventions as qrcp_mgs."""
    return _qrcp("orc_qrcp_householder", Y, kmax, tol)


def rank_guard(R: np.ndarray, J: np.ndarray, k: int, u_mode: float) -> int:
    R = np.ascontiguousarray(R, dtype=np.float64)
    return int(_load().orc_rank_guard(R.reshape(-1), R.shape[1],
                                      np.ascontiguousarray(J, dtype=np.int32), k, u_mode))


def coefficients(R: np.ndarray, J: np.ndarray, k: int) -> np.ndarray:
    """C = [I | R11^-1 R12] Z^T as a k x n array."""
    R = np.ascontiguousarray(R, dtype=np.float64)
    n = R.shape[1]
    C = np.zeros(max(k, 1) * n, dtype=np.float64)
    _load().orc_coefficients(R.reshape(-1), n, np.ascontiguousarray(J[:max(k, 1)], dtype=np.int32),
                             k, C)
    return C.reshape(max(k, 1), n)[:k]


def reconstruct_error(A: np.ndarray, J: np.ndarray, C: np.ndarray, want_ahat: bool = True):
    """A_hat = A(:,J) C, ||A - A_hat||_F^2 and ||A||_F^2."""
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    k = int(C.shape[0])
    Af = np.ascontiguousarray(A.T).reshape(-1)
    Cc = np.ascontiguousarray(C, dtype=np.float64).reshape(-1) if k > 0 else np.zeros(1)
    Jc = np.ascontiguousarray(J[:k], dtype=np.int32) if k > 0 else np.zeros(1, dtype=np.int32)
    H = np.empty((n, m), dtype=np.float64) if want_ahat else None
    e2 = ctypes.c_double(0.0)
    a2 = ctypes.c_double(0.0)
    _load().orc_reconstruct_error(Af, m, n, m, Jc, k, Cc,
                                  H.ctypes.data if want_ahat else None, m,
                                  ctypes.byref(e2), ctypes.byref(a2))
    return (H.T.copy() if want_ahat else None), float(e2.value), float(a2.value)


def error_per_qoi(A: np.ndarray, J: np.ndarray, C: np.ndarray, nq: int):
    """Per-QoI (||A_q - A_hat_q||_F^2, ||A_q||_F^2) of one box whose rows hold
    nq QoI blocks of m / nq rows each (QoI slowest): two arrays of nq."""
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    if m % nq:
        raise ValueError("m must be a multiple of nq")
    k = int(C.shape[0])
    Af = np.ascontiguousarray(A.T).reshape(-1)
    Cc = np.ascontiguousarray(C, dtype=np.float64).reshape(-1) if k > 0 else np.zeros(1)
    Jc = np.ascontiguousarray(J[:k], dtype=np.int32) if k > 0 else np.zeros(1, dtype=np.int32)
    e2 = np.zeros(nq, dtype=np.float64)
    a2 = np.zeros(nq, dtype=np.float64)
    _load().orc_error_per_qoi(Af, m, n, m, Jc, k, Cc, nq, e2, a2)
    return e2, a2


def qoi_totals(qoi, e2, a2, nqoi: int):
    """Sums of per-subdomain e2 / a2 over the subdomains of each QoI."""
    qoi = np.ascontiguousarray(qoi, dtype=np.int32)
    e2 = np.ascontiguousarray(e2, dtype=np.float64)
    a2 = np.ascontiguousarray(a2, dtype=np.float64)
    if qoi.size and (qoi.min() < 0 or qoi.max() >= nqoi):
        raise ValueError("qoi index out of range")
    ge2 = np.zeros(nqoi, dtype=np.float64)
    ga2 = np.zeros(nqoi, dtype=np.float64)
    _load().orc_qoi_totals(len(qoi), qoi, e2, a2, nqoi, ge2, ga2)
    return ge2, ga2


def compression_factor(m, n, k, stored_rows=None) -> float:
    """Aggregate CF = sum m_i n_i / sum k_i (s_i + n_i) (s_i = m_i by default)."""
    m = np.ascontiguousarray(np.atleast_1d(m), dtype=np.int64)
    n = np.ascontiguousarray(np.broadcast_to(np.atleast_1d(n), m.shape), dtype=np.int64)
    k = np.ascontiguousarray(np.atleast_1d(k), dtype=np.int32)
    srows = None
    if stored_rows is not None:
        srows = np.ascontiguousarray(np.atleast_1d(stored_rows), dtype=np.int64)
    return float(_load().orc_compression_factor(len(m), m, srows.ctypes.data if srows is not None
                                                else None, n, k))


def spid_batch(window: np.ndarray, m, n, off, ld, l: int, kmax: int, tol: float,
               u_mode: float, seed: int, want_y: bool = False) -> dict:
    """Oracle SPID over every subdomain of a flat window (any float dtype; the
    values are taken exactly into FP64).  Layout: subdomain s is the
    m[s] x n[s] column-major block at window[off[s]:] with leading dimension
    ld[s]."""
    w = np.ascontiguousarray(np.asarray(window).reshape(-1), dtype=np.float64)
    m = np.ascontiguousarray(m, dtype=np.int64)
    n = np.ascontiguousarray(n, dtype=np.int64)
    off = np.ascontiguousarray(off, dtype=np.int64)
    ld = np.ascontiguousarray(ld, dtype=np.int64)
    S = len(m)
    ntot = int(n.sum())
    J = np.full(S * kmax, -1, dtype=np.int32)
    k = np.zeros(S, dtype=np.int32)
    kqr = np.zeros(S, dtype=np.int32)
    C = np.zeros(kmax * ntot, dtype=np.float64)
    e2 = np.zeros(S, dtype=np.float64)
    a2 = np.zeros(S, dtype=np.float64)
    Y = np.zeros(l * ntot, dtype=np.float64) if want_y else None
    _load().orc_spid_batch(w, S, m, n, off, ld, l, kmax, tol, u_mode, seed,
                           Y.ctypes.data if want_y else None, J, k, kqr, C, e2, a2)
    coff = np.concatenate([[0], np.cumsum(n)])
    out = {"J": J.reshape(S, kmax), "k": k, "k_qr": kqr, "e2": e2, "a2": a2,
           "C": [C[kmax * coff[s]: kmax * coff[s + 1]].reshape(kmax, int(n[s]))
                 for s in range(S)]}
    if want_y:
        out["Y"] = [Y[l * coff[s]: l * coff[s + 1]].reshape(int(n[s]), l).T for s in range(S)]
    return out


def spid(A: np.ndarray, l: int, kmax: int, tol: float, u_mode: float, seed: int,
         want_y: bool = False) -> dict:
    """Oracle SPID on one m x n matrix."""
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    out = spid_batch(np.ascontiguousarray(A.T).reshape(-1), [m], [n], [0], [m], l, kmax, tol,
                     u_mode, seed, want_y=want_y)
    res = {"J": out["J"][0], "k": int(out["k"][0]), "k_qr": int(out["k_qr"][0]), "C": out["C"][0],
           "e2": float(out["e2"][0]), "a2": float(out["a2"][0])}
    if want_y:
        res["Y"] = out["Y"][0]
    return res


# ---------------------------------------------------------------------------
# Subsampled ID / single-pass ID on a coarse grid (Section 2, Algorithms 2-3).
# box = (nq, ez, ey, ex), stride = (sz, sy, sx); rows r = ((q ez + z) ey + y) ex + x.
# ---------------------------------------------------------------------------
def _box(box, stride):
    return (np.ascontiguousarray(box, dtype=np.int32).reshape(4),
            np.ascontiguousarray(stride, dtype=np.int32).reshape(3))


def coarse_axis(e: int, s: int) -> np.ndarray:
    """Coarse indices of an axis of e points with interval s (end point kept)."""
    lib = _load()
    cnt = int(lib.orc_coarse_axis(int(e), int(s), None))
    out = np.zeros(max(cnt, 1), dtype=np.int32)
    lib.orc_coarse_axis(int(e), int(s), out.ctypes.data)
    return out[:cnt]


def coarse_rows(box, stride) -> int:
    b, st = _box(box, stride)
    return int(_load().orc_coarse_rows(b, st))


def subsample(A: np.ndarray, box, stride) -> np.ndarray:
    """B = A(J, :) (mc x n) for an m x n matrix of one box."""
    b, st = _box(box, stride)
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    mc = coarse_rows(b, st)
    Af = np.ascontiguousarray(A.T).reshape(-1)
    out = np.zeros(mc * max(n, 1), dtype=np.float64)
    _load().orc_subsample(Af, m, n, b, st, out)
    return out[:mc * n].reshape(n, mc).T.copy()


def trilinear(G: np.ndarray, box, stride) -> np.ndarray:
    """F = M G: trilinear interpolation of a coarse mc x n matrix onto the box."""
    b, st = _box(box, stride)
    G = np.asarray(G, dtype=np.float64)
    mc, n = G.shape
    m = int(np.prod(b))
    Gf = np.ascontiguousarray(G.T).reshape(-1)
    F = np.zeros(m * max(n, 1), dtype=np.float64)
    _load().orc_trilinear(Gf, n, b, st, F, m)
    return F[:m * n].reshape(n, m).T.copy()


def subid(A: np.ndarray, box, stride, kmax: int, tol: float = 0.0, u_mode: float = 2.0 ** -53,
          want_ahat: bool = False) -> dict:
    """SubID / SPID on one box: J, k, C (k x n), Bskel (mc x k), and the squared
    errors of A(:,I_B) C_B (SubID) and M B(:,I_B) C_B (SPID)."""
    b, st = _box(box, stride)
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    assert m == int(np.prod(b))
    mc = coarse_rows(b, st)
    Af = np.ascontiguousarray(A.T).reshape(-1)
    J = np.zeros(kmax, dtype=np.int32)
    C = np.zeros(kmax * max(n, 1), dtype=np.float64)
    Bs = np.zeros(mc * kmax, dtype=np.float64)
    err = np.zeros(4, dtype=np.float64)
    H = np.zeros(m * max(n, 1), dtype=np.float64) if want_ahat else None
    k = int(_load().orc_subid(Af, m, n, b, st, kmax, float(tol), float(u_mode), J, C,
                              Bs.ctypes.data, err, H.ctypes.data if want_ahat else None))
    out = {"k": k, "J": J[:k].copy(), "J_full": J, "C": C[:kmax * n].reshape(kmax, n)[:k].copy(),
           "Bskel": Bs.reshape(kmax, mc).T[:, :k].copy(), "e2_subid": float(err[0]),
           "e2_spid": float(err[1]), "a2": float(err[2]), "mc": int(err[3])}
    if want_ahat:
        out["Ahat_spid"] = H[:m * n].reshape(n, m).T.copy()
    return out


def subid_points(A: np.ndarray, coarse_rows, interp_idx, interp_w, kmax: int, tol: float = 0.0,
                 u_mode: float = 2.0 ** -53, want_ahat: bool = False) -> dict:
    """SubID / SPID on a point set: B = A(coarse_rows, :); M given as a stencil
    (interp_idx, interp_w: m x t).  Same outputs as subid()."""
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    crow = np.ascontiguousarray(coarse_rows, dtype=np.int32)
    mc = int(crow.size)
    idx = np.ascontiguousarray(interp_idx, dtype=np.int32).reshape(m, -1)
    t = int(idx.shape[1])
    w = np.ascontiguousarray(interp_w, dtype=np.float64).reshape(m, t)
    Af = np.ascontiguousarray(A.T).reshape(-1)
    J = np.zeros(kmax, dtype=np.int32)
    C = np.zeros(kmax * max(n, 1), dtype=np.float64)
    Bs = np.zeros(mc * kmax, dtype=np.float64)
    err = np.zeros(4, dtype=np.float64)
    H = np.zeros(m * max(n, 1), dtype=np.float64) if want_ahat else None
    k = int(_load().orc_subid_points(Af, m, m, n, crow, mc, t, idx.reshape(-1), w.reshape(-1),
                                     kmax, float(tol), float(u_mode), J, C, Bs.ctypes.data, err,
                                     H.ctypes.data if want_ahat else None))
    out = {"k": k, "J": J[:k].copy(), "J_full": J, "C": C[:kmax * n].reshape(kmax, n)[:k].copy(),
           "Bskel": Bs.reshape(kmax, mc).T[:, :k].copy(), "e2_subid": float(err[0]),
           "e2_spid": float(err[1]), "a2": float(err[2]), "mc": int(err[3])}
    if want_ahat:
        out["Ahat_spid"] = H[:m * n].reshape(n, m).T.copy()
    return out


# ---------------------------------------------------------------------------
# Modified (two-stage) SPID, Section 3.3.2 / Algorithm 6.
# ---------------------------------------------------------------------------
def two_stage(A: np.ndarray, N: int, k: int, p: int, k2max: int, tol2: float, u_mode: float,
              seed: int) -> dict:
    """Stage-1 IDs of N column blocks (rank k), stage-2 ID of their skeletons
    (tolerance tol2), composed into A ~ A(:, J) C."""
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    assert n % N == 0
    nb = n // N
    Af = np.ascontiguousarray(A.T).reshape(-1)
    J = np.zeros(k2max, dtype=np.int32)
    C = np.zeros(k2max * n, dtype=np.float64)
    Jb = np.zeros(N * k, dtype=np.int32)
    kb = np.zeros(N, dtype=np.int32)
    Cb = np.zeros(N * k * nb, dtype=np.float64)
    J2 = np.zeros(k2max, dtype=np.int32)
    C1 = np.zeros(k2max * N * k, dtype=np.float64)
    err = np.zeros(2, dtype=np.float64)
    k2 = int(_load().orc_two_stage(Af, m, n, m, N, k, p, k2max, float(tol2), float(u_mode),
                                   int(seed), J, C, Jb, kb, Cb, J2, C1, err))
    return {"k": k2, "J": J[:k2].copy(), "C": C.reshape(k2max, n)[:k2].copy(),
            "Jb": Jb.reshape(N, k), "kb": kb, "Cb": Cb.reshape(N, k, nb), "J2": J2[:k2].copy(),
            "C1": C1.reshape(k2max, N * k)[:k2].copy(), "e2": float(err[0]), "a2": float(err[1])}
