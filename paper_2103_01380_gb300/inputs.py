"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds data synthesis only: flow fields, spectra and layouts.  It
contains none of the decomposition's arithmetic and is the one module that the
CUDA path's tests and the CPU oracle's tests share.

Fields follow the paper's Taylor-Green vortex cases:
  * 2D analytic TGV, Section 5.1:
      u1 = sin(x1) cos(x2) exp(-2 nu t),  u2 = -cos(x1) sin(x2) exp(-2 nu t);
  * 3D TGV initial condition of Section 5.2 (V0 = 1, L = 1, rho0 = 1,
    p0 = 100), decayed as exp(-3 nu t), plus solenoidal Fourier modes with a
    k^{-5/3} amplitude spectrum, each decaying as exp(-nu |k|^2 t) with a
    drifting phase; density and pressure from rho = 1 + 0.01 |u|^2 and the
    isentropic relation p = p0 (rho / rho0)^gamma, gamma = 1.4.

Window layout ("blocks"): subdomain s is an m_s x n_s column-major matrix
(column = snapshot) starting at element ``off[s]`` of one flat buffer with
leading dimension ``ld[s]``.  Row order inside a 3D box is
r = ((q * ez + z) * ey + y) * ex + x (x fastest, QoI slowest).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Window:
    """A flat window plus its per-subdomain block descriptors."""
    data: np.ndarray            # 1-D, float32 or float64
    m: np.ndarray               # int64 [S]
    n: np.ndarray               # int64 [S]
    off: np.ndarray             # int64 [S]
    ld: np.ndarray              # int64 [S]
    meta: dict = field(default_factory=dict)

    @property
    def num_sub(self) -> int:
        return int(len(self.m))

    def block(self, s: int) -> np.ndarray:
        """View of subdomain s as an m_s x n_s array (column j = snapshot j)."""
        m, n, off, ld = int(self.m[s]), int(self.n[s]), int(self.off[s]), int(self.ld[s])
        cols = np.lib.stride_tricks.as_strided(
            self.data[off:], shape=(n, m),
            strides=(ld * self.data.itemsize, self.data.itemsize))
        return cols.T

    def nbytes_payload(self) -> int:
        return int((self.m * self.n).sum()) * self.data.itemsize


def pack_blocks(blocks, dtype=np.float32, layout: str = "subdomain", pad_to: int = 4) -> Window:
    """Pack a list of m_s x n_s arrays into one flat window.

    layout "subdomain": [s][j][r] (each subdomain contiguous, ld = m_s rounded
    up to ``pad_to`` elements so every column starts 16-byte aligned).
    layout "snapshot": [j][s][r] (each snapshot contiguous; all n_s equal;
    ld = sum of padded m_s)."""
    S = len(blocks)
    m = np.array([b.shape[0] for b in blocks], dtype=np.int64)
    n = np.array([b.shape[1] for b in blocks], dtype=np.int64)
    mp = ((m + pad_to - 1) // pad_to) * pad_to
    if layout == "subdomain":
        ld = mp.copy()
        off = np.concatenate([[0], np.cumsum(mp * n)[:-1]]).astype(np.int64)
        total = int((mp * n).sum())
    elif layout == "snapshot":
        if len(set(n.tolist())) != 1:
            raise ValueError("snapshot layout needs equal window lengths")
        ld = np.full(S, int(mp.sum()), dtype=np.int64)
        off = np.concatenate([[0], np.cumsum(mp)[:-1]]).astype(np.int64)
        total = int(mp.sum()) * int(n[0])
    else:
        raise ValueError(layout)
    data = np.zeros(total, dtype=dtype)
    w = Window(data, m, n, off, ld, {"layout": layout})
    for s, b in enumerate(blocks):
        w.block(s)[...] = b
    return w


# --------------------------------------------------------------------------
# 2D analytic Taylor-Green vortex (Section 5.1)
# --------------------------------------------------------------------------
def tgv2d(nx: int = 64, n: int = 128, nu: float = 0.01, t_end: float = 10.0,
          noise: float = 1e-6, seed: int = 1) -> np.ndarray:
    """A (2 nx^2 x n), rows = u1 then u2 on an nx x nx grid over [0, 2pi)^2
    (x1 fastest), columns = snapshots at t_j = t_end j / (n - 1), plus i.i.d.
    N(0, noise^2) entries drawn from PCG64(seed)."""
    x = 2.0 * np.pi * np.arange(nx) / nx
    X1, X2 = np.meshgrid(x, x, indexing="xy")      # X1[b, a] = x_a
    t = t_end * np.arange(n) / max(n - 1, 1)
    g = np.exp(-2.0 * nu * t)
    u1 = (np.sin(X1) * np.cos(X2)).reshape(-1)
    u2 = (-np.cos(X1) * np.sin(X2)).reshape(-1)
    A = np.concatenate([u1, u2])[:, None] * g[None, :]
    if noise > 0:
        A = A + noise * np.random.default_rng(seed).standard_normal(A.shape)
    return A


# --------------------------------------------------------------------------
# 3D TGV-like field with Fourier modes (Section 5.2 initial condition)
# --------------------------------------------------------------------------
@dataclass
class FourierModes:
    kvec: np.ndarray     # [K, 3] integer wavevectors
    amp: np.ndarray      # [K]
    dirn: np.ndarray     # [K, 3] unit vectors orthogonal to kvec
    phase: np.ndarray    # [K]
    omega: np.ndarray    # [K]


def fourier_modes(count: int = 32, kmax: int = 8, eps_f: float = 0.05, seed: int = 2,
                  omega_range: float = 0.5) -> FourierModes:
    rng = np.random.default_rng(seed)
    ks = []
    while len(ks) < count:
        kv = rng.integers(-kmax, kmax + 1, size=3)
        if np.any(kv != 0):
            ks.append(kv)
    kvec = np.array(ks, dtype=np.float64)
    kn = np.linalg.norm(kvec, axis=1)
    spec = kn ** (-5.0 / 3.0)
    amp = eps_f * spec / spec.max()
    dirn = np.empty_like(kvec)
    for i in range(count):
        r = rng.standard_normal(3)
        r -= kvec[i] * (r @ kvec[i]) / (kvec[i] @ kvec[i])
        dirn[i] = r / np.linalg.norm(r)
    phase = rng.uniform(0.0, 2.0 * np.pi, size=count)
    omega = rng.uniform(-omega_range, omega_range, size=count)
    return FourierModes(kvec, amp, dirn, phase, omega)


def tgv3d_box(org, ext, grid: int, t: np.ndarray, modes: FourierModes, nu: float = 0.01,
              p0: float = 100.0, gamma: float = 1.4, dtype=np.float32) -> np.ndarray:
    """One box of the 3D field: (5 * ex * ey * ez) x len(t), QoIs (rho,u,v,w,p).

    The box covers grid points org + [0, ext) of a periodic grid^3 grid over
    [0, 2pi)^3 (indices wrap).  Velocity = TGV * exp(-3 nu t) + sum of modes;
    each mode is a_k d_k exp(-nu |k|^2 t) cos(k.x + phi_k + omega_k t)."""
    ex, ey, ez = (int(e) for e in ext)
    h = 2.0 * np.pi / grid
    xs = h * ((org[0] + np.arange(ex)) % grid)
    ys = h * ((org[1] + np.arange(ey)) % grid)
    zs = h * ((org[2] + np.arange(ez)) % grid)
    Z, Yg, X = np.meshgrid(zs, ys, xs, indexing="ij")         # [z][y][x]
    X, Yg, Z = X.reshape(-1), Yg.reshape(-1), Z.reshape(-1)
    npts = X.size
    K = modes.kvec.shape[0]
    # spatial basis: [TGV, cos(k.x + phi), sin(k.x + phi)] -> npts x (1 + 2K)
    arg = np.outer(X, modes.kvec[:, 0]) + np.outer(Yg, modes.kvec[:, 1]) \
        + np.outer(Z, modes.kvec[:, 2]) + modes.phase[None, :]
    cosb, sinb = np.cos(arg), np.sin(arg)
    decay = np.exp(-nu * (modes.kvec ** 2).sum(1)[:, None] * t[None, :])   # K x n
    tc = modes.amp[:, None] * decay * np.cos(np.outer(modes.omega, t))
    ts = modes.amp[:, None] * decay * np.sin(np.outer(modes.omega, t))
    g = np.exp(-3.0 * nu * t)
    tgv = [np.sin(X) * np.cos(Yg) * np.cos(Z), -np.cos(X) * np.sin(Yg) * np.cos(Z),
           np.zeros(npts)]
    vel = []
    for c in range(3):
        basis = np.concatenate([tgv[c][:, None], cosb * modes.dirn[None, :, c],
                                -sinb * modes.dirn[None, :, c]], axis=1)
        tf = np.concatenate([g[None, :], tc, ts], axis=0)
        vel.append(basis @ tf)
    speed2 = vel[0] ** 2 + vel[1] ** 2 + vel[2] ** 2
    rho = 1.0 + 0.01 * speed2
    p = p0 * rho ** gamma
    out = np.empty((5 * npts, t.size), dtype=dtype)
    for q, f in enumerate([rho, vel[0], vel[1], vel[2], p]):
        out[q * npts:(q + 1) * npts] = f
    return out


def tgv3d_window(grid: int = 64, box: int = 16, n: int = 512, t_end: float = 10.0,
                 nu: float = 0.01, modes: FourierModes | None = None, seed: int = 2,
                 dtype=np.float32, layout: str = "subdomain", boxes=None) -> Window:
    """Equal cubic boxes of edge ``box`` tiling a grid^3 periodic grid (or the
    first ``boxes`` of them), QoIs (rho,u,v,w,p), n snapshots on [0, t_end]."""
    if modes is None:
        modes = fourier_modes(seed=seed)
    nb = grid // box
    t = t_end * np.arange(n) / max(n - 1, 1)
    origins = [(bx * box, by * box, bz * box) for bz in range(nb) for by in range(nb)
               for bx in range(nb)]
    if boxes is not None:
        origins = origins[:boxes]
    m = 5 * box ** 3
    S = len(origins)
    if layout == "subdomain":
        data = np.empty(S * m * n, dtype=dtype)
        for s, o in enumerate(origins):
            data[s * m * n:(s + 1) * m * n] = tgv3d_box(o, (box,) * 3, grid, t, modes, nu,
                                                        dtype=np.float64).T.reshape(-1)
        w = Window(data, np.full(S, m, np.int64), np.full(S, n, np.int64),
                   (np.arange(S, dtype=np.int64) * m * n), np.full(S, m, np.int64),
                   {"layout": layout})
    else:
        blocks = [tgv3d_box(o, (box,) * 3, grid, t, modes, nu, dtype=np.float64)
                  for o in origins]
        w = pack_blocks(blocks, dtype=dtype, layout=layout)
    w.meta.update({"grid": grid, "box": box, "t_end": t_end, "nu": nu, "origins": origins})
    return w


def tgv3d_global(X: int, Y: int, Z: int, grid: int, t: np.ndarray,
                 modes: FourierModes | None = None, seed: int = 2, nu: float = 0.01,
                 dtype=np.float32, snap_stride: int | None = None) -> np.ndarray:
    """The 3D field on the points [0, X) x [0, Y) x [0, Z) of a periodic grid^3
    grid, laid out as a solver holds it: a flat [t][q][Z][Y][X] window (QoIs
    rho, u, v, w, p), snapshot t at element t * snap_stride (default 5 X Y Z;
    padding between snapshots stays zero)."""
    if modes is None:
        modes = fourier_modes(seed=seed)
    F = tgv3d_box((0, 0, 0), (X, Y, Z), grid, t, modes, nu, dtype=np.float64)  # [(q,z,y,x), t]
    field = 5 * X * Y * Z
    ss = field if snap_stride is None else int(snap_stride)
    out = np.zeros(ss * len(t), dtype=dtype)
    out.reshape(len(t), ss)[:, :field] = F.T
    return out


def cut_box(window: np.ndarray, nq: int, X: int, Y: int, Z: int, n: int, org, ext,
            q: int | None = None, snap_stride: int | None = None) -> np.ndarray:
    """Data matrix of the box org + [0, ext) ((x, y, z) order) of a flat
    [t][q][Z][Y][X] window: rows ((q ez + z) ey + y) ex + x with every QoI
    stacked (QoI slowest), or only QoI q's rows (z ey + y) ex + x; columns are
    the n snapshots.  A layout copy only."""
    ss = nq * X * Y * Z if snap_stride is None else int(snap_stride)
    f = window[:ss * n].reshape(n, ss)[:, :nq * X * Y * Z].reshape(n, nq, Z, Y, X)
    ox, oy, oz = (int(v) for v in org)
    ex, ey, ez = (int(v) for v in ext)
    b = f[:, :, oz:oz + ez, oy:oy + ey, ox:ox + ex]
    if q is not None:
        b = b[:, q]
    return np.ascontiguousarray(b.reshape(n, -1).T)


def uneven_boxes(count: int, edges=(8, 12, 16, 24, 32), n_range=(64, 1024), grid: int = 256,
                 t_end: float = 10.0, nu: float = 0.01, seed: int = 4,
                 modes: FourierModes | None = None):
    """Descriptors of `count` cubic boxes with uniformly drawn edges and window
    lengths, each at a uniformly random periodic offset of a grid^3 field:
    list of (origin, edge, n)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        e = int(rng.choice(edges))
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        org = tuple(int(x) for x in rng.integers(0, grid, size=3))
        out.append((org, e, n))
    return out


def uneven_window(boxes, grid: int = 256, t_end: float = 10.0, nu: float = 0.01,
                  modes: FourierModes | None = None, seed: int = 2, dtype=np.float32) -> Window:
    """Window of the boxes described by `uneven_boxes` (subdomain-major); each
    box's snapshots sample t in [0, t_end] at its own n points."""
    if modes is None:
        modes = fourier_modes(seed=seed)
    blocks = []
    for org, e, n in boxes:
        t = t_end * np.arange(n) / max(n - 1, 1)
        blocks.append(tgv3d_box(org, (e, e, e), grid, t, modes, nu, dtype=np.float64))
    w = pack_blocks(blocks, dtype=dtype)
    w.meta.update({"grid": grid, "boxes": boxes})
    return w


# --------------------------------------------------------------------------
# The same 3D field generated on the GPU (torch), for windows too large to
# build on the host.  FP32 arithmetic; every Fourier phase k . x is reduced
# exactly in integers (k and the grid indices are integers) before the
# trigonometric call, so values agree with the FP64 host generator to ~1e-6.
# --------------------------------------------------------------------------
class DeviceField:
    """Spatial basis of the TGV + Fourier field over a set of cubic boxes of a
    grid^3 periodic grid, held on the GPU; `snapshots` evaluates it at any
    batch of times.  Point order: box-major, then (z, y, x) inside the box."""

    def __init__(self, origins, edge: int, grid: int, modes: FourierModes, nu: float = 0.01,
                 device="cuda"):
        import torch
        self.torch = torch
        self.device = device
        self.edge, self.grid, self.nu, self.modes = edge, grid, nu, modes
        self.S = len(origins)
        self.npts = edge ** 3
        e = torch.arange(edge, device=device, dtype=torch.int64)
        zl, yl, xl = torch.meshgrid(e, e, e, indexing="ij")
        org = torch.tensor(origins, device=device, dtype=torch.int64)            # [S, 3] (x, y, z)
        ix = (org[:, 0, None] + xl.reshape(1, -1)) % grid                          # [S, npts]
        iy = (org[:, 1, None] + yl.reshape(1, -1)) % grid
        iz = (org[:, 2, None] + zl.reshape(1, -1)) % grid
        h = 2.0 * np.pi / grid
        x, y, z = (ix.reshape(-1).float() * h, iy.reshape(-1).float() * h, iz.reshape(-1).float() * h)
        self.tgv = torch.stack([torch.sin(x) * torch.cos(y) * torch.cos(z),
                                -torch.cos(x) * torch.sin(y) * torch.cos(z),
                                torch.zeros_like(x)], dim=1)                      # [P, 3]
        kv = torch.tensor(modes.kvec, device=device, dtype=torch.int64)            # [K, 3]
        ph = (ix.reshape(-1, 1) * kv[None, :, 0] + iy.reshape(-1, 1) * kv[None, :, 1]
              + iz.reshape(-1, 1) * kv[None, :, 2]) % grid                         # exact, [P, K]
        theta = ph.float() * h + torch.tensor(modes.phase, device=device, dtype=torch.float32)
        self.cos = torch.cos(theta)
        self.sin = torch.sin(theta)
        self.dirn = torch.tensor(modes.dirn, device=device, dtype=torch.float32)   # [K, 3]

    def snapshots(self, t: np.ndarray, p0: float = 100.0, gamma: float = 1.4):
        """Field at times t: [5, P, len(t)] (QoIs rho, u, v, w, p), FP32."""
        torch = self.torch
        md = self.modes
        decay = np.exp(-self.nu * (md.kvec ** 2).sum(1)[:, None] * t[None, :])
        tc = torch.tensor(md.amp[:, None] * decay * np.cos(np.outer(md.omega, t)),
                          device=self.device, dtype=torch.float32)                 # [K, b]
        ts = torch.tensor(md.amp[:, None] * decay * np.sin(np.outer(md.omega, t)),
                          device=self.device, dtype=torch.float32)
        g = torch.tensor(np.exp(-3.0 * self.nu * t), device=self.device, dtype=torch.float32)
        out = torch.empty((5, self.S * self.npts, len(t)), device=self.device, dtype=torch.float32)
        for c in range(3):
            d = self.dirn[:, c:c + 1]
            out[1 + c] = (self.tgv[:, c:c + 1] * g[None, :] + self.cos @ (d * tc)
                          - self.sin @ (d * ts))
        speed2 = out[1] ** 2 + out[2] ** 2 + out[3] ** 2
        out[0] = 1.0 + 0.01 * speed2
        out[4] = p0 * out[0] ** gamma
        return out

    def fill_subdomain_major(self, window, t: np.ndarray, j0: int, n_total: int):
        """Write snapshots j0 .. j0 + len(t) of every box into a subdomain-major
        window [S][n_total][5 * npts] (rows of a box in (q, z, y, x) order)."""
        b = len(t)
        f = self.snapshots(t)                                           # [5, S*P, b]
        w = window.view(self.S, n_total, 5, self.npts)
        w[:, j0:j0 + b] = f.view(5, self.S, self.npts, b).permute(1, 3, 0, 2)

    def fill_snapshot_major(self, window, t: np.ndarray, j0: int, n_total: int):
        """Write snapshots j0 .. j0 + len(t) of every box into a snapshot-major
        window [n_total][S][5 * npts] (rows of a box in (q, z, y, x) order)."""
        b = len(t)
        f = self.snapshots(t)                                           # [5, S*P, b]
        w = window.view(n_total, self.S, 5, self.npts)
        w[j0:j0 + b] = f.view(5, self.S, self.npts, b).permute(3, 1, 0, 2)


# --------------------------------------------------------------------------
# Prescribed-spectrum matrices (Haar-orthonormal factors)
# --------------------------------------------------------------------------
def haar(rows: int, cols: int, rng: np.random.Generator) -> np.ndarray:
    """rows x cols matrix with Haar-distributed orthonormal columns (QR of a
    Gaussian with the sign of diag(R) fixed positive)."""
    G = rng.standard_normal((rows, cols))
    Q, R = np.linalg.qr(G)
    return Q * np.sign(np.diag(R))[None, :]


def spectrum_matrix(m: int, n: int, sigma, seed: int) -> np.ndarray:
    """A = U diag(sigma) V^T, U (m x r) and V (n x r) Haar, r = len(sigma)."""
    sigma = np.asarray(sigma, dtype=np.float64)
    rng = np.random.default_rng(seed)
    U = haar(m, sigma.size, rng)
    V = haar(n, sigma.size, rng)
    return (U * sigma[None, :]) @ V.T


def lowrank(m: int, n: int, r: int, seed: int) -> np.ndarray:
    """Exactly rank-r Gaussian product G1 G2^T (FP64)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((m, r)) @ rng.standard_normal((r, n))


def separated_lowrank(m: int, n: int, r: int, seed: int, decay: float = 0.5,
                      noise: float = 0.0) -> np.ndarray:
    """Rank-r signal with geometrically decaying singular values plus optional
    i.i.d. noise: pivots of its sketch are well separated for small r."""
    sig = decay ** np.arange(r)
    A = spectrum_matrix(m, n, sig, seed)
    if noise > 0:
        A = A + noise * np.random.default_rng(seed + 7919).standard_normal((m, n))
    return A


def separated_columns(m: int, n: int, r: int, seed: int, ratio: float = 0.35,
                      mix: float = 0.02, noise: float = 0.0) -> np.ndarray:
    """Rank-r data whose leading columns are decided with a wide margin: column
    j < r is a random unit direction times ratio^j (nearly orthogonal for
    m >> r), every other column a random combination of those r with weights
    of size `mix`, plus optional i.i.d. noise.  A column-pivoted QR of it (or of
    a Gaussian sketch of it) picks columns 0, 1, ..., r - 1 in order, each
    residual norm about 1 / ratio times the next, so the pivots stay
    identifiable even under the ~2^-11 roundings of a TF32 sketch."""
    rng = np.random.default_rng(seed)
    D = rng.standard_normal((m, r))
    D /= np.linalg.norm(D, axis=0, keepdims=True)
    D *= ratio ** np.arange(r)[None, :]
    W = mix * rng.standard_normal((r, n - r))
    A = np.concatenate([D, D @ W], axis=1)
    if noise > 0:
        A = A + noise * rng.standard_normal((m, n))
    return A


def smooth_box_field(box, n: int, seed: int, modes: int = 6, kmax: int = 2,
                     noise: float = 0.0) -> np.ndarray:
    """m x n field of one box (nq, ez, ey, ex), rows in (q, z, y, x) order:
    per QoI a sum of `modes` separable sine/cosine products of wavenumbers
    1..kmax over the box, mode i with amplitude 2^-i and its own time signal,
    plus optional i.i.d. noise.  Smooth in space, so a coarse grid sees it."""
    nq, ez, ey, ex = (int(v) for v in box)
    rng = np.random.default_rng(seed)
    z, y, x = np.meshgrid(np.arange(ez) / ez, np.arange(ey) / ey, np.arange(ex) / ex,
                          indexing="ij")
    t = np.linspace(0.0, 1.0, n)
    A = np.zeros((nq, ez, ey, ex, n))
    for q in range(nq):
        for i in range(modes):
            kx, ky, kz = rng.integers(1, kmax + 1, size=3)
            ph = rng.uniform(0.0, 2.0 * np.pi, 3)
            sp = (np.sin(2 * np.pi * kx * x + ph[0]) * np.cos(2 * np.pi * ky * y + ph[1]) *
                  np.sin(2 * np.pi * kz * z + ph[2]))
            amp = 0.5 ** i * np.cos(2 * np.pi * (i + 1) * t + rng.uniform(0.0, 6.0))
            A[q] += sp[..., None] * amp
    A = A.reshape(-1, n)
    if noise > 0:
        A = A + noise * rng.standard_normal(A.shape)
    return A


def box_window(boxes, n, seed: int, dtype=np.float32, noise: float = 0.0, **kw) -> "Window":
    """Window of smooth_box_field blocks, one per box (nq, ez, ey, ex); n is a
    common length or one per box."""
    ns = np.broadcast_to(np.atleast_1d(n), (len(boxes),))
    blocks = [smooth_box_field(b, int(ns[i]), seed + i, noise=noise, **kw)
              for i, b in enumerate(boxes)]
    w = pack_blocks(blocks, dtype=dtype)
    w.meta["boxes"] = np.asarray(boxes, dtype=np.int32).reshape(-1, 4)
    return w


def tgv3d_u1(grid: int, t: np.ndarray, nu: float = 0.01, dtype=np.float32) -> np.ndarray:
    """u1 of the 3D TGV alone (Section 5.2 initial condition, no Fourier modes)
    on the whole grid^3 box: sin x cos y cos z exp(-3 nu t), rows (z, y, x)."""
    h = 2.0 * np.pi / grid
    c = np.arange(grid) * h
    Z, Yg, X = np.meshgrid(c, c, c, indexing="ij")
    space = (np.sin(X) * np.cos(Yg) * np.cos(Z)).reshape(-1)
    return np.outer(space, np.exp(-3.0 * nu * np.asarray(t))).astype(dtype)


# ---------------------------------------------------------------------------
# Unstructured point sets (Section 5.1 runs the ID on randomly generated
# points of the 2D TGV domain; rows of A follow the points in random order).
# The coarse subset and the interpolation stencil are inputs of the coarse-grid
# ID (the paper leaves the choice of M to the user).
# ---------------------------------------------------------------------------
def unstructured_tgv2d(npts: int, n: int, seed: int, nu: float = 0.01, t_end: float = 10.0,
                       noise: float = 0.0, qois=("u1", "u2"), smooth_modes: int = 0):
    """npts uniformly random points of [0, 2 pi)^2 (rows in random order) and
    the 2D TGV fields at them over n snapshots on [0, t_end]: returns (pts
    [npts, 2], A [len(qois) npts, n], rows QoI-major).  smooth_modes > 0 adds
    that many smooth random space-time modes of amplitude 0.1 2^-i (rank
    above one, still smooth for interpolation)."""
    rng = np.random.default_rng(seed)
    pts = rng.uniform(0.0, 2.0 * np.pi, size=(npts, 2))
    t = t_end * np.arange(n) / max(n - 1, 1)
    x1, x2 = pts[:, 0], pts[:, 1]
    g = np.exp(-2.0 * nu * t)
    fields = {"u1": np.outer(np.sin(x1) * np.cos(x2), g),
              "u2": np.outer(-np.cos(x1) * np.sin(x2), g)}
    A = np.concatenate([fields[q] for q in qois], axis=0)
    for i in range(smooth_modes):
        kx, ky = rng.integers(1, 3, size=2)
        ph = rng.uniform(0.0, 2.0 * np.pi, 3)
        sp = np.sin(kx * x1 + ph[0]) * np.cos(ky * x2 + ph[1])
        tm = 0.1 * 0.5 ** i * np.cos((i + 1) * 2.0 * np.pi * t / t_end + ph[2])
        A = A + np.outer(np.tile(sp, len(qois)), tm)
    if noise > 0:
        A = A + noise * rng.standard_normal(A.shape)
    return pts, A


def point_partitions(pts: np.ndarray, nbx: int, nby: int):
    """Indices of the points in each of nbx x nby equal blocks of [0, 2 pi)^2
    (block-row-major), each list in the points' own (random) order."""
    bx = np.minimum((pts[:, 0] / (2.0 * np.pi) * nbx).astype(int), nbx - 1)
    by = np.minimum((pts[:, 1] / (2.0 * np.pi) * nby).astype(int), nby - 1)
    return [np.nonzero((by == j) & (bx == i))[0] for j in range(nby) for i in range(nbx)]


def coarse_stencil(pts: np.ndarray, mc: int, t: int, seed: int, nq: int = 1,
                   method: str = "linear"):
    """Coarse subset and interpolation stencil of one subdomain's points (np
    points, rows QoI-major over nq QoIs): mc random coarse points per QoI
    (coarse rows listed QoI-major), and per fine row t coarse points of the same
    QoI with weights summing to one.  method "linear": barycentric weights in
    the Delaunay triangle of the coarse points that holds the point (t = 3;
    exact for fields linear in space), falling back to "idw" outside their
    hull; "idw": the t nearest coarse points with inverse-square-distance
    weights.  A coarse point takes weight one on itself.  Returns (coarse_rows
    [nq mc], idx [nq np, t], w [nq np, t])."""
    from scipy.spatial import Delaunay, cKDTree
    rng = np.random.default_rng(seed)
    npt = pts.shape[0]
    cpos = np.sort(rng.choice(npt, size=mc, replace=False))
    cp = pts[cpos]
    tree = cKDTree(cp)
    tt = min(t, mc)
    d, nb = tree.query(pts, k=tt)
    d = np.asarray(d, dtype=np.float64).reshape(npt, tt)
    nb = np.asarray(nb, dtype=np.int64).reshape(npt, tt)
    w = np.zeros((npt, t))
    idx = np.zeros((npt, t), dtype=np.int32)
    inv = np.where(d > 0.0, 1.0 / np.where(d > 0.0, d, 1.0) ** 2, 0.0)
    tot = inv.sum(axis=1, keepdims=True)
    w[:, :tt] = inv / np.where(tot > 0.0, tot, 1.0)
    idx[:, :tt] = nb
    if method == "linear" and t >= 3 and mc >= 4:
        tri = Delaunay(cp)
        simp = tri.find_simplex(pts)
        inside = simp >= 0
        T = tri.transform[simp[inside]]                    # [k, 3, 2]
        b = np.einsum("kij,kj->ki", T[:, :2, :], pts[inside] - T[:, 2, :])
        bary = np.concatenate([b, 1.0 - b.sum(axis=1, keepdims=True)], axis=1)
        w[inside] = 0.0
        w[inside, :3] = bary
        idx[inside] = 0
        idx[inside, :3] = tri.simplices[simp[inside]]
    exact = d[:, 0] == 0.0
    w[exact] = 0.0
    w[exact, 0] = 1.0
    idx[exact, 0] = nb[exact, 0]
    rows = np.concatenate([q * npt + cpos for q in range(nq)]).astype(np.int32)
    idx_all = np.concatenate([idx + q * mc for q in range(nq)]).astype(np.int32)
    w_all = np.concatenate([w] * nq)
    return rows, idx_all, w_all


def tgv2d_points_window_device(pts: np.ndarray, parts, n: int, seed: int, nu: float = 0.01,
                               t_end: float = 10.0, smooth_modes: int = 4, device="cuda"):
    """Subdomain-major FP32 window on the GPU of the 2D TGV (u1, u2) plus
    `smooth_modes` smooth space-time modes (as unstructured_tgv2d) at the
    points of each partition: block s holds rows (q, point of parts[s]), ld =
    rows rounded up to 4.  Returns (window tensor, m, n, off, ld)."""
    import torch
    rng = np.random.default_rng(seed)
    t = t_end * np.arange(n) / max(n - 1, 1)
    g = torch.tensor(np.exp(-2.0 * nu * t), device=device, dtype=torch.float32)
    modes = []
    for i in range(smooth_modes):
        kx, ky = rng.integers(1, 3, size=2)
        ph = rng.uniform(0.0, 2.0 * np.pi, 3)
        tm = 0.1 * 0.5 ** i * np.cos((i + 1) * 2.0 * np.pi * t / t_end + ph[2])
        modes.append((int(kx), int(ky), ph, torch.tensor(tm, device=device, dtype=torch.float32)))
    m = np.array([2 * len(p) for p in parts], dtype=np.int64)
    ld = (m + 3) // 4 * 4
    off = np.concatenate([[0], np.cumsum(ld * n)[:-1]]).astype(np.int64)
    win = torch.zeros(int((ld * n).sum()), device=device, dtype=torch.float32)
    P = torch.tensor(pts, device=device, dtype=torch.float64)
    for s, part in enumerate(parts):
        idx = torch.tensor(part, device=device, dtype=torch.int64)
        x1, x2 = P[idx, 0], P[idx, 1]
        sp = torch.stack([torch.sin(x1) * torch.cos(x2), -torch.cos(x1) * torch.sin(x2)])   # [2, np]
        blk = (sp.reshape(-1, 1).float() * g[None, :])
        for kx, ky, ph, tm in modes:
            mode = (torch.sin(kx * x1 + ph[0]) * torch.cos(ky * x2 + ph[1])).float()
            blk = blk + torch.cat([mode, mode]).reshape(-1, 1) * tm[None, :]
        view = win[int(off[s]):int(off[s] + ld[s] * n)].view(n, int(ld[s]))
        view[:, :int(m[s])] = blk.T
    return win, m, np.full(len(parts), n, dtype=np.int64), off, ld
