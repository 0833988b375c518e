"""Python binding of libspid (include/spid.h).

Argument marshalling only: every step of the decomposition runs in the CUDA
kernels behind the C ABI.  Device buffers are torch CUDA tensors (PyTorch is
used for device memory and streams); host results come back as numpy arrays.
There is no CPU fallback: if libspid.so is missing or cannot be loaded, every
entry point raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libspid.so")

SPID_OK = 0
STATUS_NAMES = {0: "SPID_OK", 1: "SPID_ERR_INVALID_ARG", 2: "SPID_ERR_CUDA", 3: "SPID_ERR_OOM",
                4: "SPID_ERR_STATE", 5: "SPID_ERR_TIMEOUT", 6: "SPID_ERR_NONFINITE",
                7: "SPID_ERR_UNSUPPORTED", 8: "SPID_ERR_RANK"}
SPID_ERR_RANK = 8
PREC = {"fp64": 0, "fp32": 1, "tf32": 2, "bf16": 3, "bf16x3": 4}
FLAG_PER_SUBDOMAIN = 1
FLAG_TC_ERROR = 2

# every symbol include/spid.h declares
EXPORTS = ["spid_plan_create", "spid_plan_destroy", "spid_plan_info", "spid_sketch_accumulate",
           "spid_reset",
           "spid_finalize", "spid_error", "spid_reconstruct", "spid_get_factors",
           "spid_get_sketch", "spid_device_status", "spid_omega", "spid_philox",
           "spid_compression_factor", "spid_status_string", "spid_last_error",
           "spid_sketch_fp32_noalloc",
           "spid_sub_plan_create", "spid_sub_plan_destroy", "spid_sub_plan_info",
           "spid_sub_sample", "spid_sub_finalize", "spid_sub_error", "spid_sub_reconstruct",
           "spid_sub_get_factors", "spid_sub_get_coarse", "spid_sub_device_status",
           "spid_ts_plan_create", "spid_ts_plan_destroy", "spid_ts_block", "spid_ts_finalize",
           "spid_ts_error", "spid_ts_reconstruct", "spid_ts_get_factors",
           "spid_ts_get_block_factors", "spid_ts_device_status",
           "spid_plan_get_tuning", "spid_plan_set_tuning", "spid_plan_autotune",
           "spid_plan_autotune_calls", "spid_plan_tuning_key", "spid_graph_create", "spid_graph_launch", "spid_graph_launch_host",
           "spid_graph_destroy",
           "spid_sub_plan_create_points", "spid_producer_step"]
GRAPH_SKETCH = 1
GRAPH_FINALIZE = 2
GRAPH_ERROR = 4
FORM_SPID = 0
FORM_SUBID = 1


class SpidError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)} {detail}".strip())


class _BoxLayout(ctypes.Structure):
    _fields_ = [("nq", ctypes.c_int32),
                ("X", ctypes.c_int64),
                ("Y", ctypes.c_int64),
                ("Z", ctypes.c_int64),
                ("snap_stride", ctypes.c_int64),
                ("num_box", ctypes.c_int32),
                ("org3", ctypes.POINTER(ctypes.c_int32)),
                ("ext3", ctypes.POINTER(ctypes.c_int32)),
                ("split_qoi", ctypes.c_int32)]


class _Desc(ctypes.Structure):
    _fields_ = [("num_sub", ctypes.c_int32),
                ("m", ctypes.POINTER(ctypes.c_int32)),
                ("n", ctypes.POINTER(ctypes.c_int32)),
                ("off", ctypes.POINTER(ctypes.c_int64)),
                ("ld", ctypes.POINTER(ctypes.c_int64)),
                ("k_max", ctypes.c_int32),
                ("p", ctypes.c_int32),
                ("tol", ctypes.c_double),
                ("precision", ctypes.c_int32),
                ("flags", ctypes.c_uint32),
                ("seed", ctypes.c_uint64),
                ("qoi", ctypes.POINTER(ctypes.c_int32)),
                ("num_qoi", ctypes.c_int32),
                ("boxes", ctypes.POINTER(_BoxLayout))]


class _SubDesc(ctypes.Structure):
    _fields_ = [("num_sub", ctypes.c_int32),
                ("box", ctypes.POINTER(ctypes.c_int32)),
                ("n", ctypes.POINTER(ctypes.c_int32)),
                ("off", ctypes.POINTER(ctypes.c_int64)),
                ("ld", ctypes.POINTER(ctypes.c_int64)),
                ("stride", ctypes.c_int32 * 3),
                ("k_max", ctypes.c_int32),
                ("tol", ctypes.c_double),
                ("flags", ctypes.c_uint32)]


class _Tuning(ctypes.Structure):
    _fields_ = [("sketch_pack_slices", ctypes.c_int32),
                ("sketch_stages", ctypes.c_int32),
                ("sketch_ctas_per_sm", ctypes.c_int32),
                ("error_path", ctypes.c_int32),
                ("error_rows", ctypes.c_int32),
                ("error_cols", ctypes.c_int32),
                ("sketch_slice_major", ctypes.c_int32),
                ("sketch_slice_cols", ctypes.c_int32),
                ("sketch_ms", ctypes.c_float),
                ("error_ms", ctypes.c_float)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}

    @classmethod
    def from_dict(cls, d: dict) -> "_Tuning":
        t = cls()
        for name, _ in cls._fields_:
            setattr(t, name, d.get(name, 0))
        return t


class _SubPointsDesc(ctypes.Structure):
    _fields_ = [("num_sub", ctypes.c_int32),
                ("m", ctypes.POINTER(ctypes.c_int32)),
                ("n", ctypes.POINTER(ctypes.c_int32)),
                ("off", ctypes.POINTER(ctypes.c_int64)),
                ("ld", ctypes.POINTER(ctypes.c_int64)),
                ("mc", ctypes.POINTER(ctypes.c_int32)),
                ("coarse_rows", ctypes.POINTER(ctypes.c_int32)),
                ("stencil", ctypes.c_int32),
                ("interp_idx", ctypes.POINTER(ctypes.c_int32)),
                ("interp_w", ctypes.POINTER(ctypes.c_float)),
                ("k_max", ctypes.c_int32),
                ("tol", ctypes.c_double),
                ("flags", ctypes.c_uint32)]


class _TsDesc(ctypes.Structure):
    _fields_ = [("base", _Desc),
                ("blocks", ctypes.c_int32),
                ("k2_max", ctypes.c_int32),
                ("tol2", ctypes.c_double)]


_lib = None
_lock = threading.Lock()


def load_library(path: str = LIB_PATH):
    """Load libspid.so and declare its signatures (raises if it is missing)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"libspid.so not built ({path}); run __graft_entry__.build()")
        lib = ctypes.CDLL(path)
        c = ctypes
        vp, i32, i64, u32, u64, dbl = (c.c_void_p, c.c_int32, c.c_int64, c.c_uint32, c.c_uint64,
                                       c.c_double)
        sig = {
            "spid_plan_create": ([c.POINTER(_Desc), vp, c.POINTER(vp)], c.c_int),
            "spid_plan_destroy": ([vp], c.c_int),
            "spid_plan_info": ([vp, c.POINTER(i32), c.POINTER(i32), c.POINTER(i64)], c.c_int),
            "spid_sketch_accumulate": ([vp, vp, i32, i32, vp], c.c_int),
            "spid_reset": ([vp, vp], c.c_int),
            "spid_finalize": ([vp, vp], c.c_int),
            "spid_error": ([vp, vp, vp, vp, vp], c.c_int),
            "spid_reconstruct": ([vp, vp, vp, vp], c.c_int),
            "spid_get_factors": ([vp, vp, vp, vp, vp], c.c_int),
            "spid_get_sketch": ([vp, vp, vp], c.c_int),
            "spid_device_status": ([vp, vp], c.c_int),
            "spid_omega": ([u64, i64, i32, i32, i32, vp, vp], c.c_int),
            "spid_philox": ([vp, u32, u32, vp, i64, vp], c.c_int),
            "spid_compression_factor": ([i32, vp, vp, vp], dbl),
            "spid_status_string": ([c.c_int], c.c_char_p),
            "spid_last_error": ([], c.c_char_p),
            "spid_sketch_fp32_noalloc": ([vp, i32, i32, i64, i32, u64, vp, i32, vp], c.c_int),
            "spid_sub_plan_create": ([c.POINTER(_SubDesc), c.POINTER(vp)], c.c_int),
            "spid_sub_plan_destroy": ([vp], c.c_int),
            "spid_sub_plan_info": ([vp, vp, c.POINTER(i64)], c.c_int),
            "spid_sub_sample": ([vp, vp, i32, i32, vp], c.c_int),
            "spid_sub_finalize": ([vp, vp], c.c_int),
            "spid_sub_error": ([vp, vp, i32, vp, vp, vp], c.c_int),
            "spid_sub_reconstruct": ([vp, vp, i32, vp, vp], c.c_int),
            "spid_sub_get_factors": ([vp, vp, vp, vp, vp, vp], c.c_int),
            "spid_sub_get_coarse": ([vp, vp, vp], c.c_int),
            "spid_sub_device_status": ([vp, vp], c.c_int),
            "spid_ts_plan_create": ([c.POINTER(_TsDesc), c.POINTER(vp)], c.c_int),
            "spid_ts_plan_destroy": ([vp], c.c_int),
            "spid_ts_block": ([vp, vp, i32, vp], c.c_int),
            "spid_ts_finalize": ([vp, vp, vp], c.c_int),
            "spid_ts_error": ([vp, vp, vp, vp, vp], c.c_int),
            "spid_ts_reconstruct": ([vp, vp, vp, vp], c.c_int),
            "spid_ts_get_factors": ([vp, vp, vp, vp, vp], c.c_int),
            "spid_ts_get_block_factors": ([vp, i32, vp, vp, vp, vp], c.c_int),
            "spid_ts_device_status": ([vp, vp], c.c_int),
            "spid_plan_get_tuning": ([vp, c.POINTER(_Tuning)], c.c_int),
            "spid_plan_set_tuning": ([vp, c.POINTER(_Tuning)], c.c_int),
            "spid_plan_autotune": ([vp, vp, vp, c.POINTER(_Tuning)], c.c_int),
            "spid_plan_autotune_calls": ([vp, vp, i32, vp, c.POINTER(_Tuning)], c.c_int),
            "spid_plan_tuning_key": ([vp, c.c_char_p, i32], c.c_int),
            "spid_graph_create": ([vp, vp, i32, i32, i32, u32, vp, vp, c.POINTER(vp)], c.c_int),
            "spid_graph_launch": ([vp, vp], c.c_int),
            "spid_graph_launch_host": ([vp, vp, vp, vp, vp, vp, vp, vp], c.c_int),
            "spid_graph_destroy": ([vp], c.c_int),
            "spid_sub_plan_create_points": ([c.POINTER(_SubPointsDesc), c.POINTER(vp)], c.c_int),
            "spid_producer_step": ([vp, i64, vp, i64, i32, i32, i32, c.c_float, c.c_float, vp],
                                   c.c_int),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def _check(status: int, where: str):
    if status != SPID_OK:
        detail = load_library().spid_last_error().decode(errors="replace")
        raise SpidError(status, where, detail)


def _stream_handle(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _ptr(t) -> int:
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        if not t.is_cuda:
            raise ValueError("expected a CUDA tensor")
        return t.data_ptr()
    return int(t)


def _host_ptr(t, dtype, min_bytes: int) -> int:
    """Address of a host buffer (CPU torch tensor or numpy array) holding at
    least min_bytes, contiguous, of dtype (None: any)."""
    if hasattr(t, "data_ptr"):
        if t.is_cuda:
            raise ValueError("expected a host (CPU) tensor")
        if not t.is_contiguous():
            raise ValueError("host tensor must be contiguous")
        if dtype is not None and t.element_size() != np.dtype(dtype).itemsize:
            raise ValueError(f"host tensor must hold {np.dtype(dtype).name}")
        nbytes, addr = t.numel() * t.element_size(), t.data_ptr()
    else:
        a = np.asarray(t)
        if not a.flags.c_contiguous:
            raise ValueError("host array must be contiguous")
        if dtype is not None and a.dtype != np.dtype(dtype):
            raise ValueError(f"host array must hold {np.dtype(dtype).name}")
        nbytes, addr = a.nbytes, a.ctypes.data
    if nbytes < min_bytes:
        raise ValueError(f"host buffer holds {nbytes} bytes, needs {min_bytes}")
    return addr


def producer_step(state_in, state_out, grid: int, edge: int, nq: int, dt: float, nu: float,
                  stream=None, in_box_stride: int | None = None,
                  out_box_stride: int | None = None):
    """One step of the in-situ producer (spid_producer_step) on device tensors;
    box strides default to a contiguous snapshot (nq edge^3)."""
    be = int(nq) * int(edge) ** 3
    _check(load_library().spid_producer_step(
        _ptr(state_in), int(in_box_stride or be), _ptr(state_out), int(out_box_stride or be),
        int(grid), int(edge), int(nq), float(dt), float(nu), _stream_handle(stream)),
        "spid_producer_step")


class BoxLayout:
    """Boxes of a global field [t][q][Z][Y][X] (spid_box_layout).  org, ext:
    [B, 3] arrays of (x, y, z); split_qoi: one subdomain per (box, QoI)."""

    def __init__(self, nq: int, X: int, Y: int, Z: int, org, ext, split_qoi: bool = False,
                 snap_stride: int | None = None):
        self.nq, self.X, self.Y, self.Z = int(nq), int(X), int(Y), int(Z)
        self.org = np.ascontiguousarray(org, dtype=np.int32).reshape(-1, 3)
        self.ext = np.ascontiguousarray(ext, dtype=np.int32).reshape(-1, 3)
        self.split_qoi = bool(split_qoi)
        self.snap_stride = int(snap_stride if snap_stride is not None else nq * X * Y * Z)
        self.num_box = int(self.org.shape[0])
        self.num_sub = self.num_box * (self.nq if self.split_qoi else 1)
        pts = self.ext.prod(axis=1).astype(np.int64)
        rows = pts if self.split_qoi else pts * self.nq
        self.m = np.repeat(rows, self.nq) if self.split_qoi else rows

    def struct(self) -> _BoxLayout:
        b = _BoxLayout()
        b.nq, b.X, b.Y, b.Z = self.nq, self.X, self.Y, self.Z
        b.snap_stride = self.snap_stride
        b.num_box = self.num_box
        b.org3 = self.org.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        b.ext3 = self.ext.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        b.split_qoi = int(self.split_qoi)
        return b


class Plan:
    """Batched sketched column-ID plan over a window of subdomains.

    Blocks layout: m, n, off, ld are per-subdomain rows, columns, element
    offset and leading dimension of the column-major blocks inside one flat
    window buffer.  Boxes layout: boxes = BoxLayout(...) over a global field
    (m, off, ld are then derived; pass None).  qoi / num_qoi label subdomains
    by QoI for the per-QoI error totals."""

    def __init__(self, m, n, off, ld, k_max: int, p: int = 10, tol: float = 0.0,
                 precision: str = "tf32", seed: int = 0x5EED0001, flags: int = 0,
                 qoi=None, num_qoi: int = 0, boxes: "BoxLayout | None" = None, stream=None):
        lib = load_library()
        self.boxes = boxes
        if boxes is not None:
            self.m = np.ascontiguousarray(boxes.m, dtype=np.int32)
        else:
            self.m = np.ascontiguousarray(m, dtype=np.int32)
        self.S = int(len(self.m))
        self.n = np.ascontiguousarray(np.broadcast_to(n, (self.S,)), dtype=np.int32)
        if boxes is None:
            self.off = np.ascontiguousarray(off, dtype=np.int64)
            self.ld = np.ascontiguousarray(ld, dtype=np.int64)
        self.k_max = int(k_max)
        self.p = int(p)
        self.precision = precision
        self.dtype = np.float64 if precision == "fp64" else np.float32
        self.qoi = None if qoi is None else np.ascontiguousarray(qoi, dtype=np.int32)
        self.num_qoi = int(num_qoi)
        if boxes is not None and boxes.split_qoi and qoi is None and self.num_qoi == 0:
            self.num_qoi = boxes.nq
        d = _Desc()
        d.num_sub = self.S
        d.n = self.n.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        if boxes is None:
            d.m = self.m.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
            d.off = self.off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
            d.ld = self.ld.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
        else:
            self._box_struct = boxes.struct()
            d.boxes = ctypes.pointer(self._box_struct)
        d.k_max = self.k_max
        d.p = self.p
        d.tol = float(tol)
        d.precision = PREC[precision]
        d.flags = int(flags)
        d.seed = int(seed)
        if self.qoi is not None:
            d.qoi = self.qoi.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        d.num_qoi = int(num_qoi)
        h = ctypes.c_void_p()
        _check(lib.spid_plan_create(ctypes.byref(d), _stream_handle(stream) if stream is not None
                                    else None, ctypes.byref(h)), "spid_plan_create")
        self._h = h
        l = ctypes.c_int32()
        lp = ctypes.c_int32()
        ws = ctypes.c_int64()
        _check(lib.spid_plan_info(h, ctypes.byref(l), ctypes.byref(lp), ctypes.byref(ws)),
               "spid_plan_info")
        self.l, self.l_pad, self.workspace_bytes = int(l.value), int(lp.value), int(ws.value)

    @classmethod
    def for_window(cls, win, **kw) -> "Plan":
        return cls(win.m, win.n, win.off, win.ld, **kw)

    def window_extent(self) -> int:
        """Elements from the window pointer that cover everything the plan reads
        (blocks: the exact extent; boxes: whole snapshots up to the last one)."""
        if self.boxes is not None:
            b = self.boxes
            return int(self.n.max() - 1) * b.snap_stride + b.nq * b.X * b.Y * b.Z
        return int(np.max(self.off + self.ld * (self.n.astype(np.int64) - 1) + self.m))

    @property
    def total_len(self) -> int:
        """Doubles spid_error writes to total: 4 sums plus 2 per QoI."""
        return 4 + 2 * self.num_qoi

    def per_qoi_rel_err(self, total) -> np.ndarray:
        """sqrt(sum e2 / sum a2) of each QoI from an error-total buffer."""
        t = np.asarray(total.detach().cpu().numpy() if hasattr(total, "detach") else total,
                       dtype=np.float64)
        g = t[4:4 + 2 * self.num_qoi].reshape(-1, 2)
        return np.sqrt(g[:, 0] / g[:, 1])

    def close(self):
        if getattr(self, "_h", None):
            for g in list(getattr(self, "_graphs", [])):
                g.close()
            load_library().spid_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------- tuning
    def tuning(self) -> dict:
        t = _Tuning()
        _check(load_library().spid_plan_get_tuning(self._h, ctypes.byref(t)),
               "spid_plan_get_tuning")
        return t.as_dict()

    def set_tuning(self, tuning: dict):
        t = _Tuning.from_dict(tuning)
        _check(load_library().spid_plan_set_tuning(self._h, ctypes.byref(t)),
               "spid_plan_set_tuning")

    def tuning_key(self) -> str:
        buf = ctypes.create_string_buffer(512)
        _check(load_library().spid_plan_tuning_key(self._h, buf, 512), "spid_plan_tuning_key")
        return buf.value.decode()

    def autotune(self, window, stream=None, cache: str | None = None, microbatch: int = 0) -> dict:
        """Measure the candidate tile shapes on `window`, sketched in calls of
        `microbatch` columns (0: whole-window calls), and keep the fastest.
        With `cache` (a JSON file path), a tuning stored under this plan's
        tuning key (and the call width) is applied instead of measuring, and a
        new measurement is stored there."""
        import json
        key = self.tuning_key() + (f"/calls{int(microbatch)}" if microbatch else "")
        store = {}
        if cache and os.path.exists(cache):
            with open(cache) as f:
                store = json.load(f)
            if key in store:
                self.set_tuning(store[key])
                return dict(store[key], cached=True)
        t = _Tuning()
        _check(load_library().spid_plan_autotune_calls(self._h, _ptr(window), int(microbatch),
                                                       _stream_handle(stream), ctypes.byref(t)),
               "spid_plan_autotune_calls")
        d = t.as_dict()
        if cache:
            store[key] = d
            tmp = f"{cache}.tmp{os.getpid()}"
            with open(tmp, "w") as f:
                json.dump(store, f, indent=1, sort_keys=True)
            os.replace(tmp, cache)
        return dict(d, cached=False)

    def graph(self, window, what: int = GRAPH_SKETCH | GRAPH_FINALIZE | GRAPH_ERROR, err=None,
              total=None, col0: int = 0, ncols: int | None = None,
              microbatch: int = 0) -> "Graph":
        """Capture one step (the SPID_GRAPH_* stages in `what`) as a CUDA graph."""
        if ncols is None:
            ncols = int(self.n.max()) - col0
        h = ctypes.c_void_p()
        _check(load_library().spid_graph_create(self._h, _ptr(window), int(col0), int(ncols),
                                                int(microbatch), int(what), _ptr(err), _ptr(total),
                                                ctypes.byref(h)), "spid_graph_create")
        g = Graph(self, h)
        if not hasattr(self, "_graphs"):
            self._graphs = []
        self._graphs.append(g)
        return g

    # ---------------------------------------------------------------- hot path
    def sketch_accumulate(self, window, col0: int = 0, ncols: int | None = None, stream=None):
        if ncols is None:
            ncols = int(self.n.max()) - col0
        _check(load_library().spid_sketch_accumulate(self._h, _ptr(window), int(col0),
                                                     int(ncols), _stream_handle(stream)),
               "spid_sketch_accumulate")

    sketch = sketch_accumulate

    def reset(self, stream=None):
        _check(load_library().spid_reset(self._h, _stream_handle(stream)), "spid_reset")

    def finalize(self, stream=None):
        _check(load_library().spid_finalize(self._h, _stream_handle(stream)), "spid_finalize")

    def error(self, window, err=None, total=None, stream=None):
        _check(load_library().spid_error(self._h, _ptr(window), _ptr(err), _ptr(total),
                                         _stream_handle(stream)), "spid_error")

    def reconstruct(self, window, out, stream=None):
        _check(load_library().spid_reconstruct(self._h, _ptr(window), _ptr(out),
                                               _stream_handle(stream)), "spid_reconstruct")

    # ---------------------------------------------------------------- results
    def factors(self, stream=None):
        """(k [S], J [S, k_max], C list of k_max x n_s arrays)."""
        k = np.zeros(self.S, dtype=np.int32)
        J = np.zeros((self.S, self.k_max), dtype=np.int32)
        C = np.zeros(self.k_max * int(self.n.sum()), dtype=self.dtype)
        _check(load_library().spid_get_factors(self._h, k.ctypes.data, J.ctypes.data,
                                               C.ctypes.data, _stream_handle(stream)),
               "spid_get_factors")
        coff = np.concatenate([[0], np.cumsum(self.n)]) * self.k_max
        Cs = [C[coff[s]:coff[s + 1]].reshape(self.k_max, int(self.n[s])) for s in range(self.S)]
        return k, J, Cs

    def sketches(self, stream=None):
        """List of Y_s as l x n_s arrays."""
        Y = np.zeros(self.l_pad * int(self.n.sum()), dtype=self.dtype)
        _check(load_library().spid_get_sketch(self._h, Y.ctypes.data, _stream_handle(stream)),
               "spid_get_sketch")
        yoff = np.concatenate([[0], np.cumsum(self.n)]) * self.l_pad
        return [Y[yoff[s]:yoff[s + 1]].reshape(int(self.n[s]), self.l_pad)[:, :self.l].T
                for s in range(self.S)]

    def device_status(self, stream=None) -> int:
        return int(load_library().spid_device_status(self._h, _stream_handle(stream)))


class Graph:
    """A captured step of a Plan (spid_graph_*); replay with launch()."""

    def __init__(self, plan: Plan, handle):
        self._plan = plan
        self._h = handle

    def launch(self, stream=None):
        _check(load_library().spid_graph_launch(self._h, _stream_handle(stream)),
               "spid_graph_launch")

    def launch_host(self, window_host, total_host=None, k_host=None, J_host=None, C_host=None,
                    copy_stream=None, stream=None, window_elems: int | None = None):
        """spid_graph_launch_host: copy the window from host memory (a pinned
        CPU tensor or array of at least window_elems elements, by default the
        blocks extent), run the step, copy the error sums to total_host
        (plan.total_len doubles) and the factors to k_host [S], J_host
        [S k_max] and C_host [k_max sum n] (pinned host buffers, or None);
        asynchronous."""
        p = self._plan
        if window_elems is None:
            window_elems = p.window_extent()
        win = _host_ptr(window_host, p.dtype, window_elems * np.dtype(p.dtype).itemsize)
        tot = None if total_host is None else _host_ptr(total_host, np.float64, 8 * p.total_len)
        kh = None if k_host is None else _host_ptr(k_host, np.int32, 4 * p.S)
        Jh = None if J_host is None else _host_ptr(J_host, np.int32, 4 * p.S * p.k_max)
        Ch = None if C_host is None else _host_ptr(
            C_host, p.dtype, np.dtype(p.dtype).itemsize * p.k_max * int(p.n.sum()))
        _check(load_library().spid_graph_launch_host(
            self._h, win, tot, kh, Jh, Ch, _stream_handle(copy_stream), _stream_handle(stream)),
            "spid_graph_launch_host")

    def close(self):
        if getattr(self, "_h", None):
            load_library().spid_graph_destroy(self._h)
            self._h = None
            graphs = getattr(self._plan, "_graphs", [])
            if self in graphs:
                graphs.remove(self)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class SubPlan:
    """Coarse-grid column ID (Section 2 SubID / SPID, Algorithms 2-3) over a
    window of boxes.  box: [S, 4] (nq, ez, ey, ex) per subdomain (rows of a box
    in (q, z, y, x) order, x fastest); stride: coarse interval (sz, sy, sx)."""

    def __init__(self, box, n, off, ld, stride, k_max: int, tol: float = 0.0):
        lib = load_library()
        self.box = np.ascontiguousarray(box, dtype=np.int32).reshape(-1, 4)
        self.S = int(self.box.shape[0])
        self.n = np.ascontiguousarray(np.broadcast_to(n, (self.S,)), dtype=np.int32)
        self.off = np.ascontiguousarray(off, dtype=np.int64)
        self.ld = np.ascontiguousarray(ld, dtype=np.int64)
        self.m = self.box.prod(axis=1).astype(np.int64)
        self.k_max = int(k_max)
        d = _SubDesc()
        d.num_sub = self.S
        d.box = self.box.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        d.n = self.n.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        d.off = self.off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
        d.ld = self.ld.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
        for i in range(3):
            d.stride[i] = int(stride[i])
        d.k_max = self.k_max
        d.tol = float(tol)
        d.flags = 0
        h = ctypes.c_void_p()
        _check(lib.spid_sub_plan_create(ctypes.byref(d), ctypes.byref(h)), "spid_sub_plan_create")
        self._h = h
        mc = np.zeros(self.S, dtype=np.int64)
        ws = ctypes.c_int64()
        _check(lib.spid_sub_plan_info(h, mc.ctypes.data, ctypes.byref(ws)), "spid_sub_plan_info")
        self.mc, self.workspace_bytes = mc, int(ws.value)

    @classmethod
    def from_points(cls, m, n, off, ld, coarse_rows, interp_idx, interp_w, k_max: int,
                    tol: float = 0.0) -> "SubPlan":
        """Point-set plan (spid_sub_plan_create_points): coarse_rows[s] lists the
        rows of A_s kept in B_s; interp_idx[s] / interp_w[s] are m_s x t arrays,
        fine row r = sum_q w[r, q] B_s(idx[r, q], :)."""
        lib = load_library()
        self = cls.__new__(cls)
        self.m = np.ascontiguousarray(m, dtype=np.int32)
        self.S = int(len(self.m))
        self.n = np.ascontiguousarray(np.broadcast_to(n, (self.S,)), dtype=np.int32)
        self.off = np.ascontiguousarray(off, dtype=np.int64)
        self.ld = np.ascontiguousarray(ld, dtype=np.int64)
        self.k_max = int(k_max)
        t = int(np.asarray(interp_idx[0]).reshape(int(self.m[0]), -1).shape[1])
        mc = np.array([len(c) for c in coarse_rows], dtype=np.int32)
        crow = np.ascontiguousarray(np.concatenate([np.asarray(c, dtype=np.int32)
                                                    for c in coarse_rows]))
        iidx = np.ascontiguousarray(np.concatenate([np.asarray(x, dtype=np.int32).reshape(-1)
                                                    for x in interp_idx]))
        iw = np.ascontiguousarray(np.concatenate([np.asarray(x, dtype=np.float32).reshape(-1)
                                                  for x in interp_w]))
        d = _SubPointsDesc()
        d.num_sub = self.S
        P32 = ctypes.POINTER(ctypes.c_int32)
        P64 = ctypes.POINTER(ctypes.c_int64)
        d.m = self.m.ctypes.data_as(P32)
        d.n = self.n.ctypes.data_as(P32)
        d.off = self.off.ctypes.data_as(P64)
        d.ld = self.ld.ctypes.data_as(P64)
        d.mc = mc.ctypes.data_as(P32)
        d.coarse_rows = crow.ctypes.data_as(P32)
        d.stencil = t
        d.interp_idx = iidx.ctypes.data_as(P32)
        d.interp_w = iw.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
        d.k_max = self.k_max
        d.tol = float(tol)
        d.flags = 0
        h = ctypes.c_void_p()
        _check(lib.spid_sub_plan_create_points(ctypes.byref(d), ctypes.byref(h)),
               "spid_sub_plan_create_points")
        self._h = h
        out_mc = np.zeros(self.S, dtype=np.int64)
        ws = ctypes.c_int64()
        _check(lib.spid_sub_plan_info(h, out_mc.ctypes.data, ctypes.byref(ws)), "spid_sub_plan_info")
        self.mc, self.workspace_bytes = out_mc, int(ws.value)
        return self

    @classmethod
    def for_window(cls, win, stride, **kw) -> "SubPlan":
        return cls(win.meta["boxes"], win.n, win.off, win.ld, stride, **kw)

    def close(self):
        if getattr(self, "_h", None):
            load_library().spid_sub_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sample(self, window, col0: int = 0, ncols: int | None = None, stream=None):
        if ncols is None:
            ncols = int(self.n.max()) - col0
        _check(load_library().spid_sub_sample(self._h, _ptr(window), int(col0), int(ncols),
                                              _stream_handle(stream)), "spid_sub_sample")

    def finalize(self, stream=None):
        _check(load_library().spid_sub_finalize(self._h, _stream_handle(stream)),
               "spid_sub_finalize")

    def error(self, window, form: int = FORM_SPID, err=None, total=None, stream=None):
        _check(load_library().spid_sub_error(self._h, _ptr(window), int(form), _ptr(err),
                                             _ptr(total), _stream_handle(stream)),
               "spid_sub_error")

    def reconstruct(self, window, out, form: int = FORM_SPID, stream=None):
        _check(load_library().spid_sub_reconstruct(self._h, _ptr(window), int(form), _ptr(out),
                                                   _stream_handle(stream)),
               "spid_sub_reconstruct")

    def factors(self, stream=None):
        """(k [S], J [S, k_max], C list of k_max x n_s, Bskel list of mc_s x k_max)."""
        k = np.zeros(self.S, dtype=np.int32)
        J = np.zeros((self.S, self.k_max), dtype=np.int32)
        C = np.zeros(self.k_max * int(self.n.sum()), dtype=np.float32)
        Bs = np.zeros(self.k_max * int(self.mc.sum()), dtype=np.float32)
        _check(load_library().spid_sub_get_factors(self._h, k.ctypes.data, J.ctypes.data,
                                                   C.ctypes.data, Bs.ctypes.data,
                                                   _stream_handle(stream)), "spid_sub_get_factors")
        coff = np.concatenate([[0], np.cumsum(self.n)]) * self.k_max
        soff = np.concatenate([[0], np.cumsum(self.mc)]) * self.k_max
        Cs = [C[coff[s]:coff[s + 1]].reshape(self.k_max, int(self.n[s])) for s in range(self.S)]
        Bk = [Bs[soff[s]:soff[s + 1]].reshape(self.k_max, int(self.mc[s])).T
              for s in range(self.S)]
        return k, J, Cs, Bk

    def coarse(self, stream=None):
        """List of the gathered B_s (mc_s x n_s)."""
        B = np.zeros(int((self.mc * self.n).sum()), dtype=np.float32)
        _check(load_library().spid_sub_get_coarse(self._h, B.ctypes.data, _stream_handle(stream)),
               "spid_sub_get_coarse")
        boff = np.concatenate([[0], np.cumsum(self.mc * self.n)])
        return [B[boff[s]:boff[s + 1]].reshape(int(self.n[s]), int(self.mc[s])).T
                for s in range(self.S)]

    def device_status(self, stream=None) -> int:
        return int(load_library().spid_sub_device_status(self._h, _stream_handle(stream)))


class TsPlan:
    """Modified (two-stage) SPID (Section 3.3.2, Algorithm 6): N time blocks with
    a target-rank-k sketched ID each, then a sketched ID with tolerance tol2 of
    the concatenated skeletons, composed into A ~ A(:, J) C."""

    def __init__(self, m, n, off, ld, blocks: int, k: int, k2_max: int, tol2: float,
                 p: int = 10, precision: str = "tf32", seed: int = 0x5EED0001):
        lib = load_library()
        self.m = np.ascontiguousarray(m, dtype=np.int32)
        self.n = np.ascontiguousarray(n, dtype=np.int32)
        self.off = np.ascontiguousarray(off, dtype=np.int64)
        self.ld = np.ascontiguousarray(ld, dtype=np.int64)
        self.S = int(len(self.m))
        self.N, self.k, self.k2_max = int(blocks), int(k), int(k2_max)
        self.dtype = np.float64 if precision == "fp64" else np.float32
        d = _TsDesc()
        b = d.base
        b.num_sub = self.S
        b.m = self.m.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        b.n = self.n.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        b.off = self.off.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
        b.ld = self.ld.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
        b.k_max = self.k
        b.p = int(p)
        b.tol = 0.0
        b.precision = PREC[precision]
        b.flags = 0
        b.seed = int(seed)
        d.blocks = self.N
        d.k2_max = self.k2_max
        d.tol2 = float(tol2)
        h = ctypes.c_void_p()
        _check(lib.spid_ts_plan_create(ctypes.byref(d), ctypes.byref(h)), "spid_ts_plan_create")
        self._h = h

    @classmethod
    def for_window(cls, win, **kw) -> "TsPlan":
        return cls(win.m, win.n, win.off, win.ld, **kw)

    def close(self):
        if getattr(self, "_h", None):
            load_library().spid_ts_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def block(self, window, b: int, stream=None):
        _check(load_library().spid_ts_block(self._h, _ptr(window), int(b), _stream_handle(stream)),
               "spid_ts_block")

    def finalize(self, window, stream=None):
        _check(load_library().spid_ts_finalize(self._h, _ptr(window), _stream_handle(stream)),
               "spid_ts_finalize")

    def error(self, window, err=None, total=None, stream=None):
        _check(load_library().spid_ts_error(self._h, _ptr(window), _ptr(err), _ptr(total),
                                            _stream_handle(stream)), "spid_ts_error")

    def reconstruct(self, window, out, stream=None):
        _check(load_library().spid_ts_reconstruct(self._h, _ptr(window), _ptr(out),
                                                  _stream_handle(stream)), "spid_ts_reconstruct")

    def _factors(self, fn, kmax, ncols, *pre):
        k = np.zeros(self.S, dtype=np.int32)
        J = np.zeros((self.S, kmax), dtype=np.int32)
        C = np.zeros(kmax * int(ncols.sum()), dtype=self.dtype)
        _check(fn(self._h, *pre, k.ctypes.data, J.ctypes.data, C.ctypes.data,
                  _stream_handle(None)), "spid_ts factors")
        coff = np.concatenate([[0], np.cumsum(ncols)]) * kmax
        return k, J, [C[coff[s]:coff[s + 1]].reshape(kmax, int(ncols[s])) for s in range(self.S)]

    def factors(self):
        """Final (k, J [S, k2_max] window columns, C list of k2_max x n_s)."""
        return self._factors(load_library().spid_ts_get_factors, self.k2_max, self.n)

    def block_factors(self, b: int):
        """Stage-1 (k, J local to block b, C list of k x n_s / N)."""
        return self._factors(load_library().spid_ts_get_block_factors, self.k, self.n // self.N,
                             int(b))

    def device_status(self, stream=None) -> int:
        return int(load_library().spid_ts_device_status(self._h, _stream_handle(stream)))


def omega(seed: int, r0: int, nrows: int, l: int, precision: str, out, stream=None):
    _check(load_library().spid_omega(int(seed), int(r0), int(nrows), int(l), PREC[precision],
                                     _ptr(out), _stream_handle(stream)), "spid_omega")


def philox(ctr, key0: int, key1: int, out, stream=None):
    _check(load_library().spid_philox(_ptr(ctr), int(key0), int(key1), _ptr(out),
                                      int(ctr.numel() // 4), _stream_handle(stream)), "spid_philox")


def compression_factor(m, n, k) -> float:
    m = np.ascontiguousarray(m, dtype=np.int32)
    n = np.ascontiguousarray(n, dtype=np.int32)
    k = np.ascontiguousarray(k, dtype=np.int32)
    return float(load_library().spid_compression_factor(len(m), m.ctypes.data, n.ctypes.data,
                                                        k.ctypes.data))


def sketch_fp32_noalloc(A, m: int, n: int, ld: int, l: int, seed: int, Y, ldy: int, stream=None):
    """FP32 sketch of one subdomain through the allocation-free entry point.

    For callers that cannot allocate device memory mid-run (an in-situ solver
    that owns nearly all GPU memory through its own pool, or whose time loop
    must avoid cudaMalloc/cudaFree and their device-wide synchronization): the
    split-K partials live in the library's fixed 8 MiB static device array, so
    concurrent calls on different streams race and must be serialized."""
    _check(load_library().spid_sketch_fp32_noalloc(_ptr(A), int(m), int(n), int(ld), int(l),
                                                   int(seed), _ptr(Y), int(ldy),
                                                   _stream_handle(stream)),
           "spid_sketch_fp32_noalloc")
