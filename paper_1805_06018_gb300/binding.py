"""ctypes binding of libpc (include/pc.h): the same entry points, argument
marshalling only.  Every step of an apply runs in the library's kernels.

The library is loaded on first use; if it has not been built the call raises
``LibraryMissing`` (there is no fallback path).  Device arrays are passed as
raw pointers; :class:`Operator` adds the PyTorch conveniences (data_ptr(),
current stream) on top.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libpc.so")

PC_OK, PC_ERR_ARG, PC_ERR_GRID, PC_ERR_NOMEM, PC_ERR_BUDGET, PC_ERR_CUDA, PC_ERR_TIMEOUT, \
    PC_ERR_NOT_READY, PC_ERR_UNSUPPORTED = range(9)
STATUS_NAMES = ["PC_OK", "PC_ERR_ARG", "PC_ERR_GRID", "PC_ERR_NOMEM", "PC_ERR_BUDGET", "PC_ERR_CUDA",
                "PC_ERR_TIMEOUT", "PC_ERR_NOT_READY", "PC_ERR_UNSUPPORTED"]
PC_FP64, PC_FP32, PC_BF16X3, PC_TF32X3 = range(4)
PC_SERVE_ADJOINT = 1
PRECISIONS = {"fp64": PC_FP64, "fp32": PC_FP32, "bf16x3": PC_BF16X3, "tf32x3": PC_TF32X3}


class LibraryMissing(ImportError):
    pass


class PCError(RuntimeError):
    def __init__(self, status: int, msg: str):
        self.status = status
        super().__init__("%s: %s" % (STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status, msg))


class pc_box(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int32), ("shape", ctypes.c_int64 * 3)]


class pc_grid(ctypes.Structure):
    _fields_ = [("num_cells", ctypes.c_int32), ("cells", ctypes.POINTER(ctypes.c_int32))]


class pc_tuning(ctypes.Structure):
    _fields_ = [("fft_size", ctypes.c_int32), ("tile", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("wait_limit_us", ctypes.c_int32), ("window_split", ctypes.c_int32), ("per_patch", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 2)]


class pc_operator_info(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int32), ("shape", ctypes.c_int64 * 3), ("radius", ctypes.c_int32),
                ("r", ctypes.c_int32), ("fft_size", ctypes.c_int32), ("tile", ctypes.c_int32),
                ("num_tiles", ctypes.c_int32), ("num_colors", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("spectra_bytes", ctypes.c_int64), ("device_bytes", ctypes.c_int64),
                ("build_seconds", ctypes.c_double), ("window_split", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("autotuned", ctypes.c_int32), ("tuned_candidates", ctypes.c_int32), ("tuned_ms", ctypes.c_double),
                ("num_parts", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class pc_serve_config(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_int64), ("max_inflight", ctypes.c_int32), ("streams", ctypes.c_int32),
                ("max_requests_per_launch", ctypes.c_int32), ("reserved", ctypes.c_int32 * 3)]


class pc_request_info(ctypes.Structure):
    _fields_ = [("submit_s", ctypes.c_double), ("launch_s", ctypes.c_double), ("finish_s", ctypes.c_double),
                ("nrhs", ctypes.c_int32), ("launch_requests", ctypes.c_int32), ("status", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class pc_serve_stats(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_int64), ("rhs_completed", ctypes.c_int64), ("launches", ctypes.c_int64),
                ("p50_latency_s", ctypes.c_double), ("p99_latency_s", ctypes.c_double),
                ("mean_latency_s", ctypes.c_double), ("busy_s", ctypes.c_double), ("rhs_per_s", ctypes.c_double),
                ("peak_bytes", ctypes.c_int64)]


# every entry point of include/pc.h: name -> (restype, argtypes)
_VP = ctypes.c_void_p
_PROTOS = {
    "pc_context_create": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(_VP)]),
    "pc_context_destroy": (ctypes.c_int, [_VP]),
    "pc_last_error": (ctypes.c_char_p, [_VP]),
    "pc_sample_points": (ctypes.c_int, [ctypes.POINTER(pc_box), ctypes.POINTER(pc_grid),
                                        ctypes.POINTER(ctypes.c_int32), _VP]),
    "pc_neighbourhood_boxes": (ctypes.c_int, [ctypes.POINTER(pc_box), ctypes.POINTER(pc_grid), _VP, _VP]),
    "pc_harmonic_weights": (ctypes.c_int, [ctypes.POINTER(pc_box), ctypes.POINTER(pc_grid),
                                           ctypes.POINTER(ctypes.c_int64), _VP]),
    "pc_extend_impulse": (ctypes.c_int, [ctypes.POINTER(pc_box), ctypes.POINTER(pc_grid), ctypes.c_int32,
                                         _VP, _VP]),
    "pc_build_spectra": (ctypes.c_int, [_VP, ctypes.POINTER(pc_box), ctypes.POINTER(pc_grid), ctypes.c_int32,
                                        _VP, _VP, ctypes.c_int, ctypes.POINTER(pc_tuning), ctypes.POINTER(_VP)]),
    "pc_operator_info_get": (ctypes.c_int, [_VP, ctypes.POINTER(pc_operator_info)]),
    "pc_apply": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "pc_apply_batched": (ctypes.c_int, [_VP, ctypes.c_int32, _VP, ctypes.c_int64, _VP, ctypes.c_int64, _VP]),
    "pc_apply_batched_noalloc": (ctypes.c_int, [_VP, ctypes.c_int32, _VP, ctypes.c_int64, _VP, ctypes.c_int64,
                                                 _VP]),
    "pc_noalloc_check": (ctypes.c_int, [_VP, _VP]),
    "pc_apply_plain": (ctypes.c_int, [_VP, ctypes.c_int32, _VP, ctypes.c_int64, _VP, ctypes.c_int64, _VP]),
    "pc_operator_check": (ctypes.c_int, [_VP]),
    "pc_operator_kernel_time": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_float)]),
    "pc_apply_adjoint_batched": (ctypes.c_int, [_VP, ctypes.c_int32, _VP, ctypes.c_int64, _VP, ctypes.c_int64, _VP]),
    "pc_estimate_cell_errors": (ctypes.c_int, [_VP, ctypes.c_int32, _VP, ctypes.c_int64, _VP, ctypes.c_int64,
                                                ctypes.POINTER(ctypes.c_double), _VP]),
    "pc_entries": (ctypes.c_int, [_VP, ctypes.c_int64, _VP, _VP, _VP, _VP]),
    "pc_apply_host": (ctypes.c_int, [_VP, ctypes.c_int32, _VP, ctypes.c_int64, _VP, ctypes.c_int64, ctypes.c_int32,
                                     ctypes.c_int32, _VP]),
    "pc_estimator_create": (ctypes.c_int, [_VP, ctypes.POINTER(pc_box), ctypes.c_int, ctypes.c_int32, _VP,
                                           ctypes.c_int64, _VP, ctypes.c_int64, ctypes.POINTER(_VP)]),
    "pc_estimator_update": (ctypes.c_int, [_VP, _VP, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32),
                                           _VP]),
    "pc_estimator_destroy": (ctypes.c_int, [_VP]),
    "pc_refine": (ctypes.c_int, [ctypes.POINTER(pc_box), ctypes.POINTER(pc_grid), ctypes.c_int32, _VP, _VP,
                                 ctypes.c_double, ctypes.c_double, ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                                 _VP, ctypes.POINTER(ctypes.c_int32)]),
    "pc_split_directions": (ctypes.c_int, [ctypes.POINTER(pc_box), ctypes.POINTER(pc_grid), ctypes.c_int32, _VP,
                                           ctypes.c_int32, _VP, ctypes.POINTER(ctypes.c_int32)]),
    "pc_split_is_admissible": (ctypes.c_int, [ctypes.POINTER(pc_box), ctypes.POINTER(pc_grid), ctypes.c_int32,
                                              ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]),
    "pc_block_plan_create": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, ctypes.c_int32, ctypes.POINTER(_VP)]),
    "pc_block_apply": (ctypes.c_int, [_VP, ctypes.c_int32, _VP, ctypes.c_int64, _VP, ctypes.c_int64, _VP]),
    "pc_block_plan_create_many": (ctypes.c_int, [_VP, ctypes.c_int32, _VP, _VP, _VP, _VP, ctypes.c_int32,
                                                 ctypes.POINTER(_VP)]),
    "pc_block_apply_many": (ctypes.c_int, [_VP, ctypes.c_int32, ctypes.POINTER(_VP), ctypes.POINTER(ctypes.c_int64),
                                           ctypes.POINTER(_VP), ctypes.POINTER(ctypes.c_int64), _VP]),
    "pc_block_plan_info": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
    "pc_block_plan_check": (ctypes.c_int, [_VP]),
    "pc_block_plan_destroy": (ctypes.c_int, [_VP]),
    "pc_operator_launches": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int64)]),
    "pc_operator_stage_time": (ctypes.c_int, [_VP, ctypes.c_int32, ctypes.POINTER(ctypes.c_float)]),
    "pc_operator_destroy": (ctypes.c_int, [_VP]),
    "pc_serve_create": (ctypes.c_int, [_VP, ctypes.POINTER(pc_serve_config), ctypes.POINTER(_VP)]),
    "pc_serve_submit": (ctypes.c_int, [_VP, _VP, ctypes.c_int32, _VP, _VP, ctypes.c_uint32,
                                       ctypes.POINTER(ctypes.c_uint64)]),
    "pc_serve_poll": (ctypes.c_int, [_VP, ctypes.c_uint64, ctypes.POINTER(pc_request_info)]),
    "pc_serve_stats_get": (ctypes.c_int, [_VP, ctypes.POINTER(pc_serve_stats)]),
    "pc_serve_destroy": (ctypes.c_int, [_VP]),
    "pc_autotune": (ctypes.c_int, [_VP, ctypes.POINTER(pc_box), ctypes.POINTER(pc_grid), ctypes.c_int32, _VP, _VP,
                                   ctypes.c_int, ctypes.c_int32, ctypes.POINTER(pc_tuning),
                                   ctypes.POINTER(ctypes.c_double)]),
}

_lib = None


def lib():
    """The loaded libpc (raises LibraryMissing when it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise LibraryMissing("libpc.so is not built (%s); run paper_1805_06018_gb300/build.py" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _PROTOS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(status: int, ctx=None):
    if status != PC_OK:
        msg = lib().pc_last_error(ctx)
        raise PCError(status, msg.decode() if msg else "")


def _box(shape: Sequence[int]) -> pc_box:
    b = pc_box()
    b.ndim = len(shape)
    for i in range(3):
        b.shape[i] = int(shape[i]) if i < len(shape) else 1
    return b


def _grid(cells: np.ndarray):
    arr = np.ascontiguousarray(np.asarray(cells, dtype=np.int32))
    g = pc_grid()
    g.num_cells = arr.shape[0]
    g.cells = arr.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    return g, arr   # keep arr alive


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(_VP)


def pc_sample_points(shape, cells) -> np.ndarray:
    b = _box(shape)
    g, keep = _grid(cells)
    r = ctypes.c_int32()
    _check(lib().pc_sample_points(ctypes.byref(b), ctypes.byref(g), ctypes.byref(r), None))
    out = np.zeros((r.value, len(shape)), dtype=np.int32)
    _check(lib().pc_sample_points(ctypes.byref(b), ctypes.byref(g), ctypes.byref(r), _ptr(out)))
    del keep
    return out


def pc_neighbourhood_boxes(shape, cells):
    r = len(pc_sample_points(shape, cells))
    b = _box(shape)
    g, keep = _grid(cells)
    lo = np.zeros((r, len(shape)), dtype=np.int32)
    hi = np.zeros((r, len(shape)), dtype=np.int32)
    _check(lib().pc_neighbourhood_boxes(ctypes.byref(b), ctypes.byref(g), _ptr(lo), _ptr(hi)))
    del keep
    return lo, hi


def pc_harmonic_weights(shape, cells) -> np.ndarray:
    b = _box(shape)
    g, keep = _grid(cells)
    n = ctypes.c_int64()
    _check(lib().pc_harmonic_weights(ctypes.byref(b), ctypes.byref(g), ctypes.byref(n), None))
    out = np.zeros(n.value)
    _check(lib().pc_harmonic_weights(ctypes.byref(b), ctypes.byref(g), ctypes.byref(n), _ptr(out)))
    del keep
    return out


def pc_extend_impulse(shape, cells, radius: int, impulse: np.ndarray) -> np.ndarray:
    b = _box(shape)
    g, keep = _grid(cells)
    imp = np.ascontiguousarray(impulse, dtype=np.float64)
    out = np.zeros_like(imp)
    _check(lib().pc_extend_impulse(ctypes.byref(b), ctypes.byref(g), ctypes.c_int32(radius), _ptr(imp), _ptr(out)))
    del keep
    return out


def pc_refine(shape, cells, radius: int, impulse: np.ndarray, eta_c, y_rms: float, tau: float, batch: int = 1):
    """One refinement pass of Algorithm 1: (eta_Omega, new leaf cells [n][2][d])."""
    b = _box(shape)
    g, keep = _grid(cells)
    d = len(shape)
    imp = np.ascontiguousarray(impulse, dtype=np.float64)
    eta = np.ascontiguousarray(eta_c, dtype=np.float64)
    out = np.zeros((len(cells) + batch, 2, d), dtype=np.int32)
    eo = ctypes.c_double()
    n = ctypes.c_int32()
    _check(lib().pc_refine(ctypes.byref(b), ctypes.byref(g), ctypes.c_int32(radius), _ptr(imp), _ptr(eta),
                           ctypes.c_double(y_rms), ctypes.c_double(tau), ctypes.c_int32(batch), ctypes.byref(eo),
                           _ptr(out), ctypes.byref(n)))
    del keep
    return eo.value, out[:n.value]


def pc_split_directions(shape, cells, radius: int, impulse: np.ndarray, cell: int):
    """Section 2.7's subdivision directions of leaf `cell`, best first."""
    b = _box(shape)
    g, keep = _grid(cells)
    imp = np.ascontiguousarray(impulse, dtype=np.float64)
    dirs = np.zeros(3, dtype=np.int32)
    n = ctypes.c_int32()
    _check(lib().pc_split_directions(ctypes.byref(b), ctypes.byref(g), ctypes.c_int32(radius), _ptr(imp),
                                     ctypes.c_int32(cell), _ptr(dirs), ctypes.byref(n)))
    del keep
    return [int(v) for v in dirs[:n.value]]


def pc_split_is_admissible(shape, cells, cell: int, axis: int) -> bool:
    """Whether halving leaf `cell` along `axis` keeps facet pieces at sample points."""
    b = _box(shape)
    g, keep = _grid(cells)
    ok = ctypes.c_int32()
    _check(lib().pc_split_is_admissible(ctypes.byref(b), ctypes.byref(g), ctypes.c_int32(cell), ctypes.c_int32(axis),
                                        ctypes.byref(ok)))
    del keep
    return bool(ok.value)


class Context:
    def __init__(self, device: int = 0):
        h = _VP()
        _check(lib().pc_context_create(ctypes.c_int32(device), ctypes.byref(h)))
        self.handle = h

    def noalloc_check(self, stream=None):
        """pc_noalloc_check: status of the last allocation-free apply on this device."""
        _check(lib().pc_noalloc_check(self.handle, _VP(_stream_ptr(stream))), self.handle)

    def close(self):
        if self.handle:
            lib().pc_context_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _stream_ptr(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return int(getattr(stream, "cuda_stream", stream))


class Operator:
    """A built product-convolution operator (pc_build_spectra)."""

    def __init__(self, ctx: Context, shape, cells, radius: int, impulse: np.ndarray, precision: str = "fp32",
                 weights: Optional[np.ndarray] = None, fft_size: int = 0, tile: int = 0, ctas_per_sm: int = 0,
                 wait_limit_us: int = 0, window_split: int = 0, per_patch: bool = False, autotune: bool = False):
        self.ctx = ctx
        self.shape = tuple(int(s) for s in shape)
        self.N = int(np.prod(self.shape))
        self.precision = precision
        b = _box(shape)
        g, keep = _grid(cells)
        imp = np.ascontiguousarray(impulse, dtype=np.float64)
        wts = None if weights is None else np.ascontiguousarray(weights, dtype=np.float64)
        tune = pc_tuning()
        tune.fft_size, tune.tile, tune.ctas_per_sm = fft_size, tile, ctas_per_sm
        tune.wait_limit_us, tune.window_split, tune.per_patch = wait_limit_us, window_split, int(per_patch)
        h = _VP()
        # autotune: a NULL pc_tuning asks the library to time candidate launch shapes
        _check(lib().pc_build_spectra(ctx.handle, ctypes.byref(b), ctypes.byref(g), ctypes.c_int32(radius),
                                      _ptr(imp), _ptr(wts), PRECISIONS[precision],
                                      None if autotune else ctypes.byref(tune), ctypes.byref(h)), ctx.handle)
        del keep
        self.handle = h

    def info(self) -> dict:
        inf = pc_operator_info()
        _check(lib().pc_operator_info_get(self.handle, ctypes.byref(inf)))
        return {f: (list(getattr(inf, f)) if f == "shape" else getattr(inf, f)) for f, _ in inf._fields_}

    # raw-pointer entry points -------------------------------------------------
    def pc_apply(self, x_ptr: int, y_ptr: int, stream_ptr: int):
        _check(lib().pc_apply(self.handle, _VP(x_ptr), _VP(y_ptr), _VP(stream_ptr)), self.ctx.handle)

    def pc_apply_batched(self, nrhs: int, x_ptr: int, ldx: int, y_ptr: int, ldy: int, stream_ptr: int):
        _check(lib().pc_apply_batched(self.handle, ctypes.c_int32(nrhs), _VP(x_ptr), ctypes.c_int64(ldx),
                                      _VP(y_ptr), ctypes.c_int64(ldy), _VP(stream_ptr)), self.ctx.handle)

    def pc_apply_batched_noalloc(self, nrhs: int, x_ptr: int, ldx: int, y_ptr: int, ldy: int, stream_ptr: int):
        _check(lib().pc_apply_batched_noalloc(self.handle, ctypes.c_int32(nrhs), _VP(x_ptr), ctypes.c_int64(ldx),
                                              _VP(y_ptr), ctypes.c_int64(ldy), _VP(stream_ptr)), self.ctx.handle)

    def pc_apply_adjoint_batched(self, nrhs: int, x_ptr: int, ldx: int, y_ptr: int, ldy: int, stream_ptr: int):
        _check(lib().pc_apply_adjoint_batched(self.handle, ctypes.c_int32(nrhs), _VP(x_ptr), ctypes.c_int64(ldx),
                                              _VP(y_ptr), ctypes.c_int64(ldy), _VP(stream_ptr)), self.ctx.handle)

    def pc_apply_plain(self, nrhs: int, x_ptr: int, ldx: int, y_ptr: int, ldy: int, stream_ptr: int):
        _check(lib().pc_apply_plain(self.handle, ctypes.c_int32(nrhs), _VP(x_ptr), ctypes.c_int64(ldx),
                                    _VP(y_ptr), ctypes.c_int64(ldy), _VP(stream_ptr)), self.ctx.handle)

    def check(self):
        _check(lib().pc_operator_check(self.handle), self.ctx.handle)

    def kernel_ms(self) -> float:
        """Device time of the fused kernel of the last apply (waits for it)."""
        ms = ctypes.c_float()
        _check(lib().pc_operator_kernel_time(self.handle, ctypes.byref(ms)), self.ctx.handle)
        return ms.value

    def stage_ms(self, stage: int) -> float:
        """3D BF16X3 operators: device time of stage 0 (plane FFTs), 1 (tensor-core
        first-axis DFTs) or 2 (inverse plane FFTs + overlap-add) of the last apply."""
        ms = ctypes.c_float()
        _check(lib().pc_operator_stage_time(self.handle, ctypes.c_int32(stage), ctypes.byref(ms)), self.ctx.handle)
        return ms.value

    def launches(self) -> int:
        n = ctypes.c_int64()
        _check(lib().pc_operator_launches(self.handle, ctypes.byref(n)))
        return n.value

    # torch conveniences ----------------------------------------------------------
    def _args(self, x, out):
        import torch
        if not (x.is_cuda and x.is_contiguous()):
            raise ValueError("x must be a contiguous CUDA tensor")
        want = torch.float64 if self.precision == "fp64" else torch.float32
        if x.dtype != want:
            raise ValueError("x must be %s" % want)
        B = x.numel() // self.N
        if x.numel() != B * self.N:
            raise ValueError("x does not hold whole vectors of the operator's box")
        y = torch.empty_like(x) if out is None else out
        return B, y

    def apply(self, x, out=None, stream=None):
        """y = A~ x for x of shape [B, *box] (or [*box])."""
        B, y = self._args(x, out)
        self.pc_apply_batched(B, x.data_ptr(), self.N, y.data_ptr(), self.N, _stream_ptr(stream))
        return y

    def apply_adjoint(self, x, out=None, stream=None):
        """y = A~* x (Eq. adjoint_random_z) for x of shape [B, *box] (or [*box])."""
        B, y = self._args(x, out)
        self.pc_apply_adjoint_batched(B, x.data_ptr(), self.N, y.data_ptr(), self.N, _stream_ptr(stream))
        return y

    def pc_apply_host(self, nrhs: int, x_ptr: int, ldx: int, y_ptr: int, ldy: int, adjoint: bool, chunk: int,
                      stream_ptr: int):
        _check(lib().pc_apply_host(self.handle, ctypes.c_int32(nrhs), _VP(x_ptr), ctypes.c_int64(ldx), _VP(y_ptr),
                                   ctypes.c_int64(ldy), ctypes.c_int32(int(adjoint)), ctypes.c_int32(chunk),
                                   _VP(stream_ptr)), self.ctx.handle)

    def apply_host(self, x, out=None, adjoint: bool = False, chunk: int = 0, stream=None):
        """A~ x (or A~* x) for a CPU tensor x [B, *box] (pinned for overlap);
        returns a CPU tensor.  Waits for the result unless `out` is given
        (then the caller synchronises `stream`)."""
        import torch
        want = torch.float64 if self.precision == "fp64" else torch.float32
        if x.is_cuda or not x.is_contiguous() or x.dtype != want:
            raise ValueError("x must be a contiguous CPU tensor of %s" % want)
        B = x.numel() // self.N
        if B * self.N != x.numel():
            raise ValueError("x does not hold whole vectors of the operator's box")
        y = torch.empty(x.shape, dtype=want, pin_memory=x.is_pinned()) if out is None else out
        self.pc_apply_host(B, x.data_ptr(), self.N, y.data_ptr(), self.N, adjoint, chunk, _stream_ptr(stream))
        if out is None:
            (torch.cuda.current_stream() if stream is None else stream).synchronize()
        return y

    def entries(self, rows, cols, stream=None):
        """A~[rows[i], cols[i]] (flat indices; int64 CUDA tensors) as an FP64 CUDA tensor."""
        import torch
        rows = rows.to(device="cuda", dtype=torch.int64).contiguous()
        cols = cols.to(device="cuda", dtype=torch.int64).contiguous()
        if rows.numel() != cols.numel():
            raise ValueError("rows and cols must have the same length")
        out = torch.empty(rows.numel(), dtype=torch.float64, device="cuda")
        _check(lib().pc_entries(self.handle, ctypes.c_int64(rows.numel()), _VP(rows.data_ptr()), _VP(cols.data_ptr()),
                                _VP(out.data_ptr()), _VP(_stream_ptr(stream))), self.ctx.handle)
        return out

    def estimate_cell_errors(self, z, y, num_cells: int, stream=None) -> np.ndarray:
        """eta_C for every leaf cell (Section 2.6): z, y = A* z are contiguous
        CUDA tensors [q, *box] of the operator's precision."""
        for t, name in ((z, "z"), (y, "y")):
            if not (t.is_cuda and t.is_contiguous()):
                raise ValueError("%s must be a contiguous CUDA tensor" % name)
        q = z.numel() // self.N
        if y.numel() != q * self.N:
            raise ValueError("z and y must hold the same number of vectors")
        eta = np.zeros(num_cells)
        _check(lib().pc_estimate_cell_errors(self.handle, ctypes.c_int32(q), _VP(z.data_ptr()), ctypes.c_int64(self.N),
                                             _VP(y.data_ptr()), ctypes.c_int64(self.N),
                                             eta.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                             _VP(_stream_ptr(stream))), self.ctx.handle)
        return eta

    def apply_plain(self, x, out=None, stream=None):
        B, y = self._args(x, out)
        self.pc_apply_plain(B, x.data_ptr(), self.N, y.data_ptr(), self.N, _stream_ptr(stream))
        return y

    def close(self):
        if getattr(self, "handle", None):
            h, self.handle = self.handle, None
            _check(lib().pc_operator_destroy(h), self.ctx.handle)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Estimator:
    """Incremental randomized estimator (Algorithm 1): Z and Y = A* Z are
    CUDA tensors [q, *box] kept alive by this object; update(op) returns the
    per-cell estimates of op and the number of sample points whose
    correlations were recomputed."""

    def __init__(self, ctx: Context, shape, z, y, precision: str = "fp32"):
        self.ctx = ctx
        self.z, self.y = z.contiguous(), y.contiguous()
        N = int(np.prod(shape))
        q = self.z.numel() // N
        b = _box(shape)
        h = _VP()
        _check(lib().pc_estimator_create(ctx.handle, ctypes.byref(b), PRECISIONS[precision], ctypes.c_int32(q),
                                         _VP(self.z.data_ptr()), ctypes.c_int64(N), _VP(self.y.data_ptr()),
                                         ctypes.c_int64(N), ctypes.byref(h)), ctx.handle)
        self.handle = h
        self.recomputed_total = 0

    def update(self, op: "Operator", num_cells: int, stream=None):
        eta = np.zeros(num_cells, dtype=np.float64)
        rec = ctypes.c_int32()
        _check(lib().pc_estimator_update(self.handle, op.handle, eta.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                         ctypes.byref(rec), _VP(_stream_ptr(stream))), self.ctx.handle)
        self.recomputed_total += rec.value
        return eta, rec.value

    def close(self):
        if getattr(self, "handle", None):
            h, self.handle = self.handle, None
            _check(lib().pc_estimator_destroy(h), self.ctx.handle)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BlockPlan:
    """Block apply (Section 3.3): y_T = A~[T, S] x_S, or (A~*)[T, S] x_S with
    adjoint=True, for closed boxes T = [t_lo, t_hi], S = [s_lo, s_hi]
    (pc_block_plan_create / pc_block_apply).  Bounds given as [nblocks][2]
    arrays make a plan of several blocks that apply_many runs in one launch
    (pc_block_plan_create_many / pc_block_apply_many).  The operator must
    outlive the plan."""

    def __init__(self, op: Operator, t_lo, t_hi, s_lo, s_hi, adjoint: bool = False):
        self.op = op
        d = len(op.shape)
        box = [np.ascontiguousarray(np.asarray(b, dtype=np.int64).reshape(-1, d)) for b in (t_lo, t_hi, s_lo, s_hi)]
        self.nblocks = len(box[0])
        if any(len(b) != self.nblocks for b in box):
            raise ValueError("t_lo, t_hi, s_lo, s_hi must hold the same number of blocks")
        self.t_shapes = [tuple(int(v) for v in h - l + 1) for l, h in zip(box[0], box[1])]
        self.s_shapes = [tuple(int(v) for v in h - l + 1) for l, h in zip(box[2], box[3])]
        self.t_shape, self.s_shape = self.t_shapes[0], self.s_shapes[0]
        self.adjoint = bool(adjoint)
        h = _VP()
        _check(lib().pc_block_plan_create_many(op.handle, ctypes.c_int32(self.nblocks), *[_ptr(b) for b in box],
                                               ctypes.c_int32(int(adjoint)), ctypes.byref(h)), op.ctx.handle)
        self.handle = h

    def info(self):
        """(terms, tiles): distinct k and tiles the blocks touch (summed over blocks)."""
        terms, tiles = ctypes.c_int32(), ctypes.c_int32()
        _check(lib().pc_block_plan_info(self.handle, ctypes.byref(terms), ctypes.byref(tiles)))
        return terms.value, tiles.value

    def pc_block_apply(self, nrhs: int, x_ptr: int, ldx: int, y_ptr: int, ldy: int, stream_ptr: int):
        _check(lib().pc_block_apply(self.handle, ctypes.c_int32(nrhs), _VP(x_ptr), ctypes.c_int64(ldx),
                                    _VP(y_ptr), ctypes.c_int64(ldy), _VP(stream_ptr)), self.op.ctx.handle)

    def pc_block_apply_many(self, nrhs: int, x_ptrs, ldx, y_ptrs, ldy, stream_ptr: int):
        n = self.nblocks
        xs = (_VP * n)(*[_VP(v) for v in x_ptrs])
        ys = (_VP * n)(*[_VP(v) for v in y_ptrs])
        lx = (ctypes.c_int64 * n)(*ldx)
        ly = (ctypes.c_int64 * n)(*ldy)
        _check(lib().pc_block_apply_many(self.handle, ctypes.c_int32(nrhs), xs, lx, ys, ly, _VP(stream_ptr)),
               self.op.ctx.handle)

    def _dtype(self):
        import torch
        return torch.float64 if self.op.precision == "fp64" else torch.float32

    def apply(self, x, out=None, stream=None):
        """Single-block plans: x is a contiguous CUDA tensor [B, *S] (or [*S]); returns [B, *T] (or [*T])."""
        import torch
        nS, nT = int(np.prod(self.s_shape)), int(np.prod(self.t_shape))
        want = self._dtype()
        if not (x.is_cuda and x.is_contiguous()) or x.dtype != want:
            raise ValueError("x must be a contiguous CUDA tensor of %s" % want)
        B = x.numel() // nS
        if B * nS != x.numel():
            raise ValueError("x does not hold whole vectors on S")
        shape = (B,) + self.t_shape if x.dim() > len(self.s_shape) else self.t_shape
        y = torch.empty(shape, dtype=want, device=x.device) if out is None else out
        self.pc_block_apply(B, x.data_ptr(), nS, y.data_ptr(), nT, _stream_ptr(stream))
        return y

    def apply_many(self, xs, stream=None):
        """xs: one contiguous CUDA tensor [B, *S_i] per block; returns the [B, *T_i] results."""
        import torch
        want = self._dtype()
        if len(xs) != self.nblocks:
            raise ValueError("one x per block")
        B = xs[0].shape[0]
        ys = []
        for x, sS, sT in zip(xs, self.s_shapes, self.t_shapes):
            if not (x.is_cuda and x.is_contiguous()) or x.dtype != want or tuple(x.shape) != (B,) + sS:
                raise ValueError("each x must be a contiguous CUDA tensor [B, *S_i] of %s" % want)
            ys.append(torch.empty((B,) + sT, dtype=want, device=x.device))
        self.pc_block_apply_many(B, [x.data_ptr() for x in xs], [int(np.prod(s)) for s in self.s_shapes],
                                 [y.data_ptr() for y in ys], [int(np.prod(t)) for t in self.t_shapes],
                                 _stream_ptr(stream))
        return ys

    def check(self):
        _check(lib().pc_block_plan_check(self.handle), self.op.ctx.handle)

    def close(self):
        if getattr(self, "handle", None):
            h, self.handle = self.handle, None
            _check(lib().pc_block_plan_destroy(h), self.op.ctx.handle)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pc_autotune(ctx: Context, shape, cells, radius: int, impulse: np.ndarray, precision: str = "fp32",
                nrhs: int = 8, weights: Optional[np.ndarray] = None):
    """Fastest launch shape (dict of pc_tuning fields) and its ms per batch of nrhs."""
    b = _box(shape)
    g, keep = _grid(cells)
    imp = np.ascontiguousarray(impulse, dtype=np.float64)
    wts = None if weights is None else np.ascontiguousarray(weights, dtype=np.float64)
    best = pc_tuning()
    ms = ctypes.c_double()
    _check(lib().pc_autotune(ctx.handle, ctypes.byref(b), ctypes.byref(g), ctypes.c_int32(radius), _ptr(imp),
                             _ptr(wts), PRECISIONS[precision], ctypes.c_int32(nrhs), ctypes.byref(best),
                             ctypes.byref(ms)), ctx.handle)
    del keep
    return {"fft_size": best.fft_size, "tile": best.tile, "ctas_per_sm": best.ctas_per_sm,
            "window_split": best.window_split}, ms.value


class Server:
    """pc_serve_*: batched serving of apply requests on resident operators."""

    def __init__(self, ctx: Context, budget_bytes: int, max_inflight: int = 256, streams: int = 2,
                 max_requests_per_launch: int = 32):
        self.ctx = ctx
        cfg = pc_serve_config()
        cfg.hbm_budget_bytes = int(budget_bytes)
        cfg.max_inflight = max_inflight
        cfg.streams = streams
        cfg.max_requests_per_launch = max_requests_per_launch
        h = _VP()
        _check(lib().pc_serve_create(ctx.handle, ctypes.byref(cfg), ctypes.byref(h)), ctx.handle)
        self.handle = h
        self._keep = {}

    def submit(self, op: "Operator", x, y, adjoint: bool = False) -> int:
        """Queue y = A~ x, or y = A~* x with adjoint=True (x, y: contiguous
        float32 CUDA tensors [nrhs, *box]).  The tensors are kept alive until
        poll() reports the ticket done."""
        nrhs = x.numel() // op.N
        t = ctypes.c_uint64()
        _check(lib().pc_serve_submit(self.handle, op.handle, ctypes.c_int32(nrhs), _VP(x.data_ptr()),
                                     _VP(y.data_ptr()), ctypes.c_uint32(PC_SERVE_ADJOINT if adjoint else 0),
                                     ctypes.byref(t)), self.ctx.handle)
        self._keep[t.value] = (x, y)
        return t.value

    def poll(self, ticket: int):
        """None while not ready, else the completion record (dict)."""
        info = pc_request_info()
        st = lib().pc_serve_poll(self.handle, ctypes.c_uint64(ticket), ctypes.byref(info))
        if st == PC_ERR_NOT_READY:
            return None
        self._keep.pop(ticket, None)
        _check(st, self.ctx.handle)
        return {f: getattr(info, f) for f, _ in info._fields_ if f != "reserved"}

    def stats(self) -> dict:
        st = pc_serve_stats()
        _check(lib().pc_serve_stats_get(self.handle, ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in st._fields_}

    def close(self):
        if getattr(self, "handle", None):
            lib().pc_serve_destroy(self.handle)
            self.handle = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
