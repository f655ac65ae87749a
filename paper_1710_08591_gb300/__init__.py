"""FFT beamforming of a regular antenna lattice on GB300 (arXiv 1710.08591).

Thin ctypes binding of ``libfftbf.so`` (C ABI in ``include/fftbf.h``). The functions
keep the C names without the ``fftbf_`` prefix and only marshal arguments: every step
of the computation runs in the library's CUDA kernels. There is no CPU fallback; if the
library is missing, :func:`lib` raises.

Device buffers may be passed as torch CUDA tensors or as integer device addresses;
host buffers as numpy arrays. Streams may be a ``torch.cuda.Stream``, an integer
``cudaStream_t`` or None (torch's current stream when torch is imported, else the
legacy default stream).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

__all__ = ["lib", "build", "FFTBF_OK", "PREC_FP32", "PREC_TC_FP16", "PREC_TC_BF16", "PREC_TC_FP16X3",
           "FftbfError", "Plan", "plan_create", "plan_set_precision", "execute", "execute_host", "tied_beams", "tied_set_window", "stacked_shape",
           "stacked_visibilities", "localise",
           "plan_sync", "destroy", "last_error", "last_error_code", "debug_unpack", "execute_noalloc", "debug_tc_gemm", "debug_wait_timeout", "probe_fp32", "Batch", "batch_create",
           "batch_execute", "batch_tuned_steps", "batch_grid", "batch_destroy", "Server", "server_create",
           "server_submit", "server_hold", "server_wait", "server_stats", "server_destroy"]

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libfftbf.so")

FFTBF_OK = 0
PREC_FP32, PREC_TC_FP16, PREC_TC_BF16, PREC_TC_FP16X3 = 0, 1, 2, 3
_STATUS = {0: "OK", -1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ETIMEOUT", -5: "EUNSUPPORTED"}

_lock = threading.Lock()
_lib = None


class FftbfError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"fftbf {_STATUS.get(code, code)}: {msg}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile the CUDA library for sm_103a (in-tree)."""
    from . import buildlib as _b
    return _b.build(force=force)


def lib() -> ctypes.CDLL:
    """Load libfftbf.so; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: run paper_1710_08591_gb300.build() "
                                   "(the library has no CPU fallback)")
            L = ctypes.CDLL(LIB_PATH)
            c_int, c_i64, vp = ctypes.c_int, ctypes.c_int64, ctypes.c_void_p
            L.fftbf_plan_create.restype = vp
            L.fftbf_plan_create.argtypes = [c_int] * 7 + [vp]
            L.fftbf_plan_set_precision.restype = c_int
            L.fftbf_plan_set_precision.argtypes = [vp, c_int]
            L.fftbf_execute.restype = c_int
            L.fftbf_execute.argtypes = [vp, vp, c_i64, vp, vp]
            L.fftbf_tied_beams.restype = c_int
            L.fftbf_tied_beams.argtypes = [vp, vp, c_i64, c_int, vp, vp, vp, vp]
            L.fftbf_tied_set_window.restype = c_int
            L.fftbf_tied_set_window.argtypes = [vp, vp, vp, c_int, c_int]
            L.fftbf_stacked_shape.restype = c_int
            L.fftbf_stacked_shape.argtypes = [vp, vp, vp]
            L.fftbf_stacked_visibilities.restype = c_int
            L.fftbf_stacked_visibilities.argtypes = [vp, vp, c_i64, vp, vp]
            L.fftbf_localise.restype = c_int
            L.fftbf_localise.argtypes = [vp, vp, c_i64, c_int, c_int, vp, vp]
            L.fftbf_execute_host.restype = c_int
            L.fftbf_execute_host.argtypes = [vp, vp, c_i64, vp, c_int, vp, vp, vp, vp]
            L.fftbf_plan_sync.restype = c_int
            L.fftbf_plan_sync.argtypes = [vp]
            L.fftbf_destroy.restype = None
            L.fftbf_destroy.argtypes = [vp]
            L.fftbf_last_error.restype = ctypes.c_char_p
            L.fftbf_last_error.argtypes = []
            L.fftbf_last_error_code.restype = c_int
            L.fftbf_last_error_code.argtypes = []
            L.fftbf_execute_noalloc.restype = c_int
            L.fftbf_execute_noalloc.argtypes = [c_int] * 7 + [vp, vp, c_i64, vp, vp]
            L.fftbf_batch_create.restype = vp
            L.fftbf_batch_create.argtypes = [vp, c_int]
            L.fftbf_batch_execute.restype = c_int
            L.fftbf_batch_execute.argtypes = [vp, vp, c_i64, vp, vp]
            L.fftbf_batch_tuned_steps.restype = c_int
            L.fftbf_batch_tuned_steps.argtypes = [vp, c_int]
            L.fftbf_probe_fp32.restype = c_int
            L.fftbf_probe_fp32.argtypes = [c_int, c_i64, c_int, vp, vp, vp]
            L.fftbf_batch_grid.restype = c_int
            L.fftbf_batch_grid.argtypes = [vp]
            L.fftbf_batch_destroy.restype = None
            L.fftbf_batch_destroy.argtypes = [vp]
            L.fftbf_server_create.restype = vp
            L.fftbf_server_create.argtypes = [vp, c_int, c_i64]
            L.fftbf_server_submit.restype = c_i64
            L.fftbf_server_submit.argtypes = [vp, c_int, vp, vp]
            L.fftbf_server_hold.restype = c_int
            L.fftbf_server_hold.argtypes = [vp, c_int]
            L.fftbf_server_wait.restype = c_int
            L.fftbf_server_wait.argtypes = [vp, c_i64, ctypes.c_double]
            L.fftbf_server_stats.restype = c_int
            L.fftbf_server_stats.argtypes = [vp, vp]
            L.fftbf_server_destroy.restype = None
            L.fftbf_server_destroy.argtypes = [vp]
            L.fftbf_debug_wait_timeout.restype = c_int
            L.fftbf_debug_wait_timeout.argtypes = [c_int, vp]
            L.fftbf_debug_tc_gemm.restype = c_int
            L.fftbf_debug_tc_gemm.argtypes = [vp, vp, c_int, c_int, c_int, vp, vp]
            L.fftbf_debug_unpack.restype = c_int
            L.fftbf_debug_unpack.argtypes = [vp, c_i64, vp, vp]
            _lib = L
    return _lib


def last_error() -> str:
    return lib().fftbf_last_error().decode()


def last_error_code() -> int:
    return int(lib().fftbf_last_error_code())


def _check(rc: int) -> int:
    if rc != FFTBF_OK:
        raise FftbfError(rc, last_error())
    return rc


def _dptr(x) -> int:
    """Device address of a torch CUDA tensor, or an int address."""
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_cuda:
            raise ValueError("expected a CUDA tensor")
        if not x.is_contiguous():
            raise ValueError("expected a contiguous tensor")
        return x.data_ptr()
    raise TypeError(f"cannot take a device pointer of {type(x)}")


def _stream(s) -> int:
    if s is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return 0
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _host_f64(a, n) -> np.ndarray:
    arr = np.ascontiguousarray(a, dtype=np.float64)
    if arr.size != n:
        raise ValueError(f"expected {n} values, got {arr.size}")
    return arr


class Plan:
    """Owning handle of an ``fftbf_plan``."""

    def __init__(self, nx, ny, pad_x, pad_y, npol, nfreq, n_int, weights=None):
        w = None
        if weights is not None:
            w = np.ascontiguousarray(np.asarray(weights).astype(np.complex64)).reshape(-1)
            if w.size != nx * ny:
                raise ValueError("weights must have nx*ny complex entries")
        self.shape = dict(nx=nx, ny=ny, pad_x=pad_x, pad_y=pad_y, npol=npol, nfreq=nfreq,
                          n_int=n_int)
        self._weights = w
        h = lib().fftbf_plan_create(nx, ny, pad_x, pad_y, npol, nfreq, n_int,
                                    None if w is None else w.ctypes.data)
        if not h:
            raise FftbfError(last_error_code(), last_error())
        self.handle = h

    def __getattr__(self, k):
        shape = self.__dict__.get("shape")
        if shape is not None and k in shape:
            return shape[k]
        raise AttributeError(k)

    def close(self):
        h, self.handle = getattr(self, "handle", None), None
        if h:
            lib().fftbf_destroy(h)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def plan_create(nx, ny, pad_x, pad_y, npol, nfreq, n_int, weights=None) -> Plan:
    return Plan(nx, ny, pad_x, pad_y, npol, nfreq, n_int, weights)


def plan_set_precision(plan: Plan, precision: int) -> None:
    _check(lib().fftbf_plan_set_precision(plan.handle, precision))


def execute(plan: Plan, volts, T: int, beams, stream=None) -> None:
    """Integrated FFT-beam intensities: beams[T/n_int][nfreq][pad_x][pad_y] (device)."""
    _check(lib().fftbf_execute(plan.handle, _dptr(volts), int(T), _dptr(beams), _stream(stream)))


def tied_beams(plan: Plan, beams, n_windows: int, n_tied: int, u, v, tied, stream=None) -> None:
    """Tied-array beams tied[n_windows][nfreq][n_tied] (device) from FFT-beam intensities."""
    n = plan.nfreq * n_tied
    uu, vv = _host_f64(u, n), _host_f64(v, n)
    _check(lib().fftbf_tied_beams(plan.handle, _dptr(beams), int(n_windows), int(n_tied),
                                  uu.ctypes.data, vv.ctypes.data, _dptr(tied), _stream(stream)))


def tied_set_window(plan: Plan, hx=None, hy=None, trunc_x: int = 0, trunc_y: int = 0) -> None:
    """Optimal windowed tied beams (real windows per axis) and/or truncated kernels."""
    ax = None if hx is None else _host_f64(hx, plan.nx)
    ay = None if hy is None else _host_f64(hy, plan.ny)
    _check(lib().fftbf_tied_set_window(plan.handle, None if ax is None else ax.ctypes.data,
                                       None if ay is None else ay.ctypes.data, int(trunc_x),
                                       int(trunc_y)))


def stacked_shape(plan: Plan) -> tuple[int, int]:
    dx, dy = ctypes.c_int(), ctypes.c_int()
    _check(lib().fftbf_stacked_shape(plan.handle, ctypes.byref(dx), ctypes.byref(dy)))
    return dx.value, dy.value


def stacked_visibilities(plan: Plan, beams, n_windows: int, vis, stream=None) -> None:
    """Redundancy-stacked visibilities from FFT-beam intensities into `vis` (device,
    complex64 [n_windows][nfreq][Dx][Dy], Dx, Dy = stacked_shape(plan))."""
    _check(lib().fftbf_stacked_visibilities(plan.handle, _dptr(beams), int(n_windows), _dptr(vis),
                                            _stream(stream)))


def localise(plan: Plan, beams, n_windows: int, out, n_iter: int = 5, n_taps: int = 10,
             stream=None) -> None:
    """Point-source position per (window, channel) into `out` (device float [n_windows][nfreq][3])."""
    _check(lib().fftbf_localise(plan.handle, _dptr(beams), int(n_windows), int(n_iter), int(n_taps),
                                _dptr(out), _stream(stream)))


def execute_host(plan: Plan, volts: np.ndarray, T: int, beams: np.ndarray, n_tied: int = 0,
                 u=None, v=None, tied: np.ndarray | None = None, stream=None) -> None:
    """fftbf_execute (+ fftbf_tied_beams) on host numpy buffers; stream-ordered."""
    for a in (volts, beams) + ((tied,) if n_tied else ()):
        if not (isinstance(a, np.ndarray) and a.flags.c_contiguous):
            raise ValueError("host buffers must be C-contiguous numpy arrays")
    uu = vv = None
    if n_tied:
        n = plan.nfreq * n_tied
        uu, vv = _host_f64(u, n), _host_f64(v, n)
    _check(lib().fftbf_execute_host(
        plan.handle, volts.ctypes.data, int(T), beams.ctypes.data, int(n_tied),
        None if uu is None else uu.ctypes.data, None if vv is None else vv.ctypes.data,
        None if tied is None else tied.ctypes.data, _stream(stream)))


class Batch:
    """Owning handle of an ``fftbf_batch`` over a list of plans (kept alive here)."""

    def __init__(self, plans):
        self.plans = list(plans)
        arr = (ctypes.c_void_p * len(self.plans))(*[p.handle for p in self.plans])
        h = lib().fftbf_batch_create(arr, len(self.plans))
        if not h:
            raise FftbfError(last_error_code(), last_error())
        self.handle = h

    def close(self):
        h, self.handle = getattr(self, "handle", None), None
        if h:
            lib().fftbf_batch_destroy(h)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def batch_create(plans) -> Batch:
    return Batch(plans)


def batch_execute(batch: Batch, volts, T: int, beams, stream=None) -> None:
    """One persistent launch over all plans of the batch; volts/beams: sequences of device
    buffers, one per plan."""
    n = len(batch.plans)
    if len(volts) != n or len(beams) != n:
        raise ValueError(f"need {n} voltage and beam buffers")
    va = (ctypes.c_void_p * n)(*[_dptr(v) for v in volts])
    ba = (ctypes.c_void_p * n)(*[_dptr(b) for b in beams])
    _check(lib().fftbf_batch_execute(batch.handle, va, int(T), ba, _stream(stream)))


def batch_tuned_steps(batch: Batch, i: int) -> int:
    r = lib().fftbf_batch_tuned_steps(batch.handle, i)
    if r < 0:
        raise FftbfError(r, last_error())
    return r


def batch_grid(batch: Batch) -> int:
    """CTAs of each batched launch (work items beyond it are taken from the queue in turn)."""
    return int(lib().fftbf_batch_grid(batch.handle))


def batch_destroy(batch: Batch) -> None:
    batch.close()


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("launches", ctypes.c_int64), ("peak_inflight", ctypes.c_int64),
                ("slots", ctypes.c_int64), ("max_frames_per_launch", ctypes.c_int64),
                ("max_items_per_launch", ctypes.c_int64), ("grid", ctypes.c_int64),
                ("frames_per_launch", ctypes.c_double),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("max_ms", ctypes.c_double), ("mean_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Server:
    """Owning handle of an ``fftbf_server`` (continuous batching of voltage frames)."""

    def __init__(self, lattices, hbm_budget_bytes):
        self.lattices = list(lattices)
        arr = (ctypes.c_void_p * len(self.lattices))(*[p.handle for p in self.lattices])
        h = lib().fftbf_server_create(arr, len(self.lattices), int(hbm_budget_bytes))
        if not h:
            raise FftbfError(last_error_code(), last_error())
        self.handle = h
        self._keep = {}

    def close(self):
        h, self.handle = getattr(self, "handle", None), None
        if h:
            lib().fftbf_server_destroy(h)
        self._keep = {}

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def server_create(lattices, hbm_budget_bytes) -> Server:
    return Server(lattices, hbm_budget_bytes)


def server_submit(server: Server, lattice: int, frame: np.ndarray, beams: np.ndarray) -> int:
    """Queue one frame (host uint8 array); the beams land in `beams` (host float32) on
    completion. Both arrays are kept alive by the server handle until it is closed."""
    for a in (frame, beams):
        if not (isinstance(a, np.ndarray) and a.flags.c_contiguous):
            raise ValueError("frames and beams must be C-contiguous numpy arrays")
    t = lib().fftbf_server_submit(server.handle, int(lattice), frame.ctypes.data, beams.ctypes.data)
    if t < 0:
        raise FftbfError(int(t), last_error())
    server._keep[t] = (frame, beams)
    return int(t)


def server_hold(server: Server, hold: bool) -> None:
    """Stage frames without launching while `hold` is true; releasing launches them together."""
    _check(lib().fftbf_server_hold(server.handle, 1 if hold else 0))


def server_wait(server: Server, ticket: int = -1, timeout_s: float = 60.0) -> None:
    _check(lib().fftbf_server_wait(server.handle, int(ticket), float(timeout_s)))
    if ticket >= 0:
        server._keep.pop(ticket, None)
    else:
        server._keep.clear()


def server_stats(server: Server) -> dict:
    st = ServerStats()
    _check(lib().fftbf_server_stats(server.handle, ctypes.byref(st)))
    return st.as_dict()


def server_destroy(server: Server) -> None:
    server.close()


def plan_sync(plan: Plan) -> None:
    _check(lib().fftbf_plan_sync(plan.handle))


def destroy(plan: Plan) -> None:
    plan.close()


def execute_noalloc(nx, ny, pad_x, pad_y, npol, nfreq, n_int, weights, volts, T: int, beams,
                    stream=None) -> None:
    """fftbf_execute without a plan or any device allocation (tables in static device
    memory); weights is a device tensor of nx*ny complex64 values or None."""
    _check(lib().fftbf_execute_noalloc(nx, ny, pad_x, pad_y, npol, nfreq, n_int, _dptr(weights),
                                       _dptr(volts), int(T), _dptr(beams), _stream(stream)))


def probe_fp32(packed: bool, iters: int, blocks: int, out, stream=None) -> float:
    """Launch the FP32 throughput probe (scalar FFMA or packed FFMA2) on `stream`; returns
    the flops the launch performs. `out`: device float tensor of blocks * 256 elements."""
    fl = ctypes.c_double(0.0)
    _check(lib().fftbf_probe_fp32(1 if packed else 0, int(iters), int(blocks), _dptr(out),
                                  ctypes.byref(fl), _stream(stream)))
    return fl.value


def debug_wait_timeout(limit_us: int, stream=None) -> int:
    """Run the bounded-wait test kernel; returns the status (FFTBF_ETIMEOUT expected)."""
    return int(lib().fftbf_debug_wait_timeout(int(limit_us), _stream(stream)))


def debug_tc_gemm(a, b, n: int, bf16: bool, padded: int, d, stream=None) -> None:
    """D[128][n] = A[128][32] B[n][32]^T on the tensor cores (test hook). padded: 0 K-major
    A, 1 K-major A with the stage-2 operand's padded strides, 2 MN-major A, 3 A in tensor
    memory, 4 MN-major B (3 and 4: n <= 128)."""
    _check(lib().fftbf_debug_tc_gemm(_dptr(a), _dptr(b), int(n), int(bool(bf16)), int(padded),
                                     _dptr(d), _stream(stream)))


def debug_unpack(inp, n: int, out, stream=None) -> None:
    _check(lib().fftbf_debug_unpack(_dptr(inp), int(n), _dptr(out), _stream(stream)))
