"""Seeded synthetic inputs shared by the oracle tests, the CUDA parity tests and bench.py.

This package draws inputs only; it holds none of the beamforming arithmetic. The
voltage generator is a small C library (``synth.c``) compiled on first use with gcc,
because the CHIME-like workload needs billions of Gaussian draws.

Workload recipes (the paper uses no dataset; these stand in for a CHIME-like lattice):
see :data:`WORKLOADS`.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libfftbf_synth.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile synth.c into a shared library next to it; return its path."""
    src = os.path.join(_HERE, "synth.c")
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(src):
        return _LIB
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread",
                           src, "-o", tmp, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.synth_volts.restype = ctypes.c_int
            lib.synth_volts.argtypes = [
                ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.c_double, ctypes.c_int,
                ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
            lib.synth_splitmix64_draw.restype = ctypes.c_uint64
            lib.synth_splitmix64_draw.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            _lib = lib
    return _lib


def splitmix64_draw(state: int, k: int) -> int:
    """Draw k (k >= 1) of the SplitMix64 stream started at ``state`` (C implementation)."""
    return int(_load().synth_splitmix64_draw(state, k))


def volts(nt, nfreq, npol, nx, ny, seed, sigma=2.5, sources=(), t0=0, nthreads=None,
          out=None) -> np.ndarray:
    """Quantised int4+4 voltages, uint8 [nt][nfreq][npol][nx][ny].

    ``sources`` is a sequence of (u, v, amplitude) with u, v in lattice units
    ((d/lambda) sin(theta) per axis). ``out`` may be a preallocated (e.g. pinned) uint8
    array of the right size.
    """
    shape = (nt, nfreq, npol, nx, ny)
    if out is None:
        out = np.empty(shape, dtype=np.uint8)
    else:
        assert out.dtype == np.uint8 and out.size == int(np.prod(shape)) and out.flags.c_contiguous
        out = out.reshape(shape)
    src = np.asarray(sources, dtype=np.float64).reshape(-1, 3)
    u = np.ascontiguousarray(src[:, 0])
    v = np.ascontiguousarray(src[:, 1])
    a = np.ascontiguousarray(src[:, 2])
    if nthreads is None:
        nthreads = os.cpu_count() or 1
    rc = _load().synth_volts(out.ctypes.data, t0, nt, nfreq, npol, nx, ny,
                             seed & 0xFFFFFFFFFFFFFFFF, sigma, len(src),
                             u.ctypes.data, v.ctypes.data, a.ctypes.data, nthreads)
    if rc != 0:
        raise ValueError("synth_volts rejected its arguments")
    return out


def seeded_sources(seed: int, n: int, amplitude: float):
    """n plane-wave sources at seeded directions (u, v) uniform in [0, 1)^2."""
    rng = np.random.default_rng(seed)
    uv = rng.random((n, 2))
    return [(float(uv[i, 0]), float(uv[i, 1]), float(amplitude)) for i in range(n)]


def half_sine(n: int) -> np.ndarray:
    """The half-sine window h^a = sin[pi (a + 1/2) / n] of Section 4.1 (FP64)."""
    a = np.arange(n, dtype=np.float64)
    return np.sin(np.pi * (a + 0.5) / n)


def separable_weights(hx, hy) -> np.ndarray:
    """Complex64 weights [nx][ny] = hx[ix] * hy[iy] (real window on both axes)."""
    w = np.outer(np.asarray(hx, np.float64), np.asarray(hy, np.float64))
    return w.astype(np.complex64)


def random_weights(nx, ny, seed) -> np.ndarray:
    """Seeded general complex per-feed weights (amplitude and phase), complex64 [nx][ny]."""
    rng = np.random.default_rng(seed)
    amp = 0.5 + rng.random((nx, ny))
    ph = rng.uniform(-np.pi, np.pi, (nx, ny))
    return (amp * np.exp(1j * ph)).astype(np.complex64)


def tied_pointings(seed, nfreq, n_tied, nx, ny, pad_x, pad_y):
    """Seeded tied-array pointings u, v: FP64 [nfreq][n_tied], the same at every frequency.

    On an axis whose padding is below 2n-1 the pointing is drawn on the FFT-beam grid
    (u * M an integer); otherwise it is uniform in [0, 1).
    """
    rng = np.random.default_rng(seed)

    def axis(n, m):
        if m >= 2 * n - 1:
            return rng.random(n_tied)
        return rng.integers(0, m, n_tied).astype(np.float64) / m

    u = axis(nx, pad_x)
    v = axis(ny, pad_y)
    return (np.ascontiguousarray(np.broadcast_to(u, (nfreq, n_tied))),
            np.ascontiguousarray(np.broadcast_to(v, (nfreq, n_tied))))


def next_pow2(n: int) -> int:
    p = 1
    while p < n:
        p *= 2
    return p


# Workload recipes, one per configuration of the benchmark suite. Seeds are fixed per
# workload. "sigma" is per real component; sources are (u, v, amplitude).
WORKLOADS = {
    "tiny": dict(nx=2, ny=16, pad_x=2, pad_y=32, npol=1, nfreq=8, T=1024, n_int=16,
                 sigma=2.5, n_src=1, amp=1.5, weights="uniform", seed=1),
    "chime": dict(nx=4, ny=256, pad_x=4, pad_y=512, npol=2, nfreq=1024, T=49152, n_int=384,
                  sigma=2.5, n_src=3, amp=1.5, weights="half_sine", seed=2, n_tied=2048),
    "chime_tc": dict(nx=4, ny=256, pad_x=4, pad_y=512, npol=2, nfreq=1024, T=49152,
                     n_int=384, sigma=2.5, n_src=3, amp=1.5, weights="half_sine", seed=3,
                     n_tied=2048),
}

# Lattice menu of the batched-uneven workload (nx, ny); N-S padded to 2x next pow2.
BATCH_LATTICES = [(4, 256), (8, 64), (16, 16), (2, 512), (1, 1024), (3, 128)]


def workload_weights(wl: dict) -> np.ndarray | None:
    if wl["weights"] == "uniform":
        return None
    if wl["weights"] == "half_sine":
        return separable_weights(half_sine(wl["nx"]), half_sine(wl["ny"]))
    raise ValueError(wl["weights"])
