"""Shared helpers of the GPU parity tests (inputs from synth, expectations from oracle)."""
import numpy as np

import oracle
import synth

TOL_BEAM = 1e-5     # max |P_gpu - P_ref| / P_ref over beams (FP32 form)


def make_case(nx, ny, mx, my, npol, nfreq, T, n_int, weights="uniform", seed=0, nsrc=1,
              amp=1.5, sigma=2.5):
    src = synth.seeded_sources(seed + 100, nsrc, amp)
    v = synth.volts(T, nfreq, npol, nx, ny, seed=seed, sigma=sigma, sources=src)
    if weights == "uniform":
        w = None
    elif weights == "half_sine":
        w = synth.separable_weights(synth.half_sine(nx), synth.half_sine(ny))
    elif weights == "random":
        w = synth.random_weights(nx, ny, seed + 7)
    else:
        w = np.asarray(weights, dtype=np.complex64)
    return v, w


def oracle_beams(v, w, nx, ny, mx, my, npol, nfreq, n_int, route="separable"):
    w64 = None if w is None else np.asarray(w).astype(np.complex128)
    return oracle.beams(v, nx, ny, mx, my, npol, nfreq, n_int, weights=w64, route=route)


def rel_err_per_beam(got, ref):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return np.abs(got - ref) / np.abs(ref)


def rel_err_of_mean(got, ref):
    """|P_gpu - P_ref| normalised by the mean beam power of the same (window, channel)."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    mean = ref.mean(axis=(-2, -1), keepdims=True)
    return np.abs(got - ref) / np.where(mean > 0, mean, 1.0)


def parseval_totals(v, w, n_int, mx, my):
    """Total power of every (window, channel) over the full padded grid by Parseval:
    mx * my * sum_{t in window, p, ix, iy} |w x|^2 (valid when mx >= nx and my >= ny, so
    nothing folds). v: uint8 [T][F][P][nx][ny]; w: complex [nx][ny] or None (all ones).
    |x|^2 per byte value comes from the oracle's unpack."""
    v = np.asarray(v)
    T, F, P, nx, ny = v.shape
    lut = np.abs(oracle.unpack(np.arange(256, dtype=np.uint8))) ** 2
    w2 = np.ones((nx, ny)) if w is None else np.abs(np.asarray(w, dtype=np.complex128)) ** 2
    e = lut[v].reshape(T // n_int, n_int, F, P, nx, ny).sum(axis=(1, 3))   # [J][F][nx][ny]
    return mx * my * np.einsum("jfab,ab->jf", e, w2)
