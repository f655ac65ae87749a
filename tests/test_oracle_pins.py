"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each pin is a function of the oracle module, so that the planted-mistake tests at the
bottom can run the same pins against a deliberately broken copy and see one fail.
"""
import os
import types

import numpy as np
import pytest

import oracle
from oracle import fftbf_oracle as O
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rng(seed):
    return np.random.default_rng(seed)


def _cnoise(rng, shape):
    return rng.normal(size=shape) + 1j * rng.normal(size=shape)


def _golden_printed():
    out = {}
    with open(os.path.join(GOLDEN, "paper_printed.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                k, v, tol = line.split()[:3]
                out[k] = (float(v), float(tol))
    return out


def dirichlet(n, y):
    """sin^2(n pi y) / sin^2(pi y) with its limit n^2 at integer y (Eq. pointed_beam_shape)."""
    y = np.asarray(y, dtype=np.float64)
    s = np.sin(np.pi * y)
    near = np.abs(s) < 1e-12
    safe = np.where(near, 1.0, s)
    return np.where(near, float(n * n), np.sin(n * np.pi * y) ** 2 / safe ** 2)


# --------------------------------------------------------------------------- pins ----
def pin_unpack_examples(o):
    rows = []
    with open(os.path.join(GOLDEN, "unpack_examples.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                b, re, im = line.split()
                rows.append((int(b, 16), int(re), int(im)))
    got = o.unpack(np.array([r[0] for r in rows], dtype=np.uint8))
    return bool(np.all(got.real == [r[1] for r in rows]) and
                np.all(got.imag == [r[2] for r in rows]))


def pin_unpack_exhaustive(o):
    b = np.arange(256, dtype=np.uint16).astype(np.uint8)
    # independent decode: place each nibble in the top of a signed byte, shift arithmetically
    re = (b & 0xF0).view(np.int8) >> 4
    im = ((b << 4) & 0xF0).astype(np.uint8).view(np.int8) >> 4
    got = o.unpack(b)
    return bool(np.array_equal(got.real, re.astype(np.float64)) and
                np.array_equal(got.imag, im.astype(np.float64)))


def pin_numpy_fft(o, nx=3, ny=5, mx=4, my=16, seed=0):
    """Direct sums against the library FFT of the zero-padded (or folded) weighted field."""
    rng = _rng(seed)
    x = _cnoise(rng, (2, nx, ny))
    w = _cnoise(rng, (nx, ny))
    got = o.field_separable(x, w, mx, my)
    got2 = o.field_direct(x, w, mx, my)
    wx = w * x
    grid = np.zeros((2, mx, my), dtype=np.complex128)
    for ix in range(nx):          # cyclic co-adding when M < n (Section 3.2), padding otherwise
        for iy in range(ny):
            grid[:, ix % mx, iy % my] += wx[:, ix, iy]
    ref = np.fft.fft2(grid)
    return bool(np.allclose(got, ref, rtol=0, atol=1e-11) and
                np.allclose(got2, ref, rtol=0, atol=1e-11))


def pin_routes(o, nx=3, ny=4, mx=5, my=8, n_int=3, seed=1):
    """Direct 2-D = separable = visibility route = stacked-visibility route (Eq. b2n-1)."""
    rng = _rng(seed)
    x = _cnoise(rng, (2 * n_int, 2, 2, nx, ny))
    w = _cnoise(rng, (nx, ny))
    a = o.beams_from_field(x, w, mx, my, n_int, route="direct")
    b = o.beams_from_field(x, w, mx, my, n_int, route="separable")
    c = o.beams_via_visibilities(x, w, mx, my, n_int)
    d = o.beams_via_stacked(x, w, mx, my, n_int)
    scale = np.abs(a).max()
    return bool(all(np.abs(q - a).max() <= 1e-12 * scale for q in (b, c, d)))


def pin_parseval(o, nx=4, ny=6, mx=4, my=12, seed=2):
    """sum_{A,B} P = Mx My sum |w x|^2 when M >= n on both axes (Parseval)."""
    rng = _rng(seed)
    x = _cnoise(rng, (4, 1, 2, nx, ny))
    w = _cnoise(rng, (nx, ny))
    P = o.beams_from_field(x, w, mx, my, 4)
    rhs = mx * my * np.sum(np.abs(w * x) ** 2)
    return bool(abs(P.sum() - rhs) <= 1e-12 * rhs)


def pin_plane_wave(o, nx=4, ny=8, mx=6, my=16, n_int=2, seed=3):
    """A plane wave c exp(+2 pi i (ix u + iy v)) gives
    P[A,B] = n_int npol |c|^2 D_nx(u - A/Mx) D_ny(v - B/My) (Eq. pointed_beam_shape)."""
    rng = _rng(seed)
    u, v = rng.random(2)
    c = 1.3 * np.exp(1j * 0.7)
    ix = np.arange(nx)[:, None]
    iy = np.arange(ny)[None, :]
    snap = c * np.exp(2j * np.pi * (ix * u + iy * v))
    x = np.broadcast_to(snap, (n_int, 1, 2, nx, ny)).copy()
    P = o.beams_from_field(x, None, mx, my, n_int)[0, 0]
    A = np.arange(mx)[:, None]
    B = np.arange(my)[None, :]
    ref = n_int * 2 * abs(c) ** 2 * dirichlet(nx, u - A / mx) * dirichlet(ny, v - B / my)
    return bool(np.allclose(P, ref, rtol=1e-12, atol=1e-12 * ref.max()))


def pin_plane_wave_on_grid(o, nx=4, ny=8, mx=4, my=16):
    """On the grid (u = A0/Mx, v = B0/My) a plane wave lands in beam (A0, B0) with power
    |c|^2 (nx ny)^2, and in no other beam of an unpadded axis (Eq. theta_A)."""
    A0, B0 = 3, 5
    c = 0.9 - 0.4j
    ix = np.arange(nx)[:, None]
    iy = np.arange(ny)[None, :]
    x = (c * np.exp(2j * np.pi * (ix * A0 / mx + iy * B0 / my)))[None, None, None]
    P = o.beams_from_field(x, None, mx, my, 1)[0, 0]
    peak = abs(c) ** 2 * (nx * ny) ** 2
    ok = abs(P[A0, B0] - peak) <= 1e-12 * peak
    col = np.delete(P[:, B0], A0)        # unpadded E-W axis: exact zeros elsewhere
    return bool(ok and np.all(np.abs(col) <= 1e-20 * peak))


def pin_windowed_peak(o, nx=6, ny=8, mx=6, my=16):
    """With separable half-sine weights (Section 4.1) an on-grid plane wave peaks at
    |c|^2 (sum h_x)^2 (sum h_y)^2, and sum_{a<n} sin[pi (a + 1/2)/n] = 1/sin(pi/(2n))."""
    hx, hy = synth.half_sine(nx), synth.half_sine(ny)
    w = np.outer(hx, hy)
    A0, B0 = 2, 3
    x = np.exp(2j * np.pi * (np.arange(nx)[:, None] * A0 / mx +
                             np.arange(ny)[None, :] * B0 / my))[None, None, None]
    P = o.beams_from_field(x, w, mx, my, 1)[0, 0]
    peak = 1.0 / (np.sin(np.pi / (2 * nx)) ** 2 * np.sin(np.pi / (2 * ny)) ** 2)
    return bool(abs(P[A0, B0] - peak) <= 1e-12 * peak)


def pin_asymmetric_weights(o, nx=3, ny=5, mx=4, my=8):
    """One weighted feed: P is flat at |w x|^2 in every beam, and zero weights give zero."""
    x = np.zeros((1, 1, 1, nx, ny), dtype=np.complex128)
    x[..., 2, 1] = 3 - 2j
    w = np.zeros((nx, ny), dtype=np.complex128)
    w[2, 1] = 0.5 + 0.25j
    w[1, 2] = 7.0                                   # multiplies a zero voltage
    P = o.beams_from_field(x, w, mx, my, 1)[0, 0]
    ref = abs((0.5 + 0.25j) * (3 - 2j)) ** 2
    return bool(np.allclose(P, ref, rtol=1e-13, atol=0))


def pin_linearity(o, nx=3, ny=4, mx=4, my=8, seed=4):
    rng = _rng(seed)
    x1 = _cnoise(rng, (2, nx, ny))
    x2 = _cnoise(rng, (2, nx, ny))
    w = _cnoise(rng, (nx, ny))
    a, b = 0.3 - 1.1j, 2.0 + 0.5j
    lhs = o.field_separable(a * x1 + b * x2, w, mx, my)
    rhs = a * o.field_separable(x1, w, mx, my) + b * o.field_separable(x2, w, mx, my)
    return bool(np.allclose(lhs, rhs, rtol=0, atol=1e-12))


def pin_additivity(o, nx=2, ny=4, mx=2, my=8, seed=5):
    """P sums |Y|^2 over polarisations and over the samples of each window."""
    rng = _rng(seed)
    x = _cnoise(rng, (4, 1, 2, nx, ny))
    w = _cnoise(rng, (nx, ny))
    both = o.beams_from_field(x, w, mx, my, 2)
    p0 = o.beams_from_field(x[:, :, :1], w, mx, my, 2)
    p1 = o.beams_from_field(x[:, :, 1:], w, mx, my, 2)
    one = o.beams_from_field(x, w, mx, my, 4)
    return bool(np.allclose(both, p0 + p1, rtol=1e-13) and
                np.allclose(one[0], both[0] + both[1], rtol=1e-13))


def pin_regrid_closed_form(o):
    """The regridding weights equal (1/M) sin[(2n-1) pi y]/sin(pi y) (Eq. bp_max_arbitrary)."""
    ok = True
    for n, m in ((4, 7), (16, 31), (16, 32), (32, 63)):
        y = np.linspace(-1.3, 1.7, 97) + 1e-3
        got = o.regrid_weights(n, m, y)
        yy = y[:, None] - np.arange(m)[None, :] / m
        ref = np.sin((2 * n - 1) * np.pi * yy) / np.sin(np.pi * yy) / m
        ok &= bool(np.allclose(got, ref, rtol=1e-10, atol=1e-12))
        ok &= bool(np.allclose(got.sum(axis=-1), 1.0, atol=1e-12))   # only delta = 0 survives
    return ok


def pin_regrid_identity(o, seed=6):
    """Regridded FFT-beam intensities equal the direct pointed beam when M >= 2n-1 on each
    axis; on an axis with M < 2n-1 they do for pointings on the FFT-beam grid."""
    rng = _rng(seed)
    ok = True
    for nx, ny, mx, my in ((3, 5, 5, 9), (4, 6, 4, 12), (2, 8, 4, 16)):
        n_int = 2
        x = _cnoise(rng, (2 * n_int, 2, 2, nx, ny))
        w = _cnoise(rng, (nx, ny))
        P = o.beams_from_field(x, w, mx, my, n_int)
        S = 7
        u = rng.random((2, S)) if mx >= 2 * nx - 1 else rng.integers(0, mx, (2, S)) / mx
        v = rng.random((2, S)) if my >= 2 * ny - 1 else rng.integers(0, my, (2, S)) / my
        a = o.tied_regrid(P, u, v, nx, ny)
        b = o.tied_direct(x, w, u, v, n_int)
        ok &= bool(np.allclose(a, b, rtol=1e-11, atol=1e-11 * np.abs(b).max()))
    return ok


def pin_noise_statistics(o, seed=7):
    """Var(b)/<b>^2 = 1/(n_int n_pol) for integrated Gaussian noise (Eq. var_bV), loosely."""
    rng = _rng(seed)
    nx, ny, mx, my, n_int = 2, 8, 2, 16, 8
    x = _cnoise(rng, (n_int * 400, 1, 2, nx, ny))
    P = o.beams_from_field(x, None, mx, my, n_int)[:, 0]      # [400, Mx, My]
    ratio = P.var(axis=0) / P.mean(axis=0) ** 2
    target = 1.0 / (n_int * 2)
    return bool(abs(ratio.mean() - target) < 0.15 * target)


ALL_PINS = [pin_unpack_examples, pin_unpack_exhaustive, pin_numpy_fft, pin_routes,
            pin_parseval, pin_plane_wave, pin_plane_wave_on_grid, pin_windowed_peak,
            pin_asymmetric_weights, pin_linearity, pin_additivity, pin_regrid_closed_form,
            pin_regrid_identity, pin_noise_statistics]


@pytest.mark.parametrize("pin", ALL_PINS, ids=lambda p: p.__name__)
def test_pin(pin):
    assert pin(O)


def test_numpy_fft_folded_axes():
    assert pin_numpy_fft(O, nx=6, ny=9, mx=4, my=5)      # M < n on both axes
    assert pin_numpy_fft(O, nx=1, ny=7, mx=1, my=7)


def test_routes_cyclic_and_minimal_padding():
    assert pin_routes(O, nx=3, ny=4, mx=2, my=3)          # cyclic co-adding
    assert pin_routes(O, nx=3, ny=4, mx=3, my=4)          # M = n
    assert pin_routes(O, nx=2, ny=3, mx=3, my=5)          # M = 2n - 1


def test_regrid_not_exact_without_padding():
    """With M = n the regridding identity fails off the grid: the pins above are not vacuous."""
    rng = _rng(8)
    nx, ny, mx, my = 1, 6, 1, 6
    x = _cnoise(rng, (2, 1, 1, nx, ny))
    P = O.beams_from_field(x, None, mx, my, 2)
    v = np.array([[0.31]])
    u = np.zeros((1, 1))
    direct = O.tied_direct(x, None, u, v, 2)
    yy = v[..., None] - np.arange(my) / my
    w_naive = np.sin((2 * ny - 1) * np.pi * yy) / np.sin(np.pi * yy) / my
    regrid = np.einsum("fsB,jfB->jfs", w_naive, P[:, :, 0, :])
    assert abs(regrid - direct).max() > 1e-3 * abs(direct).max()
    with pytest.raises(ValueError):
        O.regrid_weights(ny, my, v)


def test_printed_fig1_peak_ratio():
    """Fig. 1: the normalised pointed-beam peak is n, so the 32-element array peaks 4x the
    8-element one. The oracle's unnormalised P peaks at n^2 |c|^2; dividing by n (the
    1/n_ant of Eq. pointed_beam_shape) gives the paper's normalisation."""
    want, tol = _golden_printed()["fig1_peak_ratio_32_over_8"]
    peaks = {}
    for n in (32, 8):
        x = np.ones((1, 1, 1, 1, n), dtype=np.complex128)
        P = O.beams_from_field(x, None, 1, 2 * n, 1)[0, 0, 0]
        peaks[n] = P.max() / n
    assert abs(peaks[32] / peaks[8] - want) <= tol


def test_printed_naive_window_peak():
    """Section 4.1: naive half-sine windowing keeps ~83% of the unwindowed peak (n = 32).
    Normalisation of Eq. windowed_beam_shape: divide by N n with N = (1/n) sum |h|^2."""
    want, tol = _golden_printed()["naive_window_peak_fraction_n32"]
    n = 32
    h = synth.half_sine(n)
    x = np.ones((1, 1, 1, 1, n), dtype=np.complex128)
    Pw = O.beams_from_field(x, h[None, :], 1, 2 * n, 1)[0, 0, 0].max()
    Pu = O.beams_from_field(x, None, 1, 2 * n, 1)[0, 0, 0].max()
    norm = np.sum(h ** 2) / n
    frac = (Pw / (norm * n)) / (Pu / n)
    assert abs(frac - want) <= tol
    assert abs(frac - 0.811) < 0.001        # the recomputed value for the printed window


# ----------------------------------------------------- planted mistakes (CPU only) ----
def _mutant(**overrides):
    m = types.ModuleType("oracle_mutant")
    m.__dict__.update({k: v for k, v in O.__dict__.items() if not k.startswith("__")})
    m.__dict__["__builtins__"] = O.__dict__["__builtins__"]
    # rebind every function to the mutant namespace so internal calls see the overrides
    for name, fn in list(m.__dict__.items()):
        if isinstance(fn, types.FunctionType):
            m.__dict__[name] = types.FunctionType(fn.__code__, m.__dict__, name,
                                                  fn.__defaults__, fn.__closure__)
    m.__dict__.update(overrides)
    return m


def _fails_some_pin(m):
    failed = []
    for pin in ALL_PINS:
        try:
            ok = pin(m)
        except Exception:
            ok = False
        if not ok:
            failed.append(pin.__name__)
    return failed


def test_unmutated_copy_passes_every_pin():
    assert _fails_some_pin(_mutant()) == []


def test_planted_wrong_phase_sign():
    def dft_phase(n, m):
        A = np.arange(m)[:, None]
        a = np.arange(n)[None, :]
        return np.exp(+1j * O.TWO_PI * ((A * a) % m) / m)
    assert _fails_some_pin(_mutant(dft_phase=dft_phase))


def test_planted_dropped_polarisation():
    def beams_from_field(x, w, mx, my, n_int, route="separable"):
        x = np.asarray(x)
        T, F = x.shape[:2]
        y = O._field(x, w, mx, my, route)
        inten = (np.abs(y[:, :, 0]) ** 2)
        return inten.reshape(T // n_int, n_int, F, mx, my).sum(axis=1)
    assert _fails_some_pin(_mutant(beams_from_field=beams_from_field))


def test_planted_transposed_weights():
    def _weights(w, nx, ny):
        if w is None:
            return np.ones((nx, ny), dtype=np.complex128)
        return np.asarray(w).astype(np.complex128).reshape(ny, nx).T
    assert _fails_some_pin(_mutant(_weights=_weights))


def test_planted_conjugated_weights():
    def _weights(w, nx, ny):
        if w is None:
            return np.ones((nx, ny), dtype=np.complex128)
        return np.conj(np.asarray(w).astype(np.complex128).reshape(nx, ny))
    assert _fails_some_pin(_mutant(_weights=_weights))


def test_planted_swapped_nibbles():
    def unpack(volts):
        b = np.asarray(volts, dtype=np.uint8).astype(np.int64)
        lo, hi = b >> 4, b & 15
        re = np.where(hi >= 8, hi - 16, hi)
        im = np.where(lo >= 8, lo - 16, lo)
        return re + 1j * im
    assert _fails_some_pin(_mutant(unpack=unpack))


def test_planted_regrid_off_by_one():
    def regrid_weights(n, m, y):
        y = np.asarray(y, dtype=np.float64)
        yy = y[..., None] - np.arange(m) / m
        acc = np.ones(yy.shape)
        for d in range(1, n - 1):                      # drops the |delta| = n-1 terms
            acc += 2.0 * np.cos(O.TWO_PI * d * yy)
        return acc / m
    assert _fails_some_pin(_mutant(regrid_weights=regrid_weights))


def test_planted_window_sum_off_by_one():
    def beams_from_field(x, w, mx, my, n_int, route="separable"):
        x = np.asarray(x)
        T, F = x.shape[:2]
        y = O._field(x, w, mx, my, route)
        inten = (y.real ** 2 + y.imag ** 2).sum(axis=2)
        r = inten.reshape(T // n_int, n_int, F, mx, my)
        return r[:, 1:].sum(axis=1)                    # drops the first sample of a window
    assert _fails_some_pin(_mutant(beams_from_field=beams_from_field))
