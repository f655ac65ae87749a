"""FP64 CPU oracle for FFT beamforming of a regular antenna lattice (arXiv 1710.08591).

TEST INFRASTRUCTURE. Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline
and reference legs may import this module. The library's compute path never calls it,
and it imports nothing from the library: the two share no code. Inputs come from the
``synth`` generator, whose bytes are the ground truth.

Everything here is the plain definition, written in FP64 with numpy: direct DFT sums as
products with explicit phase matrices, then |.|^2, then sums over polarisation and time.
There is no FFT, no blocking and no reordering beyond what the definitions state.

Conventions (the paper is 1-D; the lattice is its separable 2-D extension):
  x[t,f,p,ix,iy]  complex voltage of feed (ix, iy) of polarisation p (Section 2: each
                  polarisation is a separate antenna).
  w[ix,iy]        complex apodisation weight, applied as w * x (Section 4.1, naive
                  windowed beam; Eq. bf uses w^a eta_a without conjugation).
  Y[A,B]          = sum_{ix,iy} w x exp(-2 pi i (A ix / Mx + B iy / My))   (Eq. fftbeamform)
  P[j,f,A,B]      = sum over the n_int samples of window j and over p of |Y|^2 (Eq. bf,
                  Eq. Vab): the unnormalised integrated FFT-beam intensity.
The paper's normalisations (1/n_samp, 1/sqrt(n_ant), c^2/(k_B nu^2)) are dropped: with
uniform weights the paper's b_A equals P / (n_samp * n_ant) for one polarisation.
When M < n on an axis the direct sum folds the feeds cyclically by itself, because
exp(-2 pi i A a / M) depends only on a mod M (Section 3.2, cyclic co-adding).
"""
from __future__ import annotations

import numpy as np

TWO_PI = 2.0 * np.pi


# --- unpacking ------------------------------------------------------------------------
def unpack(volts) -> np.ndarray:
    """Decode int4+4 bytes to complex128.

    The paper does not fix a bit layout. Reading used throughout: one byte per complex
    sample, bits 7..4 = real part, bits 3..0 = imaginary part, each a two's-complement
    4-bit integer in [-8, 7].
    """
    b = np.asarray(volts, dtype=np.uint8).astype(np.int64)
    hi = b >> 4
    lo = b & 15
    re = np.where(hi >= 8, hi - 16, hi)
    im = np.where(lo >= 8, lo - 16, lo)
    return re.astype(np.float64) + 1j * im.astype(np.float64)


# --- phase matrices -------------------------------------------------------------------
def dft_phase(n: int, m: int) -> np.ndarray:
    """E[A, a] = exp(-2 pi i A a / M) for A < M, a < n (Eq. fftbeamform, Eq. w_A^a).

    The phase is taken from the integer (A a) mod M so that it never grows.
    """
    A = np.arange(m, dtype=np.int64)[:, None]
    a = np.arange(n, dtype=np.int64)[None, :]
    return np.exp(-1j * TWO_PI * ((A * a) % m) / m)


def _weights(w, nx, ny) -> np.ndarray:
    if w is None:
        return np.ones((nx, ny), dtype=np.complex128)
    return np.asarray(w).astype(np.complex128).reshape(nx, ny)


# --- the pre-detection field Y ---------------------------------------------------------
def field_direct(x, w, mx, my) -> np.ndarray:
    """Y[..., A, B] as one 2-D direct sum with a single phase per (A, B, ix, iy).

    x: complex [..., nx, ny]. Cost O(Mx My nx ny) per snapshot: tiny lattices only.
    """
    x = np.asarray(x, dtype=np.complex128)
    nx, ny = x.shape[-2:]
    wx = _weights(w, nx, ny) * x
    A = np.arange(mx, dtype=np.int64)[:, None, None, None]
    B = np.arange(my, dtype=np.int64)[None, :, None, None]
    ix = np.arange(nx, dtype=np.int64)[None, None, :, None]
    iy = np.arange(ny, dtype=np.int64)[None, None, None, :]
    # phase / (2 pi) = (A ix mod Mx) / Mx + (B iy mod My) / My, over a common denominator
    num = ((A * ix) % mx) * my + ((B * iy) % my) * mx
    ph = np.exp(-1j * TWO_PI * (num % (mx * my)) / (mx * my))
    return np.einsum("...xy,ABxy->...AB", wx, ph)


def field_separable(x, w, mx, my) -> np.ndarray:
    """Y[..., A, B] = sum_ix E_x[A, ix] sum_iy E_y[B, iy] w x (the same sum, axis by axis)."""
    x = np.asarray(x, dtype=np.complex128)
    nx, ny = x.shape[-2:]
    wx = _weights(w, nx, ny) * x
    ex = dft_phase(nx, mx)
    ey = dft_phase(ny, my)
    z = np.matmul(ex, wx)                       # [..., Mx, ny]
    return np.matmul(z, ey.T)                   # [..., Mx, My]


def _field(x, w, mx, my, route):
    if route == "direct":
        return field_direct(x, w, mx, my)
    if route == "separable":
        return field_separable(x, w, mx, my)
    raise ValueError(route)


# --- integrated FFT-beam intensities ----------------------------------------------------
def beams_from_field(x, w, mx, my, n_int, route="separable") -> np.ndarray:
    """P[j, f, A, B] from complex voltages x [T, F, P, nx, ny] (Eq. fftbeamform, Eq. bf).

    |Y|^2 is summed over polarisation (feeds of both polarisations are separate
    antennas) and over the n_int samples of each non-overlapping window.
    """
    x = np.asarray(x)
    T, F = x.shape[:2]
    if T % n_int:
        raise ValueError("T must be a multiple of n_int")
    y = _field(x, w, mx, my, route)             # [T, F, P, Mx, My]
    inten = (y.real ** 2 + y.imag ** 2).sum(axis=2)
    return inten.reshape(T // n_int, n_int, F, mx, my).sum(axis=1)


def beams(volts, nx, ny, mx, my, npol, nfreq, n_int, weights=None, route="separable"):
    """Integrated FFT-beam intensities from packed voltages uint8 [T][F][P][nx][ny]."""
    v = np.asarray(volts, dtype=np.uint8).reshape(-1, nfreq, npol, nx, ny)
    return beams_from_field(unpack(v), weights, mx, my, n_int, route)


# --- visibility routes (tiny lattices) ---------------------------------------------------
def _feed_positions(nx, ny):
    ix, iy = np.meshgrid(np.arange(nx), np.arange(ny), indexing="ij")
    return ix.reshape(-1).astype(np.int64), iy.reshape(-1).astype(np.int64)


def visibilities(x, w, n_int) -> np.ndarray:
    """V[j, f, a, b] = sum_{t in window j, p} (w_a x_a)(w_b x_b)^* (Eq. Vab, Eq. wf).

    Unnormalised; a, b run over feeds in row-major (ix, iy) order.
    """
    x = np.asarray(x, dtype=np.complex128)
    T, F, P, nx, ny = x.shape
    wx = (_weights(w, nx, ny) * x).reshape(T // n_int, n_int, F, P, nx * ny)
    return np.einsum("jtfpa,jtfpb->jfab", wx, wx.conj())


def beams_via_visibilities(x, w, mx, my, n_int) -> np.ndarray:
    """P[A, B] = sum_{a,b} exp(-2 pi i (A (ax - bx)/Mx + B (ay - by)/My)) V_ab (Eq. b2n-1)."""
    x = np.asarray(x)
    nx, ny = x.shape[-2:]
    V = visibilities(x, w, n_int)
    px, py = _feed_positions(nx, ny)
    dx = px[:, None] - px[None, :]
    dy = py[:, None] - py[None, :]
    A = np.arange(mx, dtype=np.int64)[:, None, None, None]
    B = np.arange(my, dtype=np.int64)[None, :, None, None]
    num = ((A * dx[None, None]) % mx) * my + ((B * dy[None, None]) % my) * mx
    ph = np.exp(-1j * TWO_PI * (num % (mx * my)) / (mx * my))
    return np.einsum("jfab,ABab->jfAB", V, ph).real


def stacked_visibilities(x, w, n_int) -> np.ndarray:
    """Redundancy-stacked V~[j, f, dx, dy] = sum_alpha V_{alpha+delta, alpha} (Eq. b_V_delta).

    delta = (dx, dy) is stored at offset (dx + nx - 1, dy + ny - 1). The redundancy
    index alpha runs over [max(0, -delta), min(n, n - delta)) on each axis, which has
    n - |delta| terms (the half-open reading of the printed limits).
    """
    x = np.asarray(x)
    nx, ny = x.shape[-2:]
    V = visibilities(x, w, n_int)
    J, F = V.shape[:2]
    V = V.reshape(J, F, nx, ny, nx, ny)
    S = np.zeros((J, F, 2 * nx - 1, 2 * ny - 1), dtype=np.complex128)
    for dx in range(-(nx - 1), nx):
        for dy in range(-(ny - 1), ny):
            acc = np.zeros((J, F), dtype=np.complex128)
            for ax in range(max(0, -dx), min(nx, nx - dx)):
                for ay in range(max(0, -dy), min(ny, ny - dy)):
                    acc += V[:, :, ax + dx, ay + dy, ax, ay]
            S[:, :, dx + nx - 1, dy + ny - 1] = acc
    return S


def beams_via_stacked(x, w, mx, my, n_int) -> np.ndarray:
    """P[A, B] = sum_delta exp(-2 pi i (A dx / Mx + B dy / My)) V~_delta (Eq. b2n-1)."""
    x = np.asarray(x)
    nx, ny = x.shape[-2:]
    S = stacked_visibilities(x, w, n_int)
    dxs = np.arange(-(nx - 1), nx, dtype=np.int64)
    dys = np.arange(-(ny - 1), ny, dtype=np.int64)
    ex = np.exp(-1j * TWO_PI * ((np.arange(mx)[:, None] * dxs[None, :]) % mx) / mx)
    ey = np.exp(-1j * TWO_PI * ((np.arange(my)[:, None] * dys[None, :]) % my) / my)
    return np.einsum("Ad,Be,jfde->jfAB", ex, ey, S).real


# --- tied-array beams -----------------------------------------------------------------
def regrid_weights(n: int, m: int, y) -> np.ndarray:
    """FFT-beam regridding weights w^A for a pointing y = (d/lambda) sin(theta_p).

    Eq. bp_max_arbitrary, in the form it is derived from (Eq. b_V_delta combined with
    Eq. inv_b2n-1): w^A = (1/M) sum_{delta=-(n-1)}^{n-1} exp(-2 pi i delta (y - A/M)),
    which is real: (1/M) [1 + 2 sum_{delta>=1} cos(2 pi delta (y - A/M))].
    Valid when M >= 2n - 1. Returns [..., M] for y of shape [...].

    On an axis with M < 2n - 1 the FFT beams do not hold all of V~_delta and the
    derivation does not apply. Reading used there: only pointings on the FFT-beam grid
    (y M an integer within 1e-9) are defined, and the tied beam is the FFT beam itself,
    w^A = 1 at A = y M mod M and 0 elsewhere (Eq. theta_A: b_A is exactly the pointed
    beam at sin(theta_A) = A lambda / (M d)).
    """
    y = np.asarray(y, dtype=np.float64)
    A = np.arange(m, dtype=np.float64)
    if m >= 2 * n - 1:
        yy = y[..., None] - A / m
        acc = np.ones(yy.shape, dtype=np.float64)
        for d in range(1, n):
            acc += 2.0 * np.cos(TWO_PI * d * yy)
        return acc / m
    k = np.rint(y * m)
    if np.any(np.abs(y * m - k) > 1e-9):
        raise ValueError("pointing off the FFT-beam grid on an axis with M < 2n - 1")
    k = np.mod(k.astype(np.int64), m)
    out = np.zeros(y.shape + (m,), dtype=np.float64)
    np.put_along_axis(out, k[..., None], 1.0, axis=-1)
    return out


def tied_regrid(P, u, v, nx, ny) -> np.ndarray:
    """Tied beams from FFT-beam intensities: T[j, f, s] = sum_{A,B} w^A(u) w^B(v) P[j,f,A,B].

    P: [J, F, Mx, My]; u, v: [F, S] pointings per frequency (Eq. bp_max_arbitrary,
    applied per axis; the 2-D weight factorises because the redundancy counts do).
    """
    P = np.asarray(P, dtype=np.float64)
    mx, my = P.shape[-2:]
    wx = regrid_weights(nx, mx, u)              # [F, S, Mx]
    wy = regrid_weights(ny, my, v)              # [F, S, My]
    return np.einsum("fsA,fsB,jfAB->jfs", wx, wy, P)


def tied_direct(x, w, u, v, n_int) -> np.ndarray:
    """Direct voltage-space pointed beams (Eq. bp / Eq. c_pointed, with the apodisation):

    T[j, f, s] = sum_{t in j, p} |sum_{ix,iy} w x exp(-2 pi i (ix u_{f,s} + iy v_{f,s}))|^2.
    """
    x = np.asarray(x, dtype=np.complex128)
    T, F, P, nx, ny = x.shape
    wx = _weights(w, nx, ny) * x
    u = np.asarray(u, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    ix = np.arange(nx)
    iy = np.arange(ny)
    ex = np.exp(-1j * TWO_PI * u[:, :, None] * ix[None, None, :])   # [F, S, nx]
    ey = np.exp(-1j * TWO_PI * v[:, :, None] * iy[None, None, :])   # [F, S, ny]
    y = np.einsum("tfpxy,fsx,fsy->tfps", wx, ex, ey)
    inten = (y.real ** 2 + y.imag ** 2).sum(axis=2)
    return inten.reshape(T // n_int, n_int, F, -1).sum(axis=1)


# --- intensity-space windowing (optimal windowed beams) --------------------------------
def window_lag_coeffs(h) -> np.ndarray:
    """g_delta for delta = -(n-1) .. n-1 (index delta + n - 1) of the optimal windowed beam
    (Eq. w_opt): the window's auto-convolution sum_alpha h^(alpha+delta) h^(alpha*) divided
    by the n - |delta| redundant baselines. Unnormalised: a flat window gives g = 1, i.e.
    the plain pointed beam. Real windows give real, symmetric g."""
    h = np.asarray(h, dtype=np.complex128)
    n = h.size
    g = np.zeros(2 * n - 1, dtype=np.complex128)
    for d in range(-(n - 1), n):
        acc = 0j
        for a in range(max(0, -d), min(n, n - d)):
            acc += h[a + d] * np.conj(h[a])
        g[d + n - 1] = acc / (n - abs(d))
    return g


def windowed_regrid_weights(n: int, m: int, y, g) -> np.ndarray:
    """FFT-beam coefficients of the optimal windowed beam pointed at y (M >= 2n - 1):
    w^A = (1/M) sum_delta g_delta exp(-2 pi i delta (y - A/M)) (Eq. wA_from_wdelta applied to
    the lag weights of Eq. w_opt, in this library's unnormalised convention). Real part
    returned (g of a real window is symmetric, so the sum is real)."""
    y = np.asarray(y, dtype=np.float64)
    if m < 2 * n - 1:
        raise ValueError("windowed regridding needs M >= 2n - 1")
    yy = y[..., None] - np.arange(m, dtype=np.float64) / m
    acc = np.zeros(yy.shape, dtype=np.complex128)
    for d in range(-(n - 1), n):
        acc += g[d + n - 1] * np.exp(-1j * TWO_PI * d * yy)
    return acc.real / m


def tied_windowed_regrid(P, u, v, nx, ny, hx, hy) -> np.ndarray:
    """Optimal windowed tied beams from FFT-beam intensities, separable window hx x hy."""
    P = np.asarray(P, dtype=np.float64)
    mx, my = P.shape[-2:]
    wx = windowed_regrid_weights(nx, mx, u, window_lag_coeffs(hx))
    wy = windowed_regrid_weights(ny, my, v, window_lag_coeffs(hy))
    return np.einsum("fsA,fsB,jfAB->jfs", wx, wy, P)


def tied_windowed_visibility(x, w, u, v, n_int, hx, hy) -> np.ndarray:
    """The same beams formed directly in redundancy-stacked visibility space:
    T = sum_delta g_delta exp(-2 pi i (dx u + dy v)) V~_delta (Eq. b_V_delta with the
    optimal windowed lag weights of Eq. w_opt). Tiny lattices only."""
    x = np.asarray(x)
    nx, ny = x.shape[-2:]
    S = stacked_visibilities(x, w, n_int)                     # [J, F, 2nx-1, 2ny-1]
    gx, gy = window_lag_coeffs(hx), window_lag_coeffs(hy)
    dxs = np.arange(-(nx - 1), nx)
    dys = np.arange(-(ny - 1), ny)
    u = np.asarray(u, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    ex = gx[None, None, :] * np.exp(-1j * TWO_PI * u[:, :, None] * dxs[None, None, :])
    ey = gy[None, None, :] * np.exp(-1j * TWO_PI * v[:, :, None] * dys[None, None, :])
    return np.einsum("fsd,fse,jfde->jfs", ex, ey, S).real


def truncate_nearest(weights, y, m, k) -> np.ndarray:
    """Keep the regridding weights of the k FFT beams nearest to the pointing, zero the
    rest: beams A = first .. first + k - 1 (mod M) with first = floor(y M - (k - 1)/2 + 1/2).
    This is the compact kernel of Section 4.1 (a windowed beam needs only a few FFT beams)."""
    w = np.array(weights, dtype=np.float64, copy=True)
    y = np.asarray(y, dtype=np.float64)
    first = np.floor(y * m - (k - 1) / 2.0 + 0.5)
    rel = np.mod(np.arange(m, dtype=np.float64) - first[..., None], m)
    w[rel >= k] = 0.0
    return w


# --- visibility-space products from FFT beams ------------------------------------------
def _stack_axis(P, n, axis):
    """Inverse DFT of FFT-beam intensities along `axis` onto lags delta = -(n-1) .. n-1
    (stored at delta + n - 1): (1/M) sum_A exp(+2 pi i delta A / M) P_A (Eq. inv_b2n-1 in
    this library's unnormalised convention). Needs M >= 2n - 1."""
    m = P.shape[axis]
    d = np.arange(-(n - 1), n)
    E = np.exp(2j * np.pi * ((d[:, None] * np.arange(m)[None, :]) % m) / m) / m   # [2n-1, M]
    P = np.moveaxis(np.asarray(P), axis, -1)
    out = np.einsum("dA,...A->...d", E, P)
    return np.moveaxis(out, -1, axis)


def stacked_from_beams(P, nx, ny) -> np.ndarray:
    """Redundancy-stacked visibilities recovered from FFT-beam intensities P[..., Mx, My].

    On an axis with M >= 2n - 1 the beams are inverted onto lags (Eq. inv_b2n-1); on an
    axis with M < 2n - 1 they do not determine every lag, and the FFT-beam index is kept.
    Returns complex [..., Dx, Dy], D = 2n - 1 (lags) or M (beams) per axis."""
    P = np.asarray(P, dtype=np.float64)
    mx, my = P.shape[-2:]
    out = P.astype(np.complex128)
    if my >= 2 * ny - 1:
        out = _stack_axis(out, ny, -1)
    if mx >= 2 * nx - 1:
        out = _stack_axis(out, nx, -2)
    return out


def stacked_ew_beams(x, w, mx, n_int) -> np.ndarray:
    """N-S redundancy-stacked visibilities of each E-W FFT beam, formed from voltages:
    sum_{t,p} sum_alpha Y_A(alpha + dy) Y_A(alpha)^*, Y_A(iy) = sum_ix E_x[A, ix] w x (the
    partially stacked quantity when only the N-S axis is padded to 2n - 1). [J, F, Mx, 2ny-1]"""
    x = np.asarray(x, dtype=np.complex128)
    T, F, Pn, nx, ny = x.shape
    ya = np.einsum("Ax,tfpxy->tfpAy", dft_phase(nx, mx), _weights(w, nx, ny) * x)
    out = np.zeros((T // n_int, F, mx, 2 * ny - 1), dtype=np.complex128)
    ya = ya.reshape(T // n_int, n_int, F, Pn, mx, ny)
    for d in range(-(ny - 1), ny):
        lo, hi = max(0, -d), min(ny, ny - d)
        out[..., d + ny - 1] = np.einsum("jtfpAa,jtfpAa->jfA", ya[..., lo + d:hi + d],
                                         np.conj(ya[..., lo:hi]))
    return out


# --- localisation on FFT beams (Section 4.3) ---------------------------------------------
def baseline_moi(n: int) -> float:
    """sum_delta delta^2 (n - |delta|), the baseline moment of inertia (Eq. baseline_MOI),
    as the plain sum."""
    return float(sum(d * d * (n - abs(d)) for d in range(-(n - 1), n)))


def regrid_weight_derivative(n: int, m: int, y) -> np.ndarray:
    """d w^A / d y of the regridding weights (the sky response of the derivative beam):
    (1/M) sum_delta (-2 pi i delta) exp(-2 pi i delta (y - A/M)), real."""
    y = np.asarray(y, dtype=np.float64)
    yy = y[..., None] - np.arange(m, dtype=np.float64) / m
    acc = np.zeros(yy.shape, dtype=np.float64)
    for d in range(1, n):
        acc += -2.0 * TWO_PI * d * np.sin(TWO_PI * d * yy)
    return acc / m


def localise(P, nx, ny, n_iter=5, n_taps=10):
    """Newton estimator of a point source's position from its FFT-beam intensities
    (Section 4.3), per (window, channel) of P[J, F, Mx, My]:
      start at the strongest FFT beam (argmax taken on FP32-rounded intensities);
      on each axis with M >= 2n - 1 iterate  y <- y + T'(y) n^2 / (4 pi^2 MOI T(y)),
      where T and T' are the pointed beam and its derivative regridded from the FFT beams
      (Eq. bp_max_arbitrary and its derivative), with the curvature replaced by its value
      at the maximum (Eq. baseline_MOI) and both sums truncated to the n_taps FFT beams
      nearest the current estimate (the paper keeps ~10 beams around the source);
      an axis with M < 2n - 1 (or a single feed) keeps the beam position A/M.
    Returns [J, F, 3]: y_x, y_y (in [0, 1), lattice units) and T at the estimate."""
    P = np.asarray(P, dtype=np.float64)
    J, F, mx, my = P.shape
    out = np.zeros((J, F, 3))
    fit_x, fit_y = (mx >= 2 * nx - 1 and nx > 1), (my >= 2 * ny - 1 and ny > 1)
    for j in range(J):
        for f in range(F):
            tile = P[j, f]
            a0, b0 = np.unravel_index(np.argmax(tile.astype(np.float32)), tile.shape)
            yx, yy = a0 / mx, b0 / my
            for _ in range(n_iter):
                wx = regrid_weights(nx, mx, yx) if fit_x else np.eye(mx)[a0]
                wy = regrid_weights(ny, my, yy) if fit_y else np.eye(my)[b0]
                if fit_x:
                    wx = truncate_nearest(wx, yx, mx, min(n_taps, mx))
                if fit_y:
                    wy = truncate_nearest(wy, yy, my, min(n_taps, my))
                T = wx @ tile @ wy
                if fit_x:
                    dx = truncate_nearest(regrid_weight_derivative(nx, mx, yx), yx, mx, min(n_taps, mx))
                    yx = yx + (dx @ tile @ wy) * nx * nx / (4 * np.pi ** 2 * baseline_moi(nx) * T)
                if fit_y:
                    dy = truncate_nearest(regrid_weight_derivative(ny, my, yy), yy, my, min(n_taps, my))
                    yy = yy + (wx @ tile @ dy) * ny * ny / (4 * np.pi ** 2 * baseline_moi(ny) * T)
            wx = regrid_weights(nx, mx, yx) if fit_x else np.eye(mx)[a0]
            wy = regrid_weights(ny, my, yy) if fit_y else np.eye(my)[b0]
            out[j, f] = (np.mod(yx, 1.0), np.mod(yy, 1.0), wx @ tile @ wy)
    return out
