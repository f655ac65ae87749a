"""Pins of the oracle's intensity-space windowing (optimal windowed beams, Section 4.1)."""
import os

import numpy as np

from oracle import fftbf_oracle as O
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _printed():
    out = {}
    with open(os.path.join(GOLDEN, "paper_printed.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                k, v, tol = line.split()[:3]
                out[k] = (float(v), float(tol))
    return out


def test_flat_window_is_the_plain_pointed_beam():
    for n, m in ((4, 7), (16, 32)):
        g = O.window_lag_coeffs(np.ones(n))
        assert np.allclose(g, 1.0)
        y = np.linspace(-0.7, 1.3, 41)
        assert np.allclose(O.windowed_regrid_weights(n, m, y, g), O.regrid_weights(n, m, y),
                           atol=1e-12)


def test_lag_coeffs_closed_form_half_sine():
    # sum_alpha sin(pi(a+d+1/2)/n) sin(pi(a+1/2)/n) over n-d terms has a closed form:
    # ((n-d) cos(pi d/n) + sin(pi d/n)/sin(pi/n)) / 2
    n = 32
    g = O.window_lag_coeffs(synth.half_sine(n))
    for d in range(0, n):
        ref = ((n - d) * np.cos(np.pi * d / n) + np.sin(np.pi * d / n) / np.sin(np.pi / n)) / 2
        assert abs(g[d + n - 1] * (n - d) - ref) < 1e-10
        assert abs(g[-d + n - 1] - g[d + n - 1]) < 1e-12     # symmetric for a real window


def test_fft_beam_route_equals_visibility_route():
    """Windowed beams regridded from FFT beams equal the same lag weights applied to the
    redundancy-stacked visibilities when M >= 2n - 1 (Eq. inv_b2n-1)."""
    rng = np.random.default_rng(3)
    nx, ny, mx, my, n_int = 3, 6, 5, 12, 2
    x = rng.normal(size=(2 * n_int, 2, 2, nx, ny)) + 1j * rng.normal(size=(2 * n_int, 2, 2, nx, ny))
    hx, hy = synth.half_sine(nx), 0.3 + rng.random(ny)
    P = O.beams_from_field(x, None, mx, my, n_int)
    u, v = rng.random((2, 5)), rng.random((2, 5))
    a = O.tied_windowed_regrid(P, u, v, nx, ny, hx, hy)
    b = O.tied_windowed_visibility(x, None, u, v, n_int, hx, hy)
    assert np.allclose(a, b, rtol=1e-11, atol=1e-11 * np.abs(b).max())


def _noise(g, n):
    d = np.arange(-(n - 1), n)
    return np.sqrt(np.sum((n - np.abs(d)) * np.abs(g) ** 2))


def test_printed_optimal_window_numbers():
    """Section 4.1, n = 32 half-sine: the optimal windowed beam keeps ~95% of the peak
    of the unwindowed beam and has ~14% more sky-integrated response. Both are computed
    through the oracle chain (plane waves -> FFT beams -> windowed regridding), per unit
    noise. The printed window gives 93.8% and +15.7%; the pins allow 3 points."""
    printed = _printed()
    n, m = 32, 64
    h = synth.half_sine(n)
    g = O.window_lag_coeffs(h)
    ys = (np.arange(4 * n) + 0.37) / (4 * n)                 # source positions over a period
    y_p = 0.25
    resp_w, resp_u = [], []
    for y_s in np.concatenate([[y_p], ys]):
        x = np.exp(2j * np.pi * y_s * np.arange(n))[None, None, None, None, :]
        P = O.beams_from_field(x, None, 1, m, 1)
        resp_w.append(O.tied_windowed_regrid(P, np.zeros((1, 1)), np.full((1, 1), y_p), 1, n,
                                             np.ones(1), h)[0, 0, 0])
        resp_u.append(O.tied_regrid(P, np.zeros((1, 1)), np.full((1, 1), y_p), 1, n)[0, 0, 0])
    nw, nu = _noise(g, n), _noise(np.ones(2 * n - 1), n)
    peak = (resp_w[0] / nw) / (resp_u[0] / nu)
    integ = (np.mean(resp_w[1:]) / nw) / (np.mean(resp_u[1:]) / nu)
    want_p, tol_p = printed["optimal_window_peak_fraction_n32"]
    want_i, tol_i = printed["optimal_window_integrated_gain_n32"]
    assert abs(peak - want_p) <= tol_p
    assert abs((integ - 1.0) - want_i) <= tol_i
    assert abs(peak - 0.938) < 0.001 and abs(integ - 1.157) < 0.001


def test_truncation_rule():
    m = 64
    w = np.ones((3, m))
    y = np.array([0.1, 0.5, 0.999])
    for k in (1, 4, 5, 64):
        t = O.truncate_nearest(w, y, m, k)
        assert np.all(t.sum(axis=-1) == k)
        # the beam nearest the pointing is always kept
        near = np.mod(np.rint(y * m), m).astype(int)
        assert np.all(t[np.arange(3), near] == 1.0)


def test_windowed_kernel_is_compact():
    """A windowed regridding kernel concentrates in a few FFT beams (Section 4.1); the
    unwindowed Dirichlet kernel does not."""
    n, m = 32, 64
    y = np.array([0.2 + 0.3 / m])
    gw = O.window_lag_coeffs(synth.half_sine(n))
    ww = O.windowed_regrid_weights(n, m, y, gw)[0]
    wu = O.regrid_weights(n, m, y)[0]
    keep = O.truncate_nearest(np.ones((1, m)), y, m, 5)[0] > 0
    assert np.abs(ww[~keep]).sum() < 0.1 * np.abs(ww).sum()
    assert np.abs(wu[~keep]).sum() > 0.2 * np.abs(wu).sum()
