"""Pins of visibility-space products recovered from FFT beams (Eq. inv_b2n-1)."""
import numpy as np

from oracle import fftbf_oracle as O


def _x(rng, shape):
    return rng.normal(size=shape) + 1j * rng.normal(size=shape)


def test_inverse_recovers_stacked_visibilities():
    """With M >= 2n - 1 on both axes the FFT beams determine V~_delta exactly (Section 3.3)."""
    rng = np.random.default_rng(11)
    for nx, ny, mx, my in ((3, 4, 5, 7), (2, 5, 4, 10)):
        x = _x(rng, (4, 2, 2, nx, ny))
        w = _x(rng, (nx, ny))
        P = O.beams_from_field(x, w, mx, my, 2)
        got = O.stacked_from_beams(P, nx, ny)
        ref = O.stacked_visibilities(x, w, 2)
        assert np.allclose(got, ref, rtol=1e-11, atol=1e-11 * np.abs(ref).max())


def test_partial_stacking_on_the_padded_axis():
    """E-W unpadded, N-S padded: inverting the N-S axis gives the N-S stacked visibilities
    of each E-W FFT beam."""
    rng = np.random.default_rng(12)
    nx, ny, mx, my = 4, 6, 4, 12
    x = _x(rng, (4, 2, 2, nx, ny))
    w = _x(rng, (nx, ny))
    P = O.beams_from_field(x, w, mx, my, 2)
    got = O.stacked_from_beams(P, nx, ny)
    ref = O.stacked_ew_beams(x, w, mx, 2)
    assert got.shape == ref.shape == (2, 2, mx, 2 * ny - 1)
    assert np.allclose(got, ref, rtol=1e-11, atol=1e-11 * np.abs(ref).max())


def test_hermitian_and_zero_lag():
    rng = np.random.default_rng(13)
    nx, ny, mx, my = 3, 5, 6, 10
    x = _x(rng, (2, 1, 1, nx, ny))
    P = O.beams_from_field(x, None, mx, my, 2)
    V = O.stacked_from_beams(P, nx, ny)[0, 0]
    assert np.allclose(V, np.conj(V[::-1, ::-1]), atol=1e-10 * np.abs(V).max())   # V~_-d = V~_d^*
    assert abs(V[nx - 1, ny - 1] - np.sum(np.abs(x) ** 2)) < 1e-9 * np.abs(V).max()  # total power
