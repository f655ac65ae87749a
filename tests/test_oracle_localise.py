"""Pins of the oracle's localisation estimator (Section 4.3)."""
import numpy as np

from oracle import fftbf_oracle as O


def test_baseline_moi_closed_form():
    """Eq. baseline_MOI: 2 n^2 (n-1) [(2n-1)/6 - (n-1)/4], close to n^4/6."""
    for n in (2, 4, 32, 256):
        closed = 2 * n * n * (n - 1) * ((2 * n - 1) / 6 - (n - 1) / 4)
        assert abs(O.baseline_moi(n) - closed) < 1e-6 * closed
    assert abs(O.baseline_moi(256) / (256 ** 4 / 6) - 1) < 0.01


def test_derivative_weights_are_the_derivative():
    n, m = 16, 32
    y = np.linspace(0.013, 0.97, 23)
    h = 1e-6
    num = (O.regrid_weights(n, m, y + h) - O.regrid_weights(n, m, y - h)) / (2 * h)
    assert np.allclose(O.regrid_weight_derivative(n, m, y), num, rtol=1e-6, atol=1e-6)


def _source_beams(n, m, y_s, amp, noise, rng, nx=1, mx=1):
    """FFT-beam intensities of a point source plus independent noise on the stacked
    visibilities (simple noise model: variance (n - |delta|) per lag), built through
    Eq. b2n-1 from V~_delta = (n - |delta|) T_s exp(2 pi i delta y_s) + noise."""
    d = np.arange(-(n - 1), n)
    c = n - np.abs(d)
    V = c * amp * np.exp(2j * np.pi * d * y_s)
    if noise > 0:
        z = (rng.normal(size=n) + 1j * rng.normal(size=n)) * noise * np.sqrt(c[n - 1:] / 2)
        z[0] = z[0].real * np.sqrt(2)
        V = V + np.concatenate([np.conj(z[:0:-1]), z])
    A = np.arange(m)
    P = np.real(np.exp(-2j * np.pi * np.outer(A, d) / m) @ V)
    return P[None, None, None, :] * np.ones((1, 1, mx, 1))


def test_noiseless_source_is_found_exactly():
    rng = np.random.default_rng(0)
    n, m = 32, 64
    for y_s in (0.1234, 0.5 + 0.3 / m, 0.9871):
        P = _source_beams(n, m, y_s, 2.0, 0.0, rng)
        est = O.localise(P, 1, n, n_iter=8, n_taps=m)
        assert abs(est[0, 0, 1] - y_s) < 1e-9
        assert abs(est[0, 0, 2] - 2.0 * n * n) < 1e-6 * n * n


def test_variance_matches_cramer_rao_bound():
    """sigma(y) = sqrt(6) / (2 pi n SNR), SNR = T_s n / sigma (Section 4.3), Monte Carlo."""
    rng = np.random.default_rng(1)
    n, m, amp, noise = 32, 64, 1.0, 2.0
    snr = amp * n / noise
    ests = []
    for _ in range(600):
        y_s = rng.random()
        P = _source_beams(n, m, y_s, amp, noise, rng)
        e = O.localise(P, 1, n, n_iter=6, n_taps=10)[0, 0, 1]
        ests.append(((e - y_s + 0.5) % 1.0) - 0.5)
    sigma = np.std(ests)
    want = np.sqrt(6) / (2 * np.pi * n * snr)
    assert abs(sigma / want - 1) < 0.15
