"""The seeded input generator: determinism, layout and distribution (no method arithmetic)."""
import numpy as np

import synth

MASK = (1 << 64) - 1


def _splitmix64_py(state, k):
    z = (state + k * 0x9E3779B97F4A7C15) & MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
    return z ^ (z >> 31)


def test_splitmix64_published_first_output():
    # first output of SplitMix64 seeded with 0 (Steele, Lea and Flood 2014)
    assert synth.splitmix64_draw(0, 1) == 0xE220A8397B1DCDAF
    for s, k in ((0, 2), (12345, 7), (MASK, 3)):
        assert synth.splitmix64_draw(s, k) == _splitmix64_py(s, k)


def test_deterministic_and_time_offset():
    a = synth.volts(8, 3, 2, 4, 16, seed=11, sources=synth.seeded_sources(1, 2, 1.5))
    b = synth.volts(8, 3, 2, 4, 16, seed=11, sources=synth.seeded_sources(1, 2, 1.5),
                    nthreads=1)
    c = synth.volts(3, 3, 2, 4, 16, seed=11, sources=synth.seeded_sources(1, 2, 1.5), t0=5)
    assert a.shape == (8, 3, 2, 4, 16)
    assert np.array_equal(a, b)
    assert np.array_equal(a[5:], c)


def test_range_and_distribution():
    v = synth.volts(64, 4, 2, 4, 64, seed=3)
    hi = (v >> 4).astype(np.int64)
    lo = (v & 15).astype(np.int64)
    re = np.where(hi >= 8, hi - 16, hi)
    im = np.where(lo >= 8, lo - 16, lo)
    assert re.min() >= -7 and re.max() <= 7 and im.min() >= -7 and im.max() <= 7
    assert abs(re.mean()) < 0.05 and abs(im.mean()) < 0.05
    # rounding adds 1/12 variance; clipping at 7 removes a little
    assert 2.4 < re.std() < 2.6 and 2.4 < im.std() < 2.6


def test_source_is_coherent_across_lattice():
    # a strong on-grid source dominates: the lattice-summed field with the conjugate
    # steering phase carries n^2 |amp|^2 of power on average
    nx, ny = 2, 8
    v = synth.volts(256, 1, 1, nx, ny, seed=5, sigma=0.0, sources=[(0.5, 0.25, 6.0)])
    hi = (v >> 4).astype(np.int64)
    lo = (v & 15).astype(np.int64)
    x = np.where(hi >= 8, hi - 16, hi) + 1j * np.where(lo >= 8, lo - 16, lo)
    ix = np.arange(nx)[:, None]
    iy = np.arange(ny)[None, :]
    steer = np.exp(-2j * np.pi * (ix * 0.5 + iy * 0.25))
    y = (x[:, 0, 0] * steer).sum(axis=(1, 2))
    assert abs(np.mean(np.abs(y) ** 2) / (16 * 16 * 36) - 1) < 0.05
