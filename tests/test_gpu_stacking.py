"""Stacked visibilities recovered from FFT-beam intensities on the GPU vs the oracle."""
import numpy as np
import pytest

import oracle
from helpers import make_case, oracle_beams

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1710_08591_gb300 as fb  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fb.build()


@pytest.mark.parametrize("shape", [(3, 8, 5, 16, 2, 3, 32, 16),      # both axes invertible
                                   (4, 256, 4, 512, 2, 2, 384, 384),  # E-W kept, N-S lags
                                   (2, 16, 2, 32, 1, 8, 64, 16),      # the tiny workload
                                   (3, 40, 3, 128, 2, 2, 32, 16),     # odd E-W rows: a row paired with zeros
                                   (2, 10, 3, 24, 1, 2, 16, 8),       # N-S pad not a power of two: direct route
                                   (3, 256, 3, 512, 2, 3, 64, 32),    # warp route: two row pairs, one row alone
                                   (1, 200, 1, 512, 1, 3, 48, 16),    # warp route: one row, 8 tiles per step
                                   (8, 64, 8, 512, 1, 2, 16, 8)])     # warp route: four row pairs
def test_stacked_visibilities_match_oracle(shape):
    nx, ny, mx, my, npol, nfreq, T, n_int = shape
    v8, w = make_case(nx, ny, mx, my, npol, nfreq, T, n_int, weights="random", seed=90)
    dv = torch.from_numpy(v8.reshape(-1)).cuda()
    nwin = T // n_int
    P = torch.empty((nwin, nfreq, mx, my), device="cuda")
    with fb.plan_create(nx, ny, mx, my, npol, nfreq, n_int, weights=w) as plan:
        dx, dy = fb.stacked_shape(plan)
        vis = torch.full((nwin, nfreq, dx, dy), complex(float("nan"), 0), dtype=torch.complex64,
                         device="cuda")
        fb.execute(plan, dv, T, P)
        fb.stacked_visibilities(plan, P, nwin, vis)
        fb.plan_sync(plan)
    got = vis.cpu().numpy()
    Pref = oracle_beams(v8, w, nx, ny, mx, my, npol, nfreq, n_int)
    ref = oracle.stacked_from_beams(Pref, nx, ny)
    assert got.shape == ref.shape
    # error relative to the zero-lag (total-power) term of each (window, channel)
    scale = np.abs(ref).reshape(nwin, nfreq, -1).max(axis=-1)[..., None, None]
    assert (np.abs(got - ref) / scale).max() <= 1e-5
    if mx >= 2 * nx - 1 and my >= 2 * ny - 1:     # and the visibilities formed from voltages
        x = oracle.unpack(v8)
        vref = oracle.stacked_visibilities(x, w.astype(np.complex128), n_int)
        assert (np.abs(got - vref) / scale).max() <= 1e-5
