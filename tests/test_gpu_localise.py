"""Localisation of a point source from FFT beams on the GPU vs the oracle estimator."""
import numpy as np
import pytest

import oracle
import synth
from helpers import oracle_beams

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1710_08591_gb300 as fb  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fb.build()


@pytest.mark.parametrize("shape", [(3, 8, 5, 16, 2, 3, 64, 32),       # both axes fitted
                                   (4, 256, 4, 512, 2, 2, 384, 384),  # E-W on the grid
                                   (2, 16, 4, 32, 1, 4, 64, 16)])
def test_localise_matches_oracle(shape):
    nx, ny, mx, my, npol, nfreq, T, n_int = shape
    src = [(0.3137, 0.6021, 3.0)]                                       # one strong source
    v8 = synth.volts(T, nfreq, npol, nx, ny, seed=33, sigma=1.0, sources=src)
    dv = torch.from_numpy(v8.reshape(-1)).cuda()
    nwin = T // n_int
    P = torch.empty((nwin, nfreq, mx, my), device="cuda")
    out = torch.full((nwin, nfreq, 3), float("nan"), device="cuda")
    with fb.plan_create(nx, ny, mx, my, npol, nfreq, n_int) as plan:
        fb.execute(plan, dv, T, P)
        fb.localise(plan, P, nwin, out, n_iter=5, n_taps=10)
        fb.plan_sync(plan)
    got = out.cpu().numpy()
    ref = oracle.localise(oracle_beams(v8, None, nx, ny, mx, my, npol, nfreq, n_int), nx, ny,
                          n_iter=5, n_taps=10)
    dyx = np.abs(((got[..., 0] - ref[..., 0]) + 0.5) % 1.0 - 0.5)
    dyy = np.abs(((got[..., 1] - ref[..., 1]) + 0.5) % 1.0 - 0.5)
    assert dyx.max() < 2e-6 and dyy.max() < 2e-6
    assert np.allclose(got[..., 2], ref[..., 2], rtol=1e-5)
    # and the estimate sits near the source (quantisation and noise limit the accuracy)
    if my >= 2 * ny - 1:
        assert np.abs(((got[..., 1] - 0.6021) + 0.5) % 1.0 - 0.5).max() < 0.2 / my


@pytest.mark.parametrize("n_iter,n_taps", [(0, 10), (3, 33), (4, 64)])
def test_localise_taps_and_iterations(n_iter, n_taps):
    """More taps than lanes (33, 64: the maximum), no Newton step (the argmax beam), and an
    odd fitted E-W pad."""
    nx, ny, mx, my, npol, nfreq, T, n_int = 3, 32, 7, 64, 2, 2, 32, 16
    v8 = synth.volts(T, nfreq, npol, nx, ny, seed=41, sigma=1.0, sources=[(0.61, 0.27, 3.0)])
    dv = torch.from_numpy(v8.reshape(-1)).cuda()
    nwin = T // n_int
    P = torch.empty((nwin, nfreq, mx, my), device="cuda")
    out = torch.full((nwin, nfreq, 3), float("nan"), device="cuda")
    with fb.plan_create(nx, ny, mx, my, npol, nfreq, n_int) as plan:
        fb.execute(plan, dv, T, P)
        fb.localise(plan, P, nwin, out, n_iter=n_iter, n_taps=n_taps)
        fb.plan_sync(plan)
    got = out.cpu().numpy()
    ref = oracle.localise(oracle_beams(v8, None, nx, ny, mx, my, npol, nfreq, n_int), nx, ny,
                          n_iter=n_iter, n_taps=n_taps)
    for c in (0, 1):
        d = np.abs(((got[..., c] - ref[..., c]) + 0.5) % 1.0 - 0.5)
        assert d.max() < 2e-6, (c, d.max())
    assert np.allclose(got[..., 2], ref[..., 2], rtol=1e-5)


def test_localise_rejects_bad_taps():
    with fb.plan_create(2, 8, 2, 16, 1, 1, 4) as plan:
        P = torch.zeros((1, 1, 2, 16), device="cuda")
        out = torch.zeros((1, 1, 3), device="cuda")
        for bad in (0, 65):
            with pytest.raises(fb.FftbfError) as e:
                fb.localise(plan, P, 1, out, n_iter=2, n_taps=bad)
            assert e.value.code == -1
