"""fftbf_execute_host (host buffers, chunked copies overlapped with the transform) gives
the same beams and tied beams as the device entry points."""
import numpy as np
import pytest

import synth
from helpers import make_case

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1710_08591_gb300 as fb  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fb.build()


@pytest.mark.parametrize("pinned", [False, True])
def test_host_pipeline_matches_device_path(pinned):
    nx, ny, mx, my, npol, nfreq, n_int = 4, 256, 4, 512, 2, 64, 384
    T = 6 * n_int                                     # several chunks of whole windows
    v, w = make_case(nx, ny, mx, my, npol, nfreq, T, n_int, weights="half_sine", seed=77)
    n_tied = 33
    u, vv = synth.tied_pointings(9, nfreq, n_tied, nx, ny, mx, my)
    nwin = T // n_int
    if pinned:
        hv = torch.from_numpy(v.reshape(-1)).pin_memory().numpy()
        hb = torch.empty((nwin, nfreq, mx, my), pin_memory=True).numpy()
        ht = torch.empty((nwin, nfreq, n_tied), pin_memory=True).numpy()
    else:
        hv = np.ascontiguousarray(v.reshape(-1))
        hb = np.empty((nwin, nfreq, mx, my), np.float32)
        ht = np.empty((nwin, nfreq, n_tied), np.float32)
    with fb.plan_create(nx, ny, mx, my, npol, nfreq, n_int, weights=w) as plan:
        dv = torch.from_numpy(v.reshape(-1)).cuda()
        db = torch.empty((nwin, nfreq, mx, my), device="cuda")
        dt = torch.empty((nwin, nfreq, n_tied), device="cuda")
        fb.execute(plan, dv, T, db)
        fb.tied_beams(plan, db, nwin, n_tied, u, vv, dt)
        for _ in range(2):                            # second call reuses the staging
            hb[:] = np.nan
            fb.execute_host(plan, hv, T, hb, n_tied, u, vv, ht)
            fb.plan_sync(plan)
            assert np.array_equal(hb, db.cpu().numpy())
            assert np.array_equal(ht, dt.cpu().numpy())
