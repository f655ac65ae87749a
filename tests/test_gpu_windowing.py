"""Optimal windowed and truncated tied beams on the GPU vs the FP64 oracle."""
import numpy as np
import pytest

import oracle
import synth
from helpers import TOL_BEAM, make_case, oracle_beams

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1710_08591_gb300 as fb  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fb.build()


def _weights(n, m, y, h, trunc, grid):
    if grid:
        w = oracle.regrid_weights(n, m, y)
    elif h is None:
        w = oracle.regrid_weights(n, m, y)
    else:
        w = oracle.windowed_regrid_weights(n, m, y, oracle.window_lag_coeffs(h))
    if trunc and not grid:
        w = oracle.truncate_nearest(w, y, m, trunc)
    return w


CASES = [
    # nx, ny, mx, my, npol, nfreq, T, n_int, n_tied, window x?, window y?, trunc x, trunc y
    (3, 8, 5, 16, 2, 3, 32, 16, 37, True, True, 0, 0),      # dense windowed GEMM path
    (3, 8, 5, 16, 2, 3, 32, 16, 37, True, True, 3, 5),      # compact path, both truncated
    (3, 8, 5, 16, 2, 3, 32, 16, 37, False, True, 5, 4),     # Dirichlet x truncated, window y
    (4, 256, 4, 512, 2, 2, 384, 384, 64, False, True, 0, 5),  # grid E-W x windowed N-S, 5 taps
    (4, 256, 4, 512, 2, 2, 384, 384, 64, False, True, 0, 0),  # grid E-W x windowed N-S, dense
]


@pytest.mark.parametrize("case", CASES)
def test_windowed_tied_beams_match_oracle(case):
    nx, ny, mx, my, npol, nfreq, T, n_int, n_tied, wxo, wyo, tx, ty = case
    v8, w = make_case(nx, ny, mx, my, npol, nfreq, T, n_int, weights="random", seed=61)
    rng = np.random.default_rng(7)
    gx = mx < 2 * nx - 1
    u = rng.integers(0, mx, (nfreq, n_tied)) / mx if gx else rng.random((nfreq, n_tied))
    v = rng.random((nfreq, n_tied))
    hx = synth.half_sine(nx) if wxo else None
    hy = (0.2 + synth.half_sine(ny)) if wyo else None
    nwin = T // n_int
    dv = torch.from_numpy(v8.reshape(-1)).cuda()
    P = torch.empty((nwin, nfreq, mx, my), device="cuda")
    out = torch.full((nwin, nfreq, n_tied), float("nan"), device="cuda")
    with fb.plan_create(nx, ny, mx, my, npol, nfreq, n_int, weights=w) as plan:
        fb.execute(plan, dv, T, P)
        fb.tied_set_window(plan, hx, hy, tx, ty)
        fb.tied_beams(plan, P, nwin, n_tied, u, v, out)
        fb.plan_sync(plan)
        got = out.cpu().numpy()
        # back to the plain kernel: same as the un-windowed oracle
        fb.tied_set_window(plan)
        fb.tied_beams(plan, P, nwin, n_tied, u, v, out)
        fb.plan_sync(plan)
        plain = out.cpu().numpy()
    Pref = oracle_beams(v8, w, nx, ny, mx, my, npol, nfreq, n_int)
    wxr = _weights(nx, mx, u, hx, tx, gx)
    wyr = _weights(ny, my, v, hy, ty, False)
    ref = np.einsum("fsA,fsB,jfAB->jfs", wxr, wyr, Pref)
    scale = np.einsum("fsA,fsB,jfAB->jfs", np.abs(wxr), np.abs(wyr), Pref)
    assert np.all(np.isfinite(got))
    assert (np.abs(got - ref) / scale).max() <= TOL_BEAM
    pref = oracle.tied_regrid(Pref, u, v, nx, ny)
    pscale = np.einsum("fsA,fsB,jfAB->jfs", np.abs(oracle.regrid_weights(nx, mx, u)),
                       np.abs(oracle.regrid_weights(ny, my, v)), Pref)
    assert (np.abs(plain - pref) / pscale).max() <= TOL_BEAM


def test_window_rejected_on_unpadded_axis():
    with fb.plan_create(4, 256, 4, 512, 2, 1, 8) as plan:
        with pytest.raises(fb.FftbfError) as e:
            fb.tied_set_window(plan, hx=synth.half_sine(4))
        assert e.value.code == -1
