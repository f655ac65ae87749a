"""Tied-array beams on the tensor cores (split FP16 operands, FP32 accumulation) against
the FP64 oracle and against the CUDA-core GEMM, with the E-W axis on the FFT-beam grid:
full and partial tiles of 128 pointings and of 128 windows, one to four E-W beams."""
import numpy as np
import pytest

import oracle
from helpers import TOL_BEAM, make_case, oracle_beams

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1710_08591_gb300 as fb  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fb.build()
    fb.lib()


def _scale(P, u, v, nx, ny):
    """sum_{A,B} |w^A w^B| P: the natural size of the FP32 rounding error of a tied beam."""
    wx = np.abs(oracle.regrid_weights(nx, P.shape[-2], u))
    wy = np.abs(oracle.regrid_weights(ny, P.shape[-1], v))
    return np.einsum("fsA,fsB,jfAB->jfs", wx, wy, P)


def _tied(P_dev, shape, w, u, v, n_tied):
    nx, ny, mx, my, npol, nfreq, T, n_int = shape
    nwin = T // n_int
    out = torch.full((nwin, nfreq, n_tied), float("nan"), device="cuda")
    with fb.plan_create(nx, ny, mx, my, npol, nfreq, n_int, weights=w) as plan:
        fb.tied_beams(plan, P_dev, nwin, n_tied, u, v, out)
        fb.plan_sync(plan)
    return out.cpu().numpy()


@pytest.mark.parametrize("shape,n_tied", [((4, 256, 4, 512, 1, 2, 1024, 8), 300),   # 3 pointing tiles
                                          ((4, 64, 4, 128, 1, 3, 1040, 8), 150),    # 130 windows: 2 tiles
                                          ((2, 64, 2, 128, 2, 2, 64, 16), 200)])    # 2 E-W beams
def test_tied_tensor_core_matches_oracle_and_cuda_cores(shape, n_tied, monkeypatch):
    nx, ny, mx, my, npol, nfreq, T, n_int = shape
    v8, w = make_case(nx, ny, mx, my, npol, nfreq, T, n_int, weights="random", seed=33)
    nwin = T // n_int
    P = torch.empty((nwin, nfreq, mx, my), device="cuda")
    with fb.plan_create(nx, ny, mx, my, npol, nfreq, n_int, weights=w) as plan:
        fb.execute(plan, torch.from_numpy(v8.reshape(-1)).cuda(), T, P)
        fb.plan_sync(plan)
    rng = np.random.default_rng(9)
    u = rng.integers(0, mx, (nfreq, n_tied)) / mx            # E-W on the FFT-beam columns
    v = rng.random((nfreq, n_tied))
    got = _tied(P, shape, w, u, v, n_tied)
    assert np.all(np.isfinite(got))
    Pn = P.cpu().numpy().astype(np.float64)
    scale = _scale(Pn, u, v, nx, ny)
    # against the regridding of the same FP32 beams in FP64, and of the oracle's beams
    assert (np.abs(got - oracle.tied_regrid(Pn, u, v, nx, ny)) / scale).max() <= TOL_BEAM
    Pref = oracle_beams(v8, w, nx, ny, mx, my, npol, nfreq, n_int)
    assert (np.abs(got - oracle.tied_regrid(Pref, u, v, nx, ny)) / scale).max() <= TOL_BEAM
    monkeypatch.setenv("FFTBF_TIED_TC", "0")                 # the CUDA-core GEMM
    simt = _tied(P, shape, w, u, v, n_tied)
    assert (np.abs(got - simt) / scale).max() <= TOL_BEAM


def test_tied_falls_back_to_cuda_cores_when_split_tables_do_not_fit(monkeypatch):
    """With the split tables unallocatable (a test hook makes tied_tc_build report
    FFTBF_ENOMEM without touching the allocator), the call succeeds on the CUDA-core GEMM,
    matches the oracle's regridding and leaves no error behind on the thread."""
    shape = (4, 256, 4, 512, 1, 2, 256, 8)
    nx, ny, mx, my, npol, nfreq, T, n_int = shape
    v8, w = make_case(nx, ny, mx, my, npol, nfreq, T, n_int, weights="random", seed=44)
    nwin, n_tied = T // n_int, 130
    P = torch.empty((nwin, nfreq, mx, my), device="cuda")
    with fb.plan_create(nx, ny, mx, my, npol, nfreq, n_int, weights=w) as plan:
        fb.execute(plan, torch.from_numpy(v8.reshape(-1)).cuda(), T, P)
        fb.plan_sync(plan)
    rng = np.random.default_rng(12)
    u = rng.integers(0, mx, (nfreq, n_tied)) / mx
    v = rng.random((nfreq, n_tied))
    monkeypatch.setenv("FFTBF_TEST_TIED_TC_NOMEM", "1")
    got = _tied(P, shape, w, u, v, n_tied)
    assert fb.last_error_code() == 0 and fb.last_error() == ""
    Pn = P.cpu().numpy().astype(np.float64)
    scale = _scale(Pn, u, v, nx, ny)
    assert np.all(np.isfinite(got))
    assert (np.abs(got - oracle.tied_regrid(Pn, u, v, nx, ny)) / scale).max() <= TOL_BEAM
    monkeypatch.setenv("FFTBF_TIED_TC", "0")
    simt = _tied(P, shape, w, u, v, n_tied)
    assert np.array_equal(got, simt)                         # the same CUDA-core kernel ran
