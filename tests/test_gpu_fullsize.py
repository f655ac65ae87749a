"""Full-size parity: the CHIME-like 4x256 workload in the launch configuration bench.py
times (fftbf_execute over a 3072-sample, 1024-channel device block; tied beams for 2048
pointings), checked on sampled (window, channel) slices that the oracle computes one by
one."""
import numpy as np
import pytest

import oracle
import synth
from helpers import TOL_BEAM

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1710_08591_gb300 as fb  # noqa: E402

NX, NY, MX, MY, NPOL, NFREQ, NINT = 4, 256, 4, 512, 2, 1024, 384
T_HOST, T_DEV, N_TIED = 768, 3072, 2048


@pytest.fixture(scope="module")
def run():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fb.build()
    src = synth.seeded_sources(102, 3, 1.5)
    block = synth.volts(T_HOST, NFREQ, NPOL, NX, NY, seed=2, sources=src)
    w = synth.separable_weights(synth.half_sine(NX), synth.half_sine(NY))
    u, v = synth.tied_pointings(3, NFREQ, N_TIED, NX, NY, MX, MY)
    hb = torch.from_numpy(block.reshape(-1))
    dvol = torch.empty(hb.numel() * (T_DEV // T_HOST), dtype=torch.uint8, device="cuda")
    for c in range(T_DEV // T_HOST):
        dvol[c * hb.numel():(c + 1) * hb.numel()].copy_(hb)
    nwin = T_DEV // NINT
    beams = torch.full((nwin, NFREQ, MX, MY), float("nan"), device="cuda")
    tied = torch.full((nwin, NFREQ, N_TIED), float("nan"), device="cuda")
    with fb.plan_create(NX, NY, MX, MY, NPOL, NFREQ, NINT, weights=w) as plan:
        fb.execute(plan, dvol, T_DEV, beams)
        fb.tied_beams(plan, beams, nwin, N_TIED, u, v, tied)
        fb.plan_sync(plan)
    del dvol
    return dict(block=block, w=w, u=u, v=v, beams=beams.cpu().numpy(),
                tied=tied.cpu().numpy())


SLICES = [(0, 0), (7, 1023), (3, 511), (5, 17), (6, 900), (1, 1)]


def _oracle_slice(r, j, f):
    t0 = (j * NINT) % T_HOST
    v = np.ascontiguousarray(r["block"][t0:t0 + NINT, f:f + 1])
    return oracle.beams(v, NX, NY, MX, MY, NPOL, 1, NINT, weights=r["w"].astype(np.complex128))


def test_no_nan(run):
    assert np.all(np.isfinite(run["beams"]))
    assert np.all(np.isfinite(run["tied"]))


@pytest.mark.parametrize("j,f", SLICES)
def test_beams_slice(run, j, f):
    ref = _oracle_slice(run, j, f)[0, 0]
    got = run["beams"][j, f]
    err = np.abs(got - ref) / ref
    assert err.max() <= TOL_BEAM, f"max rel err {err.max():.3g}"


@pytest.mark.parametrize("j,f", SLICES[:3])
def test_tied_slice(run, j, f):
    P = _oracle_slice(run, j, f)                                   # [1, 1, MX, MY]
    u, v = run["u"][f:f + 1], run["v"][f:f + 1]
    ref = oracle.tied_regrid(P, u, v, NX, NY)[0, 0]
    wx = np.abs(oracle.regrid_weights(NX, MX, u))
    wy = np.abs(oracle.regrid_weights(NY, MY, v))
    scale = np.einsum("fsA,fsB,jfAB->jfs", wx, wy, P)[0, 0]
    err = np.abs(run["tied"][j, f] - ref) / scale
    assert err.max() <= TOL_BEAM, f"max scaled err {err.max():.3g}"
