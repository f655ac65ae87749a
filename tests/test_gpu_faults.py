"""Failure detection without faulting the GPU: bounded device waits return an error
status the host reads and the context stays usable; host-side faults of the server
(bad frames, a frame that cannot complete in time) give error statuses and leave the
other frames' results unchanged."""
import time

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


def test_bounded_wait_runs_out_and_context_survives():
    t0 = time.perf_counter()
    rc = fb.debug_wait_timeout(20000)            # 20 ms on a barrier nothing arrives on
    dt = time.perf_counter() - t0
    assert rc == -4                               # FFTBF_ETIMEOUT
    assert "ran out" in fb.last_error()
    assert dt < 10.0
    # the context is intact: a normal transform still runs and is correct
    nx, ny, mx, my, npol, nfreq, T, n_int = 4, 256, 4, 512, 2, 2, 32, 16
    v, w = make_case(nx, ny, mx, my, npol, nfreq, T, n_int, weights="half_sine", seed=3)
    dv = torch.from_numpy(v.reshape(-1)).cuda()
    out = torch.empty((T // n_int, nfreq, mx, my), device="cuda")
    with fb.plan_create(nx, ny, mx, my, npol, nfreq, n_int, weights=w) as plan:
        fb.plan_set_precision(plan, fb.PREC_TC_FP16)
        fb.execute(plan, dv, T, out)
        fb.plan_sync(plan)
    assert torch.isfinite(out).all()


def test_server_faults_leave_other_frames_unchanged():
    nx, ny, nf, n_int = 8, 64, 4, 32
    plan = fb.plan_create(nx, ny, nx, 128, 2, nf, n_int)
    good = [synth.volts(n_int, nf, 2, nx, ny, seed=70 + i) for i in range(3)]
    with fb.server_create([plan], 1 << 28) as sv:
        ref = []
        for fr in good:
            out = np.empty((nf, nx, 128), np.float32)
            fb.server_wait(sv, fb.server_submit(sv, 0, fr, out), 60.0)
            ref.append(out)
        # malformed requests are refused up front
        with pytest.raises(fb.FftbfError):
            fb.server_submit(sv, 3, good[0], np.empty((nf, nx, 128), np.float32))
        with pytest.raises(ValueError):
            fb.server_submit(sv, 0, good[0][:, ::2], np.empty((nf, nx, 128), np.float32))
        # a wait that cannot be met in time reports ETIMEOUT (the server is held, so the
        # frames are staged but not launched); released, the frames still complete
        outs = []
        tickets = []
        fb.server_hold(sv, True)
        for fr in good:
            o = np.empty((nf, nx, 128), np.float32)
            tickets.append(fb.server_submit(sv, 0, fr, o))
            outs.append(o)
        with pytest.raises(fb.FftbfError) as e:
            fb.server_wait(sv, tickets[-1], 0.05)
        assert e.value.code == -4
        # a ticket that was never issued is refused, not waited for
        with pytest.raises(fb.FftbfError) as e:
            fb.server_wait(sv, tickets[-1] + 1000, 0.05)
        assert e.value.code == -1
        fb.server_hold(sv, False)
        fb.server_wait(sv, -1, 60.0)
        for o, r in zip(outs, ref):
            assert np.array_equal(o, r)
    plan.close()
