"""Continuous-batching server: every frame's beams are the same alone and in a mix of
concurrent frames from several lattices, match the oracle, and admission stays within
the device-slot budget."""
import numpy as np
import pytest

import synth
from helpers import TOL_BEAM, oracle_beams

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1710_08591_gb300 as fb  # noqa: E402

# serving lattices (nx, ny); one frame = n_int samples x NFREQ channels x 2 pols
SERVE_LATTICES = [(4, 256), (8, 64), (16, 16)]
NFREQ, NINT, NPOL = 4, 64, 2


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fb.build()
    plans, frames, weights = [], [], []
    for k, (nx, ny) in enumerate(SERVE_LATTICES):
        w = synth.separable_weights(synth.half_sine(nx), synth.half_sine(ny))
        plans.append(fb.plan_create(nx, ny, nx, 2 * synth.next_pow2(ny), NPOL, NFREQ, NINT, weights=w))
        weights.append(w)
        frames.append([synth.volts(NINT, NFREQ, NPOL, nx, ny, seed=500 + 10 * k + j,
                                   sources=synth.seeded_sources(600 + k + j, 2, 1.5))
                       for j in range(3)])
    yield plans, frames, weights
    for p in plans:
        p.close()


def _out(plan):
    return np.full((plan.nfreq, plan.pad_x, plan.pad_y), np.nan, dtype=np.float32)


def test_frames_same_alone_and_in_mix(setup):
    plans, frames, weights = setup
    budget = 1 << 30
    # alone: one frame at a time
    alone = {}
    with fb.server_create(plans, budget) as sv:
        for k in range(len(plans)):
            for j in range(3):
                out = _out(plans[k])
                t = fb.server_submit(sv, k, frames[k][j], out)
                fb.server_wait(sv, t, 60.0)
                alone[(k, j)] = out
    # mix: everything submitted while the server is held, interleaved across lattices,
    # twice over, then released: the frames go out together
    mixed = {}
    with fb.server_create(plans, budget) as sv:
        fb.server_hold(sv, True)
        for rep in range(2):
            for j in range(3):
                for k in range(len(plans)):
                    out = _out(plans[k])
                    fb.server_submit(sv, k, frames[k][j], out)
                    mixed[(k, j, rep)] = out
        fb.server_hold(sv, False)
        fb.server_wait(sv, -1, 120.0)
        st = fb.server_stats(sv)
    assert st["completed"] == st["submitted"] == 18
    # a mix happened: frames of all three lattices shared launches and were in flight together
    assert st["max_frames_per_launch"] > 1 and st["frames_per_launch"] > 1, st
    assert st["launches"] < st["submitted"] and st["peak_inflight"] > 1, st
    assert st["p99_ms"] >= st["p50_ms"] > 0.0
    for (k, j, rep), out in mixed.items():
        assert np.array_equal(out, alone[(k, j)]), (k, j, rep)
    # and each lattice's frames match the FP64 oracle
    for k, (nx, ny) in enumerate(SERVE_LATTICES):
        my = 2 * synth.next_pow2(ny)
        ref = oracle_beams(frames[k][0], weights[k], nx, ny, nx, my, NPOL, NFREQ, NINT)[0]
        err = np.abs(alone[(k, 0)] - ref) / ref
        assert err.max() <= TOL_BEAM


def test_admission_bounded_by_budget(setup):
    plans, frames, _ = setup
    nx, ny = SERVE_LATTICES[0]
    slot = NINT * NFREQ * NPOL * nx * ny + NFREQ * nx * 2 * synth.next_pow2(ny) * 4
    budget = 3 * slot + 4096                         # three slots
    outs = []
    with fb.server_create(plans, budget) as sv:
        for i in range(12):
            out = _out(plans[i % 3])
            fb.server_submit(sv, i % 3, frames[i % 3][i % 3 % 3], out)
            outs.append(out)
        fb.server_wait(sv, -1, 120.0)
        st = fb.server_stats(sv)
    assert st["slots"] <= 3 and st["peak_inflight"] <= st["slots"]
    assert st["completed"] == 12
    assert all(np.all(np.isfinite(o)) for o in outs)


def test_bad_lattice_index_rejected(setup):
    plans, frames, _ = setup
    with fb.server_create(plans, 1 << 28) as sv:
        with pytest.raises(fb.FftbfError) as e:
            fb.server_submit(sv, 7, frames[0][0], _out(plans[0]))
        assert e.value.code == -1


def test_burst_beyond_the_grid_same_as_alone():
    """A held burst of 63 frames of 16 channels each (1008 work items in one launch, more
    than the launch's CTAs, so CTAs take several items from the queue): every frame's
    beams are bit-identical to the same frame served alone."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fb.build()
    nf, nint = 16, 32
    plans, frames = [], []
    for k, (nx, ny) in enumerate(SERVE_LATTICES):
        w = synth.separable_weights(synth.half_sine(nx), synth.half_sine(ny))
        plans.append(fb.plan_create(nx, ny, nx, 2 * synth.next_pow2(ny), NPOL, nf, nint, weights=w))
        frames.append([synth.volts(nint, nf, NPOL, nx, ny, seed=700 + 10 * k + j,
                                   sources=synth.seeded_sources(800 + k + j, 2, 1.5))
                       for j in range(3)])
    try:
        alone = {}
        with fb.server_create(plans, 1 << 30) as sv:
            for k in range(3):
                for j in range(3):
                    out = _out(plans[k])
                    fb.server_wait(sv, fb.server_submit(sv, k, frames[k][j], out), 60.0)
                    alone[(k, j)] = out
        burst = []
        with fb.server_create(plans, 1 << 30) as sv:
            fb.server_hold(sv, True)
            for i in range(63):
                k, j = i % 3, (i // 3) % 3
                out = _out(plans[k])
                fb.server_submit(sv, k, frames[k][j], out)
                burst.append((k, j, out))
            fb.server_hold(sv, False)
            fb.server_wait(sv, -1, 120.0)
            st = fb.server_stats(sv)
        assert st["max_frames_per_launch"] == 63 and st["launches"] == 1, st
        assert st["max_items_per_launch"] == 63 * nf > st["grid"], st
        for k, j, out in burst:
            assert np.array_equal(out, alone[(k, j)]), (k, j)
    finally:
        for p in plans:
            p.close()
