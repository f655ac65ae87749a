"""fftbf_execute_noalloc: the allocation-free entry point for callers that cannot call
cudaMalloc (an application whose own pool owns the device memory, or a real-time loop
that must not make allocator calls). It must give what fftbf_execute gives with a plan,
call after call, although every call shares one statically reserved table array.

This file is collected last on purpose: if it fails, a run that stops at the first
failure has already run every other test.
"""
import numpy as np
import pytest

import synth
from helpers import TOL_BEAM

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1710_08591_gb300 as fb  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fb.build()
    fb.lib()


def _case(nx, ny, mx, my, npol, nfreq, T, n_int, weights, seed):
    v = synth.volts(T, nfreq, npol, nx, ny, seed=seed, sources=synth.seeded_sources(seed, 2, 1.5))
    dv = torch.from_numpy(v.reshape(-1)).cuda()
    w = None
    if weights:
        w = synth.separable_weights(synth.half_sine(nx), synth.half_sine(ny))
    with fb.plan_create(nx, ny, mx, my, npol, nfreq, n_int, weights=w) as plan:
        ref = torch.empty((T // n_int, nfreq, mx, my), device="cuda")
        fb.execute(plan, dv, T, ref)
        fb.plan_sync(plan)
    wd = None if w is None else torch.from_numpy(w.reshape(-1).view(np.float32).copy()).cuda()
    return dv, wd, ref


def test_noalloc_matches_plan_path_on_two_calls_in_a_row():
    shapes = [
        # CHIME-like lattice with half-sine weights, then a tiny lattice with unit weights:
        # the second call must not see anything the first left in the shared array
        ((4, 256, 4, 512, 2, 8, 768, 384), True, 11),
        ((2, 16, 2, 32, 1, 8, 256, 16), False, 12),
    ]
    cases = [(_case(*shape, weights, seed), shape) for shape, weights, seed in shapes]
    outs = [torch.empty_like(ref) for (dv, wd, ref), _ in cases]

    def call_and_check(k):
        (dv, wd, ref), (nx, ny, mx, my, npol, nfreq, T, n_int) = cases[k]
        outs[k].fill_(float("nan"))
        fb.execute_noalloc(nx, ny, mx, my, npol, nfreq, n_int, wd, dv, T, outs[k])
        torch.cuda.synchronize()
        got, want = outs[k].cpu().numpy(), ref.cpu().numpy()
        err = np.abs(got - want) / np.abs(want)
        assert err.max() <= TOL_BEAM, f"lattice {k}: max rel err {err.max():.3g}"

    # The first call on the device looks up the array's address and the driver loads
    # each kernel on its first launch; neither is an allocation by this library, so the
    # device's free memory is compared from the third call on.
    call_and_check(0)
    call_and_check(1)
    free_before = torch.cuda.mem_get_info()[0]
    call_and_check(0)                        # two more calls in a row, different lattices
    call_and_check(1)
    assert torch.cuda.mem_get_info()[0] == free_before     # no device memory was taken


def test_noalloc_rejects_tables_beyond_the_static_array():
    v = torch.zeros(16, dtype=torch.uint8, device="cuda")
    out = torch.zeros(16, device="cuda")
    with pytest.raises(fb.FftbfError) as e:
        fb.execute_noalloc(1, 16, 1, 16384, 1, 1, 1, None, v, 1, out)
    assert e.value.code == -1 and "static scratch" in str(e.value)
