"""Tensor-core form: the tcgen05 GEMM building block against numpy, and the fused
tensor-core beam kernel against the FP64 oracle (its error is reported and bounded)."""
import numpy as np
import pytest

from helpers import make_case, oracle_beams

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1710_08591_gb300 as fb  # noqa: E402

# Stated bounds of the 16-bit forms, max over beams of |P_tc - P_ref| / P_ref on the
# CHIME-like lattice with half-sine weights (two roundings of the complex field to
# 11-bit (FP16) or 8-bit (BF16) significands, before each GEMM stage).
TOL_TC = {"fp16": 5e-3, "bf16": 3e-2}
RMS_TC = {"fp16": 1e-3, "bf16": 6e-3}
# The split-FP16 form (hi + lo operands, three products per stage) is held to the FP32
# form's bound: 1e-5 of each beam.
TOL_TC["fp16x3"] = 1e-5
RMS_TC["fp16x3"] = 2e-6
PREC = {"fp16": fb.PREC_TC_FP16, "bf16": fb.PREC_TC_BF16, "fp16x3": fb.PREC_TC_FP16X3}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fb.build()
    fb.lib()


@pytest.mark.parametrize("bf16", [False, True], ids=["fp16", "bf16"])
@pytest.mark.parametrize("padded", [0, 1, 2, 3, 4], ids=["canon", "padded", "mn-major", "a-tmem", "b-mn-major"])
@pytest.mark.parametrize("n", [32, 64, 128])
def test_tc_gemm_building_block(bf16, padded, n):
    rng = np.random.default_rng(n + 2 * padded + bf16)
    dt = torch.bfloat16 if bf16 else torch.float16
    A = torch.from_numpy(rng.normal(size=(128, 32)).astype(np.float32)).to(dt)
    B = torch.from_numpy(rng.normal(size=(n, 32)).astype(np.float32)).to(dt)
    # distinct exact rows/columns so that a transposed or shifted layout cannot pass
    A[:, 0] = torch.arange(128, dtype=torch.float32).to(dt)
    B[:, 1] = torch.arange(n, dtype=torch.float32).to(dt)
    ref = A.float().numpy().astype(np.float64) @ B.float().numpy().astype(np.float64).T
    da = A.cuda().view(torch.int16)
    db = B.cuda().view(torch.int16)
    d = torch.full((128, n), float("nan"), device="cuda")
    fb.debug_tc_gemm(da, db, n, bf16, padded, d)
    got = d.cpu().numpy()
    assert np.all(np.isfinite(got))
    assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max()


def run_tc(v, w, shape, form):
    nx, ny, mx, my, npol, nfreq, T, n_int = shape
    dv = torch.from_numpy(np.ascontiguousarray(v).reshape(-1)).cuda()
    out = torch.full((T // n_int, nfreq, mx, my), float("nan"), device="cuda")
    with fb.plan_create(nx, ny, mx, my, npol, nfreq, n_int, weights=w) as plan:
        fb.plan_set_precision(plan, PREC[form])
        fb.execute(plan, dv, T, out)
        fb.plan_sync(plan)
    return out.cpu().numpy()


SHAPES = [
    ((4, 256, 4, 512, 2, 3, 768, 384), "half_sine"),    # CHIME-like lattice
    ((4, 256, 4, 512, 1, 2, 30, 5), "random"),          # one pol, ragged: 5 snapshots, 2 per step
    ((3, 200, 4, 512, 2, 2, 32, 16), "random"),         # E-W padded 3 -> 4, 200 N-S feeds
    ((4, 200, 4, 512, 2, 2, 32, 16), "half_sine"),      # real weights, rows of 200 feeds
    ((4, 160, 4, 512, 1, 2, 16, 8), "half_sine"),       # real weights, rows of 160 feeds
]


@pytest.mark.parametrize("form", ["fp16", "bf16", "fp16x3"])
@pytest.mark.parametrize("shape,wk", SHAPES, ids=lambda x: "x".join(map(str, x)) if isinstance(x, tuple) else x)
def test_tc_beams_match_oracle(form, shape, wk):
    v, w = make_case(*shape, weights=wk, seed=31)
    got = run_tc(v, w, shape, form)
    nx, ny, mx, my, npol, nfreq, T, n_int = shape
    ref = oracle_beams(v, w, nx, ny, mx, my, npol, nfreq, n_int)
    assert np.all(np.isfinite(got))
    rel = np.abs(got - ref) / ref
    rms = float(np.sqrt(np.mean(rel ** 2)))
    print(f"\n[tc error] form={form} shape={shape} weights={wk}: max rel {rel.max():.3e}, "
          f"rms rel {rms:.3e}")
    assert rel.max() <= TOL_TC[form]
    assert rms <= RMS_TC[form]


@pytest.mark.parametrize("form", ["fp16", "bf16"])
def test_tc_serial_kernel_matches_pipelined(form, monkeypatch):
    """The serial kernel (FFTBF_TC_KERNEL=serial; the default for BF16) and the first
    warp-specialised kernel (FFTBF_TC_PIPE=1) compute the same sums in the same order:
    bit-identical results."""
    shape = (4, 256, 4, 512, 2, 3, 96, 48)
    v, w = make_case(*shape, weights="half_sine", seed=8)
    monkeypatch.setenv("FFTBF_TC_KERNEL", "serial")
    serial = run_tc(v, w, shape, form)
    monkeypatch.delenv("FFTBF_TC_KERNEL")
    monkeypatch.setenv("FFTBF_TC_PIPE", "1")
    piped = run_tc(v, w, shape, form)
    diff = np.abs(piped - serial) / np.abs(serial)
    assert np.array_equal(piped, serial), f"max rel diff {diff.max():.3e} at {np.argmax(diff)}"


@pytest.mark.parametrize("form", ["fp16", "bf16"])
@pytest.mark.parametrize("wk", ["half_sine", "random"])
@pytest.mark.parametrize("npol,n_int,T", [(2, 48, 96), (1, 5, 30), (2, 3, 12)],
                         ids=["2pol", "1pol-odd", "2pol-short"])
def test_tc_16bit_kernels_agree_with_oracle(form, wk, npol, n_int, T, monkeypatch):
    """The grouped kernel (default for aligned 4x256 voltages), the pair-wise
    warp-specialised kernel and the serial kernel of the FP16 and BF16 forms, each against
    the oracle at the form's bounds, on
    real and complex weights, one or two polarisations and an odd snapshot count (a pair
    with one snapshot)."""
    shape = (4, 256, 4, 512, npol, 3, T, n_int)
    v, w = make_case(*shape, weights=wk, seed=9 + npol + n_int)
    ref = oracle_beams(v, w, 4, 256, 4, 512, npol, 3, n_int)
    for kern in ("grouped", "ws", "serial"):
        monkeypatch.setenv("FFTBF_TC_KERNEL", kern)
        got = run_tc(v, w, shape, form)
        rel = np.abs(got - ref) / ref
        assert np.all(np.isfinite(got)), kern
        assert rel.max() <= TOL_TC[form], (kern, rel.max())
        assert np.sqrt(np.mean(rel ** 2)) <= RMS_TC[form], kern


def test_tc_bit_identical_alone_and_in_batch():
    shape = (4, 256, 4, 512, 2, 4, 128, 32)
    v, w = make_case(*shape, weights="half_sine", seed=5)
    full = run_tc(v, w, shape, "fp16")
    again = run_tc(v, w, shape, "fp16")
    assert np.array_equal(full, again)
    one = run_tc(v[32:64], w, (4, 256, 4, 512, 2, 4, 32, 32), "fp16")
    assert np.array_equal(one[0], full[1])


def test_tc_rejects_unsupported_lattice():
    with fb.plan_create(2, 16, 2, 32, 1, 2, 4) as plan:
        with pytest.raises(fb.FftbfError) as e:
            fb.plan_set_precision(plan, fb.PREC_TC_FP16)
        assert e.value.code == -5
