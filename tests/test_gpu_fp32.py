"""Parity of the FP32 CUDA path (through the C ABI) with the FP64 oracle."""
import zlib

import numpy as np
import pytest

import oracle
import synth
from helpers import TOL_BEAM, make_case, oracle_beams, rel_err_of_mean, rel_err_per_beam

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1710_08591_gb300 as fb  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fb.build()
    fb.lib()


def run_beams(v, w, nx, ny, mx, my, npol, nfreq, n_int):
    T = v.shape[0]
    dv = torch.from_numpy(np.ascontiguousarray(v).reshape(-1)).cuda()
    out = torch.full((T // n_int, nfreq, mx, my), float("nan"), device="cuda")
    with fb.plan_create(nx, ny, mx, my, npol, nfreq, n_int, weights=w) as plan:
        fb.execute(plan, dv, T, out)
        fb.plan_sync(plan)
    return out.cpu().numpy()


def test_unpack_exhaustive_bit_exact():
    b = np.arange(256, dtype=np.uint16).astype(np.uint8)
    din = torch.from_numpy(b).cuda()
    dout = torch.empty(512, device="cuda")
    fb.debug_unpack(din, 256, dout)
    torch.cuda.synchronize()
    got = dout.cpu().numpy().reshape(256, 2)
    ref = oracle.unpack(b)
    assert np.array_equal(got[:, 0], ref.real.astype(np.float32))
    assert np.array_equal(got[:, 1], ref.imag.astype(np.float32))


CASES = [
    # nx, ny, mx, my, npol, nfreq, T, n_int, weights
    (2, 16, 2, 32, 1, 8, 1024, 16, "uniform"),       # the tiny workload, in full
    (4, 256, 4, 512, 2, 3, 768, 384, "half_sine"),  # CHIME-like lattice
    (4, 64, 4, 128, 2, 2, 96, 24, "random"),
    (3, 128, 3, 256, 2, 2, 64, 16, "half_sine"),    # E-W size 3: folded DFT matrix
    (8, 64, 8, 128, 2, 2, 64, 32, "half_sine"),
    (16, 16, 16, 32, 2, 3, 64, 16, "half_sine"),    # radix-16 E-W butterfly
    (2, 512, 2, 1024, 2, 2, 32, 16, "half_sine"),
    (1, 1024, 1, 2048, 2, 2, 32, 16, "half_sine"),
    (6, 20, 4, 8, 1, 2, 48, 16, "random"),          # cyclic co-adding on both axes
    (4, 32, 7, 63, 1, 2, 32, 8, "random"),          # M = 2n - 1: direct-DFT kernel
    (5, 12, 5, 24, 2, 2, 40, 10, "uniform"),        # E-W size 5: direct-DFT kernel
    (4, 256, 4, 512, 1, 2, 15, 5, "random"),        # ragged: 5 snapshots, 2 per step
    (1, 1, 1, 1, 1, 2, 8, 4, "random"),             # one antenna, one beam
    (1, 2, 1, 4, 1, 3, 12, 3, "uniform"),
    (4, 8, 8, 16, 2, 2, 32, 8, "random"),           # E-W padded: not a plain DFT
    (1, 256, 1, 512, 2, 3, 30, 5, "random"),        # 512-beam kernel, 4 snapshots/step, ragged
    (2, 200, 2, 512, 1, 2, 14, 7, "half_sine"),     # 512-beam kernel, 200 feeds, ragged
    (8, 256, 8, 512, 2, 2, 16, 8, "random"),        # 512-beam kernel, 8 warps
    (3, 256, 4, 512, 2, 2, 16, 8, "random"),        # 512-beam kernel, E-W padded 3 -> 4
    (1, 50, 1, 128, 2, 3, 48, 16, "random"),        # warp path: 128 beams, 8 snapshots/step
    (2, 100, 2, 256, 1, 2, 30, 10, "half_sine"),    # warp path: ragged (10 snapshots, 4/step)
    (5, 128, 3, 256, 2, 2, 24, 12, "random"),       # warp path: E-W 5 folded onto 3
    (1, 300, 1, 1024, 2, 2, 16, 8, "random"),       # warp path: 1024 beams, E-W 1
    (4, 33, 4, 128, 2, 2, 16, 8, "random"),         # warp path: 33 feeds, 2 snapshots/step
    (2, 700, 2, 2048, 1, 2, 12, 6, "random"),       # 2048 beams, a warp pair per transform
    (12, 10, 16, 32, 2, 2, 40, 20, "random"),       # 32 beams, a lane per transform; E-W 12 -> 16
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "x".join(map(str, c[:4])) + f"_p{c[4]}_n{c[7]}_{c[8]}")
def test_beams_match_oracle(case):
    nx, ny, mx, my, npol, nfreq, T, n_int, wk = case
    v, w = make_case(nx, ny, mx, my, npol, nfreq, T, n_int, weights=wk, seed=zlib.crc32(repr(case).encode()) % 1000)
    got = run_beams(v, w, nx, ny, mx, my, npol, nfreq, n_int)
    ref = oracle_beams(v, w, nx, ny, mx, my, npol, nfreq, n_int)
    assert got.shape == ref.shape
    assert np.all(np.isfinite(got))
    err = rel_err_per_beam(got, ref)
    assert err.max() <= TOL_BEAM, f"max rel err {err.max():.3g}"


@pytest.mark.parametrize("case", [c for c in CASES if c[3] in (32, 128, 256, 512, 1024, 2048) and 2 * c[1] <= c[3]],
                         ids=lambda c: "x".join(map(str, c[:4])))
def test_generic_kernel_on_warp_shapes(case, monkeypatch):
    """The generic Stockham kernel, forced on shapes the warp-per-transform kernels (and
    the 512-beam kernel) normally take."""
    monkeypatch.setenv("FFTBF_FP32_GENERIC", "1")
    nx, ny, mx, my, npol, nfreq, T, n_int, wk = case
    v, w = make_case(nx, ny, mx, my, npol, nfreq, T, n_int, weights=wk, seed=4)
    got = run_beams(v, w, nx, ny, mx, my, npol, nfreq, n_int)
    ref = oracle_beams(v, w, nx, ny, mx, my, npol, nfreq, n_int)
    assert rel_err_per_beam(got, ref).max() <= TOL_BEAM


def test_tiny_matches_visibility_route():
    nx, ny, mx, my, npol, nfreq, T, n_int = 2, 16, 2, 32, 1, 8, 256, 16
    v, w = make_case(nx, ny, mx, my, npol, nfreq, T, n_int, seed=1)
    got = run_beams(v, w, nx, ny, mx, my, npol, nfreq, n_int)
    x = oracle.unpack(v)
    ref = oracle.beams_via_visibilities(x, None, mx, my, n_int)
    assert rel_err_per_beam(got, ref).max() <= TOL_BEAM


def test_plane_wave_on_grid_exact_zeros():
    """A noiseless on-grid plane wave with integer components lands in one beam; every
    other beam of the unpadded axes is zero (Eq. theta_A)."""
    nx = ny = mx = my = 4
    A0, B0, n_int = 1, 3, 8
    ix = np.arange(nx)[:, None]
    iy = np.arange(ny)[None, :]
    x = 3 * (1j ** ((ix * A0 + iy * B0) % 4))
    re = np.rint(x.real).astype(np.int64) & 15
    im = np.rint(x.imag).astype(np.int64) & 15
    snap = ((re << 4) | im).astype(np.uint8)
    v = np.broadcast_to(snap, (n_int, 1, 1, nx, ny)).copy()
    got = run_beams(v, None, nx, ny, mx, my, 1, 1, n_int)[0, 0]
    peak = n_int * 9 * (nx * ny) ** 2
    assert got[A0, B0] == pytest.approx(peak, rel=1e-6)
    mask = np.ones_like(got, dtype=bool)
    mask[A0, B0] = False
    assert np.abs(got[mask]).max() <= 1e-5 * peak / (mx * my)


def test_zero_input_gives_zero():
    v = np.zeros((16, 2, 2, 4, 256), dtype=np.uint8)
    got = run_beams(v, synth.random_weights(4, 256, 3), 4, 256, 4, 512, 2, 2, 8)
    assert np.all(got == 0.0)


def test_bit_identical_alone_and_in_batch():
    """Each window's result does not depend on what else the launch carries."""
    nx, ny, mx, my, npol, nfreq, n_int = 4, 256, 4, 512, 2, 4, 32
    T = 4 * n_int
    v, w = make_case(nx, ny, mx, my, npol, nfreq, T, n_int, weights="half_sine", seed=9)
    full = run_beams(v, w, nx, ny, mx, my, npol, nfreq, n_int)
    again = run_beams(v, w, nx, ny, mx, my, npol, nfreq, n_int)
    assert np.array_equal(full, again)
    for j in range(T // n_int):
        one = run_beams(v[j * n_int:(j + 1) * n_int], w, nx, ny, mx, my, npol, nfreq, n_int)
        assert np.array_equal(one[0], full[j])


def test_execute_rejects_partial_window():
    v = torch.zeros(10 * 2 * 32, dtype=torch.uint8, device="cuda")
    out = torch.zeros(4096, device="cuda")
    with fb.plan_create(2, 16, 2, 32, 1, 2, 4) as plan:
        with pytest.raises(fb.FftbfError) as e:
            fb.execute(plan, v, 10, out)
        assert e.value.code == -1
        fb.execute(plan, v, 0, out)          # T = 0 is a no-op


# ----------------------------------------------------------------- tied beams ----
def run_tied(P_dev, plan, nwin, u, v, n_tied):
    out = torch.full((nwin, plan.nfreq, n_tied), float("nan"), device="cuda")
    fb.tied_beams(plan, P_dev, nwin, n_tied, u, v, out)
    fb.plan_sync(plan)
    return out.cpu().numpy()


def tied_scale(P, u, v, nx, ny):
    """sum_{A,B} |w^A w^B| P: the natural size of the FP32 rounding error of a tied beam."""
    wx = np.abs(oracle.regrid_weights(nx, P.shape[-2], u))
    wy = np.abs(oracle.regrid_weights(ny, P.shape[-1], v))
    return np.einsum("fsA,fsB,jfAB->jfs", wx, wy, P)


@pytest.mark.parametrize("shape", [(3, 8, 5, 16, 2, 4, 64, 16, 37),      # both axes dense
                                   (4, 256, 4, 512, 2, 3, 768, 384, 100),  # E-W on the grid
                                   (2, 16, 2, 32, 1, 8, 1024, 16, 70)])   # the tiny workload
def test_tied_beams_match_oracle(shape):
    nx, ny, mx, my, npol, nfreq, T, n_int, n_tied = shape
    v8, w = make_case(nx, ny, mx, my, npol, nfreq, T, n_int, weights="random", seed=21)
    dv = torch.from_numpy(v8.reshape(-1)).cuda()
    nwin = T // n_int
    P = torch.empty((nwin, nfreq, mx, my), device="cuda")
    rng = np.random.default_rng(5)

    def axis(n, m):
        if m >= 2 * n - 1:
            return rng.random((nfreq, n_tied))
        return rng.integers(0, m, (nfreq, n_tied)) / m

    u, vv = axis(nx, mx), axis(ny, my)
    with fb.plan_create(nx, ny, mx, my, npol, nfreq, n_int, weights=w) as plan:
        fb.execute(plan, dv, T, P)
        got = run_tied(P, plan, nwin, u, vv, n_tied)
        again = run_tied(P, plan, nwin, u, vv, n_tied)     # cached tables
        assert np.array_equal(got, again)
    Pref = oracle_beams(v8, w, nx, ny, mx, my, npol, nfreq, n_int)
    ref = oracle.tied_regrid(Pref, u, vv, nx, ny)
    scale = tied_scale(Pref, u, vv, nx, ny)
    assert (np.abs(got - ref) / scale).max() <= TOL_BEAM
    # the regridded beams are the direct pointed beams of the apodised voltages
    direct = oracle.tied_direct(oracle.unpack(v8), None if w is None else w.astype(np.complex128),
                                u, vv, n_int)
    assert (np.abs(got - direct) / scale).max() <= TOL_BEAM


def test_tied_rejects_off_grid_pointing():
    with fb.plan_create(4, 256, 4, 512, 2, 1, 8) as plan:
        P = torch.zeros((1, 1, 4, 512), device="cuda")
        out = torch.zeros((1, 1, 1), device="cuda")
        with pytest.raises(fb.FftbfError) as e:
            fb.tied_beams(plan, P, 1, 1, np.array([0.3]), np.array([0.5]), out)
        assert e.value.code == -1 and "off the FFT-beam grid" in str(e.value)


@pytest.mark.parametrize("shape,prec", [((4, 256, 4, 512, 2, 2, 32, 16), "fp32"),
                                        ((3, 128, 3, 256, 2, 2, 32, 16), "fp32"),
                                        ((8, 64, 8, 128, 2, 2, 32, 16), "fp32"),
                                        ((4, 256, 4, 512, 2, 2, 32, 16), "tc_fp16_serial"),
                                        ((4, 256, 4, 512, 2, 2, 32, 16), "tc_bf16_serial"),
                                        ((4, 256, 4, 512, 2, 2, 32, 16), "tc_fp16x3")])
def test_misaligned_voltages_give_identical_beams(shape, prec, monkeypatch):
    """A voltage pointer off the 16-byte boundary is accepted (staged byte by byte instead
    of with 16-byte copies) and gives bit-identical beams. The aligned call runs the
    constant-size instance of the 4x256 lattice (or of an exactly 2x-padded warp-path
    shape), the misaligned one the runtime-size instance, so this also checks that both
    sum in the same order. (tc_fp16_serial, tc_bf16_serial: the serial tensor-core kernel,
    which serves misaligned FP16 and BF16 calls; aligned calls run the warp-specialised
    kernel, checked against the oracle in test_misaligned_tensor_core_kernels_agree.)"""
    if prec.endswith("_serial"):
        monkeypatch.setenv("FFTBF_TC_KERNEL", "serial")
        prec = prec[:-len("_serial")]
    nx, ny, mx, my, npol, nfreq, T, n_int = shape
    v, w = make_case(nx, ny, mx, my, npol, nfreq, T, n_int, weights="half_sine", seed=77)
    flat = torch.from_numpy(np.ascontiguousarray(v).reshape(-1))
    base = torch.zeros(flat.numel() + 16, dtype=torch.uint8, device="cuda")
    outs = []
    for off in (0, 3):
        base[off:off + flat.numel()].copy_(flat)
        out = torch.full((T // n_int, nfreq, mx, my), float("nan"), device="cuda")
        with fb.plan_create(nx, ny, mx, my, npol, nfreq, n_int, weights=w) as plan:
            if prec != "fp32":
                fb.plan_set_precision(plan, {"tc_fp16": fb.PREC_TC_FP16, "tc_bf16": fb.PREC_TC_BF16,
                                             "tc_fp16x3": fb.PREC_TC_FP16X3}[prec])
            fb.execute(plan, base[off:off + flat.numel()], T, out)
            fb.plan_sync(plan)
        outs.append(out.cpu().numpy())
    assert np.all(np.isfinite(outs[0]))
    assert np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("form,tol", [("fp16", 5e-3), ("bf16", 3e-2)])
def test_misaligned_tensor_core_kernels_agree(form, tol):
    """FP16 or BF16 on the 4x256 lattice: an aligned voltage pointer runs the
    warp-specialised tensor-core kernel (bulk copies need 16-byte alignment), a misaligned
    one the serial kernel. Their roundings differ, so both are held to the form's bound
    against the oracle (5e-3 or 3e-2 of each beam)."""
    shape = (4, 256, 4, 512, 2, 2, 32, 16)
    nx, ny, mx, my, npol, nfreq, T, n_int = shape
    v, w = make_case(nx, ny, mx, my, npol, nfreq, T, n_int, weights="half_sine", seed=78)
    ref = oracle_beams(v, w, nx, ny, mx, my, npol, nfreq, n_int)
    flat = torch.from_numpy(np.ascontiguousarray(v).reshape(-1))
    base = torch.zeros(flat.numel() + 16, dtype=torch.uint8, device="cuda")
    outs = []
    for off in (0, 3):
        base[off:off + flat.numel()].copy_(flat)
        out = torch.full((T // n_int, nfreq, mx, my), float("nan"), device="cuda")
        with fb.plan_create(nx, ny, mx, my, npol, nfreq, n_int, weights=w) as plan:
            fb.plan_set_precision(plan, fb.PREC_TC_FP16 if form == "fp16" else fb.PREC_TC_BF16)
            fb.execute(plan, base[off:off + flat.numel()], T, out)
            fb.plan_sync(plan)
        outs.append(out.cpu().numpy())
    for o in outs:
        assert np.all(np.isfinite(o))
        assert (np.abs(o - ref) / ref).max() <= tol
    assert (np.abs(outs[0] - outs[1]) / ref).max() <= 1e-2
