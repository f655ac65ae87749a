"""Full-size parity: the CHIME-like 4x256 workload in the launch configuration bench.py
times (fftbf_execute over a 3072-sample, 1024-channel device block; tied beams for 2048
pointings), checked on sampled (window, channel) slices that the oracle computes one by
one, and on every (window, channel) item through Parseval's identity.

Every form runs here: the FP32 form, the three tensor-core forms and the warp-specialised
tensor-core kernel. One call has 8 windows x 1024 channels = 8192 work items and the
persistent kernels launch at most 152 SMs x 8 CTAs, so every CTA takes several items in
turn (the cross-item prefetch and accumulator reuse run here, as in the bench)."""
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
NWIN = T_DEV // NINT

# Per-beam bounds of the 16-bit forms, as in test_gpu_tc.py (max and rms over beams of
# |P - P_ref| / P_ref); the split form is held to the FP32 bound.
TOL_FORM = {"fp32": (TOL_BEAM, 2e-6), "fp16": (5e-3, 1e-3), "bf16": (3e-2, 6e-3),
            "fp16x3": (1e-5, 2e-6)}
# Parseval: the relative error of each item's total power. A total is a sum of 2048
# positive beams whose rounding errors are independent, so it sits far inside the
# per-beam bound; the gate is the form's rms bound. For the FP32 form the gate (1e-6) is
# also far below the spread of the totals between items (~1.6e-3 for 786k samples of
# sigma 2.5), so a dropped, repeated or misplaced item fails it; the 16-bit forms are
# checked item by item against the FP32 form's beams for that.
PARSEVAL = {"fp32": 1e-6, "fp16": 1e-3, "bf16": 6e-3, "fp16x3": 2e-6}


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
    beams = torch.full((NWIN, NFREQ, MX, MY), float("nan"), device="cuda")
    tied = torch.full((NWIN, NFREQ, N_TIED), float("nan"), device="cuda")
    with fb.plan_create(NX, NY, MX, MY, NPOL, NFREQ, NINT, weights=w) as plan:
        fb.execute(plan, dvol, T_DEV, beams)
        fb.tied_beams(plan, beams, NWIN, N_TIED, u, v, tied)
        fb.plan_sync(plan)
    r = dict(block=block, w=w, u=u, v=v, dvol=dvol, beams=beams.cpu().numpy(),
             tied=tied.cpu().numpy())
    r["parseval"] = _parseval_rhs(block, w)
    r["oracle"] = {}
    yield r
    del r["dvol"]


def _parseval_rhs(block, w):
    """Mx My sum_{t in window, p, ix, iy} |w x|^2 for both windows of the host block and
    every channel: the total power of each item over the full padded grid (M >= n on both
    axes, so nothing folds). |x|^2 per byte value comes from the oracle's unpack; the
    gathers and sums run in FP64 with torch on the device (the block is 1.6 GB)."""
    lut = np.abs(oracle.unpack(np.arange(256, dtype=np.uint8))) ** 2
    lut_d = torch.from_numpy(lut).cuda()
    w2 = torch.from_numpy(np.abs(np.asarray(w, dtype=np.complex128)) ** 2).cuda()   # [NX][NY]
    out = np.zeros((T_HOST // NINT, NFREQ))
    hb = torch.from_numpy(block)                                                    # [T][F][P][NX][NY]
    for j in range(T_HOST // NINT):
        for f0 in range(0, NFREQ, 128):
            chunk = hb[j * NINT:(j + 1) * NINT, f0:f0 + 128].cuda()
            e = lut_d[chunk.int()]                                                 # |x|^2
            s = (e.sum(dim=(0, 2)) * w2).sum(dim=(-2, -1))                         # [128]
            out[j, f0:f0 + 128] = s.cpu().numpy()
    return out * MX * MY


SLICES = [(0, 0), (7, 1023), (3, 511), (5, 17), (6, 900), (1, 1)]


def _oracle_slice(r, j, f):
    key = ((j * NINT) % T_HOST, f)
    if key not in r["oracle"]:
        t0 = key[0]
        v = np.ascontiguousarray(r["block"][t0:t0 + NINT, f:f + 1])
        r["oracle"][key] = oracle.beams(v, NX, NY, MX, MY, NPOL, 1, NINT,
                                        weights=r["w"].astype(np.complex128))
    return r["oracle"][key]


def _check_parseval(r, got, form):
    tot = got.astype(np.float64).sum(axis=(-2, -1))                    # [NWIN][NFREQ]
    ref = r["parseval"][np.arange(NWIN) % (T_HOST // NINT)]
    rel = np.abs(tot - ref) / ref
    assert rel.max() <= PARSEVAL[form], f"{form}: Parseval max rel {rel.max():.3g}"
    return rel.max()


def test_no_nan(run):
    assert np.all(np.isfinite(run["beams"]))
    assert np.all(np.isfinite(run["tied"]))


@pytest.mark.parametrize("j,f", SLICES)
def test_beams_slice(run, j, f):
    ref = _oracle_slice(run, j, f)[0, 0]
    got = run["beams"][j, f]
    err = np.abs(got - ref) / ref
    assert err.max() <= TOL_BEAM, f"max rel err {err.max():.3g}"


def test_beams_parseval_every_item(run):
    _check_parseval(run, run["beams"], "fp32")


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


FORMS = [("fp16", None), ("bf16", None), ("fp16x3", None), ("fp16", "ws"), ("bf16", "ws"),
         ("fp16", "pipe"), ("bf16", "pipe")]


@pytest.mark.parametrize("form,pipe", FORMS,
                         ids=["fp16", "bf16", "fp16x3", "fp16-ws", "bf16-ws", "fp16-pipe", "bf16-pipe"])
def test_tensor_core_form_full_size(run, form, pipe, monkeypatch):
    """A tensor-core form over the bench's 8192-item launch: sampled slices against the
    oracle, every item against the FP32 form's beams (both within the form's per-beam
    bound of the oracle) and against Parseval."""
    monkeypatch.delenv("FFTBF_TC_KERNEL", raising=False)
    if pipe == "pipe":
        monkeypatch.setenv("FFTBF_TC_PIPE", "1")
    else:
        monkeypatch.delenv("FFTBF_TC_PIPE", raising=False)
        if pipe == "ws":
            monkeypatch.setenv("FFTBF_TC_KERNEL", "ws")
    prec = {"fp16": fb.PREC_TC_FP16, "bf16": fb.PREC_TC_BF16, "fp16x3": fb.PREC_TC_FP16X3}[form]
    beams = torch.full((NWIN, NFREQ, MX, MY), float("nan"), device="cuda")
    with fb.plan_create(NX, NY, MX, MY, NPOL, NFREQ, NINT, weights=run["w"]) as plan:
        fb.plan_set_precision(plan, prec)
        fb.execute(plan, run["dvol"], T_DEV, beams)
        fb.plan_sync(plan)
    got = beams.cpu().numpy()
    del beams
    assert np.all(np.isfinite(got))
    tol, rms_tol = TOL_FORM[form]
    worst = []
    for j, f in SLICES:
        ref = _oracle_slice(run, j, f)[0, 0]
        rel = np.abs(got[j, f] - ref) / ref
        worst.append((float(rel.max()), float(np.sqrt(np.mean(rel ** 2)))))
    # every item: the FP32 form (itself within 1e-5 of the oracle) as the yardstick
    rel_all = np.abs(got - run["beams"]) / run["beams"]
    tot = got.astype(np.float64).sum(axis=(-2, -1))
    pref = run["parseval"][np.arange(NWIN) % (T_HOST // NINT)]
    prel = np.abs(tot - pref) / pref
    print(f"\n[full-size {form}{' ' + pipe if pipe else ''}] oracle slices: max rel "
          f"{max(x[0] for x in worst):.3e}, rms {max(x[1] for x in worst):.3e}; every item vs "
          f"FP32 form: max rel {rel_all.max():.3e}, rms {np.sqrt(np.mean(rel_all ** 2)):.3e}; "
          f"Parseval max rel {prel.max():.3e}")
    for (j, f), (mx_, rms) in zip(SLICES, worst):
        assert mx_ <= tol, (form, j, f, mx_)
        assert rms <= rms_tol, (form, j, f, rms)
    assert rel_all.max() <= tol + TOL_BEAM, (form, float(rel_all.max()))
    assert prel.max() <= PARSEVAL[form], (form, float(prel.max()))
