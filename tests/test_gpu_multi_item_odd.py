"""Persistent beam kernels on the 4x256 lattice with several work items per CTA and odd
snapshot counts, against the FP64 oracle (Eq. fftbeamform, Eq. bf).

One polarisation and n_int = 5 give 5 snapshots per (window, channel) item: the FP32
kernel's last iteration of every item holds a single snapshot, and the tensor-core kernels'
last snapshot pair of every item holds one. With 2 windows x 400 channels = 800 items, the
CTAs of the FP32 kernel (4 per SM) and of the tensor-core kernels (1 or 2 per SM) each take
several items in turn; in the warp-specialised FP16 kernel, whose input warps work on two
pairs per round, a CTA with 3 items has 9 pairs, so rounds straddle item boundaries and the
last round holds one pair; in the grouped kernel (four snapshots per group, one CTA per
SM) a CTA with 5 or 6 items has 25 or 30 snapshots, so groups straddle items and the last
group holds one or two snapshots."""
import numpy as np
import pytest

from helpers import TOL_BEAM, make_case, oracle_beams, rel_err_per_beam

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1710_08591_gb300 as fb  # noqa: E402

SHAPE = (4, 256, 4, 512, 1, 400, 10, 5)           # nx, ny, mx, my, npol, nfreq, T, n_int
TOL_FP16, RMS_FP16 = 5e-3, 1e-3                   # the FP16 form's stated bounds
TOL_BF16, RMS_BF16 = 3e-2, 6e-3


@pytest.fixture(scope="module")
def case():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fb.build()
    nx, ny, mx, my, npol, nfreq, T, n_int = SHAPE
    v, w = make_case(nx, ny, mx, my, npol, nfreq, T, n_int, weights="random", seed=31)
    ref = oracle_beams(v, w, nx, ny, mx, my, npol, nfreq, n_int)
    return v, w, ref


def run(v, w, prec=None):
    nx, ny, mx, my, npol, nfreq, T, n_int = SHAPE
    dv = torch.from_numpy(np.ascontiguousarray(v).reshape(-1)).cuda()
    out = torch.full((T // n_int, nfreq, mx, my), float("nan"), device="cuda")
    with fb.plan_create(nx, ny, mx, my, npol, nfreq, n_int, weights=w) as plan:
        if prec is not None:
            fb.plan_set_precision(plan, prec)
        fb.execute(plan, dv, T, out)
        fb.plan_sync(plan)
    return out.cpu().numpy()


def test_fp32_several_items_per_cta_odd_snapshots(case):
    v, w, ref = case
    got = run(v, w)
    assert np.all(np.isfinite(got))
    assert rel_err_per_beam(got, ref).max() <= TOL_BEAM


@pytest.mark.parametrize("kern", ["grouped", "ws", "serial"])
def test_fp16_several_items_per_cta_odd_pairs(case, kern, monkeypatch):
    v, w, ref = case
    monkeypatch.setenv("FFTBF_TC_KERNEL", kern)
    got = run(v, w, fb.PREC_TC_FP16)
    rel = np.abs(got - ref) / ref
    assert np.all(np.isfinite(got)), kern
    assert rel.max() <= TOL_FP16, (kern, rel.max())
    assert np.sqrt(np.mean(rel ** 2)) <= RMS_FP16, kern


@pytest.mark.parametrize("kern", ["grouped", "ws", "serial"])
def test_bf16_several_items_per_cta_odd_pairs(case, kern, monkeypatch):
    v, w, ref = case
    monkeypatch.setenv("FFTBF_TC_KERNEL", kern)
    got = run(v, w, fb.PREC_TC_BF16)
    rel = np.abs(got - ref) / ref
    assert np.all(np.isfinite(got))
    assert rel.max() <= TOL_BF16
    assert np.sqrt(np.mean(rel ** 2)) <= RMS_BF16
