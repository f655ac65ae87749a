"""Batched uneven lattices in one persistent launch: parity with the oracle per array,
bit-identical results alone and in the mix, graph replay, autotuned tiles."""
import numpy as np
import pytest

import synth
from helpers import TOL_BEAM, make_case, oracle_beams, parseval_totals

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1710_08591_gb300 as fb  # noqa: E402

# (nx, ny): N-S padded to twice the next power of two, E-W unpadded
LATTICES = synth.BATCH_LATTICES


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fb.build()
    fb.lib()


def _arrays(nfreqs, T, n_int, npol=2, seed=40):
    arrs = []
    for k, ((nx, ny), nf) in enumerate(zip(LATTICES, nfreqs)):
        mx, my = nx, 2 * synth.next_pow2(ny)
        v, w = make_case(nx, ny, mx, my, npol, nf, T, n_int,
                         weights="half_sine" if k % 2 == 0 else "random", seed=seed + k)
        arrs.append(dict(shape=(nx, ny, mx, my, npol, nf, n_int), v=v, w=w))
    return arrs


def _run(arrs, T, stream=None, repeat=1):
    plans = [fb.plan_create(*a["shape"], weights=a["w"]) for a in arrs]
    dvs = [torch.from_numpy(a["v"].reshape(-1)).cuda() for a in arrs]
    outs = [torch.full((T // a["shape"][6], a["shape"][5], a["shape"][2], a["shape"][3]),
                       float("nan"), device="cuda") for a in arrs]
    with fb.batch_create(plans) as b:
        steps = [fb.batch_tuned_steps(b, i) for i in range(len(plans))]
        for _ in range(repeat):
            fb.batch_execute(b, dvs, T, outs, stream)
        torch.cuda.synchronize()
    res = [o.cpu().numpy() for o in outs]
    for p in plans:
        p.close()
    return res, steps


def test_batch_matches_oracle_every_array():
    T, n_int = 32, 16
    arrs = _arrays([3, 2, 4, 2, 2, 3], T, n_int)
    got, steps = _run(arrs, T)
    assert all(s >= 1 for s in steps)
    for a, g in zip(arrs, got):
        nx, ny, mx, my, npol, nf, n_int_ = a["shape"]
        ref = oracle_beams(a["v"], a["w"], nx, ny, mx, my, npol, nf, n_int_)
        err = np.abs(g - ref) / ref
        assert err.max() <= TOL_BEAM, (a["shape"], err.max())


@pytest.mark.parametrize("path", ["generic", "warp"])
def test_batch_each_path_matches_oracle(path, monkeypatch):
    """Both transform paths of the batch kernel, forced in turn (the warp-per-transform
    path covers the 2x-padded 4x512, 8x128, 2x1024 and 3x256 shapes; the others stay
    generic)."""
    monkeypatch.setenv("FFTBF_BATCH_PATH", path)
    T, n_int = 24, 12
    arrs = _arrays([2, 3, 2, 2, 1, 3], T, n_int, seed=70)
    got, _ = _run(arrs, T)
    for a, g in zip(arrs, got):
        nx, ny, mx, my, npol, nf, n_int_ = a["shape"]
        ref = oracle_beams(a["v"], a["w"], nx, ny, mx, my, npol, nf, n_int_)
        assert (np.abs(g - ref) / ref).max() <= TOL_BEAM, (path, a["shape"])


def test_batch_bit_identical_alone_and_in_mix_and_replayed():
    T, n_int = 64, 32
    arrs = _arrays([2, 3, 2, 2, 1, 2], T, n_int, seed=50)
    s = torch.cuda.Stream()
    mix, _ = _run(arrs, T, stream=s, repeat=3)          # captured once, replayed
    for k in (0, 4, 5):
        alone, _ = _run([arrs[k]], T, stream=s)
        assert np.array_equal(alone[0], mix[k])


def test_batch_constant_size_and_runtime_instances_bit_identical():
    """Aligned voltages run the constant-size instances of the exactly 2x-padded shapes
    (all six lattices), voltages 3 bytes off the 16-byte boundary the runtime-size ones:
    the beams must be bit-identical."""
    T, n_int = 32, 16
    arrs = _arrays([2, 2, 2, 2, 1, 2], T, n_int, seed=90)
    res = []
    for off in (0, 3):
        plans = [fb.plan_create(*a["shape"], weights=a["w"]) for a in arrs]
        dvs = []
        for a in arrs:
            flat = torch.from_numpy(np.ascontiguousarray(a["v"]).reshape(-1))
            base = torch.zeros(flat.numel() + 16, dtype=torch.uint8, device="cuda")
            base[off:off + flat.numel()].copy_(flat)
            dvs.append(base[off:off + flat.numel()])
        outs = [torch.full((T // a["shape"][6], a["shape"][5], a["shape"][2], a["shape"][3]),
                           float("nan"), device="cuda") for a in arrs]
        with fb.batch_create(plans) as b:
            fb.batch_execute(b, dvs, T, outs, None)
            torch.cuda.synchronize()
        res.append([o.cpu().numpy() for o in outs])
        for p_ in plans:
            p_.close()
    for k, (x, y) in enumerate(zip(*res)):
        assert np.all(np.isfinite(x)), arrs[k]["shape"]
        assert np.array_equal(x, y), arrs[k]["shape"]


def test_batch_every_cta_takes_several_items():
    """Items outnumber the launch grid several times over, so every CTA takes items from
    the queue again and again, as in the bench: sampled (window, channel) slices of every
    array against the oracle, every item against Parseval, and one array alone
    bit-identical to its place in the mix."""
    T, n_int, nf = 64, 16, 160
    arrs = _arrays([nf] * 6, T, n_int, seed=120)
    plans = [fb.plan_create(*a["shape"], weights=a["w"]) for a in arrs]
    dvs = [torch.from_numpy(a["v"].reshape(-1)).cuda() for a in arrs]
    outs = [torch.full((T // n_int, nf, a["shape"][2], a["shape"][3]), float("nan"),
                       device="cuda") for a in arrs]
    with fb.batch_create(plans) as b:
        grid = fb.batch_grid(b)
        items = sum(o.shape[0] * o.shape[1] for o in outs)
        assert items >= 3 * grid, (items, grid)
        fb.batch_execute(b, dvs, T, outs, None)
        torch.cuda.synchronize()
    got = [o.cpu().numpy() for o in outs]
    rng = np.random.default_rng(3)
    for a, g in zip(arrs, got):
        nx, ny, mx, my, npol, _, _ = a["shape"]
        assert np.all(np.isfinite(g)), a["shape"]
        tot = parseval_totals(a["v"], a["w"], n_int, mx, my)
        prel = np.abs(g.astype(np.float64).sum(axis=(-2, -1)) - tot) / tot
        assert prel.max() <= 1e-6, (a["shape"], prel.max())
        for j, f in [(0, 0), (T // n_int - 1, nf - 1)] + [tuple(rng.integers(0, (T // n_int, nf)))]:
            v = np.ascontiguousarray(a["v"][j * n_int:(j + 1) * n_int, f:f + 1])
            ref = oracle_beams(v, a["w"], nx, ny, mx, my, npol, 1, n_int)[0, 0]
            err = np.abs(g[j, f] - ref) / ref
            assert err.max() <= TOL_BEAM, (a["shape"], j, f, err.max())
    alone, _ = _run([arrs[2]], T)
    assert np.array_equal(alone[0], got[2])
    for p_ in plans:
        p_.close()


def test_batch_rejects_unsupported_shape():
    with fb.plan_create(5, 12, 5, 24, 1, 2, 4) as p:
        with pytest.raises(fb.FftbfError) as e:
            fb.batch_create([p])
        assert e.value.code == -5
