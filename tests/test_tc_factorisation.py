"""The two-stage factorisation the grouped tensor-core kernel computes (Eq. fftbeamform on
the 4x256 lattice, N-S zero-padded to 512 as Eq. b2n-1 recommends), restated with numpy
matrices in FP64 and held to numpy.fft of the zero-padded lattice.

Stage 1 is one real matrix F1 (rows (A, k1), columns (ix, re/im, n1)) holding the E-W DFT
and the pruned 32-point N-S DFT, applied to data columns (snapshot, re/im of the output,
n2) in which each snapshot appears twice: (re; im) for the real part and (im; -re) for the
imaginary part. Each row then carries its own W512^(n2 k1) twiddle, and stage 2 is the
real-embedded 16-point DFT over n2 (columns (re/im, k2)). If any of these pieces had a
wrong sign, a transposed index or a dropped factor, the beams would not match the FFT."""
import numpy as np

NX, NY, MX, MY = 4, 256, 4, 512


def f1_matrix():
    f1 = np.zeros((128, 128))
    for m in range(128):
        A, k1 = divmod(m, 32)
        for k in range(128):
            ix, r = divmod(k, 32)
            ci, n1 = divmod(r, 16)
            c = np.exp(-2j * np.pi * ((8 * A * ix + n1 * k1) % 32) / 32)
            f1[m, k] = c.real if ci == 0 else -c.imag
    return f1


def data_columns(z):
    """z: [4 ix][256 iy] complex -> B [128 (ix, ci, n1)][32 (co, n2)]."""
    b = np.zeros((128, 32))
    for ix in range(4):
        for n1 in range(16):
            x = z[ix, 16 * n1:16 * n1 + 16]               # n2 = 0..15
            b[32 * ix + n1, :16] = x.real                  # ci 0, co 0
            b[32 * ix + 16 + n1, :16] = x.imag             # ci 1, co 0
            b[32 * ix + n1, 16:] = x.imag                  # ci 0, co 1
            b[32 * ix + 16 + n1, 16:] = -x.real            # ci 1, co 1
    return b


def f2_matrix():
    """[32 (ci, n2)][32 (co, k2)]: out = in x W16^(n2 k2), real-embedded."""
    f2 = np.zeros((32, 32))
    for n2 in range(16):
        for k2 in range(16):
            w = np.exp(-2j * np.pi * ((n2 * k2) % 16) / 16)
            f2[n2, k2], f2[16 + n2, k2] = w.real, -w.imag
            f2[n2, 16 + k2], f2[16 + n2, 16 + k2] = w.imag, w.real
    return f2


def grouped_beams(z):
    d1 = f1_matrix() @ data_columns(z)                     # [128 (A, k1)][32 (co, n2)]
    y = d1[:, :16] + 1j * d1[:, 16:]
    k1 = np.arange(128) % 32
    y = y * np.exp(-2j * np.pi * ((np.arange(16)[None, :] * k1[:, None]) % 512) / 512)
    d2 = np.concatenate([y.real, y.imag], axis=1) @ f2_matrix()   # [128][(co, k2)]
    p = d2[:, :16] ** 2 + d2[:, 16:] ** 2                  # [(A, k1)][k2]
    out = np.zeros((MX, MY))
    for m in range(128):
        A, kk1 = divmod(m, 32)
        out[A, kk1 + 32 * np.arange(16)] = p[m]
    return out


def test_grouped_factorisation_matches_padded_fft():
    rng = np.random.default_rng(20)
    for _ in range(3):
        z = rng.standard_normal((NX, NY)) + 1j * rng.standard_normal((NX, NY))
        ref = np.abs(np.fft.fft(np.fft.fft(z, n=MX, axis=0), n=MY, axis=1)) ** 2
        got = grouped_beams(z)
        assert np.allclose(got, ref, rtol=1e-10, atol=1e-10 * ref.max())


def test_grouped_factorisation_plane_wave_lands_in_its_beam():
    # a plane wave on the grid (A0, B0) puts (nx ny)^2 |c|^2 in that beam and ~0 elsewhere
    A0, B0, c = 1, 77, 0.5 - 1.5j
    ix, iy = np.meshgrid(np.arange(NX), np.arange(NY), indexing="ij")
    z = c * np.exp(2j * np.pi * (A0 * ix / MX + B0 * iy / MY))
    got = grouped_beams(z)
    assert np.isclose(got[A0, B0], (NX * NY) ** 2 * abs(c) ** 2, rtol=1e-12)
    # the N-S axis is padded 2x, so the neighbours of the peak carry sidelobes; the E-W
    # axis is unpadded, so every other E-W beam is exactly empty
    assert np.all(np.delete(got, A0, axis=0) < 1e-18 * got[A0, B0])
