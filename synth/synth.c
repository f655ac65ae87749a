/*
 * Seeded synthetic channelised voltages for FFT-beamforming tests and benchmarks.
 *
 * This file holds no part of the beamforming method: it only draws inputs.
 * Both the CPU oracle and the CUDA path read the bytes it writes, and the bytes are the
 * ground truth of every comparison.
 *
 * Signal model (the antenna response of the paper's Section 2, eq:feed, with isotropic
 * antennas): each complex sample is receiver noise plus a few plane-wave sources,
 *   eta[t,f,p,ix,iy] = n + sum_s amp_s * exp(i phi[t,f,p,s]) * exp(+2 pi i (ix u_s + iy v_s)).
 * The source phase phi is drawn per (t, f, p, s), so each source is a noise-like signal
 * that is coherent across the lattice. The noise is complex Gaussian with standard
 * deviation sigma per real component. Each component is rounded half-to-even, clipped to
 * [-7, 7] and packed as one byte: bits 7..4 hold the real part and bits 3..0 the
 * imaginary part, both two's-complement 4-bit integers.
 *
 * Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014) used as a counter-based generator: the
 * k-th draw of stream s is mix64(s + k * 0x9E3779B97F4A7C15). Gaussians use the
 * Box-Muller transform in FP64.
 *
 * Output layout: uint8 [nt][nfreq][npol][nx][ny], time index t0 .. t0+nt-1.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define GOLDEN_GAMMA 0x9E3779B97F4A7C15ULL
#define TWO_PI 6.283185307179586476925286766559

static inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* Draw number k (k >= 1) of the SplitMix64 stream started at state s. */
static inline uint64_t draw(uint64_t s, uint64_t k) { return mix64(s + k * GOLDEN_GAMMA); }

/* Uniform on (0, 1] with 53 random bits. */
static inline double u01(uint64_t h) { return (double)((h >> 11) + 1) * 0x1.0p-53; }

uint64_t synth_splitmix64_draw(uint64_t s, uint64_t k) { return draw(s, k); }

typedef struct {
  uint8_t* out;
  int64_t t0, nt;
  int nfreq, npol, nx, ny;
  uint64_t seed_noise, seed_src;
  double sigma;
  int nsrc;
  const double* amp;
  const double* steer; /* [nsrc][nx*ny][2] exp(+2 pi i (ix u + iy v)) */
  int64_t row_lo, row_hi; /* rows are (t, f) pairs */
} job_t;

static inline int quantise(double x) {
  double r = nearbyint(x); /* default rounding mode: half to even */
  if (r > 7.0) r = 7.0;
  if (r < -7.0) r = -7.0;
  return (int)r;
}

static void* run_rows(void* arg) {
  job_t* J = (job_t*)arg;
  const int nant = J->nx * J->ny;
  double* ph = (double*)malloc(sizeof(double) * 2 * (J->nsrc > 0 ? J->nsrc : 1));
  for (int64_t row = J->row_lo; row < J->row_hi; ++row) {
    const int64_t tl = row / J->nfreq;
    const int f = (int)(row % J->nfreq);
    const int64_t t = J->t0 + tl;
    for (int p = 0; p < J->npol; ++p) {
      const uint64_t snap = ((uint64_t)t * J->nfreq + f) * J->npol + p;
      for (int s = 0; s < J->nsrc; ++s) {
        const double phi = TWO_PI * u01(draw(J->seed_src, snap * J->nsrc + s + 1));
        ph[2 * s] = J->amp[s] * cos(phi);
        ph[2 * s + 1] = J->amp[s] * sin(phi);
      }
      uint8_t* dst = J->out + ((tl * J->nfreq + f) * (int64_t)J->npol + p) * nant;
      const uint64_t e0 = snap * (uint64_t)nant;
      for (int a = 0; a < nant; ++a) {
        const uint64_t e = e0 + a;
        const double r = J->sigma * sqrt(-2.0 * log(u01(draw(J->seed_noise, 2 * e + 1))));
        const double th = TWO_PI * u01(draw(J->seed_noise, 2 * e + 2));
        double re = r * cos(th), im = r * sin(th);
        for (int s = 0; s < J->nsrc; ++s) {
          const double* g = J->steer + ((int64_t)s * nant + a) * 2;
          re += ph[2 * s] * g[0] - ph[2 * s + 1] * g[1];
          im += ph[2 * s] * g[1] + ph[2 * s + 1] * g[0];
        }
        const int qr = quantise(re), qi = quantise(im);
        dst[a] = (uint8_t)(((qr & 15) << 4) | (qi & 15));
      }
    }
  }
  free(ph);
  return NULL;
}

/*
 * Fill out[nt][nfreq][npol][nx][ny] with quantised voltages for times t0 .. t0+nt-1.
 * src_u, src_v are the source directions in lattice units ((d/lambda) sin theta per axis),
 * src_amp their amplitudes. Returns 0, or -1 on a bad argument.
 */
int synth_volts(uint8_t* out, int64_t t0, int64_t nt, int nfreq, int npol, int nx, int ny,
                uint64_t seed, double sigma, int nsrc, const double* src_u,
                const double* src_v, const double* src_amp, int nthreads) {
  if (!out || nt < 0 || nfreq < 1 || npol < 1 || nx < 1 || ny < 1 || nsrc < 0) return -1;
  if (nsrc > 0 && (!src_u || !src_v || !src_amp)) return -1;
  const int nant = nx * ny;
  double* steer = (double*)malloc(sizeof(double) * 2 * (size_t)(nsrc > 0 ? nsrc : 1) * nant);
  if (!steer) return -1;
  for (int s = 0; s < nsrc; ++s)
    for (int ix = 0; ix < nx; ++ix)
      for (int iy = 0; iy < ny; ++iy) {
        double ang = TWO_PI * (ix * src_u[s] + iy * src_v[s]);
        steer[((int64_t)s * nant + ix * ny + iy) * 2] = cos(ang);
        steer[((int64_t)s * nant + ix * ny + iy) * 2 + 1] = sin(ang);
      }
  if (nthreads < 1) nthreads = 1;
  const int64_t rows = nt * nfreq;
  if (rows < nthreads) nthreads = rows > 0 ? (int)rows : 1;
  job_t* jobs = (job_t*)calloc((size_t)nthreads, sizeof(job_t));
  pthread_t* th = (pthread_t*)calloc((size_t)nthreads, sizeof(pthread_t));
  for (int i = 0; i < nthreads; ++i) {
    job_t* J = &jobs[i];
    J->out = out; J->t0 = t0; J->nt = nt; J->nfreq = nfreq; J->npol = npol;
    J->nx = nx; J->ny = ny; J->sigma = sigma; J->nsrc = nsrc; J->amp = src_amp;
    J->steer = steer;
    J->seed_noise = mix64(seed);
    J->seed_src = mix64(seed ^ 0xD1B54A32D192ED03ULL);
    J->row_lo = rows * i / nthreads;
    J->row_hi = rows * (i + 1) / nthreads;
  }
  for (int i = 1; i < nthreads; ++i) pthread_create(&th[i], NULL, run_rows, &jobs[i]);
  run_rows(&jobs[0]);
  for (int i = 1; i < nthreads; ++i) pthread_join(th[i], NULL);
  free(th);
  free(jobs);
  free(steer);
  return 0;
}
