/*
 * fx_oracle.c -- plain, slow FP64 CPU oracle of the FX correlator hot path.
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark call this file.  It shares no code, header, table or
 * constant with the CUDA library; it is written from the paper and from the
 * readings listed below, step by step, in the order the method runs.
 *
 * The paper (Abstract) defines the correlator as an FX correlator: each
 * station's samples are first Fourier transformed, then every station pair is
 * cross-multiplied and accumulated.  Sec. 2 says the delay model (Calc,
 * extended for a moving spacecraft and the spacecraft -> tracking-station
 * leg) supplies each station's delay; here that delay enters as polynomial
 * segments tau(t) = sum_i c_i (t - t0)^i.  Everything the paper leaves open
 * is fixed by these readings:
 *
 *   packing   code of stream j at sample-time t sits at bit 2*(t*G + j) of a
 *             little-endian bit stream (LSB first); G = nsub*npol streams,
 *             j = sb*npol + pol; a 4-entry table maps codes to levels.
 *   frames    (selectable) Mark5B-style framing: the station's bytes are frames
 *             of a 16-byte header and P payload bytes; the payloads in frame
 *             order form the bit stream above; a frame is valid when its first
 *             header word (32-bit little-endian) is the sync word 0xABADDEED.
 *   time      seconds relative to the scan epoch; block b spans geocentric
 *             samples [b*N, b*N + N), centre t_c = (b*N + N/2)/fs.
 *   delay     segment = largest t0 <= t_c; tau by Horner from c5 with fma at
 *             every step; n_b = floor(fma(tau, fs, 0.5)); eps = tau - n_b/fs;
 *             the block reads station samples [b*N + n_b, b*N + n_b + N).
 *   validity  a block is valid at a station when its window lies inside the
 *             station's samples and t_c >= the first segment's t0 (and, for
 *             framed input, every frame holding one of its samples is valid);
 *             a baseline's weight counts blocks valid at both ends.
 *   integr.   block b belongs to integration floor(b*N / SPI), with
 *             SPI = fs*tint samples per integration (an integer).
 *   spectrum  X[k] = sum_n x[n] exp(-2 pi i k n / N), k = 0..N/2-1 (DC kept,
 *             Nyquist dropped), unnormalised, rectangular window.
 *   rotation  post-F (the default) at the block centre:
 *             X[k] *= exp(+2 pi i (phi + f_k eps)), phi = frac(nu0 * tau), f_k = k*fs/N.
 *             pre-F (selectable): the fringe phase is applied per sample before
 *             the transform, linear about the block centre,
 *               y[n] = x[n] exp(+2 pi i (phi + nu0 tau'(t_c) (n - N/2) / fs)),
 *             tau' the derivative of the delay polynomial at t_c; then the
 *             complex N-point transform Y[k] = sum_n y[n] exp(-2 pi i k n / N),
 *             k = 0..N/2-1, and the fractional-delay slope Y[k] *= exp(+2 pi i f_k eps).
 *   X-step    V_ab[k] = sum over blocks of X_a[k] conj(X_b[k]) for a <= b,
 *             parallel hands (stream by stream); baselines (0,0),(0,1),..,(1,1),..
 *             With both hands of two polarisations (selectable, npol = 2):
 *             V_ab^pq[k] = sum over blocks of X_a^p[k] conj(X_b^q[k]) for every
 *             a <= b and p, q in {0, 1}, hand products ordered pq = 00, 01, 10, 11.
 *   output    V_ab / (W_ab * N); zero where W_ab = 0.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (the FP64 delay
 * arithmetic must not be contracted beyond the fma calls written here).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* Scan description (flat arrays so that ctypes can pass it).               */

typedef struct {
  int S, nsub, npol, nchan;
  double fs, tint;
  double lut[4];
  const double *nu0;      /* [nsub] sky frequency per subband (Hz)          */
  const int *nseg;        /* [S] segment count per station                  */
  const double *seg_t0;   /* [S * maxseg]                                   */
  const double *seg_c;    /* [S * maxseg * 6]                               */
  int maxseg;
  const uint8_t *bytes;   /* all stations' packed bytes, concatenated       */
  const int64_t *byte_off;/* [S] offset of each station's bytes             */
  const int64_t *sample0; /* [S] station sample index of the first group    */
  const int64_t *nsamp;   /* [S] number of sample-time groups present       */
  int rotation;           /* 0: post-F fringe rotation, 1: pre-F            */
  int frame_payload;      /* 0: plain packed bytes; P > 0: frames of 16 + P bytes */
} oracle_scan;

#define ORACLE_SYNC 0xABADDEEDu
#define ORACLE_HEADER 16

/* ------------------------------------------------------------------------ */
/* Unpacking (the packing reading above).                                   */

int oracle_code(const uint8_t *bytes, int G, int64_t t, int j) {
  int64_t bit = 2 * (t * (int64_t)G + j);
  return (bytes[bit >> 3] >> (bit & 7)) & 3;
}

/* The same code from a framed stream: payload byte q of the bit stream sits in
 * frame q / P at offset 16 + q % P. */
static int framed_code(const uint8_t *raw, int P, int G, int64_t t, int j) {
  int64_t bit = 2 * (t * (int64_t)G + j);
  int64_t q = bit >> 3;
  int64_t f = q / P;
  return (raw[f * (ORACLE_HEADER + P) + ORACLE_HEADER + (q - f * P)] >> (bit & 7)) & 3;
}

static int frame_valid(const uint8_t *raw, int P, int64_t f) {
  const uint8_t *h = raw + f * (int64_t)(ORACLE_HEADER + P);
  uint32_t w = (uint32_t)h[0] | ((uint32_t)h[1] << 8) | ((uint32_t)h[2] << 16) | ((uint32_t)h[3] << 24);
  return w == ORACLE_SYNC;
}

static int sample_code(const oracle_scan *sc, int s, int64_t t, int j) {
  const uint8_t *bytes = sc->bytes + sc->byte_off[s];
  const int G = sc->nsub * sc->npol;
  return sc->frame_payload > 0 ? framed_code(bytes, sc->frame_payload, G, t, j) : oracle_code(bytes, G, t, j);
}

/* codes of stream j for sample-time groups [t0, t0+count) of one station. */
void oracle_unpack_codes(const uint8_t *bytes, int G, int j, int64_t t0, int64_t count, uint8_t *out) {
  for (int64_t n = 0; n < count; ++n) out[n] = (uint8_t)oracle_code(bytes, G, t0 + n, j);
}

/* ------------------------------------------------------------------------ */
/* Delay model: segment selection, Horner in FP64, integer and fractional   */
/* delay, absolute fringe phase.                                            */

typedef struct {
  int64_t nstart;  /* n_b: integer-sample delay                            */
  double tau;      /* delay at the block centre (s)                        */
  double rate;     /* d tau / dt at the block centre (s/s)                 */
  double eps;      /* tau - n_b/fs (s)                                     */
  int covered;     /* t_c lies at or after the first segment's t0          */
} oracle_delay;

static oracle_delay block_delay(const oracle_scan *sc, int s, int64_t b) {
  oracle_delay d;
  const int N = 2 * sc->nchan;
  double tc = (double)(b * (int64_t)N + N / 2) / sc->fs;
  const double *t0 = sc->seg_t0 + (size_t)s * sc->maxseg;
  int ns = sc->nseg[s];
  int seg = -1;
  for (int i = 0; i < ns; ++i)
    if (t0[i] <= tc) seg = i;
  d.covered = seg >= 0;
  if (seg < 0) seg = 0;
  const double *c = sc->seg_c + ((size_t)s * sc->maxseg + seg) * 6;
  double u = tc - t0[seg];
  double tau = c[5];
  for (int i = 4; i >= 0; --i) tau = fma(tau, u, c[i]);
  d.tau = tau;
  /* derivative of the same polynomial, sum_{i>=1} i c_i u^(i-1) */
  double rate = 0.0;
  for (int i = 5; i >= 1; --i) rate = rate * u + (double)i * c[i];
  d.rate = rate;
  d.nstart = (int64_t)floor(fma(tau, sc->fs, 0.5));
  d.eps = tau - (double)d.nstart / sc->fs;
  return d;
}

static int block_valid(const oracle_scan *sc, int s, int64_t b, const oracle_delay *d) {
  const int N = 2 * sc->nchan;
  int64_t i0 = b * (int64_t)N + d->nstart;
  if (!(d->covered && i0 >= sc->sample0[s] && i0 + N <= sc->sample0[s] + sc->nsamp[s])) return 0;
  if (sc->frame_payload > 0) {
    /* every frame holding a sample of the window must be valid */
    const int G = sc->nsub * sc->npol, P = sc->frame_payload;
    const uint8_t *raw = sc->bytes + sc->byte_off[s];
    for (int64_t t = i0 - sc->sample0[s]; t < i0 - sc->sample0[s] + N; ++t)
      for (int j = 0; j < G; ++j) {
        int64_t q = (2 * (t * (int64_t)G + j)) >> 3;
        if (!frame_valid(raw, P, q / P)) return 0;
      }
  }
  return 1;
}

/* Per (station, block): n_b, eps, tau, validity and (if rate != NULL) the
 * delay rate for blocks [b0, b0+nb). */
void oracle_delays_ex(const oracle_scan *sc, int64_t b0, int64_t nb, int64_t *nstart, double *eps,
                      double *tau, uint8_t *valid, double *rate) {
  for (int s = 0; s < sc->S; ++s)
    for (int64_t i = 0; i < nb; ++i) {
      oracle_delay d = block_delay(sc, s, b0 + i);
      size_t o = (size_t)s * nb + i;
      nstart[o] = d.nstart;
      eps[o] = d.eps;
      tau[o] = d.tau;
      valid[o] = (uint8_t)block_valid(sc, s, b0 + i, &d);
      if (rate) rate[o] = d.rate;
    }
}

/* Per (station, block): n_b, eps, tau and validity for blocks [b0, b0+nb). */
void oracle_delays(const oracle_scan *sc, int64_t b0, int64_t nb,
                   int64_t *nstart, double *eps, double *tau, uint8_t *valid) {
  oracle_delays_ex(sc, b0, nb, nstart, eps, tau, valid, NULL);
}

/* Absolute fringe phase in turns, frac(nu0 * tau), in FP64. */
static double fringe_turns(double nu0, double tau) {
  double p = nu0 * tau;
  return p - floor(p);
}

/* ------------------------------------------------------------------------ */
/* FFT: iterative radix-2 Cooley-Tukey (1965), decimation in time, FP64,    */
/* forward sign exp(-2 pi i k n / N); inverse uses exp(+...) unscaled.       */

void oracle_fft(double *re, double *im, int n, int inverse) {
  for (int i = 1, j = 0; i < n; ++i) {
    int bit = n >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) {
      double t = re[i]; re[i] = re[j]; re[j] = t;
      t = im[i]; im[i] = im[j]; im[j] = t;
    }
  }
  double sgn = inverse ? 1.0 : -1.0;
  for (int len = 2; len <= n; len <<= 1) {
    int half = len >> 1;
    for (int k = 0; k < half; ++k) {
      double ang = sgn * 2.0 * ORACLE_PI * (double)k / (double)len;
      double wr = cos(ang), wi = sin(ang);
      for (int i = 0; i < n; i += len) {
        double ar = re[i + k], ai = im[i + k];
        double br = re[i + k + half], bi = im[i + k + half];
        double tr = br * wr - bi * wi;
        double ti = br * wi + bi * wr;
        re[i + k] = ar + tr; im[i + k] = ai + ti;
        re[i + k + half] = ar - tr; im[i + k + half] = ai - ti;
      }
    }
  }
}

/* ------------------------------------------------------------------------ */
/* One station's rotated spectrum for one stream and block (F step).        */
/* Returns 0 when the block is not valid at that station (spectrum zeroed). */

static int station_spectrum(const oracle_scan *sc, int s, int j, int64_t b,
                            double *re, double *im, double *xr, double *xi) {
  const int N = 2 * sc->nchan, G = sc->nsub * sc->npol;
  oracle_delay d = block_delay(sc, s, b);
  if (!block_valid(sc, s, b, &d)) {
    memset(xr, 0, sizeof(double) * sc->nchan);
    memset(xi, 0, sizeof(double) * sc->nchan);
    return 0;
  }
  int64_t t0 = b * (int64_t)N + d.nstart - sc->sample0[s];
  double nu0 = sc->nu0[j / sc->npol];
  double phi = fringe_turns(nu0, d.tau);
  if (sc->rotation == 1) {
    /* pre-F: per-sample fringe phase, linear about the block centre */
    double per_sample = nu0 * d.rate / sc->fs;
    for (int n = 0; n < N; ++n) {
      double a = 2.0 * ORACLE_PI * (phi + per_sample * (double)(n - N / 2));
      double x = sc->lut[sample_code(sc, s, t0 + n, j)];
      re[n] = x * cos(a);
      im[n] = x * sin(a);
    }
    oracle_fft(re, im, N, 0);
    for (int k = 0; k < sc->nchan; ++k) {
      double fk = (double)k * sc->fs / (double)N;
      double a = 2.0 * ORACLE_PI * fk * d.eps;
      double c = cos(a), sn = sin(a);
      xr[k] = re[k] * c - im[k] * sn;
      xi[k] = re[k] * sn + im[k] * c;
    }
    return 1;
  }
  for (int n = 0; n < N; ++n) {
    re[n] = sc->lut[sample_code(sc, s, t0 + n, j)];
    im[n] = 0.0;
  }
  oracle_fft(re, im, N, 0);
  for (int k = 0; k < sc->nchan; ++k) {
    double fk = (double)k * sc->fs / (double)N;
    double a = 2.0 * ORACLE_PI * (phi + fk * d.eps);
    double c = cos(a), sn = sin(a);
    xr[k] = re[k] * c - im[k] * sn;
    xi[k] = re[k] * sn + im[k] * c;
  }
  return 1;
}

/* Exported single spectrum (for comparing one F-step output in isolation). */
int oracle_spectrum(const oracle_scan *sc, int s, int j, int64_t b, double *out /* [nchan][2] */) {
  const int N = 2 * sc->nchan;
  double *re = malloc(sizeof(double) * N), *im = malloc(sizeof(double) * N);
  double *xr = malloc(sizeof(double) * sc->nchan), *xi = malloc(sizeof(double) * sc->nchan);
  int v = station_spectrum(sc, s, j, b, re, im, xr, xi);
  for (int k = 0; k < sc->nchan; ++k) { out[2 * k] = xr[k]; out[2 * k + 1] = xi[k]; }
  free(re); free(im); free(xr); free(xi);
  return v;
}

/* ------------------------------------------------------------------------ */
/* Integration boundaries: first block of integration i = ceil(i*SPI/N).    */

static int64_t integ_first_block(int64_t i, int64_t spi, int N) {
  return (i * spi + N - 1) / N;
}

/* ------------------------------------------------------------------------ */
/* The full FX path for integrations [i0, i0+ni) and streams [j0, j0+nj).   */
/* vis: [ni][nbl][nj][nchan][2]; weights: [ni][nbl] (blocks valid at both). */
/* full != 0 also computes b < a (for the Hermitian-structure test); then   */
/* vis is [ni][S*S][nj][nchan][2] in row-major (a, b).                       */

int oracle_correlate_ex(const oracle_scan *sc, int64_t i0, int ni, int j0, int nj,
                        int full, double *vis, double *weights) {
  const int S = sc->S, N = 2 * sc->nchan, nch = sc->nchan;
  const int nbl = full ? S * S : S * (S + 1) / 2;
  int64_t spi = llround(sc->fs * sc->tint);
  if (fabs(sc->fs * sc->tint - (double)spi) > 1e-6 || spi <= 0) return -1;
  memset(vis, 0, sizeof(double) * 2 * (size_t)ni * nbl * nj * nch);
  if (weights) memset(weights, 0, sizeof(double) * (size_t)ni * nbl);

#pragma omp parallel for schedule(dynamic, 1)
  for (int jj = 0; jj < nj; ++jj) {
    int j = j0 + jj;
    double *re = malloc(sizeof(double) * N), *im = malloc(sizeof(double) * N);
    double *xr = malloc(sizeof(double) * (size_t)S * nch), *xi = malloc(sizeof(double) * (size_t)S * nch);
    double *acc = malloc(sizeof(double) * 2 * (size_t)nbl * nch);
    int *ok = malloc(sizeof(int) * S);
    for (int ii = 0; ii < ni; ++ii) {
      int64_t bfirst = integ_first_block(i0 + ii, spi, N);
      int64_t bend = integ_first_block(i0 + ii + 1, spi, N);
      memset(acc, 0, sizeof(double) * 2 * (size_t)nbl * nch);
      double *w = malloc(sizeof(double) * nbl);
      memset(w, 0, sizeof(double) * nbl);
      for (int64_t b = bfirst; b < bend; ++b) {
        for (int s = 0; s < S; ++s)
          ok[s] = station_spectrum(sc, s, j, b, re, im, xr + (size_t)s * nch, xi + (size_t)s * nch);
        int bl = 0;
        for (int a = 0; a < S; ++a)
          for (int c = full ? 0 : a; c < S; ++c, ++bl) {
            if (!(ok[a] && ok[c])) continue;
            w[bl] += 1.0;
            const double *ar = xr + (size_t)a * nch, *ai = xi + (size_t)a * nch;
            const double *cr = xr + (size_t)c * nch, *ci = xi + (size_t)c * nch;
            double *o = acc + 2 * (size_t)bl * nch;
            for (int k = 0; k < nch; ++k) {
              /* X_a conj(X_c) */
              o[2 * k] += ar[k] * cr[k] + ai[k] * ci[k];
              o[2 * k + 1] += ai[k] * cr[k] - ar[k] * ci[k];
            }
          }
      }
      for (int bl = 0; bl < nbl; ++bl) {
        double scale = w[bl] > 0 ? 1.0 / (w[bl] * (double)N) : 0.0;
        double *dst = vis + 2 * ((((size_t)ii * nbl + bl) * nj + jj) * nch);
        const double *src = acc + 2 * (size_t)bl * nch;
        for (int k = 0; k < 2 * nch; ++k) dst[k] = src[k] * scale;
        if (weights && jj == 0) weights[(size_t)ii * nbl + bl] = w[bl];
      }
      free(w);
    }
    free(re); free(im); free(xr); free(xi); free(acc); free(ok);
  }
  return 0;
}

int oracle_correlate(const oracle_scan *sc, int64_t i0, int ni, int j0, int nj,
                     double *vis, double *weights) {
  return oracle_correlate_ex(sc, i0, ni, j0, nj, 0, vis, weights);
}

/* ------------------------------------------------------------------------ */
/* Both hands of two polarisations, for integrations [i0, i0+ni):           */
/* vis [ni][nbl][nsub][4][nchan][2], hand product pq = 2p + q, i.e.         */
/* V_ab^pq = sum over blocks of X_a^p conj(X_b^q); weights [ni][nbl].       */

int oracle_correlate_cross(const oracle_scan *sc, int64_t i0, int ni, double *vis, double *weights) {
  const int S = sc->S, N = 2 * sc->nchan, nch = sc->nchan, nsub = sc->nsub;
  const int nbl = S * (S + 1) / 2;
  if (sc->npol != 2) return -2;
  int64_t spi = llround(sc->fs * sc->tint);
  if (fabs(sc->fs * sc->tint - (double)spi) > 1e-6 || spi <= 0) return -1;
  memset(vis, 0, sizeof(double) * 2 * (size_t)ni * nbl * nsub * 4 * nch);
  if (weights) memset(weights, 0, sizeof(double) * (size_t)ni * nbl);

#pragma omp parallel for schedule(dynamic, 1)
  for (int sb = 0; sb < nsub; ++sb) {
    double *re = malloc(sizeof(double) * N), *im = malloc(sizeof(double) * N);
    /* spectra of both pols of every station: [p][s][k] */
    double *xr = malloc(sizeof(double) * 2 * (size_t)S * nch), *xi = malloc(sizeof(double) * 2 * (size_t)S * nch);
    double *acc = malloc(sizeof(double) * 2 * (size_t)nbl * 4 * nch);
    int *ok = malloc(sizeof(int) * S);
    for (int ii = 0; ii < ni; ++ii) {
      int64_t bfirst = integ_first_block(i0 + ii, spi, N);
      int64_t bend = integ_first_block(i0 + ii + 1, spi, N);
      memset(acc, 0, sizeof(double) * 2 * (size_t)nbl * 4 * nch);
      double *w = malloc(sizeof(double) * nbl);
      memset(w, 0, sizeof(double) * nbl);
      for (int64_t b = bfirst; b < bend; ++b) {
        for (int p = 0; p < 2; ++p)
          for (int s = 0; s < S; ++s) {
            size_t o = ((size_t)p * S + s) * nch;
            /* validity depends on the station and block only */
            ok[s] = station_spectrum(sc, s, sb * 2 + p, b, re, im, xr + o, xi + o);
          }
        int bl = 0;
        for (int a = 0; a < S; ++a)
          for (int c = a; c < S; ++c, ++bl) {
            if (!(ok[a] && ok[c])) continue;
            w[bl] += 1.0;
            for (int p = 0; p < 2; ++p)
              for (int q = 0; q < 2; ++q) {
                const double *ar = xr + ((size_t)p * S + a) * nch, *ai = xi + ((size_t)p * S + a) * nch;
                const double *cr = xr + ((size_t)q * S + c) * nch, *ci = xi + ((size_t)q * S + c) * nch;
                double *o = acc + 2 * ((size_t)bl * 4 + 2 * p + q) * nch;
                for (int k = 0; k < nch; ++k) {
                  /* X_a^p conj(X_c^q) */
                  o[2 * k] += ar[k] * cr[k] + ai[k] * ci[k];
                  o[2 * k + 1] += ai[k] * cr[k] - ar[k] * ci[k];
                }
              }
          }
      }
      for (int bl = 0; bl < nbl; ++bl) {
        double scale = w[bl] > 0 ? 1.0 / (w[bl] * (double)N) : 0.0;
        for (int pq = 0; pq < 4; ++pq) {
          double *dst = vis + 2 * (((((size_t)ii * nbl + bl) * nsub + sb) * 4 + pq) * nch);
          const double *src = acc + 2 * ((size_t)bl * 4 + pq) * nch;
          for (int k = 0; k < 2 * nch; ++k) dst[k] = src[k] * scale;
        }
        if (weights && sb == 0) weights[(size_t)ii * nbl + bl] = w[bl];
      }
      free(w);
    }
    free(re); free(im); free(xr); free(xi); free(acc); free(ok);
  }
  return 0;
}

int oracle_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
