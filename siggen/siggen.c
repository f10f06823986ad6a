/*
 * siggen.c -- seeded synthetic signals that stand in for the paper's four signal
 * domains (biomedical EEG, seismic traces, power-grid telemetry, meteorological
 * series; Sec. 5.2, Table 2).  The real datasets are not available, so every
 * input of the tests and of the benchmark is drawn here from a seed.
 *
 * This module holds none of the codec's arithmetic (no transform, no quantizer,
 * no entropy coder).  It is shared by the FP64 oracle (tests) and by the
 * benchmark, and by nothing else.
 *
 * PRNG: xoshiro256** (Blackman & Vigna) seeded through SplitMix64; uniform
 * doubles from the top 53 bits; normals by the Box-Muller transform (both
 * outputs of each pair are used).  Stream i of workload c uses the seed
 * splitmix64(0xF97C0000 + 1000003*c + i).
 *
 * Compile with -ffp-contract=off so that x86 and Arm hosts produce the same
 * values for the same seed (up to libm differences in sin/cos/exp/log).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ---- PRNG ------------------------------------------------------------- */

static uint64_t sm64_step(uint64_t *state) {
  uint64_t z = (*state += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* One SplitMix64 output for state x (used to derive per-stream seeds). */
uint64_t sg_splitmix64(uint64_t x) {
  uint64_t s = x;
  return sm64_step(&s);
}

uint64_t sg_stream_seed(uint32_t config, uint64_t index) {
  return sg_splitmix64(0xF97C0000ull + 1000003ull * (uint64_t)config + index);
}

typedef struct {
  uint64_t s[4];
  double spare;
  int have_spare;
} sg_rng;

static uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static void rng_seed(sg_rng *r, uint64_t seed) {
  uint64_t sm = seed;
  for (int i = 0; i < 4; ++i) r->s[i] = sm64_step(&sm);
  r->have_spare = 0;
  r->spare = 0.0;
}

static uint64_t rng_next(sg_rng *r) {
  uint64_t *s = r->s;
  const uint64_t out = rotl64(s[1] * 5u, 7) * 9u;
  const uint64_t t = s[1] << 17;
  s[2] ^= s[0];
  s[3] ^= s[1];
  s[1] ^= s[2];
  s[0] ^= s[3];
  s[2] ^= t;
  s[3] = rotl64(s[3], 45);
  return out;
}

/* uniform in [0, 1) */
static double rng_uniform(sg_rng *r) { return (double)(rng_next(r) >> 11) * 0x1.0p-53; }

static double rng_range(sg_rng *r, double lo, double hi) { return lo + (hi - lo) * rng_uniform(r); }

static double rng_normal(sg_rng *r) {
  if (r->have_spare) {
    r->have_spare = 0;
    return r->spare;
  }
  double u1 = 1.0 - rng_uniform(r); /* (0, 1] so the log is finite */
  double u2 = rng_uniform(r);
  double rad = sqrt(-2.0 * log(u1));
  r->spare = rad * sin(2.0 * M_PI * u2);
  r->have_spare = 1;
  return rad * cos(2.0 * M_PI * u2);
}

/* Exported for tests of the generator itself. */
void sg_rng_fill_u64(uint64_t seed, uint64_t *out, uint64_t n) {
  sg_rng r;
  rng_seed(&r, seed);
  for (uint64_t i = 0; i < n; ++i) out[i] = rng_next(&r);
}

void sg_rng_fill_normal(uint64_t seed, double *out, uint64_t n) {
  sg_rng r;
  rng_seed(&r, seed);
  for (uint64_t i = 0; i < n; ++i) out[i] = rng_normal(&r);
}

/* ---- domain generators --------------------------------------------------- */

/* EEG-like channel, 256 Hz: 8 sinusoids (f ~ U[1,40] Hz, amplitude ~ U[5,50] uV,
 * phase ~ U[0,2pi)) plus pink noise (Voss-McCartney, 16 rows) rescaled to an
 * empirical standard deviation of 10 uV. */
void sg_eeg(uint64_t seed, float *x, uint64_t S) {
  sg_rng r;
  rng_seed(&r, seed);
  double f[8], a[8], ph[8];
  for (int j = 0; j < 8; ++j) {
    f[j] = rng_range(&r, 1.0, 40.0);
    a[j] = rng_range(&r, 5.0, 50.0);
    ph[j] = rng_range(&r, 0.0, 2.0 * M_PI);
  }
  if (S == 0) return;
  /* pink noise into x first */
  double rows[16];
  double acc = 0.0;
  for (int j = 0; j < 16; ++j) {
    rows[j] = rng_normal(&r);
    acc += rows[j];
  }
  double s1 = 0.0, s2 = 0.0;
  for (uint64_t n = 0; n < S; ++n) {
    if (n > 0) {
      int z = __builtin_ctzll(n);
      if (z < 16) {
        double v = rng_normal(&r);
        acc += v - rows[z];
        rows[z] = v;
      }
    }
    float p = (float)acc;
    x[n] = p;
    s1 += p;
    s2 += (double)p * (double)p;
  }
  double mean = s1 / (double)S;
  double var = s2 / (double)S - mean * mean;
  double scale = var > 0.0 ? 10.0 / sqrt(var) : 0.0;
  /* sinusoids: exact phase at the start of every 256-sample block, then a
   * complex rotation per sample inside the block */
  double cr[8], sr[8];
  for (int j = 0; j < 8; ++j) {
    cr[j] = cos(2.0 * M_PI * f[j] / 256.0);
    sr[j] = sin(2.0 * M_PI * f[j] / 256.0);
  }
  for (uint64_t b0 = 0; b0 < S; b0 += 256) {
    double c[8], sn[8];
    for (int j = 0; j < 8; ++j) {
      double ph0 = 2.0 * M_PI * f[j] * ((double)b0 / 256.0) + ph[j];
      c[j] = cos(ph0);
      sn[j] = sin(ph0);
    }
    uint64_t b1 = b0 + 256 < S ? b0 + 256 : S;
    for (uint64_t n = b0; n < b1; ++n) {
      double v = 0.0;
      for (int j = 0; j < 8; ++j) {
        v += a[j] * sn[j];
        double c2 = c[j] * cr[j] - sn[j] * sr[j];
        sn[j] = sn[j] * cr[j] + c[j] * sr[j];
        c[j] = c2;
      }
      x[n] = (float)(v + scale * (double)x[n]);
    }
  }
}

/* Seismic trace, 1 kHz: Ricker wavelets r(t) = (1 - 2 pi^2 f^2 t^2) exp(-pi^2 f^2 t^2)
 * at Poisson event times (rate 10 / s), peak frequency f ~ U[10,60] Hz,
 * amplitude ~ N(0,1), support |t| <= 1.5 / f; plus white Gaussian noise at
 * SNR 20 dB (noise variance = mean clean power / 100). */
void sg_seismic(uint64_t seed, float *x, uint64_t S) {
  sg_rng r;
  rng_seed(&r, seed);
  const double fs = 1000.0;
  const double dur = (double)S / fs;
  for (uint64_t n = 0; n < S; ++n) x[n] = 0.0f;
  double t = 0.0;
  for (;;) {
    t += -log(1.0 - rng_uniform(&r)) / 10.0;
    if (t >= dur) break;
    double f = rng_range(&r, 10.0, 60.0);
    double amp = rng_normal(&r);
    double half = 1.5 / f;
    int64_t n0 = (int64_t)ceil((t - half) * fs);
    int64_t n1 = (int64_t)floor((t + half) * fs);
    if (n0 < 0) n0 = 0;
    if (n1 > (int64_t)S - 1) n1 = (int64_t)S - 1;
    double pf2 = M_PI * M_PI * f * f;
    for (int64_t n = n0; n <= n1; ++n) {
      double tau = (double)n / fs - t;
      double tt = pf2 * tau * tau;
      x[n] = (float)((double)x[n] + amp * (1.0 - 2.0 * tt) * exp(-tt));
    }
  }
  double p = 0.0;
  for (uint64_t n = 0; n < S; ++n) p += (double)x[n] * (double)x[n];
  double sigma = S ? sqrt(p / (double)S / 100.0) : 0.0;
  for (uint64_t n = 0; n < S; ++n) x[n] = (float)((double)x[n] + sigma * rng_normal(&r));
}

/* Power-grid series, one sample per minute: 100 + A_d sin(2 pi t/1440 + phi_d)
 * + A_w sin(2 pi t/10080 + phi_w) + AR(1) noise (phi = 0.95, innovation std 2);
 * A_d ~ U[20,40], A_w ~ U[5,15]. */
void sg_power(uint64_t seed, float *x, uint64_t S) {
  sg_rng r;
  rng_seed(&r, seed);
  double ad = rng_range(&r, 20.0, 40.0);
  double aw = rng_range(&r, 5.0, 15.0);
  double pd = rng_range(&r, 0.0, 2.0 * M_PI);
  double pw = rng_range(&r, 0.0, 2.0 * M_PI);
  double ar = 0.0;
  for (uint64_t n = 0; n < S; ++n) {
    ar = 0.95 * ar + 2.0 * rng_normal(&r);
    double tn = (double)n;
    double v = 100.0 + ad * sin(2.0 * M_PI * tn / 1440.0 + pd) + aw * sin(2.0 * M_PI * tn / 10080.0 + pw) + ar;
    x[n] = (float)v;
  }
}

/* Meteorological series, one sample per 10 minutes: 15 + A_s sin(2 pi t/52560 + phi)
 * + random walk (step std 0.01) + white noise (std 0.5); A_s ~ U[5,15]. */
void sg_met(uint64_t seed, float *x, uint64_t S) {
  sg_rng r;
  rng_seed(&r, seed);
  double as = rng_range(&r, 5.0, 15.0);
  double ph = rng_range(&r, 0.0, 2.0 * M_PI);
  double walk = 0.0;
  for (uint64_t n = 0; n < S; ++n) {
    if (n > 0) walk += 0.01 * rng_normal(&r);
    double v = 15.0 + as * sin(2.0 * M_PI * (double)n / 52560.0 + ph) + walk + 0.5 * rng_normal(&r);
    x[n] = (float)v;
  }
}

/* domain: 0 = EEG, 1 = seismic, 2 = power, 3 = meteorological */
int sg_signal(int domain, uint64_t seed, float *x, uint64_t S) {
  switch (domain) {
    case 0: sg_eeg(seed, x, S); return 0;
    case 1: sg_seismic(seed, x, S); return 0;
    case 2: sg_power(seed, x, S); return 0;
    case 3: sg_met(seed, x, S); return 0;
    default: return -1;
  }
}

/* Many signals at once (OpenMP over signals); signal i goes to out + offsets[i]. */
int sg_signal_many(const int32_t *domains, const uint64_t *seeds, const uint64_t *lengths,
                   const uint64_t *offsets, uint64_t count, float *out, int n_threads) {
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads > 0 ? n_threads : 1) reduction(| : bad)
  for (int64_t i = 0; i < (int64_t)count; ++i) {
    bad |= sg_signal(domains[i], seeds[i], out + offsets[i], lengths[i]) != 0;
  }
  return bad ? -1 : 0;
}

/* Layout of the mixed-domain batch: n signals with lengths floor(exp(U[ln lo, ln hi]))
 * and domains dealt round-robin (n/4 each) and then shuffled (Fisher-Yates). */
void sg_mixed_layout(uint64_t seed, uint64_t n, uint64_t lo, uint64_t hi, uint64_t *lengths, int32_t *domains) {
  sg_rng r;
  rng_seed(&r, seed);
  double llo = log((double)lo), lhi = log((double)hi);
  for (uint64_t i = 0; i < n; ++i) {
    uint64_t s = (uint64_t)floor(exp(rng_range(&r, llo, lhi)));
    if (s < lo) s = lo;
    if (s > hi) s = hi;
    lengths[i] = s;
    domains[i] = (int32_t)(i % 4);
  }
  for (uint64_t i = n; i > 1; --i) {
    uint64_t j = rng_next(&r) % i;
    int32_t tmp = domains[i - 1];
    domains[i - 1] = domains[j];
    domains[j] = tmp;
  }
}
