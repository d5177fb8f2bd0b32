/*
 * Seeded synthetic 8-bit filterbank generator.
 *
 * This module only makes INPUT data. It holds none of the dedispersion or
 * single-pulse-search arithmetic: where a pulse is dispersed, the caller
 * passes the per-channel arrival sample of that pulse, computed elsewhere.
 * Both the CPU oracle's tests and the GPU path's tests and benchmark draw
 * their inputs from here, so the two sides always see identical bytes.
 *
 * Layout: time-major filterbank, x[t][c] (t = sample, c = channel), uint8,
 * the order in which a telescope back end writes spectra.
 *
 * Noise model (fully integer, identical on every host architecture):
 *   u_k, k = 0..11   twelve uniform 16-bit integers taken from three
 *                    splitmix64 outputs keyed by (seed, beam, channel, t)
 *   v = 128*4096 + (sum_k u_k - 12*32768) + amp_q12
 *   x = clamp(floor((v + 2048) / 4096), 0, 255)
 * The Irwin-Hall sum of twelve uniforms is a standard Gaussian approximation;
 * divided by 65536 it has unit variance, so the noise has mean ~128 and
 * standard deviation ~16 (bounded at +-6 sigma, inside the 0..255 clip).
 * amp_q12 is the summed pulse amplitude at (c, t) in units of 1/4096 LSB.
 */
#include <stdint.h>
#include <stddef.h>

static inline uint64_t splitmix64(uint64_t z) {
  /* Steele, Lea & Flood (2014) SplitMix64 finaliser. */
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

static inline int32_t noise_q12(uint64_t key) {
  int32_t s = 0;
  for (int k = 0; k < 3; ++k) {
    uint64_t r = splitmix64(key * 3u + (uint64_t)k);
    s += (int32_t)(r & 0xFFFF) + (int32_t)((r >> 16) & 0xFFFF) + (int32_t)((r >> 32) & 0xFFFF) +
         (int32_t)(r >> 48);
  }
  return s - 12 * 32768;
}

/*
 * Fill out[t - t0][c] for t in [t0, t0 + nsamp), c in [0, nchans).
 *   seed, beam       : RNG stream selection
 *   npulses          : number of injected boxcar pulses
 *   arrival          : [npulses][nchans] int64, first sample of pulse p in channel c
 *   width            : [npulses] boxcar length in samples (>= 1)
 *   amp_q12          : [npulses] amplitude per channel in 1/4096 LSB
 * Generating any sub-range [t0, t0 + nsamp) yields exactly the bytes of the
 * same range of a longer generation, so chunks can be made independently.
 */
void synth_filterbank(uint8_t* out, int64_t t0, int64_t nsamp, int32_t nchans, uint64_t seed,
                      uint64_t beam, int32_t npulses, const int64_t* arrival, const int32_t* width,
                      const int32_t* amp_q12) {
  const uint64_t base = splitmix64(seed ^ splitmix64(beam + 0x51ED270B1Dull));
#pragma omp parallel for schedule(static)
  for (int64_t tt = 0; tt < nsamp; ++tt) {
    const int64_t t = t0 + tt;
    for (int32_t c = 0; c < nchans; ++c) {
      uint64_t key = base + (((uint64_t)t << 16) | (uint64_t)c);
      int64_t v = 128 * 4096 + (int64_t)noise_q12(key);
      for (int32_t p = 0; p < npulses; ++p) {
        int64_t a = arrival[(size_t)p * (size_t)nchans + (size_t)c];
        if (t >= a && t < a + width[p]) v += amp_q12[p];
      }
      /* v + 2048 >= 0 unless a negative pulse amplitude is injected; clamp first so the
         floor division below only ever sees non-negative values */
      int64_t q = v + 2048 < 0 ? 0 : (v + 2048) / 4096;
      out[(size_t)tt * (size_t)nchans + (size_t)c] = (uint8_t)(q > 255 ? 255 : q);
    }
  }
}
