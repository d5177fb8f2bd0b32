/*
 * CPU ORACLE for brute-force incoherent dedispersion + boxcar single-pulse search.
 *
 * TEST INFRASTRUCTURE ONLY. This file is the plain, slow, obviously correct
 * statement of what the GPU path computes. Only the test-suite, the smoke
 * check and the benchmark's CPU-baseline leg may load it. It shares no code,
 * header or table with the GPU library, and the GPU library never calls it.
 *
 * The paper (Novotny, Adamek & Armour, "Implementing CUDA Streams into
 * AstroAccelerate", Sec. 1 and Sec. 2) names the two phases -- dedispersion of
 * time-chunked 8-bit data, then single pulse search (SPDT) -- but prints no
 * formula. Every formula below is the textbook definition, and each choice
 * the paper leaves open is marked READING.
 *
 * Arithmetic: FP64 for the delay table and the SNR, exact integers elsewhere.
 * Build with -ffp-contract=off so that no multiply-add is fused and the FP64
 * results are the same on every host.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* READING: cold-plasma dispersion constant k_DM = 4.148808e3 s MHz^2 pc^-1 cm^3
 * (delay in seconds for DM in pc cm^-3 and frequencies in MHz). */
#define OR_KDM 4.148808e3

/*
 * Dispersion delay table (Sec. 1: the DM-trial plan of the dedispersion phase; Sec. 3: the
 * ~6000-trial plan over 0-3000 pc cm^-3).
 *   DM_i   = dm_start + i * dm_step                      (READING: not accumulated)
 *   tau_c  = k_DM * DM_i * (1/f_c^2 - 1/f_ref^2),  f_ref = max_c f_c   (READING)
 *   s[i][c] = floor(tau_c / (tsamp * d) + 0.5)           (READING: round half up,
 *                                                          units of decimated samples)
 * Evaluation order, one IEEE operation at a time:
 *   dm = dm_start + (i * dm_step); a = 1/(f_c*f_c); b = 1/(f_ref*f_ref);
 *   tau = (k_DM * dm) * (a - b);  x = tau / (tsamp * d) + 0.5;  s = floor(x).
 * out: [n_trials][nchans] int32. Returns 0, or -1 if a shift does not fit int32.
 */
int or_shift_table(const double* freqs, int32_t nchans, double tsamp, double dm_start,
                   double dm_step, int32_t n_trials, int32_t decimation, int32_t* out) {
  double fref = freqs[0];
  for (int32_t c = 1; c < nchans; ++c)
    if (freqs[c] > fref) fref = freqs[c];
  const double b = 1.0 / (fref * fref);
  const double unit = tsamp * (double)decimation;
  for (int32_t i = 0; i < n_trials; ++i) {
    const double dm = dm_start + (double)i * dm_step;
    for (int32_t c = 0; c < nchans; ++c) {
      const double a = 1.0 / (freqs[c] * freqs[c]);
      const double tau = (OR_KDM * dm) * (a - b);
      const double s = floor(tau / unit + 0.5);
      if (!(s >= -2147483648.0 && s <= 2147483647.0)) return -1;
      out[(size_t)i * nchans + c] = (int32_t)s;
    }
  }
  return 0;
}

/* Delay in seconds of channel c at dispersion measure dm relative to the highest frequency
 * (same formula as above, before division by the sample time). */
void or_delay_seconds(const double* freqs, int32_t nchans, double dm, double* out) {
  double fref = freqs[0];
  for (int32_t c = 1; c < nchans; ++c)
    if (freqs[c] > fref) fref = freqs[c];
  const double b = 1.0 / (fref * fref);
  for (int32_t c = 0; c < nchans; ++c) {
    const double a = 1.0 / (freqs[c] * freqs[c]);
    out[c] = (OR_KDM * dm) * (a - b);
  }
}

/*
 * Time decimation (READING: exact sum of d consecutive samples, windows aligned at global
 * sample 0; the paper is silent, the DM plan's "decimation" factors need a rule).
 * x: time-major uint8 filterbank [nsamp_in][nchans] whose row 0 is global sample t_in0.
 * out[c][j] = sum_{k<d} x[(t_first + j*d + k) - t_in0][c],  j in [0, n_out),
 * with t_first = j_first * d (j_first = first decimated index wanted).
 * The result is channel-major [nchans][n_out] uint32 (a plain re-indexing of the input).
 * Returns -1 if the requested window is not inside the input.
 */
int or_decimate(const uint8_t* x, int64_t t_in0, int64_t nsamp_in, int32_t nchans, int32_t d,
                int64_t j_first, int64_t n_out, uint32_t* out) {
  const int64_t t_first = j_first * d;
  if (t_first < t_in0 || t_first + n_out * d > t_in0 + nsamp_in) return -1;
#pragma omp parallel for schedule(static)
  for (int32_t c = 0; c < nchans; ++c) {
    for (int64_t j = 0; j < n_out; ++j) {
      uint32_t acc = 0;
      for (int32_t k = 0; k < d; ++k)
        acc += x[(size_t)(t_first + j * d + k - t_in0) * nchans + c];
      out[(size_t)c * n_out + j] = acc;
    }
  }
  return 0;
}

/*
 * Brute-force incoherent dedispersion (Sec. 1, Sec. 2.1: "dedispersion of data").
 *   y[i][j] = sum_{c < nchans} xd[c][(j0 + j) + s[i][c] - base]
 * xd: channel-major decimated data [nchans][nd], whose column 0 is decimated index `base`.
 * Outputs the global decimated indices j0 .. j0+nout-1 of the trials listed in `trials`
 * (indices into the shift table rows). y: [ntrials_out][nout] int32; sums are exact
 * (the caller keeps nchans * max(xd) < 2^31). Returns -1 if an index leaves xd.
 */
int or_dedisperse(const uint32_t* xd, int64_t base, int64_t nd, int32_t nchans,
                  const int32_t* shifts, const int32_t* trials, int32_t ntrials_out, int64_t j0,
                  int64_t nout, int32_t* y) {
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
  for (int32_t ii = 0; ii < ntrials_out; ++ii) {
    const int32_t* s = shifts + (size_t)trials[ii] * nchans;
    for (int64_t j = 0; j < nout; ++j) {
      int64_t acc = 0;
      for (int32_t c = 0; c < nchans; ++c) {
        const int64_t k = j0 + j + s[c] - base;
        if (k < 0 || k >= nd) {
          bad = 1;
          continue;
        }
        acc += xd[(size_t)c * nd + k];
      }
      y[(size_t)ii * nout + j] = (int32_t)acc;
    }
  }
  return bad ? -1 : 0;
}

/*
 * Moments of one dedispersed series over a window of n samples (Sec. 2.2, single pulse
 * search; READING: plain mean/variance from exact sums): S1 = sum y (int64),
 * S2 = sum y^2 (unsigned 128-bit, returned as lo/hi 64-bit words).
 */
void or_moments(const int32_t* y, int64_t n, int64_t* s1, uint64_t* s2lo, uint64_t* s2hi) {
  int64_t a = 0;
  unsigned __int128 b = 0;
  for (int64_t j = 0; j < n; ++j) {
    a += y[j];
    b += (unsigned __int128)((int64_t)y[j] * (int64_t)y[j]);
  }
  *s1 = a;
  *s2lo = (uint64_t)b;
  *s2hi = (uint64_t)(b >> 64);
}

typedef struct {
  int32_t trial;   /* trial index within its range */
  int32_t range;
  int64_t t_start; /* first original sample of the boxcar (global) */
  int32_t width;   /* boxcar width in original samples */
  int32_t pad;
  double snr;
} or_cand_t;

/*
 * Boxcar single-pulse search of one window of dedispersed series (Sec. 2.2; READINGs):
 *  - trailing boxcar of w decimated samples ending at window index j (j >= w-1):
 *      B_w[j] = P[j+1] - P[j+1-w],  P = int64 prefix sum of the window;
 *  - SNR_w[j] = (n*B_w[j] - w*S1) / (sqrt(w) * sqrt(n*S2 - S1^2)), FP64 from exact integers,
 *    i.e. (B - w*mean) / (sigma*sqrt(w)) with the window's own mean and population sigma;
 *    when n*S2 - S1^2 == 0 the series has no candidates;
 *  - per aligned block of `block` window samples [b*block, (b+1)*block), the maximum SNR over
 *    j in the block and all widths; ties go to the smaller j, then the smaller w;
 *  - the block maximum is a candidate when SNR >= threshold.
 * y: [ntr][n] series of trials `trial_ids` of range `range`, decimation d; widths_dec are
 * decimated widths (ascending); window sample j has global decimated index J0 + j.
 * Writes at most cap candidates; returns the total number found.
 */
int64_t or_sps(const int32_t* y, int32_t ntr, int64_t n, const int32_t* trial_ids, int32_t range,
               int32_t d, int64_t J0, const int32_t* widths_dec, int32_t nw, int32_t block,
               double threshold, or_cand_t* out, int64_t cap) {
  if (n <= 0 || ntr <= 0) return 0;
  /* trials are independent: each keeps its own candidate list, concatenated in trial order */
  or_cand_t** lists = (or_cand_t**)calloc((size_t)ntr, sizeof(or_cand_t*));
  int64_t* counts = (int64_t*)calloc((size_t)ntr, sizeof(int64_t));
  const int64_t nblocks = (n + block - 1) / block;
#pragma omp parallel
  {
    int64_t* P = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
#pragma omp for schedule(dynamic, 1)
    for (int32_t ii = 0; ii < ntr; ++ii) {
      const int32_t* yi = y + (size_t)ii * n;
      int64_t s1;
      uint64_t lo, hi;
      or_moments(yi, n, &s1, &lo, &hi);
      const unsigned __int128 s2 = ((unsigned __int128)hi << 64) | lo;
      const unsigned __int128 s1sq = (unsigned __int128)((__int128)s1 * (__int128)s1);
      const unsigned __int128 v = (unsigned __int128)n * s2 - s1sq;
      if (v == 0) continue;
      const double sq = sqrt((double)v);
      P[0] = 0;
      for (int64_t j = 0; j < n; ++j) P[j + 1] = P[j] + yi[j];
      or_cand_t* mine = NULL;
      int64_t cnt = 0;
      for (int64_t b0 = 0; b0 < n; b0 += block) {
        int have = 0;
        int64_t bj = 0;
        int32_t bw = 0;
        double best = 0.0;
        const int64_t b1 = b0 + block < n ? b0 + block : n;
        for (int64_t j = b0; j < b1; ++j) {
          for (int32_t k = 0; k < nw; ++k) {
            const int32_t w = widths_dec[k];
            if (j < w - 1) continue;
            const int64_t bsum = P[j + 1] - P[j + 1 - w];
            const int64_t num = n * bsum - (int64_t)w * s1;
            const double snr = (double)num / (sqrt((double)w) * sq);
            if (!have || snr > best) {
              have = 1;
              best = snr;
              bj = j;
              bw = w;
            }
          }
        }
        if (have && best >= threshold) {
          if (mine == NULL) mine = (or_cand_t*)malloc(sizeof(or_cand_t) * (size_t)nblocks);
          or_cand_t* o = mine + cnt++;
          o->trial = trial_ids[ii];
          o->range = range;
          o->t_start = (J0 + bj - bw + 1) * (int64_t)d;
          o->width = bw * d;
          o->pad = 0;
          o->snr = best;
        }
      }
      lists[ii] = mine;
      counts[ii] = cnt;
    }
    free(P);
  }
  int64_t total = 0;
  for (int32_t ii = 0; ii < ntr; ++ii) {
    for (int64_t k = 0; k < counts[ii]; ++k) {
      if (total < cap) out[total] = lists[ii][k];
      ++total;
    }
    free(lists[ii]);
  }
  free(lists);
  free(counts);
  return total;
}

/*
 * Clipped (robust) moments of one boxcar-filtered series (Sec. 2.2 names the SPDT estimators of
 * the single pulse search, whose definition is not in the paper; READING: iterative
 * kappa-sigma clipping, a standard robust estimator, applied per boxcar width).
 *   values : B_w[j] = sum_{k=j-w+1..j} y[k] for window samples j = w-1 .. n-1 (m = n-w+1 of
 *            them); none when m <= 0
 *   step 0 : N, T1 = sum B, T2 = sum B^2 (exact, T2 as 128 bits) over every value
 *   step i : (i = 1 .. iters) mu = T1 / N and sd = sqrt(N*T2 - T1^2) / N in FP64 (the 128-bit
 *            variance numerator converted to double with correct rounding);
 *            lo = ceil(mu - kappa*sd), hi = floor(mu + kappa*sd); N, T1, T2 recomputed over
 *            the values with lo <= B <= hi. A step whose previous variance is 0 (or N is 0)
 *            keeps the previous statistics; the loop stops there.
 * Returns the final N, T1 and T2 (lo/hi words).
 */
void or_clipped_moments(const int32_t* y, int64_t n, int32_t w, double kappa, int32_t iters,
                        int64_t* n_out, int64_t* t1_out, uint64_t* t2lo, uint64_t* t2hi) {
  int64_t N = 0, T1 = 0;
  unsigned __int128 T2 = 0;
  const int64_t m = n - w + 1;
  int64_t* B = NULL;
  if (m > 0) {
    B = (int64_t*)malloc(sizeof(int64_t) * (size_t)m);
    int64_t run = 0;
    for (int64_t k = 0; k < w - 1; ++k) run += y[k];
    for (int64_t j = w - 1; j < n; ++j) {
      run += y[j];
      if (j - w >= 0) run -= y[j - w];
      B[j - (w - 1)] = run;
    }
    for (int64_t k = 0; k < m; ++k) {
      N += 1;
      T1 += B[k];
      T2 += (unsigned __int128)((__int128)B[k] * (__int128)B[k]);
    }
  }
  for (int32_t it = 0; it < iters && N > 0; ++it) {
    const unsigned __int128 V = (unsigned __int128)N * T2 -
                                (unsigned __int128)((__int128)T1 * (__int128)T1);
    if (V == 0) break;
    const double mu = (double)T1 / (double)N;
    const double sd = sqrt((double)V) / (double)N;
    const double lo = ceil(mu - kappa * sd), hi = floor(mu + kappa * sd);
    int64_t N2 = 0, S1 = 0;
    unsigned __int128 S2 = 0;
    for (int64_t k = 0; k < m; ++k) {
      const double b = (double)B[k];
      if (b >= lo && b <= hi) {
        N2 += 1;
        S1 += B[k];
        S2 += (unsigned __int128)((__int128)B[k] * (__int128)B[k]);
      }
    }
    N = N2;
    T1 = S1;
    T2 = S2;
  }
  free(B);
  *n_out = N;
  *t1_out = T1;
  *t2lo = (uint64_t)T2;
  *t2hi = (uint64_t)(T2 >> 64);
}

/*
 * Boxcar single-pulse search with per-width clipped statistics (Sec. 2.2; READINGs as in
 * or_sps, except the noise statistic): for width w the SNR of B_w[j] is
 *      (N_w * B_w[j] - T1_w) / sqrt(N_w * T2_w - T1_w^2)
 * i.e. (B - mu_w) / sd_w with the clipped mean and population deviation of B_w itself
 * (or_clipped_moments; kappa, iters). A width whose clipped variance is 0 contributes nothing.
 * Block peaks, ties, threshold and output as in or_sps.
 */
int64_t or_sps_clipped(const int32_t* y, int32_t ntr, int64_t n, const int32_t* trial_ids,
                       int32_t range, int32_t d, int64_t J0, const int32_t* widths_dec, int32_t nw,
                       int32_t block, double threshold, double kappa, int32_t iters,
                       or_cand_t* out, int64_t cap) {
  if (n <= 0 || ntr <= 0) return 0;
  or_cand_t** lists = (or_cand_t**)calloc((size_t)ntr, sizeof(or_cand_t*));
  int64_t* counts = (int64_t*)calloc((size_t)ntr, sizeof(int64_t));
  const int64_t nblocks = (n + block - 1) / block;
#pragma omp parallel
  {
    int64_t* P = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
    int64_t* Nw = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nw > 0 ? nw : 1));
    int64_t* T1w = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nw > 0 ? nw : 1));
    double* den = (double*)malloc(sizeof(double) * (size_t)(nw > 0 ? nw : 1));
#pragma omp for schedule(dynamic, 1)
    for (int32_t ii = 0; ii < ntr; ++ii) {
      const int32_t* yi = y + (size_t)ii * n;
      for (int32_t k = 0; k < nw; ++k) {
        uint64_t lo, hi;
        or_clipped_moments(yi, n, widths_dec[k], kappa, iters, &Nw[k], &T1w[k], &lo, &hi);
        const unsigned __int128 t2 = ((unsigned __int128)hi << 64) | lo;
        const unsigned __int128 v = (unsigned __int128)Nw[k] * t2 -
                                    (unsigned __int128)((__int128)T1w[k] * (__int128)T1w[k]);
        den[k] = (Nw[k] > 0 && v > 0) ? sqrt((double)v) : 0.0;
      }
      P[0] = 0;
      for (int64_t j = 0; j < n; ++j) P[j + 1] = P[j] + yi[j];
      or_cand_t* mine = NULL;
      int64_t cnt = 0;
      for (int64_t b0 = 0; b0 < n; b0 += block) {
        int have = 0;
        int64_t bj = 0;
        int32_t bw = 0;
        double best = 0.0;
        const int64_t b1 = b0 + block < n ? b0 + block : n;
        for (int64_t j = b0; j < b1; ++j) {
          for (int32_t k = 0; k < nw; ++k) {
            const int32_t w = widths_dec[k];
            if (j < w - 1 || den[k] == 0.0) continue;
            const int64_t bsum = P[j + 1] - P[j + 1 - w];
            const int64_t num = Nw[k] * bsum - T1w[k];
            const double snr = (double)num / den[k];
            if (!have || snr > best) {
              have = 1;
              best = snr;
              bj = j;
              bw = w;
            }
          }
        }
        if (have && best >= threshold) {
          if (mine == NULL) mine = (or_cand_t*)malloc(sizeof(or_cand_t) * (size_t)nblocks);
          or_cand_t* o = mine + cnt++;
          o->trial = trial_ids[ii];
          o->range = range;
          o->t_start = (J0 + bj - bw + 1) * (int64_t)d;
          o->width = bw * d;
          o->pad = 0;
          o->snr = best;
        }
      }
      lists[ii] = mine;
      counts[ii] = cnt;
    }
    free(P);
    free(Nw);
    free(T1w);
    free(den);
  }
  int64_t total = 0;
  for (int32_t ii = 0; ii < ntr; ++ii) {
    for (int64_t k = 0; k < counts[ii]; ++k) {
      if (total < cap) out[total] = lists[ii][k];
      ++total;
    }
    free(lists[ii]);
  }
  free(lists);
  free(counts);
  return total;
}

/*
 * Friends-of-friends grouping of candidates (Sec. 2.2: the single pulse search reports
 * candidates; READING: candidates of one pulse seen at neighbouring DM trials, times and widths
 * are merged into one group, as a single-pulse search's candidate clustering does).
 *   DM of a candidate : dm_start[range] + trial * dm_step[range] (FP64, as the delay table)
 *   friends(a, b)     : |DM_a - DM_b| <= dm_link  and  their boxcars [t_start, t_start + width)
 *                       overlap or the later one starts at most t_link samples after the
 *                       earlier one's last sample: t_a <= t_b + w_b - 1 + t_link and
 *                       t_b <= t_a + w_a - 1 + t_link
 *   groups            : connected components of the friendship graph
 * label[k] receives the smallest index of candidate k's group. Plain O(n^2) union of pairs.
 * Returns the number of groups.
 */
int64_t or_fof(const or_cand_t* c, int64_t n, const double* dm_start, const double* dm_step,
               double dm_link, int64_t t_link, int64_t* label) {
  for (int64_t k = 0; k < n; ++k) label[k] = k;
  /* repeated relaxation: every pair of friends takes the smaller label, until nothing moves */
  int changed = 1;
  while (changed) {
    changed = 0;
    for (int64_t a = 0; a < n; ++a) {
      const double dma = dm_start[c[a].range] + (double)c[a].trial * dm_step[c[a].range];
      for (int64_t b = a + 1; b < n; ++b) {
        const double dmb = dm_start[c[b].range] + (double)c[b].trial * dm_step[c[b].range];
        if (fabs(dma - dmb) > dm_link) continue;
        if (c[a].t_start > c[b].t_start + c[b].width - 1 + t_link) continue;
        if (c[b].t_start > c[a].t_start + c[a].width - 1 + t_link) continue;
        if (label[a] != label[b]) {
          const int64_t m = label[a] < label[b] ? label[a] : label[b];
          label[a] = label[b] = m;
          changed = 1;
        }
      }
    }
  }
  int64_t groups = 0;
  for (int64_t k = 0; k < n; ++k) groups += label[k] == k;
  return groups;
}
