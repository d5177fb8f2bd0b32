/*
 * dd.h -- C ABI of the GB300 (sm_103a) dedispersion + single-pulse-search library.
 *
 * The operations follow the problem statement of Novotny, Adamek & Armour,
 * "Implementing CUDA Streams into AstroAccelerate -- A Case Study":
 *   - Sec. 1 (time chunking over CUDA streams) and Sec. 2 (pinned memory, asynchronous copies,
 *     stream IDs, no implicit synchronisation in the compute loop);
 *   - Sec. 2.1 (the dedispersion phase, streamed);
 *   - Sec. 2.2 (the single-pulse-search phase; all allocation moved to the planning phase);
 *   - Sec. 3 (the DM-trial plan: ~6000 trials over 0-3000 pc cm^-3, SKA-like input).
 * The paper prints no formulas. The readings used here:
 *   delay      s[i][c] = floor(k_DM*DM_i*(f_c^-2 - f_ref^-2) / (tsamp*d) + 0.5),
 *              k_DM = 4.148808e3 s MHz^2 pc^-1 cm^3, f_ref = max f_c, DM_i = dm_start + i*dm_step
 *   decimation x_d[c][m] = sum_{k<d} x[c][m*d + k]   (windows aligned at global sample 0)
 *   dedisp.    y[i][j]  = sum_c x_d[c][j + s[i][c]]   (exact integer sum, int32)
 *   search     trailing boxcars B_w[j] (w decimated samples), SNR = (n*B - w*S1) /
 *              (sqrt(w)*sqrt(n*S2 - S1^2)) over the chunk window's own moments, one candidate
 *              per aligned block of `peak_block` samples (max over samples and widths; ties go to
 *              the earlier sample, then the narrower width) when SNR >= threshold.
 *
 * Conventions
 *   - Every function returns DD_OK (0) or a negative DD_ERR_* code; dd_last_error() gives a
 *     message for the calling thread's last failure.
 *   - All device and pinned host memory is allocated in dd_plan (Sec. 2.2: allocation moved out of
 *     the compute phase) and released by dd_plan_destroy. dd_run / sps_run / dd_candidates
 *     allocate nothing.
 *   - A plan is used from one host thread at a time.
 *   - Layouts: filterbank chunks are time-major uint8, x[t][c] (row = one spectrum of nchans
 *     bytes, channel 0 first). Series are int32 [trial][sample] of one range.
 */
#ifndef DD_H
#define DD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DD_OK 0
#define DD_ERR_ARG (-1)     /* invalid argument or plan parameter */
#define DD_ERR_NOMEM (-2)   /* device or pinned host allocation failed in dd_plan */
#define DD_ERR_CUDA (-3)    /* a CUDA runtime call or kernel failed */
#define DD_ERR_TIMEOUT (-4) /* a bounded wait for the GPU ran out */
#define DD_ERR_CAP (-5)     /* more candidates than the buffer holds; *ncands = the true count */
#define DD_ERR_STATE (-6)   /* call out of order (e.g. candidates of a chunk already recycled) */

/* Plan option flags. */
#define DD_FLAG_TIMING 1u   /* bracket every dedispersion launch with CUDA events (dd_stats) */
#define DD_FLAG_NAIVE 2u    /* use the one-thread-per-output dedispersion kernel (testing aid) */
#define DD_FLAG_DEVICE_INPUT 4u /* chunks are always in device memory: no staging buffer is
                                   allocated and host chunks are refused (DD_ERR_ARG) */
#define DD_FLAG_TILE256 8u  /* plan the tiled kernel with 256-sample time tiles only (testing
                               aid; 512-sample tiles are tried first otherwise) */
#define DD_FLAG_TRIALS32 16u /* plan the tiled kernel with 32-trial tiles only (testing aid;
                                64-trial tiles are tried first otherwise) */
#define DD_FLAG_AUTOTUNE 32u /* dd_plan times every tile shape that fits each range (trials x
                                outputs x threads: 64 x 512 x 512, 64 x 512 x 1024, 64 x 256 x
                                512, 32 x 256 x 512) on the plan's own buffers and keeps the
                                fastest (adds a few launches per range to planning) */
#define DD_FLAG_WARPS32 64u /* plan the tiled kernel with 1024-thread CTAs only (testing aid) */

typedef struct dd_plan_s* dd_plan_t;

/* One DM range of the trial plan (Sec. 3): trials dm_start + i*dm_step, i < n_trials, searched
 * on data decimated by `decimation` (a power of two, 1..256). */
typedef struct {
  double dm_start;
  double dm_step;
  int32_t n_trials;
  int32_t decimation;
} dd_range_t;

typedef struct {
  int64_t chunk_len;   /* most new samples one dd_run call may deliver (Sec. 1: a time chunk);
                          a multiple of 256, at most 65535 * 256 = 16776960 */
  int32_t n_streams;   /* CUDA streams the chunks rotate over (Sec. 2: stream IDs), 1..16 */
  int32_t max_width;   /* largest boxcar width (original samples) sps_run will be given */
  int32_t peak_block;  /* samples per candidate block (decimated samples of each range), >= 1 */
  int32_t device;      /* CUDA device ordinal */
  int64_t max_cands;   /* device candidate buffer per chunk; 0 = default (1<<20) */
  uint32_t flags;      /* DD_FLAG_* */
  int32_t staging_threads; /* > 0: chunks in pageable host memory are first copied into a small
                              pinned buffer per stream by this many host threads, then sent
                              asynchronously (Sec. 2.1: pinned staging buffers filled by CPU
                              threads); 0: the CUDA driver copies pageable chunks itself */
} dd_opts_t;

/* One single-pulse candidate (Sec. 2.2). */
typedef struct {
  int32_t trial;   /* trial index within its range */
  int32_t range;   /* range index in the plan */
  int64_t t_start; /* first original sample of the boxcar, counted from the first sample ever
                      given to dd_run */
  int32_t width;   /* boxcar width in original samples */
  int32_t pad;
  double snr;      /* FP64 SNR */
} dd_cand_t;

/*
 * dd_plan -- build a plan (Sec. 1 "mapping of tasks ... allocation of all necessary memory";
 * Sec. 3 DM plan).
 *   freqs_mhz : host [nchans] channel-centre frequencies in MHz (any order; f_ref = the largest)
 *   tsamp_s   : sample time in seconds (> 0)
 *   ranges    : host [nranges] DM ranges; n_trials >= 1; decimation a power of two <= 256
 *   opts      : host, see dd_opts_t
 *   out       : receives the plan handle (owned by the caller, release with dd_plan_destroy)
 * Builds the delay table on the GPU, derives the overlap O (original samples of history every
 * chunk needs: the largest delay of any range, rounded up to the largest decimation), creates
 * n_streams CUDA streams and allocates every device and pinned buffer used later.
 * Errors: DD_ERR_ARG (bad sizes, nchans*255*max(width, decimation) >= 2^31, delays beyond
 * int32), DD_ERR_NOMEM, DD_ERR_CUDA.
 */
int dd_plan(const double* freqs_mhz, int32_t nchans, double tsamp_s, const dd_range_t* ranges,
            int32_t nranges, const dd_opts_t* opts, dd_plan_t* out);

/*
 * dd_plan_info -- plan facts.
 *   overlap  : O in original samples (may be NULL)
 *   ntrials  : total trials over all ranges (may be NULL)
 *   shifts   : receives a plan-owned HOST pointer to the delay table, int32
 *              [sum_r n_trials_r][nchans], ranges in plan order, valid until dd_plan_destroy
 *              (may be NULL)
 */
int dd_plan_info(dd_plan_t plan, int64_t* overlap, int32_t* ntrials, const int32_t** shifts);

/*
 * dd_plan_kernel -- which dedispersion kernel range `range` (0-based, plan order) runs on.
 *   kind         : DD_KERNEL_TILED (delay classes shared by a trial tile), DD_KERNEL_DIRECT
 *                  (the fallback where the range's delay classes or decimation exceed the tiled
 *                  kernel's limits: coarse channels, decimation above x16) or
 *                  DD_KERNEL_PER_OUTPUT (one thread per output, with DD_FLAG_NAIVE) (may be NULL)
 *   tile_samples : outputs per time tile of the tiled kernel, 0 for the others (may be NULL)
 * Errors: DD_ERR_ARG (NULL plan, range out of bounds).
 */
#define DD_KERNEL_TILED 1
#define DD_KERNEL_DIRECT 2
#define DD_KERNEL_PER_OUTPUT 3
int dd_plan_kernel(dd_plan_t plan, int32_t range, int32_t* kind, int32_t* tile_samples);

/*
 * dd_plan_model -- the work of one dedispersion launch of range `range` over a window of `nout`
 * outputs, counted on the host (no GPU work); it is what roofline fractions divide by.
 *   kind, tile_samples : as dd_plan_kernel
 *   tile_trials        : trials per tile of the tiled kernel (64 or 32), else 0
 *   cta_threads        : threads per CTA of the tiled kernel (512 or 1024), else 0
 *   ctas_per_sm        : CTAs of the tiled kernel's tile shape per SM (1 or 2), else 0
 *   outputs            : DM-trial*samples, n_trials * nout
 *   adds               : algorithmic channel-adds of the brute-force sum (Sec. 2.1), outputs*nchans
 *   fused              : 1 when the range's search is fused into the kernel (dd_fuse_search)
 *   dram_bytes         : algorithmic DRAM bytes: each channel's window of decimated input
 *                        (nout + the range's largest delay samples) read once, the int32 series
 *                        written once (fused: a 4-byte sum and a 1-byte sample per trial, width
 *                        and peak block instead, plus the series if they are kept)
 *   smem_wavefronts    : tiled kernel only (else 0): warp-wide shared-memory accesses the launch
 *                        issues (one wavefront each: the kernel's accesses have no bank
 *                        conflicts), counted from the plan-time tables
 *   copy_bytes         : tiled kernel only: bytes its tensor and bulk copies write into shared
 *                        memory
 * Errors: DD_ERR_ARG.
 */
typedef struct {
  int32_t kind;
  int32_t tile_samples;
  int32_t tile_trials;
  int32_t cta_threads;
  int32_t ctas_per_sm;
  int32_t fused;
  int64_t outputs;
  double adds;
  double dram_bytes;
  double smem_wavefronts;
  double copy_bytes;
} dd_launch_model_t;
int dd_plan_model(dd_plan_t plan, int32_t range, int64_t nout, dd_launch_model_t* out);

/*
 * dd_run -- enqueue the dedispersion of the next time chunk (Sec. 1, Sec. 2.1).
 *   chunk       : time-major uint8 [nsamp][nchans]; a host pointer (pinned memory gives
 *                 asynchronous copies, Sec. 2.1) or a device pointer. Read-only; it must stay
 *                 valid and unchanged until this chunk's dd_candidates returns or dd_sync.
 *                 With opts.staging_threads > 0 a pageable chunk is copied into the slot's
 *                 pinned staging buffer before dd_run returns (the host copy of the next chunk
 *                 overlaps the GPU work of this one) and may be reused as soon as it returns.
 *   nsamp       : new samples, 0 < nsamp <= chunk_len, a multiple of the largest decimation
 *   cuda_stream : NULL = the plan's own streams (chunk k runs on stream k mod n_streams);
 *                 otherwise every stage of this chunk is enqueued on that cudaStream_t.
 * The plan keeps O samples of history on the device, so consecutive chunks dedisperse exactly
 * like one long input. After the chunk, the outputs of range r are the global decimated indices
 * j with j*d_r in [max(0, T-O), max(0, T+nsamp-O)), T = samples delivered before this chunk.
 * Returns immediately (asynchronous). The chunk is numbered 0, 1, 2, ... in call order;
 * its results stay available until n_streams further chunks have been run.
 * Errors: DD_ERR_ARG, DD_ERR_CUDA.
 */
int dd_run(dd_plan_t plan, const uint8_t* chunk, int64_t nsamp, void* cuda_stream);

/*
 * dd_series -- device view of the most recent chunk's dedispersed series of one range.
 *   dev_ptr : receives a plan-owned DEVICE pointer to int32 [n_trials_r][stride]
 *   len     : samples of the chunk window (row j = global decimated index *j0 + j)
 *   stride  : row stride in elements;  j0 : global decimated index of sample 0 (may be NULL)
 * The data is complete once the chunk's stream has finished (dd_sync or dd_candidates).
 * Errors: DD_ERR_ARG, DD_ERR_STATE (no chunk has been run, or the range's search is fused and
 * its series are not kept: dd_fuse_search).
 */
int dd_series(dd_plan_t plan, int32_t range, const int32_t** dev_ptr, int64_t* len,
              int64_t* stride, int64_t* j0);

/* Exact moments of one dedispersed series over its chunk window (Sec. 2.2: the statistics that
 * normalise the single pulse search): s1 = sum y, s2 = sum y^2 as an unsigned 128-bit value
 * (s2hi * 2^64 + s2lo). 32 bytes per record. */
typedef struct {
  int64_t s1;
  uint64_t s2lo;
  uint64_t s2hi;
  uint64_t pad;
} dd_moments_t;

/*
 * dd_moments -- device view of the most recent chunk's moments of one range (Sec. 2.2).
 *   dev_ptr : receives a plan-owned DEVICE pointer to dd_moments_t [n_trials_r], trial order
 *   n       : samples of the chunk window the moments cover (0: an empty window, for which the
 *             records are not written and must not be read)
 * The moments are accumulated by the dedispersion kernels with exact integer arithmetic and are
 * complete once the chunk's stream has finished (dd_sync or dd_candidates); they stay valid
 * until the chunk's slot is reused n_streams chunks later.
 * Errors: DD_ERR_ARG (NULL plan, bad range), DD_ERR_STATE (no chunk has been run).
 */
int dd_moments(dd_plan_t plan, int32_t range, const dd_moments_t** dev_ptr, int64_t* n);

/*
 * dd_fuse_search -- fuse the search's position pass into the dedispersion kernel (Sec. 2.1 sums
 * followed by the Sec. 2.2 boxcars), so that the int32 series need not be written to HBM and
 * read back. From the plan's first dd_run on, every range whose widths (those of `widths` that
 * are multiples of its decimation d, divided by d) are all <= 512 and whose kernel is the tiled
 * one is dedispersed by the fused form (re-planned on the 64-trial x 512-sample tile if the plan
 * chose another shape): after each tile, per (trial, width, peak block) the block's largest
 * boxcar sum and its earliest sample are recorded, boxcars reaching into the previous tile
 * included. sps_run then turns the records into candidates with the window moments; they are
 * the candidates the plain search finds (same statistics, evaluation order and tie rules).
 *   widths, nwidths : the search's widths (original samples), as sps_run; every later sps_run
 *                     on the plan must pass exactly these
 *   fuse_flags      : 0 or DD_FUSE_KEEP_SERIES (fused ranges also write their series, for
 *                     dd_series and the clipped estimator)
 *   nfused          : receives the number of fused ranges (may be NULL); ranges not fused keep
 *                     the plain path
 * Call once, after dd_plan and before the first dd_run. It allocates the record buffers (per
 * stream slot: 5 bytes per trial, width and peak block, plus the segment edges) and, without
 * DD_FUSE_KEEP_SERIES, gives up the fused ranges' series buffers: dd_series on such a range
 * returns DD_ERR_STATE, as does sps_run_ex with DD_EST_CLIPPED.
 * Errors: DD_ERR_ARG (widths, flags), DD_ERR_STATE (a chunk was run, or called twice),
 * DD_ERR_NOMEM, DD_ERR_CUDA; on an error the plan is unchanged.
 */
#define DD_FUSE_KEEP_SERIES 1u
int dd_fuse_search(dd_plan_t plan, const int32_t* widths, int32_t nwidths, uint32_t fuse_flags,
                   int32_t* nfused);

/*
 * sps_run -- enqueue the single pulse search of the most recent chunk (Sec. 2.2).
 *   widths    : host [nwidths] boxcar widths in original samples, strictly increasing,
 *               1 <= w <= max_width. Range r searches the widths w with w >= d_r and
 *               w % d_r == 0, as w/d_r decimated samples.
 *   threshold : candidates have SNR >= threshold
 * Enqueued on the chunk's own stream after its dedispersion (stream-ordered; no cross-stream
 * wait on atomics). Asynchronous; collect the result with dd_candidates. On a plan whose search
 * is fused (dd_fuse_search) the widths must be the fused ones, and the fused ranges' candidates
 * come from the block records of the dedispersion kernel.
 * Errors: DD_ERR_ARG (also: other widths than a fused plan's), DD_ERR_STATE (no chunk, or
 * already searched), DD_ERR_CUDA.
 */
int sps_run(dd_plan_t plan, const int32_t* widths, int32_t nwidths, float threshold);

/*
 * sps_run_ex -- sps_run with a choice of noise statistic (Sec. 2.2 names the SPDT estimators of
 * the search without defining them; both choices here are readings).
 *   how->estimator  : DD_EST_WINDOW: the chunk window's mean and deviation of the series, with
 *                     sqrt(w) scaling (sps_run; how may be NULL for it);
 *                     DD_EST_CLIPPED: per boxcar width, the mean and population deviation of the
 *                     boxcar sums B_w themselves, made robust by clip_iters steps of
 *                     kappa-sigma clipping: each step keeps the sums within
 *                     ceil(mu - kappa*sd) .. floor(mu + kappa*sd) of the previous step's (FP64
 *                     mu = T1/N, sd = sqrt(N*T2 - T1^2)/N from exact integer sums). The SNR is
 *                     (N*B - T1) / sqrt(N*T2 - T1^2); a width with no variance left gives none.
 *   how->clip_iters : 0 .. 16 clipping steps;  how->clip_kappa : the bound in deviations (> 0)
 * Errors: those of sps_run; DD_ERR_ARG for an unknown estimator or bad clipping parameters.
 */
#define DD_EST_WINDOW 0
#define DD_EST_CLIPPED 1
typedef struct {
  int32_t estimator;
  int32_t clip_iters;
  double clip_kappa;
} dd_sps_opts_t;
int sps_run_ex(dd_plan_t plan, const int32_t* widths, int32_t nwidths, float threshold,
               const dd_sps_opts_t* how);

/*
 * dd_candidates -- wait for chunk `seq`'s search and copy its candidates.
 *   seq    : chunk number (0-based dd_run call count); must be one of the last n_streams chunks
 *   out    : caller-owned host array of cap entries, sorted by (range, trial, t_start, width)
 *   ncands : receives the number of candidates found
 *   timeout_ms : bound on the wait (<= 0: 600000)
 * Errors: DD_ERR_STATE (unknown, recycled or unsearched chunk), DD_ERR_TIMEOUT (the wait ran
 * out, or a dedispersion kernel of this chunk ran out of its bounded device-side wait, so the
 * chunk's results are not valid; later chunks are not affected), DD_ERR_CAP (more than cap or
 * than opts.max_cands; *ncands holds the true count, out holds the first cap in sorted order of
 * those kept; when more than opts.max_cands were found, which ones the device buffer kept
 * depends on the order the search's blocks ran in, so only the count is reproducible),
 * DD_ERR_CUDA.
 */
int dd_candidates(dd_plan_t plan, int64_t seq, dd_cand_t* out, int64_t cap, int64_t* ncands,
                  int64_t timeout_ms);

/* dd_sync -- wait for all enqueued work of the plan. Errors: DD_ERR_CUDA. */
int dd_sync(dd_plan_t plan);

/*
 * dd_stats -- counters of the plan since creation or the last reset.
 *   launches      : kernels launched by the plan
 *   dedisp_ms     : device time during which at least one dedispersion launch was running (the
 *                   union of the launches' intervals, so launches of chunks that overlap on
 *                   different streams count once); needs DD_FLAG_TIMING; measured with CUDA
 *                   events on each launching stream; complete after dd_sync
 *   dedisp_launches : dedispersion launches timed
 *   reset         : non-zero = zero the counters after reading
 */
int dd_stats(dd_plan_t plan, int64_t* launches, double* dedisp_ms, int64_t* dedisp_launches,
             int32_t reset);

/*
 * dd_stats_range -- the dedispersion timing of dd_stats restricted to the launches of one range:
 * the union of their intervals (ms) and their number, since creation or the last reset of
 * dd_stats. Needs DD_FLAG_TIMING; complete after dd_sync. Errors: DD_ERR_ARG, DD_ERR_CUDA.
 */
int dd_stats_range(dd_plan_t plan, int32_t range, double* dedisp_ms, int64_t* dedisp_launches);

/*
 * dd_sps_static -- the single pulse search of dd_candidates, on caller-provided device series,
 * with no memory allocated by the library. The paper has no counterpart: this entry point exists
 * for callers that cannot let a library allocate device memory at run time -- a real-time
 * pipeline that reserves its whole GPU memory budget at start-up and must never take the
 * implicit synchronisation of cudaMalloc/cudaFree in its processing loop, or a plug-in whose
 * host framework owns every device allocation.
 *   series     : DEVICE int32 [n_trials][stride], window samples 0..n-1 of one range
 *                (e.g. from dd_series); read-only
 *   n_trials   : 1 .. 16384 (the capacity of the fixed scratch; larger counts are rejected)
 *   range, decimation, j0 : copied into the candidates (range index, d_r, global decimated
 *                index of window sample 0), exactly as the plan's search reports them
 *   widths, nwidths, threshold, peak_block : as in sps_run / dd_opts_t (widths on the HOST)
 *   cands      : DEVICE dd_cand_t [cap], caller-owned; filled in no particular order
 *   count      : DEVICE unsigned long long, caller-owned; set to the number of candidates
 *                found (entries beyond cap are counted but not written)
 *   cuda_stream: cudaStream_t the work is enqueued on (NULL = the default stream); returns
 *                without waiting
 * Scratch: per-trial moments in a fixed device array of 16384 records (512 KB), which every GPU
 * that loads the library holds until the process exits. The first call in each CUDA context
 * looks up that array's device address (cudaGetSymbolAddress) with the device current and keeps
 * it for that context, so make the first call on each device (and again after a context has
 * been destroyed and re-created, e.g. by cudaDeviceReset) before any stream capture. Every call
 * shares the array and leaves its contents behind: calls whose work may overlap on the GPU
 * (different streams, or several host threads) race on it and must be serialised by the
 * caller. The count is cleared by the call; the moments are recomputed in full.
 * Errors (dd_last_error explains): DD_ERR_ARG (NULL pointer, sizes outside the limits above,
 * bad widths, a threshold that is not finite), DD_ERR_CUDA (no device or a failed launch).
 */
int dd_sps_static(const int32_t* series, int32_t n_trials, int64_t n, int64_t stride,
                  int32_t range, int32_t decimation, int64_t j0, const int32_t* widths,
                  int32_t nwidths, float threshold, int32_t peak_block, dd_cand_t* cands,
                  int64_t cap, unsigned long long* count, void* cuda_stream);

/*
 * dd_group_candidates -- friends-of-friends grouping of candidates (Sec. 2.2: one pulse is
 * reported at neighbouring DM trials, times and widths; reading: a single-pulse search's
 * candidate clustering). Host only, no GPU work.
 *   cands, n   : host candidates, e.g. one chunk's from dd_candidates (sorted as it returns
 *                them; any order works, indices refer to this order)
 *   ranges     : host [nranges] the plan's DM ranges (the DM of a candidate is
 *                dm_start + trial * dm_step of its range)
 *   dm_link    : candidates whose DMs differ by at most this much (pc cm^-3) ...
 *   t_link     : ... and whose boxcars [t_start, t_start + width) overlap or leave at most
 *                t_link original samples between the earlier one's last sample and the later
 *                one's first, are friends; groups are the connected components of friendship
 *   out, cap   : host dd_group_t [cap]: one record per group in order of its smallest index:
 *                rep (index of the member with the largest SNR; ties to the smaller index),
 *                members, the DM extent and the first and last original sample of its boxcars
 *   ngroups    : receives the number of groups
 *   label      : host int64 [n] or NULL: receives each candidate's group as the smallest index
 *                of its members
 * Errors: DD_ERR_ARG (bad sizes, a candidate's range or width, non-finite or negative links),
 * DD_ERR_CAP (more groups than cap; *ngroups holds the true count).
 */
typedef struct {
  int64_t rep;
  int64_t members;
  double dm_lo;
  double dm_hi;
  int64_t t_lo;
  int64_t t_hi;
} dd_group_t;
int dd_group_candidates(const dd_cand_t* cands, int64_t n, const dd_range_t* ranges,
                        int32_t nranges, double dm_link, int64_t t_link, dd_group_t* out,
                        int64_t cap, int64_t* ngroups, int64_t* label);

/* dd_plan_destroy -- wait for the plan's work and free everything it allocated. NULL is a no-op. */
void dd_plan_destroy(dd_plan_t plan);

/* ---------------------------------------------------------------- serving
 * Many beams, each with a plan of its own, whose chunks arrive at arbitrary times (Sec. 1: work
 * split over CUDA streams, applied across beams; Sec. 2.2: every buffer allocated when a beam is
 * planned). A dispatcher thread owned by the server makes every plan call: a submitted chunk
 * waits in its beam's queue and is started, oldest first across beams, as soon as fewer chunks
 * are on the GPU than the admission limit and its beam has a free stream slot (at most
 * n_streams chunks of one beam in flight); chunks of different beams then run concurrently,
 * each beam on its own streams, and a chunk gives the same candidates as it would with its
 * beam alone. Admission limit: with at most two requests waiting, two chunks may be on the GPU
 * and the newer one's dedispersion is ordered after the older one's search (its copy, corner
 * turn and decimation overlap it), so that chunks finish in arrival order close to their own
 * service time; with a longer backlog, as many chunks as are waiting (at most max_inflight) run
 * unordered, so that their launches fill each other's gaps. */
typedef struct dd_server_s* dd_server_t;

typedef struct {
  int64_t ticket;    /* from dd_serve_submit */
  int32_t beam;
  int32_t status;    /* DD_OK or the error of dd_run / sps_run / dd_candidates */
  int64_t seq;       /* chunk number within its beam */
  int64_t ncands;    /* candidates found (those beyond cap are counted, not copied) */
  double queue_ms;   /* submission -> start on the GPU */
  double latency_ms; /* submission -> candidates in the caller's buffer */
} dd_serve_result_t;

/* dd_serve_create -- start a server on `device` that keeps at most max_inflight chunks on the
 * GPU (the cap of the admission limit above) and accepts beams whose plans fit hbm_budget_bytes of device memory in total.
 * Errors: DD_ERR_ARG. */
int dd_serve_create(int32_t max_inflight, int64_t hbm_budget_bytes, int32_t device,
                    dd_server_t* out);

/* dd_serve_add_beam -- plan a beam (arguments as in dd_plan; opts->device is ignored, the
 * server's device is used) and its search (widths, threshold as in sps_run, checked here so
 * that a chunk's search cannot be refused after its dedispersion was enqueued). *beam receives
 * its index. Errors: those of dd_plan; DD_ERR_ARG for widths outside 1..opts->max_width, not
 * strictly increasing or more than 16 of them, or a threshold that is not finite;
 * DD_ERR_NOMEM when the plan would exceed the HBM budget (the plan is released again).
 * Should enqueueing a chunk of a beam still fail (a CUDA error), the beam's plan is drained and
 * the beam is marked failed: that chunk, its chunks then on the GPU and every later chunk of
 * the beam are reported with the error as their status. */
int dd_serve_add_beam(dd_server_t server, const double* freqs_mhz, int32_t nchans,
                      double tsamp_s, const dd_range_t* ranges, int32_t nranges,
                      const dd_opts_t* opts, const int32_t* widths, int32_t nwidths,
                      float threshold, int32_t* beam);

/* dd_serve_submit -- queue the next chunk of a beam (as dd_run: time-major uint8
 * [nsamp][nchans], host or device memory, caller-owned and unchanged until its result is
 * polled). The chunk's candidates are copied to out (host, cap entries, sorted as by
 * dd_candidates) before its result is reported. Returns without waiting for the GPU (the
 * dispatcher holds the server's lock only to move requests between queues, never across a copy,
 * a launch or a sort); the submission time, from which queue_ms and latency_ms are measured, is
 * taken on entry. Errors: DD_ERR_ARG. */
int dd_serve_submit(dd_server_t server, int32_t beam, const uint8_t* chunk, int64_t nsamp,
                    dd_cand_t* out, int64_t cap, int64_t* ticket);

/* dd_serve_poll -- take up to max finished results (oldest first), waiting up to timeout_ms
 * for the first when none is ready (0: do not wait). *n receives the number taken. */
int dd_serve_poll(dd_server_t server, dd_serve_result_t* out, int32_t max, int32_t* n,
                  int64_t timeout_ms);

/* ---------------------------------------------------------------- batches
 * Many beams of uneven length and channel count processed in one step, each from its first
 * sample: chunks are enqueued round-robin over the beams (each beam with a plan of its own and
 * its own streams), so the beams' work overlaps on the device; every (beam, chunk) keeps its own
 * candidates. DD_BATCH_GRAPH captures the step once as a CUDA graph that every dd_batch_run
 * replays (the inputs stay at their device addresses; refill them between steps).
 * DD_BATCH_AUTOTUNE picks the tile shape of every plan's ranges by timing the candidates.
 * DD_BATCH_PERSISTENT runs the step in rounds on one stream instead: round c takes chunk c of
 * every beam that has one (copies, corner turns, decimations), then ONE persistent dedispersion
 * launch per kernel instance (uint8 / uint16 data) whose CTAs, one per SM, take (beam, range,
 * trial tile, time tile) items from a device work list until it is empty, then the searches. */
#define DD_BATCH_GRAPH 1u
#define DD_BATCH_AUTOTUNE 2u
#define DD_BATCH_PERSISTENT 4u

typedef struct dd_batch_s* dd_batch_t;

typedef struct {
  const double* freqs_mhz; /* host [nchans] */
  int32_t nchans;
  int32_t pad;
  double tsamp_s;
  int64_t nsamp;           /* samples of the beam, a multiple of the largest decimation */
  const uint8_t* input;    /* DEVICE time-major [nsamp][nchans], caller-owned */
} dd_batch_beam_t;

/* dd_batch_create -- plan every beam (ranges and opts shared; opts->chunk_len is the chunk
 * length; DD_FLAG_TIMING is refused), allocate cap_per_chunk candidates for every (beam, chunk)
 * and, with DD_BATCH_GRAPH, capture one step. Errors: those of dd_plan, DD_ERR_ARG,
 * DD_ERR_NOMEM, DD_ERR_CUDA. */
int dd_batch_create(int32_t nbeams, const dd_batch_beam_t* beams, const dd_range_t* ranges,
                    int32_t nranges, const dd_opts_t* opts, const int32_t* widths,
                    int32_t nwidths, float threshold, int64_t cap_per_chunk, uint32_t flags,
                    dd_batch_t* out);

/* dd_batch_run -- enqueue one step (asynchronous); dd_batch_wait waits for it (bounded).
 * dd_batch_wait errors: DD_ERR_TIMEOUT when the step does not finish within timeout_ms (<= 0:
 * 600000), and also when a dedispersion kernel of the step ran out of its bounded device-side
 * wait (the step's candidates are then not valid and dd_batch_candidates refuses them until a
 * later step succeeds), DD_ERR_CUDA. */
int dd_batch_run(dd_batch_t batch);
int dd_batch_wait(dd_batch_t batch, int64_t timeout_ms);

/* dd_batch_info -- chunks of a beam, its DM-trial*samples per step, and the time tile chosen
 * for its first range (0: the simple kernel). */
int dd_batch_info(dd_batch_t batch, int32_t beam, int64_t* nchunks, int64_t* outputs,
                  int32_t* tile_samples);

/* dd_batch_candidates -- after dd_batch_wait: the candidates of one (beam, chunk), sorted as by
 * dd_candidates. Errors: DD_ERR_ARG, DD_ERR_STATE (no finished step), DD_ERR_CAP. */
int dd_batch_candidates(dd_batch_t batch, int32_t beam, int64_t chunk, dd_cand_t* out,
                        int64_t cap, int64_t* ncands);

/* dd_batch_destroy -- wait and release everything. NULL is a no-op. */
void dd_batch_destroy(dd_batch_t batch);

/* dd_serve_pending -- chunks queued but not started, and chunks on the GPU. */
int dd_serve_pending(dd_server_t server, int64_t* queued, int32_t* inflight);

/* dd_serve_destroy -- stop the dispatcher (queued chunks are dropped, chunks on the GPU
 * finish) and release every beam's plan. NULL is a no-op. */
void dd_serve_destroy(dd_server_t server);

/*
 * dd_tiled_plan_check -- host-only check of the tiled kernel's plan for one range (no GPU, no
 * CUDA call). Builds the plan-time tables the tiled kernel would use from a delay table and
 * verifies them against it: each trial's pair words lie in one plane (even or odd words) of its
 * delay class and stand for class words that add, in every channel, the sample at that trial's
 * own delay; class word ranges are aligned; every read stays inside the staged rows; the build
 * work lists cover every block of every class once.
 *   shifts       : int32 [n_trials][cpad], delays of one range in decimated samples, channels
 *                  padded to cpad (a multiple of 8) by repeating the last channel
 *   tile_samples : 512 or 256 (outputs per time tile)
 *   tile_trials  : 64 or 32 (trials per tile)
 *   ok           : receives 1 if the tiled kernel can run the range, else 0
 *   violations   : receives the number of violated checks (0 expected; 0 when ok is 0)
 * Errors: DD_ERR_ARG.
 */
int dd_tiled_plan_check(const int32_t* shifts, int32_t n_trials, int32_t cpad,
                        int32_t decimation, int32_t tile_samples, int32_t tile_trials,
                        int32_t* ok, int64_t* violations);

/*
 * dd_selftest_wait -- failure-detection self-test of the device-side bounded wait. The tiled
 * dedispersion kernel waits on each stage's copy barrier for at most 2 s (or 2^26 polls); when
 * that runs out it sets an error bit that dd_candidates reports as DD_ERR_TIMEOUT, waits (again
 * bounded) for its copies in flight and returns, so the CUDA context stays usable. This call
 * runs the same wait in one thread on a barrier that nothing completes, on its own stream, and
 * reports the outcome. It allocates 4 bytes of device memory for the duration of the call.
 *   device    : CUDA device to run on
 *   timed_out : receives 1 if the wait ran out and was reported (the designed outcome), else 0
 *   waited_ms : receives the call's host-measured duration (may be NULL)
 * Errors: DD_ERR_ARG (NULL timed_out), DD_ERR_NOMEM, DD_ERR_CUDA.
 */
int dd_selftest_wait(int32_t device, int32_t* timed_out, double* waited_ms);

/*
 * dd_measure_peaks -- measure, on `device`, the issue rates that bound the dedispersion kernels
 * (the denominators of their roofline; not part of the paper's method). Two CTAs of 16 warps per
 * SM run independent dependency chains of one instruction kind; rates are per SM and per SM
 * clock, averaged over the SMs:
 *   alu_lanes_per_clk      : LOP3 lane-instructions (the integer ALU pipe)
 *   dp_lanes_per_clk       : DP2A lane-instructions (the integer dot-product pipe)
 *   int_lanes_per_clk      : LOP3 and DP2A interleaved: integer lane-instructions of both pipes
 *   add_per_clk            : 32-bit additions of plain add chains
 *   lds_wavefronts_per_clk : warp-wide 32-bit shared-memory loads of 32 consecutive words (one
 *                            128-byte wavefront each)
 *   sm_mhz                 : the SM clock during the runs (cycles over nanoseconds)
 *   sms                    : multiprocessors
 * Takes a few milliseconds; allocates a few bytes of device memory for the duration of the call.
 * Errors: DD_ERR_ARG (NULL out, no such device), DD_ERR_NOMEM, DD_ERR_CUDA.
 */
typedef struct {
  int32_t sms;
  int32_t pad;
  double sm_mhz;
  double alu_lanes_per_clk;
  double dp_lanes_per_clk;
  double int_lanes_per_clk;
  double add_per_clk;
  double lds_wavefronts_per_clk;
} dd_peaks_t;
int dd_measure_peaks(int32_t device, dd_peaks_t* out);

/* dd_last_error -- message of the calling thread's last error ("" if none). Library-owned. */
const char* dd_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* DD_H */
