// Internal declarations shared by the library's translation units (not part of the C ABI).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "dd.h"

namespace ddk {

constexpr int kMaxRanges = 64;
constexpr int kMaxWidths = 16;

// Exact moments of one (range, trial) series over a chunk window: S1 = sum y, S2 = sum y^2 as a
// 128-bit value (s2lo, s2hi). 32 bytes so one trial's record is one sector.
struct Moments {
  unsigned long long s1, s2lo, s2hi, pad;
};
static_assert(sizeof(Moments) == sizeof(dd_moments_t), "dd_moments views the device records");

// Clipped statistics of one (trial, width) boxcar series: N values, T1 = their sum, T2 = the sum
// of their squares as 128 bits (t2lo, t2hi). 32 bytes.
struct WidthStats {
  long long n, t1;
  unsigned long long t2lo, t2hi;
};

// One launch of the clipped-statistics kernel: every trial of one range of one chunk.
struct ClipArgs {
  const int32_t* y;        // [n_trials][stride]
  int64_t stride;
  int64_t n;               // window length
  int32_t n_trials;
  int32_t nw;
  int32_t wd[kMaxWidths];  // decimated widths, increasing
  int32_t hist;            // largest decimated width - 1, rounded up to 256
  int32_t iters;           // clipping steps
  double kappa;            // clipping bound in deviations
  WidthStats* out;         // [n_trials][nw]
};

// Per-range parameters of the delay-table kernel.
struct ShiftRange {
  double dm_start, dm_step;
  int32_t n_trials, decimation, row0, pad;
};

// One launch of the search kernel handles one range of one chunk.
struct SpsArgs {
  const int32_t* y;        // [n_trials][stride]
  int64_t stride;
  int64_t n;               // window length
  const Moments* mom;      // [n_trials]
  int32_t n_trials;
  int32_t range;
  int32_t d;
  int32_t block;           // samples per candidate block (power of two <= 32)
  int64_t J0;              // global decimated index of window sample 0
  int32_t nw;
  int32_t hist;            // largest decimated width - 1, rounded up to 256
  int32_t wd[kMaxWidths];  // decimated widths, increasing
  float threshold;
  int32_t pad;
  dd_cand_t* cands;
  unsigned long long* count;
  int64_t cap;
  const WidthStats* wst;   // [n_trials][nw] per-width statistics; nullptr: the window's moments
};

// Per-range geometry of one chunk for the tiled dedispersion kernel.
struct DedispRange {
  const void* xd;          // decimated ring: uint8 (d == 1) or uint16 [Cp][xd_stride]
  int64_t xd_stride;       // elements
  int64_t m0;              // ring column of window sample 0
  int64_t nout;            // window length
  int32_t* y;              // [n_trials][y_stride]
  int64_t y_stride;
  Moments* mom;            // [n_trials]
  const int32_t* shifts;   // [n_trials][Cp]
  int32_t n_trials;
  int32_t is_u16;
};

// Arguments of the tiled dedispersion kernel (dd_dedisp.cu), one launch per range.
struct TiledArgs {
  const void* xd;          // decimated ring, uint8 (d == 1) or uint16, [Cp][xd_stride]
  int64_t xd_stride;       // elements
  int64_t m0;              // ring column of window sample 0
  int64_t nout;            // window length
  int32_t* y;              // [n_trials][y_stride]
  int64_t y_stride;
  Moments* mom;            // [n_trials], zeroed before the launch
  const int32_t* shifts;   // [n_trials][Cp], non-decreasing in the trial index
  int32_t n_trials;
  int32_t cpad;
  int32_t row_slot;        // elements per staged channel row
  int32_t zcap;            // pair words per stage buffer
  int32_t nstage;          // staging buffers (3 or 4)
  const uint8_t* tabs;     // delay-class tables of the range, one per (trial tile, stage)
  int32_t* err;            // bit 0: a bounded wait ran out
  CUtensorMap rows;        // the ring as [Cp][xd_stride / seg][seg] (make_ring_map)
};

// Search fused into the tiled kernel (64 x 512 tiles, 16 warps): one CTA walks a segment of
// consecutive time tiles of one trial tile and, after each tile, records per (trial, width,
// peak block) the block's largest boxcar sum and its earliest sample. Boxcars that reach back
// into the previous tile read that tile's prefix sums from the CTA's tail buffer; the first tile
// of a segment has none, and its boxcars that start before the segment are completed by
// k_fused_edges from the previous segment's tail and this segment's head.
struct FusedArgs {
  uint32_t* key;           // [n_trials][nw][nblk]: 1 + the largest boxcar sum, 0 = no sample
  uint8_t* off;            // [n_trials][nw][nblk]: its earliest sample within the block
  uint32_t* edge;          // [nsegs][trial tiles][2][64][hist]: head, tail prefix sums per CTA
  int64_t nblk;            // peak blocks of the window, ceil(nout / block)
  int32_t nw;              // widths (decimated), increasing, the last <= 512
  int32_t hist;            // the largest width: prefix sums kept from the previous tile
  int32_t hp;              // hist rounded up to 32
  int32_t block;           // samples per peak block (power of two <= 32)
  int32_t seg_tiles;       // time tiles per segment
  int32_t nsegs;           // segments (gridDim.y)
  int32_t keep_series;     // also write the series
  int32_t e_off;           // shared-memory byte offset of the per-warp prefix-sum rows
  int32_t wd[kMaxWidths];
};

// The search's last step for a fused range: per (trial, peak block) the FP64 SNR of each
// width's recorded maximum, the best over widths, and the candidate (as k_sps).
struct SpsFusedArgs {
  const uint32_t* key;     // FusedArgs::key
  const uint8_t* off;
  int64_t nblk;
  int64_t n;               // window length
  const Moments* mom;      // [n_trials]
  int32_t n_trials;
  int32_t range;
  int32_t d;
  int32_t block;
  int64_t J0;
  int32_t nw;
  int32_t wd[kMaxWidths];
  float threshold;
  dd_cand_t* cands;
  unsigned long long* count;
  int64_t cap;
};

// Arguments of the persistent tiled kernel: a device work list over many ranges (of many plans)
// of one instance (data type, tile shape, staging buffers). Segment k covers every tile of
// descs[seg_desc[k]]: items seg_first[k] .. seg_first[k + 1] - 1 (trial tiles fastest).
struct PersistArgs {
  const TiledArgs* descs;      // device [ndesc], 64-byte aligned (tensor maps inside)
  const int32_t* seg_desc;     // device [nseg]
  const int64_t* seg_first;    // device [nseg + 1]
  int32_t nseg;
  int32_t pad;
  unsigned long long* counter; // device, zeroed before the launch
};

// Plan of the tiled kernel for one range (host): tile shape, shared-memory sizes and the
// delay-class tables the kernel copies in per stage. ok = false: the range does not fit.
struct TiledPlan {
  bool ok = false;
  int tt = 0;
  int trials = 0;          // trials per tile (64 or 32)
  int threads = 0;         // threads per CTA (512 or 1024)
  int ctas = 0;            // CTAs per SM the tile shape is compiled for
  int nseg = 0;            // 128-byte segments per staged channel row
  int nstage = 0;          // staging buffers
  int row_slot = 0;
  int zcap = 0;
  size_t smem = 0;
  size_t tab_bytes = 0;
  std::vector<uint8_t> tabs;
  // Shared-memory work of one row of time tiles (every trial tile of the range, TT outputs),
  // counted from the tables as the kernel issues it: warp-wide shared-memory instructions
  // (wavefronts of the LSU data pipe: accumulation loads, pair-word build loads and stores,
  // table reads, addressing stores) and the bytes the tensor and bulk copies write.
  int64_t lsu_wavefronts = 0;
  int64_t copy_bytes = 0;
};

TiledPlan tiled_plan(const int32_t* shifts, int ntr, int cpad, int decimation, int tt,
                     int trials, int threads);
int64_t tiled_plan_check(const int32_t* shifts, int ntr, int cpad, int decimation, int tt,
                         int trials, int* ok);
cudaError_t prepare_tiled(int is_u16, int tt, int nstage, int trials, int threads, size_t smem);
// One CTA waits, with the tiled kernel's bound, on a barrier nothing completes; sets *err bit 0
// when the bound runs out.
cudaError_t launch_wait_selftest(int32_t* err, cudaStream_t st);
cudaError_t launch_tiled(const TiledArgs& a, int is_u16, int tt, int trials, int threads,
                         cudaStream_t st);
// The persistent form over a work list; smem = the largest staging arrangement of its
// descriptors (smem_bytes), grid = ctas (one per SM).
cudaError_t launch_tiled_persistent(const PersistArgs& p, int is_u16, int tt, int nstage,
                                    int trials, int threads, size_t smem, int ctas,
                                    cudaStream_t st);
size_t tiled_smem_bytes(int is_u16, int row_slot, int zcap, int nstage);
// Fused search (64 x 512 x 512 instances): where the per-warp prefix-sum rows go in shared
// memory (inside the staging area when it is large enough, else after it) and the launch's
// dynamic shared memory; false if that exceeds what a CTA may plan for.
bool fused_smem(int is_u16, int row_slot, int zcap, int nstage, int hp, int32_t* e_off,
                size_t* smem);
cudaError_t prepare_fused(int is_u16, int nstage, size_t smem);
// Time segments of a fused launch: minimises (waves of one CTA per SM) x (tiles per segment)
// for ntx trial tiles and ntt time tiles, at most smax segments.
int fused_segments(int ntx, int ntt, int sms, int smax);
// The fused dedispersion launch, grid (trial tiles, f.nsegs), then the segment-edge pass.
cudaError_t launch_fused(const TiledArgs& a, const FusedArgs& f, int is_u16, size_t smem,
                         cudaStream_t st);
cudaError_t launch_sps_fused(const SpsFusedArgs& a, cudaStream_t st);

// Tensor map of a channel-major ring (uint8, or uint16 when is_u16) for the tiled kernel's
// stage copies: dims {128-byte segment, segments per row, cpad rows}, box {segment, nseg, 16}.
// The row stride must be a multiple of 128 bytes. Host only; no device work.
cudaError_t make_ring_map(CUtensorMap* map, const void* ring, int is_u16, int64_t stride,
                          int32_t cpad, int nseg);

// Record `msg` as the calling thread's last error (dd_last_error) and return `code`.
int report_error(int code, const char* msg);

// 1 when chunk `seq` of the plan has been searched and its candidates are ready, 0 while its
// work is pending, DD_ERR_STATE if it is not a searched chunk still held by the plan.
int chunk_state(dd_plan_s* plan, int64_t seq);

// Batch support: wait for the plan and start its stream again at sample 0; the plan's streams;
// outputs (DM-trial*samples) of a stream of nsamp samples; the search of the latest chunk into
// caller-chosen device buffers (count cleared first; no host readback); choose each tiled
// range's time tile by timing the candidates; the chosen tile (0: simple kernel); send the
// dedispersion kernels' error bits to a caller-owned device word (the caller clears and reads
// it) instead of the slot's own, which dd_run clears for each chunk.
int plan_reset(dd_plan_s* plan);
void plan_streams(dd_plan_s* plan, std::vector<cudaStream_t>* out);
int64_t plan_outputs(dd_plan_s* plan, int64_t nsamp);
int sps_enqueue(dd_plan_s* plan, const int32_t* widths, int32_t nwidths, float threshold,
                dd_cand_t* cands, unsigned long long* count, int64_t cap);
int plan_autotune(dd_plan_s* plan);
int range_tile(dd_plan_s* plan, int r);
void plan_redirect_errors(dd_plan_s* plan, int32_t* err);
// A tiled dedispersion launch handed back by run_deferred for a persistent launch.
struct DeferredTile {
  TiledArgs args;
  int32_t is_u16;
  int32_t nstage;
  size_t smem;
};
// dd_run on stream `st`, except that the range launches of the 64 x 512 x 512 tile shape are
// appended to *out instead of being made (every other launch is made as dd_run makes it).
int run_deferred(dd_plan_s* plan, const uint8_t* chunk, int64_t nsamp, cudaStream_t st,
                 std::vector<DeferredTile>* out);
// Serving support: make the next dd_run's dedispersion wait (once) for an event of another
// plan on the same device; the event recorded when chunk `seq` of a plan has been searched
// (nullptr if that chunk is not a searched chunk still held by the plan).
void plan_gate_next(dd_plan_s* plan, cudaEvent_t ev);
cudaEvent_t chunk_done_event(dd_plan_s* plan, int64_t seq);

// ---- launchers (dd_kernels.cu); each returns the cudaGetLastError() of its launch
cudaError_t launch_shift_table(const double* freqs, int32_t nchans, int32_t cpad, double fref,
                               double tsamp, const ShiftRange* ranges, int32_t nranges,
                               int32_t total_rows, int32_t* shifts, int32_t* err,
                               cudaStream_t st);
cudaError_t launch_corner_turn(const uint8_t* in, int64_t n, int32_t nchans, uint8_t* ring,
                               int64_t ring_stride, int64_t col0, cudaStream_t st);
cudaError_t launch_decimate(const void* in, int in_is_u16, int64_t in_stride, uint16_t* out,
                            int64_t out_stride, int32_t cpad, int64_t n_out, cudaStream_t st);
cudaError_t launch_dedisp_naive(const DedispRange& r, int32_t cpad, cudaStream_t st);
cudaError_t launch_dedisp_direct(const DedispRange& r, int32_t cpad, cudaStream_t st);
cudaError_t launch_moments(const int32_t* y, int32_t ntr, int64_t n, int64_t stride, Moments* mom,
                           cudaStream_t st);
cudaError_t launch_sps(const SpsArgs& a, cudaStream_t st);
cudaError_t launch_clip_stats(const ClipArgs& a, cudaStream_t st);

}  // namespace ddk
