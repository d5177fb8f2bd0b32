// Tiled brute-force dedispersion for sm_103a (Sec. 2.1 "dedispersion of data"; the sum is the
// plain definition y[i][j] = sum_c x_d[c][j + s[i][c]], computed exactly in integers).
//
// One CTA owns a tile of D consecutive DM trials x TT output samples of one range and walks the
// channels in stages of kNG groups of eight channels. Tile shapes (the plan picks the first that
// fits, or times them all): 64 x 512 with 16 warps (128 registers per thread, 64 accumulators
// per lane), the same tile with 32 warps (64 registers, 32 accumulators: twice the warps on the
// same tables and shared memory), and 64 x 256 or 32 x 256 with 16 warps, two CTAs per SM.
//
//   * Delay classes. For an 8-channel group the tile's trials fall into a few classes by the
//     relative delays (r0..r7) of the eight channels. A class shares one sequence of sums
//        S_p[u] = x[c0][a+u+r0] + .. + x[c7][a+u+r7]
//     that each of its trials reads at its own base offset, stored as "pair words"
//        Z_p[u] = S_p[u] | S_p[u+1] << 16
//     (exact in 16-bit lanes: two groups' sums stay below 2^16 for d <= 16). The even and odd
//     pair words are kept in two planes, so a lane that owns outputs 2m and 2m+1 of a trial
//     reads one word, and consecutive lanes read consecutive words. The classes depend on the
//     delay table only, so the plan computes them once (tiled_plan, below) as one fixed-size
//     table per (trial tile, stage), together with a balanced split of the stage's word building
//     over the warps; the kernel never searches for them.
//   * TMA brings each stage's 16 channel rows (one 3-D tensor copy: every row from the same
//     128-byte segment on, so each lands contiguous) and its class table into shared memory
//     NS - 1 stages ahead (NS = 4 staging buffers, or 3 where 4 do not fit shared memory);
//     completion is tracked by mbarriers with bounded waits.
//   * The main loop adds, per (trial, output pair), the two groups' pair words with one IADD
//     and splits the sum over the two outputs with two DP2As: one 32-bit shared-memory load per
//     sixteen channel-adds, for uint8 and uint16 (decimated) data alike.
//
// Software pipeline, one __syncthreads per stage s:
//     TMA for stage s+NS-1 | build the words of stage s+1 | accumulate stage s
// Words are built from 32-bit loads and funnel shifts; the eight-channel sums are formed in SWAR
// lanes (bytes split into 16-bit lanes for uint8 data). Where each class's channel rows start in
// a stage buffer (row word and funnel shift) depends on where the stage's copy starts, so the
// CTA works it out once per stage, one (class, channel) per thread, two stages ahead. Exact
// moments (S1, 128-bit S2) of every series are added in the epilogue with integer atomics, so
// the search needs no second statistics pass.
#include <cudaTypedefs.h>

#include <algorithm>
#include <climits>
#include <cstring>
#include <mutex>

#include "dd_internal.h"

namespace ddk {

namespace {

constexpr int kMaxTileTrials = 64;         // trials per tile: 64 or 32
constexpr int kThreads = 512;               // threads of the 16-warp shapes
constexpr int kWarps = kThreads / 32;       // work lists of a stage's build (one per warp, or
                                            // shared by two warps in 32-warp CTAs)
constexpr int kG = 8;                       // channels per group (one delay class)
constexpr int kNG = 2;                      // groups per stage
constexpr int kRows = kG * kNG;             // channel rows per stage
constexpr int kMaxNStage = 4;               // staging buffers (rows + class table), at most
constexpr int kMaxCls = 16;                 // classes per group
constexpr int kMaxWork = 8;                 // build ranges per warp and stage
constexpr int kSegBytes = 128;              // inner extent of a staged-row copy (tensor map)
constexpr size_t kSmemLimit = 220 * 1024;   // dynamic shared memory a CTA may plan for
constexpr size_t kSmemLimit2 = 110 * 1024;  // ... when two CTAs share an SM

// CTAs per SM a tile shape is compiled for (its register budget: 65536 / (NT x CTAs)).
__host__ __device__ constexpr int tile_ctas(int D, int TT, int NT) {
  return (NT == 1024 || (D == 64 && TT == 512)) ? 1 : 2;
}

// One delay class: its channels' first staged sample relative to the tile's first trial
// (rel), and its pair words in the stage's word region.
struct ClsEntry {
  int16_t rel[kG];
  int16_t zoff;  // first word (multiple of 4)
  int16_t zlen;  // words (multiple of 4)
  int32_t pad;
};

// Entry of trial t of a tile in GroupTab::zstart for a CTA of W warps with tpw trials per warp:
// warp t mod W reads its trials t, t + W, ... as tpw consecutive entries.
__host__ __device__ constexpr int trial_slot(int t, int W, int tpw) { return (t % W) * tpw + t / W; }

struct GroupTab {
  int16_t zstart[kMaxTileTrials];  // stage word offset of each trial's sequence (0: no trial),
                                   // warp-major: entry trial_slot(t) (a warp's trials contiguous)
  ClsEntry cls[kMaxCls];
  int32_t ncls, pad0, pad1, pad2;
};

// The stage's pair-word build, cut at plan time into blocks of 32 units (one per lane) and
// dealt to the warps in near-equal contiguous shares. A share is a few ranges, each within one
// class: group << 4 | class, first block << 8, blocks << 16.
struct StageTab {
  GroupTab g[kNG];
  uint32_t work[kWarps][kMaxWork];
  uint8_t nwork[kWarps];
  int32_t xmin;  // smallest delay of the stage's rows for the tile's first trial
  int32_t pad[3];
};
static_assert(sizeof(StageTab) % 16 == 0, "class tables are copied in 16-byte units");

// Row addressing of every class of one stage: for each of its eight channels, the byte offset
// of the row word holding the class's first sample within the stage buffer (8 x uint16) and the
// funnel shift in bits that brings that sample to bit 0 (8 x uint8).
struct AddrTab {
  uint4 addr[kNG][kMaxCls];
  uint2 sh[kNG][kMaxCls];
};
constexpr int kAddrEntries = kNG * kMaxCls * kG;  // one per thread of the first half of the CTA
static_assert(kAddrEntries <= kThreads, "one addressing entry per thread");

__host__ __device__ constexpr size_t align16(size_t v) { return (v + 15) & ~size_t(15); }

struct SmemLayout {
  size_t raw, z, tab, addr, mbar, total;
};

// The mbarriers come first, at the same place for every tile shape and range (a persistent CTA
// re-initialises them between tiles of different ranges); the staged rows start 128-byte aligned.
__host__ __device__ inline SmemLayout smem_layout(int es, int zes, int row_slot, int zcap,
                                                  int nst) {
  SmemLayout L;
  L.mbar = 0;
  size_t off = 128;
  L.raw = off;
  off = align16(off + (size_t)nst * kRows * row_slot * es);
  L.z = off;
  off = align16(off + (size_t)2 * zcap * zes);
  L.tab = off;
  off = align16(off + sizeof(StageTab) * nst);
  L.addr = off;
  off = align16(off + sizeof(AddrTab) * 2);
  L.total = off;
  return L;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

template <int OFF>  // 32-bit shared-memory load at a byte address + OFF
__device__ __forceinline__ uint32_t lds(uint32_t addr) {
  uint32_t v;
  asm volatile("ld.shared.u32 %0, [%1+%2];" : "=r"(v) : "r"(addr), "n"(OFF));
  return v;
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait for a stage with a bound: at most 2 s and 2^26 polls; false if it ran out.
__device__ bool mbar_wait_bounded(unsigned long long* bar, uint32_t parity) {
  const unsigned long long t0 = globaltimer_ns();
  for (int it = 0; it < (1 << 26); ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255) == 255 && globaltimer_ns() - t0 > 2000000000ull) return false;
  }
  return false;
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// First row segment of a stage's copy: every row is copied from the segment holding sample
// m0 + j0 + xmin on, xmin being the smallest delay of the stage's rows.
template <typename T>
__device__ __forceinline__ int64_t first_seg(const TiledArgs& a, int64_t j0, int32_t xmin) {
  constexpr int SEG = kSegBytes / (int)sizeof(T);  // elements per segment
  return (a.m0 + j0 + xmin) / SEG;
}

__device__ __forceinline__ int32_t stage_xmin(const TiledArgs& a, int stage, int nstages,
                                              int tile) {
  if (stage >= nstages) return 0;
  return __ldg(&reinterpret_cast<const StageTab*>(a.tabs)[(size_t)tile * nstages + stage].xmin);
}

// Issue of one stage by one thread: one tensor copy of the stage's 16 rows (segments
// [first_seg, first_seg + nseg) of each; rows past the padded channels read as zeros) and one
// bulk copy of its class table, after arming the stage's mbarrier with their bytes.
template <typename T>
__device__ __forceinline__ void issue_stage(const TiledArgs& a, int stage, int nstages,
                                            T* raw_buf, StageTab* tab_buf,
                                            unsigned long long* bar, int32_t xmin, int64_t j0,
                                            int tile) {
  const uint32_t row_bytes = (uint32_t)a.row_slot * (uint32_t)sizeof(T);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  mbar_arrive_expect_tx(bar, kRows * row_bytes + (uint32_t)sizeof(StageTab));
  const int32_t seg = (int32_t)first_seg<T>(a, j0, xmin);
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(raw_buf)),
      "l"(reinterpret_cast<uint64_t>(&a.rows)), "r"(0), "r"(seg), "r"(stage * kRows),
      "r"(smem_addr(bar))
      : "memory");
  bulk_g2s(tab_buf, a.tabs + ((size_t)tile * nstages + stage) * sizeof(StageTab),
           (uint32_t)sizeof(StageTab), bar);
}

// One addressing entry of a stage: entry e = (group, class, channel). The row's copy starts at
// segment first_seg (issue_stage), so the class's first sample sits
// m0 + j0 + s_first - first_seg * (segment elements) + rel elements into the row. Its inputs come
// from the class table and the delay table in global memory (the staged copy of the table may
// still be in flight), loaded one iteration before the entry is formed.
struct AddrInputs {
  int32_t ncls;  // classes of the entry's group (0: no such group)
  int32_t rel;
  int32_t smin;
  int32_t xmin;
};

__device__ __forceinline__ AddrInputs addr_inputs(const TiledArgs& a, int stage, int nstages,
                                                  int ngroups, int trial0, int e, int tile) {
  AddrInputs in{0, 0, 0, 0};
  const int gl = e / (kMaxCls * kG), p = (e / kG) % kMaxCls, k = e % kG;
  if (stage < nstages && stage * kNG + gl < ngroups) {
    const StageTab* st =
        &reinterpret_cast<const StageTab*>(a.tabs)[(size_t)tile * nstages + stage];
    const GroupTab* gt = &st->g[gl];
    in.xmin = __ldg(&st->xmin);
    in.ncls = __ldg(&gt->ncls);
    in.rel = __ldg(&gt->cls[p].rel[k]);  // the table is zero past the group's classes
    in.smin = __ldg(a.shifts + (int64_t)trial0 * a.cpad + stage * kRows + gl * kG + k);
  }
  return in;
}

template <typename T>
__device__ __forceinline__ void addr_entry(const TiledArgs& a, const AddrInputs& in, int64_t j0,
                                           int e, AddrTab* at) {
  constexpr int SEG = kSegBytes / (int)sizeof(T);
  const int gl = e / (kMaxCls * kG), p = (e / kG) % kMaxCls, k = e % kG;
  if (p >= in.ncls) return;
  const int row = gl * kG + k;
  const int ph = (int)(a.m0 + j0 + in.smin - first_seg<T>(a, j0, in.xmin) * SEG);
  const uint32_t byte = (uint32_t)(row * a.row_slot + in.rel + ph) * (uint32_t)sizeof(T);
  reinterpret_cast<uint16_t*>(&at->addr[gl][p])[k] = (uint16_t)(byte & ~3u);
  reinterpret_cast<uint8_t*>(&at->sh[gl][p])[k] = (uint8_t)((byte & 3u) * 8u);
}

// The eight channel rows of one class, as one lane reads them: shared-memory byte address of
// the row word holding its first unit, and the funnel shift of each channel.
struct RowItem {
  uint32_t addr[kG];
  uint32_t sh[kG];
};

template <typename T>
struct Word;

// Row words of channel k at byte offset OFF: the word holding the class's first sample and the
// next one.
template <int OFF>
__device__ __forceinline__ void row_words(const RowItem& it, int k, uint32_t& w0, uint32_t& w1) {
  w0 = lds<OFF>(it.addr[k]);
  w1 = lds<OFF + 4>(it.addr[k]);
}

// uint8 data. Unit u covers pair words 4u .. 4u + 3, i.e. the eight-channel sums
// S[4u .. 4u + 4] (one more than its words, which the last pair word needs). Each channel's two
// row words are funnel-shifted to the class's first sample; bytes are split into even/odd
// 16-bit lanes so that eight channels add without carries (8 x 255 < 2^16). The fifth sum is
// the next unit's first one, S[4(u + 1)]: the next lane's, taken with one shuffle. So a block of
// 32 lanes stores 31 units (lanes 0 .. 30); lane 31 computes the next block's first unit only
// to hand its first sum to lane 30 (kBlock = 31). The pair words go to the class's even plane
// (4u, 4u + 2) and odd plane (4u + 1, 4u + 3); lanes take consecutive units, so every load and
// store is free of bank conflicts. Every lane of the warp runs the unit (the shuffle needs them
// all); `live` says whether this lane's words are stored.
template <>
struct Word<uint8_t> {
  static constexpr int kUnit = 4;   // pair words per unit
  static constexpr int kBlock = 31; // units stored per 32-lane block
  template <int OFF>
  static __device__ __forceinline__ void unit(const RowItem& it, uint32_t* ev, uint32_t* od,
                                              bool live) {
    uint32_t e = 0, o = 0;
#pragma unroll
    for (int k = 0; k < kG; ++k) {
      uint32_t w0, w1;
      row_words<OFF>(it, k, w0, w1);
      const uint32_t a = __funnelshift_r(w0, w1, it.sh[k]);  // samples 0..3 in bytes 0..3
      e += a & 0x00FF00FFu;                                  // samples 0, 2
      o += __byte_perm(a, 0, 0x4341);                        // samples 1, 3
    }
    const uint32_t nx = __shfl_down_sync(0xffffffffu, e, 1);  // low half: S4 (next unit's S0)
    if (live) {
      uint2 x, y;
      x.x = __byte_perm(e, o, 0x5410);   // S0 | S1 << 16
      x.y = __byte_perm(e, o, 0x7632);   // S2 | S3 << 16
      y.x = __byte_perm(o, e, 0x7610);   // S1 | S2 << 16
      y.y = __byte_perm(o, nx, 0x5432);  // S3 | S4 << 16
      *reinterpret_cast<uint2*>(ev) = x;
      *reinterpret_cast<uint2*>(od) = y;
    }
  }
};

// uint16 data. Unit u covers pair words 2u, 2u + 1 (sums S[2u .. 2u + 2]) from two row words
// per channel; 16-bit lanes add eight channels without carries (8 x 255 x d < 2^16), and the
// third sample, halfword (shift / 16) of the second row word, is added by a DP2A on the
// rotated word.
template <>
struct Word<uint16_t> {
  static constexpr int kUnit = 2;
  static constexpr int kBlock = 32;  // units per 32-lane block
  template <int OFF>
  static __device__ __forceinline__ void unit(const RowItem& it, uint32_t* ev, uint32_t* od,
                                              bool /*live: always, lanes past the class skip*/) {
    uint32_t e = 0, s2 = 0;
#pragma unroll
    for (int k = 0; k < kG; ++k) {
      uint32_t w0, w1;
      row_words<OFF>(it, k, w0, w1);
      e += __funnelshift_r(w0, w1, it.sh[k]);                  // samples 0, 1
      s2 = __dp2a_lo(__funnelshift_r(w1, w1, it.sh[k]), 1u, s2);  // sample 2
    }
    *ev = e;                           // S0 | S1 << 16
    *od = __byte_perm(e, s2, 0x5432);  // S1 | S2 << 16
  }
};

// Add one pair word (S[u] | S[u + 1] << 16, or the sum of two groups' words) to the two
// outputs it serves.
__device__ __forceinline__ void pair_add(uint32_t z, uint32_t& even, uint32_t& odd) {
  even = __dp2a_lo(z, 0x0001u, even);  // + low half
  odd = __dp2a_lo(z, 0x0100u, odd);    // + high half
}

// Build every pair word of one stage: a warp walks the ranges of work list `list`; lane l builds
// unit 32 * b + l of every block b of a range. With HALVES = 1 the warp builds every block, two
// per pass; with HALVES = 2 two warps share the list, warp `half` building blocks b0 + half,
// b0 + half + 2, ...
template <typename T, int HALVES>
__device__ __forceinline__ void build_stage(const StageTab& tb, const AddrTab& at, uint32_t rawb,
                                            uint32_t* Zs, int list, int lane, int half) {
  constexpr int U = Word<T>::kUnit;
  const int nw = tb.nwork[list];
  for (int w = 0; w < nw; ++w) {
    const uint32_t wk = tb.work[list][w];
    const int gi = (int)((wk >> 4) & 1), p = (int)(wk & 15);
    const int b0 = (int)((wk >> 8) & 255), nb = (int)(wk >> 16);
    const int zlen = tb.g[gi].cls[p].zlen;
    constexpr int B = Word<T>::kBlock;  // units per block
    int u = B * (b0 + (HALVES == 2 ? half : 0)) + lane;
    const uint4 ad = at.addr[gi][p];
    const uint2 sv = at.sh[gi][p];
    const uint32_t base = rawb + 4u * (uint32_t)u;  // one row word per unit
    RowItem it;
    it.addr[0] = base + (ad.x & 0xFFFFu);
    it.addr[1] = base + (ad.x >> 16);
    it.addr[2] = base + (ad.y & 0xFFFFu);
    it.addr[3] = base + (ad.y >> 16);
    it.addr[4] = base + (ad.z & 0xFFFFu);
    it.addr[5] = base + (ad.z >> 16);
    it.addr[6] = base + (ad.w & 0xFFFFu);
    it.addr[7] = base + (ad.w >> 16);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      it.sh[k] = sv.x >> (8 * k);
      it.sh[k + 4] = sv.y >> (8 * k);
    }
    // even plane: pair words 0, 2, 4, ... of the class; odd plane: 1, 3, 5, ...
    uint32_t* ev = Zs + tb.g[gi].cls[p].zoff + (U / 2) * u;
    uint32_t* od = ev + zlen / 2;
    if constexpr (B == 31) {
      // uint8: every lane runs every unit (shuffles); lanes 0 .. 30 store the block's units.
      // Lanes past the class compute nothing they store; their loads stay inside the CTA's
      // shared memory (the staged rows are followed by the word planes).
      const bool store_lane = lane < 31;
      if (HALVES == 1) {
        for (int b = 0; b < nb; b += 2) {
          Word<T>::template unit<0>(it, ev, od, store_lane && u * U < zlen);
          if (b + 1 < nb)
            Word<T>::template unit<4 * B>(it, ev + B * U / 2, od + B * U / 2,
                                          store_lane && (u + B) * U < zlen);
#pragma unroll
          for (int k = 0; k < kG; ++k) it.addr[k] += 8u * B;  // two blocks further
          u += 2 * B;
          ev += B * U;
          od += B * U;
        }
      } else {
        for (int b = half; b < nb; b += 2) {
          Word<T>::template unit<0>(it, ev, od, store_lane && u * U < zlen);
#pragma unroll
          for (int k = 0; k < kG; ++k) it.addr[k] += 8u * B;
          u += 2 * B;
          ev += B * U;
          od += B * U;
        }
      }
    } else {
      // uint16: lanes past the class skip their units
      if (HALVES == 1) {
        for (int b = 0; b < nb; b += 2) {
          if (u * U < zlen) Word<T>::template unit<0>(it, ev, od, true);
          if (b + 1 < nb && (u + B) * U < zlen)
            Word<T>::template unit<4 * B>(it, ev + B * U / 2, od + B * U / 2, true);
#pragma unroll
          for (int k = 0; k < kG; ++k) it.addr[k] += 8u * B;  // two blocks further
          u += 2 * B;
          ev += B * U;
          od += B * U;
        }
      } else {
        for (int b = half; b < nb; b += 2) {
          if (u * U < zlen) Word<T>::template unit<0>(it, ev, od, true);
#pragma unroll
          for (int k = 0; k < kG; ++k) it.addr[k] += 8u * B;
          u += 2 * B;
          ev += B * U;
          od += B * U;
        }
      }
    }
  }
}

// ---- search fused into the tile (Sec. 2.2 boxcars over the series the tile has just summed)
//
// Per trial the warp forms the tile's inclusive prefix sums P[j] (uint32, relative to the tile's
// start: exact differences since every boxcar sum is < 2^31) in a shared-memory row, preceded by
// the `hist` prefix sums of the previous tile in this tile's frame (P[m] = -(sum of the previous
// tile's outputs after m), m = -hist .. -1). Then B_w[j] = P[j] - P[j - w] for every width, and
// per peak block the largest B_w + 1 (0: no valid sample) and its earliest sample are stored.
// Valid samples: inside the window, j >= w - 1 in the window (the boxcars of Sec. 2.2 reading),
// and, in the first tile of a segment (no previous tile), boxcars inside the tile only; the
// others are k_fused_edges' work.

// L2 evict-last access policy for the tail buffers: rewritten every tile and read back one tile
// later, while the streamed channel rows pass through L2 in between.
__device__ __forceinline__ uint64_t l2_keep_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ uint32_t ld_keep(const uint32_t* p, uint64_t pol) {
  uint32_t v;
  asm volatile("ld.global.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ void st_keep(uint32_t* p, uint32_t v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.u32 [%0], %1, %2;" ::"l"(p), "r"(v), "l"(pol) : "memory");
}

// Largest key over aligned groups of B lanes (B a power of two <= 32) and, for the group's
// first lane, the group's earliest lane holding it.
__device__ __forceinline__ uint32_t group_max(uint32_t key, int B, int lane, int* first) {
  uint32_t mx = key;
  if (B == 32) {
    mx = __reduce_max_sync(0xffffffffu, key);
  } else {
    for (int o = B >> 1; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  const uint32_t bal = __ballot_sync(0xffffffffu, key == mx);
  const uint32_t gm = B == 32 ? 0xffffffffu : ((1u << B) - 1u);
  *first = __ffs((bal >> (lane & ~(B - 1))) & gm) - 1;
  return mx;
}

// Head and tail buffers of CTA (trial tile bx, segment seg): [64][hist] each.
__device__ __forceinline__ uint32_t* fused_edge(const FusedArgs& f, int ntx, int bx, int seg) {
  return f.edge + ((size_t)seg * ntx + bx) * 2 * kMaxTileTrials * (size_t)f.hist;
}

template <int TT, int W, int kTPW, int KT>
__device__ __forceinline__ void fused_search(const TiledArgs& a, const FusedArgs& f,
                                             const uint32_t (&acc)[kTPW][KT],
                                             unsigned char* smem, int bx, int by, bool first,
                                             int trial0, int ntr, int64_t j0, int warp,
                                             int lane) {
  constexpr int KP = KT / 2;
  const int hist = f.hist, HP = f.hp, Bk = f.block, nw = f.nw;
  const int wmax = f.wd[nw - 1];
  const int ntx = (a.n_trials + kMaxTileTrials - 1) / kMaxTileTrials;
  const int seg = by / f.seg_tiles;
  uint32_t* head = fused_edge(f, ntx, bx, seg);
  uint32_t* tail = head + kMaxTileTrials * (size_t)hist;
  uint32_t* E = reinterpret_cast<uint32_t*>(smem + f.e_off) + (size_t)warp * (HP + TT) + HP;
  const int64_t nout = a.nout;
  const uint64_t pol = l2_keep_policy();
#pragma unroll
  for (int q = 0; q < kTPW; ++q) {  // unrolled: acc stays in registers
    const int t = warp + W * q;
    if (t >= ntr) break;  // uniform in the warp; later q only larger
    uint32_t* tl = tail + (size_t)t * hist;
    uint32_t hv[16];  // hist <= 512; independent loads, all in flight before the scan
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const int i = lane + 32 * r;
      hv[r] = (!first && i < hist) ? ld_keep(tl + i, pol) : 0u;
    }
    // inclusive prefix sums of the tile; lane l holds outputs 2(l + 32k) and 2(l + 32k) + 1
    uint32_t carry = 0;
#pragma unroll
    for (int k = 0; k < KP; ++k) {
      const uint32_t ev = acc[q][2 * k], od = acc[q][2 * k + 1];
      uint32_t incl = ev + od;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t x = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += x;
      }
      const uint32_t po = carry + incl;
      *reinterpret_cast<uint2*>(E + 2 * (lane + 32 * k)) = make_uint2(po - od, po);
      carry += __shfl_sync(0xffffffffu, incl, 31);
    }
    // the previous tile's prefix sums in this tile's frame (none before a segment's first tile:
    // no valid boxcar reads them there)
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const int i = lane + 32 * r;
      if (i < hist) E[i - hist] = hv[r];
    }
    __syncwarp();
    if (first && seg > 0) {
      uint32_t* hd = head + (size_t)t * hist;
      for (int i = lane; i < hist; i += 32) hd[i] = E[i];
    }
    // this tile's last prefix sums in the next tile's frame (P[TT + m] - P[TT - 1])
    for (int i = lane; i < hist; i += 32) st_keep(tl + i, E[TT - hist + i] - carry, pol);
    const int64_t rowk = (int64_t)(trial0 + t) * nw;
    // one lane per item: a 32-sample block is two items of 16 samples (lanes b and b + 16), a
    // smaller block one item; each lane visits its samples from (lane mod P) on, so the 32 lanes
    // of a load read 32 different banks, and keeps per width the largest key and, on ties, the
    // earliest sample
    const int P = Bk == 32 ? 16 : Bk;
    const int nitems = (TT / Bk) * (Bk == 32 ? 2 : 1);
    const bool interior = j0 >= wmax - 1 && !first && j0 + TT <= nout;
#pragma unroll 1
    for (int it = lane; it < nitems; it += 32) {
      const int b = Bk == 32 ? (it & 15) : it;
      const int h = Bk == 32 ? (it >> 4) : 0;
      const int o0 = h * P;  // the item's first sample within its block
      const int jl0 = b * Bk + o0;
      uint32_t best[kMaxWidths];
      int boff[kMaxWidths];
#pragma unroll
      for (int k = 0; k < kMaxWidths; ++k) best[k] = 0u, boff[k] = 32;
#pragma unroll 1
      for (int i = 0; i < P; ++i) {
        const int pi = (i + lane) & (P - 1);
        const int jl = jl0 + pi, o = o0 + pi;
        const int64_t jg = j0 + jl;
        const uint32_t p1 = E[jl] + 1u;
#pragma unroll
        for (int k = 0; k < kMaxWidths; ++k) {
          if (k < nw) {
            const int w = f.wd[k];
            uint32_t key = p1 - E[jl - w];
            if (!interior) {
              const bool valid = jg < nout && jg >= w - 1 && (!first || jl >= w - 1);
              key = valid ? key : 0u;
            }
            const bool take = key > best[k] || (key == best[k] && o < boff[k]);
            best[k] = take ? key : best[k];
            boff[k] = take ? o : boff[k];
          }
        }
      }
      if (Bk == 32) {  // every lane has an item: combine the two halves of each block
#pragma unroll
        for (int k = 0; k < kMaxWidths; ++k) {
          if (k < nw) {
            const uint32_t ob = __shfl_xor_sync(0xffffffffu, best[k], 16);
            const int oo = __shfl_xor_sync(0xffffffffu, boff[k], 16);
            const bool take = ob > best[k] || (ob == best[k] && oo < boff[k]);
            best[k] = take ? ob : best[k];
            boff[k] = take ? oo : boff[k];
          }
        }
      }
      const int64_t jb = j0 + (int64_t)b * Bk;  // the block's first window sample
      if (h == 0 && jb < nout) {
        const int64_t blk = jb / Bk;
#pragma unroll
        for (int k = 0; k < kMaxWidths; ++k) {
          if (k < nw) {
            const int64_t idx = (rowk + k) * f.nblk + blk;
            f.key[idx] = best[k];
            f.off[idx] = (uint8_t)(best[k] ? boff[k] : 0);
          }
        }
      }
    }
    __syncwarp();  // the row is rewritten for the warp's next trial
  }
  // the rows overlay the staging buffers that the next tile's tensor copies fill
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Boxcars of a segment's first tile that start in the previous segment: per (boundary, trial),
// width w, samples j < w - 1 of the tile, B = head[j] - tail[hist + j - w], merged into the
// block's record (these samples precede every sample the fused pass saw in the block, so they
// win ties). CTA (4 x trial tile + quarter, boundary) takes 16 trials of the trial tile, one per
// warp; a warp first copies its trial's head and tail into shared memory (independent loads, all
// in flight), then works from there.
constexpr int kEdgeTrials = 16;

__global__ void __launch_bounds__(512) k_fused_edges(const __grid_constant__ TiledArgs a,
                                                     const __grid_constant__ FusedArgs f) {
  extern __shared__ __align__(16) uint32_t edge_rows[];  // [16 warps][2][hist]
  const int bx = blockIdx.x / 4, quarter = blockIdx.x % 4, seg = blockIdx.y + 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t J = (int64_t)seg * f.seg_tiles * 512;
  if (J >= a.nout) return;
  const int ntx = gridDim.x / 4;
  const int hist = f.hist, Bk = f.block;
  const int t = quarter * kEdgeTrials + warp;  // trial within the trial tile
  const int trial = bx * kMaxTileTrials + t;
  if (trial >= a.n_trials) return;  // warp-uniform; no barrier follows
  const uint32_t* hd = fused_edge(f, ntx, bx, seg) + (size_t)t * hist;
  const uint32_t* tl =
      fused_edge(f, ntx, bx, seg - 1) + kMaxTileTrials * (size_t)hist + (size_t)t * hist;
  uint32_t* H = edge_rows + (size_t)warp * 2 * hist;
  uint32_t* T = H + hist;
#pragma unroll 4
  for (int i = lane; i < hist; i += 32) {
    H[i] = __ldcg(hd + i);
    T[i] = __ldcg(tl + i);
  }
  __syncwarp();
  for (int k = 0; k < f.nw; ++k) {
    const int w = f.wd[k];
    for (int jb = 0; jb < w - 1; jb += 32) {
      const int jl = jb + lane;
      const int64_t jg = J + jl;
      const bool valid = jl < w - 1 && jg < a.nout;
      const uint32_t key = valid ? H[jl] + 1u - T[hist + jl - w] : 0u;
      int fo;
      const uint32_t mx = group_max(key, Bk, lane, &fo);
      if ((lane & (Bk - 1)) == 0 && jg < a.nout && mx != 0) {
        const int64_t idx = ((int64_t)trial * f.nw + k) * f.nblk + jg / Bk;
        if (mx >= f.key[idx]) {
          f.key[idx] = mx;
          f.off[idx] = (uint8_t)fo;
        }
      }
    }
  }
}

template <typename T, int TT, int NS, int D, int NT, bool FUSED = false>
__device__ __forceinline__ bool tile_body(const TiledArgs& a, int bx, int by,
                                          unsigned char* smem, bool reuse,
                                          const FusedArgs* f = nullptr, bool first = false) {
  constexpr int KT = TT / 32;       // outputs per lane and trial
  constexpr int KP = TT / 64;       // pair words per lane and trial
  constexpr int W = NT / 32;        // warps
  constexpr int kTPW = D / W;       // trials per warp
  constexpr int HALVES = W / kWarps;  // warps sharing a build work list
  const SmemLayout SL = smem_layout(sizeof(T), 4, a.row_slot, a.zcap, NS);
  T* raw = reinterpret_cast<T*>(smem + SL.raw);
  uint32_t* Zbuf = reinterpret_cast<uint32_t*>(smem + SL.z);
  StageTab* tab = reinterpret_cast<StageTab*>(smem + SL.tab);
  AddrTab* atab = reinterpret_cast<AddrTab*>(smem + SL.addr);
  unsigned long long* mbar = reinterpret_cast<unsigned long long*>(smem + SL.mbar);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int trial0 = bx * D;
  const int ntr = min(D, a.n_trials - trial0);
  const int64_t j0 = (int64_t)by * TT;
  const int ngroups = a.cpad / kG;
  const int nstages = (ngroups + kNG - 1) / kNG;
  const size_t stage_elems = (size_t)kRows * a.row_slot;

  if (tid == 0) {
    for (int s = 0; s < NS; ++s) {
      if (reuse) asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(&mbar[s]))
                              : "memory");
      mbar_init(&mbar[s], 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  // row addressing of stages 0 and 1; stage s + 2 is formed during iteration s from inputs
  // loaded during iteration s - 1 (the prologue for s = 0)
  AddrInputs ain{0, 0, 0, 0};
  {
    const int s0 = tid / kAddrEntries;
    if (s0 < 2) {
      const AddrInputs in0 =
          addr_inputs(a, s0, nstages, ngroups, trial0, tid % kAddrEntries, bx);
      addr_entry<T>(a, in0, j0, tid % kAddrEntries, &atab[s0]);
    }
    if (tid < kAddrEntries) ain = addr_inputs(a, 2, nstages, ngroups, trial0, tid, bx);
  }
  __syncthreads();
  // stages whose copies have been issued: NS in the prologue, then one per iteration s >= 1
  // (the same count in every thread)
  int issued = min(NS, nstages);
  int32_t xmin_next = 0;  // first delay of the next stage to issue (issuing thread)
  if (tid == NT - 32) {
    for (int s = 0; s < NS && s < nstages; ++s)
      issue_stage<T>(a, s, nstages, raw + (size_t)s * stage_elems, &tab[s], &mbar[s],
                     stage_xmin(a, s, nstages, bx), j0, bx);
    xmin_next = stage_xmin(a, NS, nstages, bx);
  }
  bool ok0 = mbar_wait_bounded(&mbar[0], 0);
  if (ok0) build_stage<T, HALVES>(tab[0], atab[0], smem_addr(raw), Zbuf, warp % kWarps, lane,
                                  warp / kWarps);
  bool aborted = __syncthreads_or(!ok0);
  int s_abort = 0;  // first stage whose copies may still be in flight

  uint32_t acc[kTPW][KT];
#pragma unroll
  for (int q = 0; q < kTPW; ++q)
#pragma unroll
    for (int k = 0; k < KT; ++k) acc[q][k] = 0;

  for (int s = 0; s < nstages && !aborted; ++s) {
    const int ng = min(kNG, ngroups - s * kNG);
    // (1) TMA for stage s + NS - 1 into the buffers stage s - 1 used (its words were built
    //     during stage s - 2 and its table last read by the accumulation of stage s - 1)
    if (s >= 1 && s + NS - 1 < nstages) {
      const int s2 = s + NS - 1;
      const int b2 = s2 % NS;
      if (tid == NT - 32) {
        issue_stage<T>(a, s2, nstages, raw + (size_t)b2 * stage_elems, &tab[b2], &mbar[b2],
                       xmin_next, j0, bx);
        xmin_next = stage_xmin(a, s2 + 1, nstages, bx);
      }
      issued = s2 + 1;
    }
    // row addressing of stage s + 2, into the buffer stage s used (read during iteration s - 1)
    if (tid < kAddrEntries) {
      if (s + 2 < nstages) addr_entry<T>(a, ain, j0, tid, &atab[s & 1]);
      ain = addr_inputs(a, s + 3, nstages, ngroups, trial0, tid, bx);
    }
    // (2) pair words of stage s + 1
    bool ok = true;
    if (s + 1 < nstages) {
      const int b1 = (s + 1) % NS;
      ok = mbar_wait_bounded(&mbar[b1], (uint32_t)(((s + 1) / NS) & 1));
      if (ok)
        build_stage<T, HALVES>(tab[b1], atab[(s + 1) & 1],
                               smem_addr(raw + (size_t)b1 * stage_elems),
                               Zbuf + (size_t)((s + 1) & 1) * a.zcap, warp % kWarps, lane,
                               warp / kWarps);
    }
    // (3) accumulate stage s: lane l of the warp reads, for each of its trials, pair word
    //     l + 32k of the trial's plane in both groups (outputs 2(l + 32k) and 2(l + 32k) + 1)
    {
      const StageTab& tc = tab[s % NS];
      const uint32_t* Zs = Zbuf + (size_t)(s & 1) * a.zcap + lane;
      const uint32_t* zp[kTPW];
      const uint32_t* zq[kTPW];
      static_assert(kTPW == 4 || kTPW == 2, "a warp's offsets are one 8- or 4-byte load");
      if constexpr (kTPW == 4) {
        const uint2 e0 = *reinterpret_cast<const uint2*>(tc.g[0].zstart + warp * 4);
        const uint2 e1 = *reinterpret_cast<const uint2*>(tc.g[1].zstart + warp * 4);
        zp[0] = Zs + (e0.x & 0xFFFFu); zp[1] = Zs + (e0.x >> 16);
        zp[2] = Zs + (e0.y & 0xFFFFu); zp[3] = Zs + (e0.y >> 16);
        zq[0] = Zs + (e1.x & 0xFFFFu); zq[1] = Zs + (e1.x >> 16);
        zq[2] = Zs + (e1.y & 0xFFFFu); zq[3] = Zs + (e1.y >> 16);
      } else {
        const uint32_t e0 = *reinterpret_cast<const uint32_t*>(tc.g[0].zstart + warp * 2);
        const uint32_t e1 = *reinterpret_cast<const uint32_t*>(tc.g[1].zstart + warp * 2);
        zp[0] = Zs + (e0 & 0xFFFFu); zp[1] = Zs + (e0 >> 16);
        zq[0] = Zs + (e1 & 0xFFFFu); zq[1] = Zs + (e1 >> 16);
      }
      if (ng == kNG) {  // uniform; only the last stage may hold one group
#pragma unroll
        for (int k = 0; k < KP; ++k)
#pragma unroll
          for (int q = 0; q < kTPW; ++q)
            pair_add(zp[q][32 * k] + zq[q][32 * k], acc[q][2 * k], acc[q][2 * k + 1]);
      } else {
#pragma unroll
        for (int k = 0; k < KP; ++k)
#pragma unroll
          for (int q = 0; q < kTPW; ++q) pair_add(zp[q][32 * k], acc[q][2 * k], acc[q][2 * k + 1]);
      }
    }
    if (__syncthreads_or(!ok)) {
      aborted = true;
      s_abort = s + 1;
    }
  }

  if (aborted) {
    if (tid == 0) {
      atomicOr(a.err, 1);
      // let every copy still in flight land before the CTA's shared memory goes away
      for (int s = s_abort; s < issued; ++s)
        mbar_wait_bounded(&mbar[s % NS], (uint32_t)((s / NS) & 1));
    }
    return false;
  }

  // ---- epilogue: series + exact moments
#pragma unroll
  for (int q = 0; q < kTPW; ++q) {
    const int t = warp + W * q;
    if (t < ntr) {
      int32_t* yr = a.y + (int64_t)(trial0 + t) * a.y_stride;
      unsigned long long s1 = 0, lo = 0, hi = 0;
      const bool store = !FUSED || f->keep_series;
#pragma unroll
      for (int k = 0; k < KP; ++k) {
        const int64_t j = j0 + 2 * (lane + 32 * k);
        if (!store) {
        } else if (j + 1 < a.nout) {
          *reinterpret_cast<int2*>(yr + j) = make_int2((int32_t)acc[q][2 * k],
                                                       (int32_t)acc[q][2 * k + 1]);
        } else if (j < a.nout) {
          yr[j] = (int32_t)acc[q][2 * k];
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          if (j + h < a.nout) {
            const uint32_t v = acc[q][2 * k + h];
            s1 += v;
            const unsigned long long sq = (unsigned long long)v * v;
            lo += sq;
            hi += (lo < sq) ? 1ull : 0ull;
          }
        }
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        s1 += __shfl_xor_sync(0xffffffffu, s1, off);
        const unsigned long long olo = __shfl_xor_sync(0xffffffffu, lo, off);
        const unsigned long long ohi = __shfl_xor_sync(0xffffffffu, hi, off);
        const unsigned long long nlo = lo + olo;
        hi = hi + ohi + (nlo < lo ? 1ull : 0ull);
        lo = nlo;
      }
      if (lane == 0) {
        Moments* m = a.mom + trial0 + t;
        atomicAdd(&m->s1, s1);
        const unsigned long long old = atomicAdd(&m->s2lo, lo);
        atomicAdd(&m->s2hi, hi + ((old + lo < old) ? 1ull : 0ull));
      }
    }
  }
  if constexpr (FUSED)
    fused_search<TT, W, kTPW, KT>(a, *f, acc, smem, bx, by, first, trial0, ntr, j0, warp, lane);
  return true;
}

// One launch per range: CTA (x, y) runs trial tile x, time tile y.
template <typename T, int TT, int NS, int D, int NT>
__global__ void __launch_bounds__(NT, tile_ctas(D, TT, NT))
    k_dedisp_tiled(const __grid_constant__ TiledArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];  // tensor copies land 128-aligned
  tile_body<T, TT, NS, D, NT>(a, blockIdx.x, blockIdx.y, smem, false);
}

// Persistent form: one CTA per SM takes tiles from a device work list that spans many ranges of
// many plans (beams), until the list is exhausted. Segment k of the list holds every tile of
// descriptor seg_desc[k] (trial tiles fastest, as the per-range grid orders them), items
// seg_first[k] .. seg_first[k + 1] - 1. The shared-memory arrangement of each tile follows its
// own descriptor; the launch provides the largest any descriptor needs.
template <typename T, int TT, int NS, int D, int NT>
__global__ void __launch_bounds__(NT, 1) k_dedisp_persistent(const __grid_constant__ PersistArgs p) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ long long item_s;
  const int64_t total = p.seg_first[p.nseg];
  bool reuse = false;
  for (;;) {
    if (threadIdx.x == 0) item_s = (long long)atomicAdd(p.counter, 1ull);
    __syncthreads();
    const int64_t item = item_s;
    if (item >= total) break;  // uniform
    int lo = 0, hi = p.nseg - 1;  // the segment holding the item
    while (lo < hi) {
      const int mid = (lo + hi + 1) / 2;
      if (p.seg_first[mid] <= item) lo = mid; else hi = mid - 1;
    }
    const TiledArgs& a = p.descs[p.seg_desc[lo]];
    // the tensor map was written to global memory by a copy: acquire it for the tensor proxy
    // before the tile's first copy uses it
    if (threadIdx.x == NT - 32)
      asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(&a.rows)
                   : "memory");
    const int64_t local = item - p.seg_first[lo];
    const int ntx = (a.n_trials + D - 1) / D;
    if (!tile_body<T, TT, NS, D, NT>(a, (int)(local % ntx), (int)(local / ntx), smem, reuse))
      break;  // a bounded wait ran out (uniform): the error bit is set
    reuse = true;
  }
}

// Fused form: CTA (x, y) runs trial tile x over time tiles y * seg_tiles .. (y + 1) * seg_tiles
// - 1 in order, each tile's search reading the previous tile's prefix sums (FusedArgs).
template <typename T, int NS>
__global__ void __launch_bounds__(512, 1)
    k_dedisp_fused(const __grid_constant__ TiledArgs a, const __grid_constant__ FusedArgs f) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int ntt = (int)((a.nout + 511) / 512);
  const int y0 = blockIdx.y * f.seg_tiles, y1 = min(ntt, y0 + f.seg_tiles);
  for (int y = y0; y < y1; ++y)
    if (!tile_body<T, 512, NS, 64, 512, true>(a, blockIdx.x, y, smem, y > y0, &f, y == y0))
      break;  // a bounded wait ran out (uniform): the error bit is set
}

template <typename T, int TT, int NS, int D, int NT>
cudaError_t launch_tiled_t(const TiledArgs& a, cudaStream_t st) {
  const SmemLayout SL = smem_layout(sizeof(T), 4, a.row_slot, a.zcap, NS);
  dim3 grid((unsigned)((a.n_trials + D - 1) / D), (unsigned)((a.nout + TT - 1) / TT));
  k_dedisp_tiled<T, TT, NS, D, NT><<<grid, NT, SL.total, st>>>(a);
  return cudaGetLastError();
}

// Ranges sharing an instance need different amounts of shared memory, so the instance is
// allowed the device's opt-in maximum once (a launch still only reserves what it asks for).
template <typename T, int TT, int NS, int D, int NT>
cudaError_t prepare_t(size_t smem) {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  if (smem > (size_t)optin) return cudaErrorInvalidValue;
  e = cudaFuncSetAttribute(k_dedisp_tiled<T, TT, NS, D, NT>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
  // the whole unified L1 as shared memory, so that two CTAs of a two-CTA shape fit an SM
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_dedisp_tiled<T, TT, NS, D, NT>,
                             cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
  return e;
}

}  // namespace

namespace {

// Cut a stage's classes into blocks of B units (U pair words each; B = 31 for uint8 data, 32
// for uint16: Word<T>::kBlock) and deal them to the warps in contiguous shares of
// ceil(blocks / warps); false if a share needs more ranges than a warp's list holds or a class
// more blocks than a range can name.
bool deal_work(StageTab& st, int U, int B) {
  int total = 0;
  for (int gl = 0; gl < kNG; ++gl)
    for (int p = 0; p < st.g[gl].ncls; ++p) total += (st.g[gl].cls[p].zlen / U + B - 1) / B;
  const int share = (total + kWarps - 1) / kWarps;
  int w = 0, used = 0;
  for (int gl = 0; gl < kNG; ++gl)
    for (int p = 0; p < st.g[gl].ncls; ++p) {
      const int nb = (st.g[gl].cls[p].zlen / U + B - 1) / B;
      if (nb > 255) return false;
      int b = 0;
      while (b < nb) {
        const int take = std::min(nb - b, share - used);
        if (w >= kWarps || st.nwork[w] >= kMaxWork) return false;
        st.work[w][st.nwork[w]++] =
            (uint32_t)(gl << 4 | p) | (uint32_t)b << 8 | (uint32_t)take << 16;
        b += take;
        used += take;
        if (used == share) {
          ++w;
          used = 0;
        }
      }
    }
  return true;
}

// Self-test of the bounded wait above: one thread arms a fresh mbarrier that nothing ever
// completes and waits on it; when the bound runs out it records the error bit, as the tiled
// kernel does for a copy that never lands.
__global__ void k_wait_selftest(int32_t* err) {
  __shared__ unsigned long long bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (!mbar_wait_bounded(&bar, 0)) atomicOr(err, 1);
  }
}

}  // namespace

cudaError_t launch_wait_selftest(int32_t* err, cudaStream_t st) {
  k_wait_selftest<<<1, 32, 0, st>>>(err);
  return cudaGetLastError();
}

// Host: the shared-memory work of one row of time tiles, instruction by instruction as
// k_dedisp_tiled issues it (one wavefront per warp-wide access: the kernel's loads and stores are
// free of bank conflicts; a 64-bit store of 32 lanes is two wavefronts). Per (trial tile, stage):
//   accumulation : every warp loads, for its kTPW trials and TT / 64 pair-word columns, one word
//                  per group present (trials past the range's end load too), plus the trials'
//                  zstart entries;
//   build        : per block (31 units for uint8 data, 32 for uint16), 2 row words for each of
//                  the 8 channels and the two plane stores; per work range, its descriptor,
//                  class entry and addressing words;
//   addressing   : two stores per (group, class, channel) entry, by the first 8 warps;
//   copies       : the tensor copy of the 16 staged rows and the bulk copy of the stage table.
static void tiled_smem_work(TiledPlan& P, int ntiles, int nstages, int ngroups, bool u16) {
  const StageTab* tabs = reinterpret_cast<const StageTab*>(P.tabs.data());
  const int W = P.threads / 32, halves = W / kWarps;
  const int KP = P.tt / 64, kTPW = P.trials / W;
  const int sts_per_block = u16 ? 2 : 4;
  int64_t lsu = 0, bytes = 0;
  for (int ti = 0; ti < ntiles; ++ti)
    for (int s = 0; s < nstages; ++s) {
      const StageTab& st = tabs[(size_t)ti * nstages + s];
      const int ng = std::min(kNG, ngroups - s * kNG);
      lsu += (int64_t)W * kTPW * KP * ng;             // accumulation words
      lsu += (int64_t)W * ng;                         // zstart entries (one load per group)
      lsu += W;                                       // nwork
      for (int w = 0; w < kWarps; ++w)
        for (int k = 0; k < st.nwork[w]; ++k) {
          const uint32_t wk = st.work[w][k];
          const int nb = (int)(wk >> 16);
          lsu += 5 * halves;                          // descriptor, zlen, zoff, addr, shift
          lsu += (int64_t)nb * (2 * kG + sts_per_block);
        }
      lsu += (int64_t)(kAddrEntries / 32) * 2;        // addressing stores
      bytes += (int64_t)kRows * P.row_slot * (u16 ? 2 : 1) + (int64_t)sizeof(StageTab);
    }
  P.lsu_wavefronts = lsu;
  P.copy_bytes = bytes;
}

// Host: delay classes of every (trial tile, stage) of one range, as the kernel reads them.
// Classes are numbered in order of their first trial; a class's zlen pair words start at a
// multiple of 4 within the stage, groups one after another, the even plane (pair words 0, 2,
// 4, ...) in the first zlen / 2 words and the odd plane after it. A trial whose sequence starts
// o words into its class reads plane (o mod 2) from word o / 2 on. Fails (ok = false) where the
// kernel's limits do not hold: a 16-bit lane holds the sum of two groups' eight channels of
// values up to 255 x decimation, so decimation must stay at or below 16; delays must be
// monotone in the trial within a channel; classes, work lists and the staged rows must fit
// their fixed-size tables and shared memory.
TiledPlan tiled_plan(const int32_t* tab, int ntr, int cpad, int decimation, int tt, int D,
                     int nt) {
  TiledPlan P;
  P.ok = false;
  const bool u16 = decimation > 1;
  if (decimation < 1 || kRows * 255 * decimation > 65535 || cpad % kG) return P;
  if ((D != 64 && D != 32) || (tt != 512 && tt != 256) || (nt != 512 && nt != 1024)) return P;
  const int NG = kNG, U = u16 ? 2 : 4;
  const int ngroups = cpad / kG, nstages = (ngroups + NG - 1) / NG;
  const int ntiles = (ntr + D - 1) / D;
  int64_t spread = 0, zcap = 0, span = 0;
  std::vector<StageTab> out((size_t)ntiles * nstages);
  for (int ti = 0; ti < ntiles; ++ti) {
    const int t0 = ti * D, n = std::min(D, ntr - t0);
    for (int c = 0; c < cpad; ++c) {
      for (int i = 1; i < n; ++i)
        if (tab[(int64_t)(t0 + i) * cpad + c] < tab[(int64_t)(t0 + i - 1) * cpad + c]) return P;
      spread = std::max<int64_t>(spread, tab[(int64_t)(t0 + n - 1) * cpad + c] -
                                             tab[(int64_t)t0 * cpad + c]);
    }
    for (int s = 0; s < nstages; ++s) {
      StageTab& st = out[(size_t)ti * nstages + s];
      std::memset(&st, 0, sizeof st);
      // the rows' common copy window: from the smallest first-trial delay to the largest
      // last-trial delay of the stage's channels
      int32_t xmin = INT32_MAX, xmax = 0;
      for (int c = s * kRows; c < std::min(cpad, (s + 1) * kRows); ++c) {
        xmin = std::min(xmin, tab[(int64_t)t0 * cpad + c]);
        xmax = std::max(xmax, tab[(int64_t)(t0 + n - 1) * cpad + c]);
      }
      st.xmin = xmin;
      span = std::max<int64_t>(span, (int64_t)xmax - xmin);
      int words = 0;
      for (int gl = 0; gl < NG && s * NG + gl < ngroups; ++gl) {
        const int g = s * NG + gl;
        GroupTab& gt = st.g[gl];
        const int32_t* first = tab + (int64_t)t0 * cpad + kG * g;
        int b[kMaxTileTrials], cls_of[kMaxTileTrials];
        int32_t ckey[kMaxCls][kG];
        int cmin[kMaxCls], cmax[kMaxCls];
        int ncls = 0;
        for (int i = 0; i < n; ++i) {
          const int32_t* sv = tab + (int64_t)(t0 + i) * cpad + kG * g;
          b[i] = *std::min_element(sv, sv + kG);
          int32_t key[kG];
          for (int q = 0; q < kG; ++q) {
            const int64_t r = (int64_t)sv[q] - b[i];
            if (r > 32767) return P;
            key[q] = (int32_t)r;
          }
          int p = 0;
          while (p < ncls && !std::equal(key, key + kG, ckey[p])) ++p;
          if (p == ncls) {
            if (ncls == kMaxCls) return P;
            std::copy(key, key + kG, ckey[ncls]);
            cmin[ncls] = cmax[ncls] = b[i];
            ++ncls;
          } else {
            cmin[p] = std::min(cmin[p], b[i]);
            cmax[p] = std::max(cmax[p], b[i]);
          }
          cls_of[i] = p;
        }
        int zoff[kMaxCls], zlens[kMaxCls];
        for (int p = 0; p < ncls; ++p) {
          const int zlen = (tt + cmax[p] - cmin[p] + 3) & ~3;
          zoff[p] = words;
          ClsEntry& e = gt.cls[p];
          for (int q = 0; q < kG; ++q) {
            const int64_t rel = (int64_t)cmin[p] + ckey[p][q] - first[q];
            if (rel < 0 || rel > 32767) return P;
            e.rel[q] = (int16_t)rel;
          }
          e.zoff = (int16_t)words;
          e.zlen = (int16_t)zlen;
          zlens[p] = zlen;
          words += zlen;
          if (words > 32767) return P;
        }
        for (int i = 0; i < n; ++i) {
          const int p = cls_of[i], o = b[i] - cmin[p];
          gt.zstart[trial_slot(i, nt / 32, D / (nt / 32))] =
              (int16_t)(zoff[p] + (o % 2) * (zlens[p] / 2) + o / 2);
        }
        gt.ncls = ncls;
      }
      if (!deal_work(st, U, u16 ? 32 : 31)) return P;
      zcap = std::max<int64_t>(zcap, words);
    }
  }
  if (spread > 65536) return P;
  const int SEG = kSegBytes / (u16 ? 2 : 1);
  P.tt = tt;
  P.trials = D;
  P.threads = nt;
  P.ctas = tile_ctas(D, tt, nt);
  // staged row: the stage's window (span + tt samples) from up to SEG - 1 samples into its
  // first segment, and 32 samples the word-wise build may read past the last word it uses
  P.nseg = (int)((span + tt + 32 + 2 * SEG - 2) / SEG);
  if (P.nseg > 255) return P;
  P.row_slot = P.nseg * SEG;
  P.zcap = (int)((std::max<int64_t>(zcap, 4) + 3) / 4 * 4);
  P.tab_bytes = out.size() * sizeof(StageTab);
  P.tabs.resize(P.tab_bytes);
  std::memcpy(P.tabs.data(), out.data(), P.tab_bytes);
  // addressing entries hold byte offsets within a stage buffer as uint16
  if ((size_t)kRows * P.row_slot * (u16 ? 2 : 1) > 65535) return P;
  // as many staging buffers as fit (4, else 3: a copy is then issued two stages ahead)
  const size_t limit = P.ctas == 2 ? kSmemLimit2 : kSmemLimit;
  for (int nst = kMaxNStage; nst >= 3 && !P.ok; --nst) {
    P.nstage = nst;
    P.smem = smem_layout(u16 ? 2 : 1, 4, P.row_slot, P.zcap, nst).total;
    P.ok = P.smem <= limit;
  }
  if (P.ok) tiled_smem_work(P, ntiles, nstages, ngroups, u16);
  return P;
}

// Instances: uint8/uint16 data x 4/3 staging buffers x the tile shapes (outputs, trials,
// threads): 512 x 64 with 512 or 1024 threads, 256 x 64 and 256 x 32 with 512.
#define DD_TILED_SHAPES(X, T, U16)                                                  \
  X(T, U16, 512, 4, 64, 512) X(T, U16, 512, 3, 64, 512) X(T, U16, 512, 4, 64, 1024) \
  X(T, U16, 512, 3, 64, 1024) X(T, U16, 256, 4, 64, 512) X(T, U16, 256, 3, 64, 512) \
  X(T, U16, 256, 4, 32, 512) X(T, U16, 256, 3, 32, 512)
#define DD_TILED_INSTANCES(X) DD_TILED_SHAPES(X, uint8_t, 0) DD_TILED_SHAPES(X, uint16_t, 1)
// The persistent form exists for the 64 x 512 tile with 16 warps (the shape every plan measured
// so far runs fastest on).
#define DD_PERSIST_INSTANCES(X)                                                   \
  X(uint8_t, 0, 512, 4, 64, 512) X(uint8_t, 0, 512, 3, 64, 512)                   \
  X(uint16_t, 1, 512, 4, 64, 512) X(uint16_t, 1, 512, 3, 64, 512)

// Host: plan one range and verify the tables against the delay table they were built from,
// independently of how they were built. Returns the number of violations of:
//   - every trial's tt / 2 pair words lie inside one plane of its class, and the class word
//     they stand for (o = 2 x plane position + plane) adds, in every channel of the group, the
//     sample at the trial's own delay (rel + o);
//   - class word ranges start and end on 16-byte boundaries;
//   - the stage's copy start is the smallest first-trial delay of its rows, and every read of
//     every trial stays inside the staged row;
//   - the build work lists cover every block (31 units for uint8 data, 32 for uint16) of every
//     class exactly once.
int64_t tiled_plan_check(const int32_t* tab, int ntr, int cpad, int decimation, int tt, int D,
                         int* ok) {
  const TiledPlan P = tiled_plan(tab, ntr, cpad, decimation, tt, D, kThreads);
  *ok = P.ok ? 1 : 0;
  if (!P.ok) return 0;
  const bool u16 = decimation > 1;
  const int U = u16 ? 2 : 4, SEG = kSegBytes / (u16 ? 2 : 1), B = u16 ? 32 : 31;
  const int ngroups = cpad / kG, nstages = (ngroups + kNG - 1) / kNG;
  const int ntiles = (ntr + D - 1) / D;
  const StageTab* tabs = reinterpret_cast<const StageTab*>(P.tabs.data());
  int64_t bad = 0;
  for (int ti = 0; ti < ntiles; ++ti) {
    const int t0 = ti * D, n = std::min(D, ntr - t0);
    for (int s = 0; s < nstages; ++s) {
      const StageTab& st = tabs[(size_t)ti * nstages + s];
      int32_t xmin = INT32_MAX;
      for (int c = s * kRows; c < std::min(cpad, (s + 1) * kRows); ++c)
        xmin = std::min(xmin, tab[(int64_t)t0 * cpad + c]);
      bad += st.xmin != xmin;
      for (int t = t0; t < t0 + n; ++t)
        for (int c = s * kRows; c < std::min(cpad, (s + 1) * kRows); ++c)
          bad += (int64_t)tab[(int64_t)t * cpad + c] - xmin + tt + 32 + SEG - 1 > P.row_slot;
      std::vector<int> covered;  // blocks of every (group, class), in order
      std::vector<int> first_block(kNG * kMaxCls + 1, 0);
      for (int gl = 0; gl < kNG; ++gl)
        for (int p = 0; p < kMaxCls; ++p) {
          const int nb = p < st.g[gl].ncls ? (st.g[gl].cls[p].zlen / U + B - 1) / B : 0;
          first_block[gl * kMaxCls + p + 1] = first_block[gl * kMaxCls + p] + nb;
        }
      covered.assign(first_block.back(), 0);
      for (int w = 0; w < kWarps; ++w)
        for (int k = 0; k < st.nwork[w]; ++k) {
          const uint32_t wk = st.work[w][k];
          const int gl = (int)((wk >> 4) & 1), p = (int)(wk & 15);
          const int b0 = (int)((wk >> 8) & 255), nb = (int)(wk >> 16);
          for (int b = b0; b < b0 + nb; ++b) {
            const int idx = first_block[gl * kMaxCls + p] + b;
            if (p >= st.g[gl].ncls || idx >= first_block[gl * kMaxCls + p + 1]) {
              ++bad;
            } else {
              ++covered[idx];
            }
          }
        }
      for (int v : covered) bad += v != 1;
      for (int gl = 0; gl < kNG && s * kNG + gl < ngroups; ++gl) {
        const GroupTab& gt = st.g[gl];
        const int c0 = (s * kNG + gl) * kG;
        for (int p = 0; p < gt.ncls; ++p) bad += (gt.cls[p].zoff % 4) + (gt.cls[p].zlen % 4) != 0;
        for (int i = 0; i < n; ++i) {
          const int z = gt.zstart[trial_slot(i, kWarps, D / kWarps)];
          int p = 0, o = -1;
          for (; p < gt.ncls; ++p) {
            const int zo = gt.cls[p].zoff, half = gt.cls[p].zlen / 2;
            if (zo <= z && z + tt / 2 <= zo + half) {
              o = 2 * (z - zo);  // even plane
              break;
            }
            if (zo + half <= z && z + tt / 2 <= zo + 2 * half) {
              o = 2 * (z - zo - half) + 1;  // odd plane
              break;
            }
          }
          if (p == gt.ncls) {
            ++bad;
            continue;
          }
          for (int q = 0; q < kG; ++q) {
            const int64_t want = (int64_t)tab[(int64_t)(t0 + i) * cpad + c0 + q] -
                                 tab[(int64_t)t0 * cpad + c0 + q];
            bad += (int64_t)gt.cls[p].rel[q] + o != want;
          }
        }
      }
    }
  }
  return bad;
}

size_t tiled_smem_bytes(int is_u16, int row_slot, int zcap, int nstage) {
  return smem_layout(is_u16 ? 2 : 1, 4, row_slot, zcap, nstage).total;
}

cudaError_t launch_tiled_persistent(const PersistArgs& p, int is_u16, int tt, int nstage, int D,
                                    int nt, size_t smem, int ctas, cudaStream_t st) {
  if (p.nseg <= 0 || ctas <= 0) return cudaSuccess;
#define DD_PERSIST(T, U16, TT, NS, DT, NTH)                                     \
  if (is_u16 == U16 && tt == TT && nstage == NS && D == DT && nt == NTH) {       \
    cudaError_t e = cudaFuncSetAttribute(k_dedisp_persistent<T, TT, NS, DT, NTH>, \
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                         (int)smem);                            \
    if (e != cudaSuccess) return e;                                             \
    k_dedisp_persistent<T, TT, NS, DT, NTH><<<ctas, NTH, smem, st>>>(p);        \
    return cudaGetLastError();                                                  \
  }
  DD_PERSIST_INSTANCES(DD_PERSIST)
#undef DD_PERSIST
  return cudaErrorInvalidValue;
}

cudaError_t prepare_tiled(int is_u16, int tt, int nstage, int D, int nt, size_t smem) {
#define DD_PREPARE(T, U16, TT, NS, DT, NTH)                                     \
  if (is_u16 == U16 && tt == TT && nstage == NS && D == DT && nt == NTH) \
    return prepare_t<T, TT, NS, DT, NTH>(smem);
  DD_TILED_INSTANCES(DD_PREPARE)
#undef DD_PREPARE
  return cudaErrorInvalidValue;
}

namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

}  // namespace

cudaError_t make_ring_map(CUtensorMap* map, const void* ring, int is_u16, int64_t stride,
                          int32_t cpad, int nseg) {
  const int es = is_u16 ? 2 : 1;
  const int64_t seg = kSegBytes / es;
  if ((stride * es) % kSegBytes || nseg < 1 || nseg > 255 || cpad < 1 ||
      (reinterpret_cast<uintptr_t>(ring) & 15))
    return cudaErrorInvalidValue;
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  const cuuint64_t dims[3] = {(cuuint64_t)seg, (cuuint64_t)(stride / seg), (cuuint64_t)cpad};
  const cuuint64_t strides[2] = {(cuuint64_t)kSegBytes, (cuuint64_t)(stride * es)};
  const cuuint32_t box[3] = {(cuuint32_t)seg, (cuuint32_t)nseg, (cuuint32_t)kRows};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r =
      fn(map, is_u16 ? CU_TENSOR_MAP_DATA_TYPE_UINT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8, 3,
         const_cast<void*>(ring), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
         CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

bool fused_smem(int is_u16, int row_slot, int zcap, int nstage, int hp, int32_t* e_off,
                size_t* smem) {
  const SmemLayout L = smem_layout(is_u16 ? 2 : 1, 4, row_slot, zcap, nstage);
  const size_t rows = (size_t)kWarps * (hp + 512) * sizeof(uint32_t);
  size_t total = L.total, off = L.raw;
  if (L.tab - L.raw < rows) {  // the staging area is too small: the rows go after it
    off = L.total;
    total = L.total + rows;
  }
  if (total > kSmemLimit) return false;
  *e_off = (int32_t)off;
  *smem = total;
  return true;
}

namespace {

template <typename T, int NS>
cudaError_t prepare_fused_t() {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_dedisp_fused<T, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             optin);
  return e;
}

}  // namespace

cudaError_t prepare_fused(int is_u16, int nstage, size_t smem) {
  if (smem > kSmemLimit) return cudaErrorInvalidValue;
  const cudaError_t e = cudaFuncSetAttribute(k_fused_edges,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)((512 / 32) * 2 * 512 * sizeof(uint32_t)));
  if (e != cudaSuccess) return e;
  if (!is_u16 && nstage == 4) return prepare_fused_t<uint8_t, 4>();
  if (!is_u16 && nstage == 3) return prepare_fused_t<uint8_t, 3>();
  if (is_u16 && nstage == 4) return prepare_fused_t<uint16_t, 4>();
  if (is_u16 && nstage == 3) return prepare_fused_t<uint16_t, 3>();
  return cudaErrorInvalidValue;
}

int fused_segments(int ntx, int ntt, int sms, int smax) {
  int best = 1;
  int64_t best_cost = -1;
  for (int s = 1; s <= std::min(ntt, std::max(1, smax)); ++s) {
    const int seg = (ntt + s - 1) / s;
    const int used = (ntt + seg - 1) / seg;  // segments that get tiles
    const int64_t waves = ((int64_t)ntx * used + sms - 1) / sms;
    const int64_t cost = waves * seg;
    if (best_cost < 0 || cost < best_cost) {
      best_cost = cost;
      best = used;
    }
  }
  return best;
}

cudaError_t launch_fused(const TiledArgs& a, const FusedArgs& f, int is_u16, size_t smem,
                         cudaStream_t st) {
  if (a.nout <= 0 || a.n_trials <= 0) return cudaSuccess;
  const int ntx = (a.n_trials + kMaxTileTrials - 1) / kMaxTileTrials;
  const int ntt = (int)((a.nout + 511) / 512);
  if (f.nsegs < 1 || (int64_t)f.nsegs * f.seg_tiles < ntt ||
      (int64_t)(f.nsegs - 1) * f.seg_tiles >= ntt || f.hist < 1 || f.hist > 512 ||
      f.hp < f.hist || f.nw < 1 || f.wd[f.nw - 1] != f.hist)
    return cudaErrorInvalidValue;
  const dim3 grid((unsigned)ntx, (unsigned)f.nsegs);
  if (!is_u16 && a.nstage == 4) k_dedisp_fused<uint8_t, 4><<<grid, 512, smem, st>>>(a, f);
  else if (!is_u16 && a.nstage == 3) k_dedisp_fused<uint8_t, 3><<<grid, 512, smem, st>>>(a, f);
  else if (is_u16 && a.nstage == 4) k_dedisp_fused<uint16_t, 4><<<grid, 512, smem, st>>>(a, f);
  else if (is_u16 && a.nstage == 3) k_dedisp_fused<uint16_t, 3><<<grid, 512, smem, st>>>(a, f);
  else return cudaErrorInvalidValue;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || f.nsegs < 2) return e;
  const size_t esmem = (size_t)(512 / 32) * 2 * f.hist * sizeof(uint32_t);
  k_fused_edges<<<dim3((unsigned)ntx * 4, (unsigned)(f.nsegs - 1)), 512, esmem, st>>>(a, f);
  return cudaGetLastError();
}

cudaError_t launch_tiled(const TiledArgs& a, int is_u16, int tt, int D, int nt,
                         cudaStream_t st) {
  if (a.nout <= 0 || a.n_trials <= 0) return cudaSuccess;
#define DD_LAUNCH(T, U16, TT, NS, DT, NTH)                                        \
  if (is_u16 == U16 && tt == TT && a.nstage == NS && D == DT && nt == NTH) \
    return launch_tiled_t<T, TT, NS, DT, NTH>(a, st);
  DD_TILED_INSTANCES(DD_LAUNCH)
#undef DD_LAUNCH
  return cudaErrorInvalidValue;
}

}  // namespace ddk
