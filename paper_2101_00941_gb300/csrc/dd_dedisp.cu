// Tiled brute-force dedispersion for sm_103a (Sec. 2.1 "dedispersion of data"; the sum is the
// plain definition y[i][j] = sum_c x_d[c][j + s[i][c]], computed exactly in integers).
//
// One CTA (16 warps) owns a tile of kTileTrials consecutive DM trials x TT output samples of one
// range and walks the channels in stages of kNG groups of eight channels.
//
//   * Delay classes. For an 8-channel group the tile's trials fall into a few classes by the
//     relative delays (r0..r7) of the eight channels. A class shares one "pattern word" sequence
//        Z_p[u] = (x[c0][a+u+r0] + .. + x[c3][a+u+r3]) | (x[c4][a+u+r4] + .. + x[c7][..]) << 16
//     -- two 16-bit lanes, each the exact sum of four channels (4 x 255 x d < 2^16 for d <= 64)
//     -- that each of its trials reads at its own base offset. The classes depend on the delay
//     table only, so the plan computes them once (tiled_plan, below) as one fixed-size table per
//     (trial tile, stage); the kernel never searches for them.
//   * TMA (cp.async.bulk) brings each stage's 16 channel rows and its class table into shared
//     memory kNStage stages ahead; completion is tracked by mbarriers with bounded waits.
//   * The main loop adds one pattern word per (trial, sample) with one DP2A: one 32-bit
//     shared-memory load per eight channel-adds, for uint8 and uint16 (decimated) data alike.
//
// Software pipeline, one __syncthreads per stage s:
//     TMA for stage s+kNStage-1 | build the words of stage s+1 | accumulate stage s
// Words are built from aligned 32-bit loads and funnel shifts; the four-channel sums are formed
// in SWAR lanes (bytes split into 16-bit lanes for uint8 data). Exact moments (S1, 128-bit S2)
// of every series are added in the epilogue with integer atomics, so the search needs no second
// statistics pass.
#include <algorithm>
#include <cstring>

#include "dd_internal.h"

namespace ddk {

namespace {

constexpr int kTileTrials = 64;
constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;
constexpr int kTPW = kTileTrials / kWarps;  // trials per warp
constexpr int kG = 8;                       // channels per group (one pattern word)
constexpr int kNG = 2;                      // groups per stage
constexpr int kRows = kG * kNG;             // channel rows per stage
constexpr int kNStage = 4;                  // staging buffers (rows + class table)
constexpr int kMaxCls = 16;                 // classes per group
constexpr int kMaxItems = 64;               // build items (64 units of one class) per group

// One delay class: its channels' first staged sample relative to the tile's first trial
// (rel), and its words in the stage's pattern-word region.
struct ClsEntry {
  int16_t rel[kG];
  int16_t zoff;  // first word (multiple of 4)
  int16_t zlen;  // words (multiple of 4)
  int32_t pad;
};

struct GroupTab {
  int16_t zstart[kTileTrials];  // stage word offset of each trial's sequence (0 for no trial)
  ClsEntry cls[kMaxCls];
  uint16_t item[kMaxItems];     // class << 8 | segment of 64 units
  int32_t ncls, nitem, pad0, pad1;
};

struct StageTab {
  GroupTab g[kNG];
};
static_assert(sizeof(StageTab) % 16 == 0, "class tables are copied in 16-byte units");

__host__ __device__ constexpr size_t align16(size_t v) { return (v + 15) & ~size_t(15); }

struct SmemLayout {
  size_t raw, z, tab, phase, mbar, total;
};

__host__ __device__ inline SmemLayout smem_layout(int es, int zes, int row_slot, int zcap) {
  SmemLayout L;
  size_t off = 0;
  L.raw = off;
  off = align16(off + (size_t)kNStage * kRows * row_slot * es);
  L.z = off;
  off = align16(off + (size_t)2 * zcap * zes);
  L.tab = off;
  off = align16(off + sizeof(StageTab) * kNStage);
  L.phase = off;
  off = align16(off + sizeof(int32_t) * kNStage * kRows);
  L.mbar = off;
  off = align16(off + sizeof(unsigned long long) * kNStage);
  L.total = off;
  return L;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
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

// Warp-cooperative issue of one stage (one warp): lane k < kRows copies channel row k --
// whole 16-byte units covering [m0 + j0 + s_first, m0 + j0 + s_last + TT) -- and records the
// sample's phase within the first unit; lane kRows copies the stage's class table. Lane 0 first
// arms the stage's mbarrier with the total byte count.
template <typename T, int TT>
__device__ void issue_stage(const TiledArgs& a, int stage, int nstages, T* raw_buf,
                            StageTab* tab_buf, int32_t* phase_buf, unsigned long long* bar,
                            int trial0, int ntr, int64_t j0, int lane) {
  constexpr int A = 16 / (int)sizeof(T);  // elements per 16 bytes
  const int c = stage * kRows + lane;
  const bool mine = lane < kRows && c < a.cpad;
  int64_t a0 = 0;
  uint32_t nb = 0;
  if (mine) {
    const int32_t smin = __ldg(a.shifts + (int64_t)trial0 * a.cpad + c);
    const int32_t smax = __ldg(a.shifts + (int64_t)(trial0 + ntr - 1) * a.cpad + c);
    const int64_t start = a.m0 + j0 + smin;
    a0 = start & ~(int64_t)(A - 1);
    const int64_t end = a.m0 + j0 + smax + TT;
    nb = (uint32_t)(((end - a0) * (int64_t)sizeof(T) + 15) & ~int64_t(15));
    phase_buf[lane] = (int32_t)(start - a0);
  }
  if (lane == kRows) nb = (uint32_t)sizeof(StageTab);
  __syncwarp();  // the phases written above are released by lane 0's arrive below
  uint32_t total = nb;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) total += __shfl_xor_sync(0xffffffffu, total, off);
  if (lane == 0) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_arrive_expect_tx(bar, total);
  }
  __syncwarp();
  if (mine)
    bulk_g2s(raw_buf + (size_t)lane * a.row_slot,
             static_cast<const T*>(a.xd) + (int64_t)c * a.xd_stride + a0, nb, bar);
  if (lane == kRows)
    bulk_g2s(tab_buf, a.tabs + ((size_t)blockIdx.x * nstages + stage) * sizeof(StageTab),
             (uint32_t)sizeof(StageTab), bar);
}

template <typename T>
struct Word;

// Row access shared by both data types: for each of the group's eight channels, the row word
// holding the class's sample 0 and the bit phase of that sample in it. A build unit starts on a
// multiple of the samples per row word, so the phase is fixed per class: set once per item.
struct RowItem {
  const uint32_t* rp[kG];
  uint32_t sh[kG];
};

template <int EPW>  // elements per 32-bit row word
__device__ __forceinline__ RowItem row_item(const uint32_t* rows, int row_words, int g,
                                            const int (&col)[kG]) {
  RowItem it;
#pragma unroll
  for (int k = 0; k < kG; ++k) {
    it.rp[k] = rows + (size_t)(kG * g + k) * row_words + col[k] / EPW;
    it.sh[k] = (uint32_t)(col[k] % EPW) * (32u / EPW);
  }
  return it;
}

// uint8 data: a lane builds 8 consecutive pattern words (two units of 4) from three row words
// per channel; bytes are split into even/odd 16-bit lanes so that four channels add without
// carries, then the two four-channel sums of each sample are paired into its word.
template <>
struct Word<uint8_t> {
  static constexpr int kUnit = 4;  // pattern words per unit
  static constexpr int kEPW = 4;
  static __device__ __forceinline__ void sums(const uint32_t (&v)[kG], uint4& out) {
    uint32_t elo = 0, olo = 0, ehi = 0, ohi = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      elo += v[k] & 0x00FF00FFu;             // samples 0, 2
      olo += __byte_perm(v[k], 0, 0x4341);   // samples 1, 3
      ehi += v[k + 4] & 0x00FF00FFu;
      ohi += __byte_perm(v[k + 4], 0, 0x4341);
    }
    out.x = __byte_perm(elo, ehi, 0x5410);  // sample 0: (ch0-3 sum) | (ch4-7 sum) << 16
    out.y = __byte_perm(olo, ohi, 0x5410);  // sample 1
    out.z = __byte_perm(elo, ehi, 0x7632);  // sample 2
    out.w = __byte_perm(olo, ohi, 0x7632);  // sample 3
  }
  // units 2p and 2p + 1 = pattern words 8p .. 8p + 7
  static __device__ __forceinline__ void build2(const RowItem& it, int p, bool second,
                                                uint32_t* dst) {
    uint32_t a[kG], b[kG];
#pragma unroll
    for (int k = 0; k < kG; ++k) {
      const uint32_t w0 = it.rp[k][2 * p], w1 = it.rp[k][2 * p + 1], w2 = it.rp[k][2 * p + 2];
      a[k] = __funnelshift_r(w0, w1, it.sh[k]);
      b[k] = __funnelshift_r(w1, w2, it.sh[k]);
    }
    uint4 o;
    sums(a, o);
    reinterpret_cast<uint4*>(dst)[2 * p] = o;
    if (second) {
      sums(b, o);
      reinterpret_cast<uint4*>(dst)[2 * p + 1] = o;
    }
  }
};

// uint16 data: a lane builds 4 consecutive pattern words (two units of 2): 16-bit lanes add
// four channels without carries (4 x 255 x d < 2^16).
template <>
struct Word<uint16_t> {
  static constexpr int kUnit = 2;
  static constexpr int kEPW = 2;
  // units 2p and 2p + 1 = pattern words 4p .. 4p + 3
  static __device__ __forceinline__ void build2(const RowItem& it, int p, bool second,
                                                uint32_t* dst) {
    uint32_t alo = 0, ahi = 0, blo = 0, bhi = 0;
#pragma unroll
    for (int k = 0; k < kG; ++k) {
      const uint32_t w0 = it.rp[k][2 * p], w1 = it.rp[k][2 * p + 1], w2 = it.rp[k][2 * p + 2];
      const uint32_t a = __funnelshift_r(w0, w1, it.sh[k]);  // samples 0, 1
      const uint32_t b = __funnelshift_r(w1, w2, it.sh[k]);  // samples 2, 3
      if (k < 4) {
        alo += a;
        blo += b;
      } else {
        ahi += a;
        bhi += b;
      }
    }
    uint2 o;
    o.x = __byte_perm(alo, ahi, 0x5410);  // sample 0
    o.y = __byte_perm(alo, ahi, 0x7632);  // sample 1
    reinterpret_cast<uint2*>(dst)[2 * p] = o;
    if (second) {
      o.x = __byte_perm(blo, bhi, 0x5410);  // sample 2
      o.y = __byte_perm(blo, bhi, 0x7632);  // sample 3
      reinterpret_cast<uint2*>(dst)[2 * p + 1] = o;
    }
  }
};

__device__ __forceinline__ uint32_t dot(uint32_t z, uint32_t acc) {
  return __dp2a_lo(z, 0x0101u, acc);  // acc + (ch0-3 sum) + (ch4-7 sum)
}

// Build every pattern word of one stage. The plan cut the work into items of 64 units of one
// class; warp w takes items w, w + kWarps, ... and each lane builds two adjacent units.
template <typename T>
__device__ __forceinline__ void build_stage(const StageTab& tb, int ng, const T* rawb,
                                            const int32_t* phase, int row_slot, uint32_t* Zs,
                                            int warp, int lane) {
  constexpr int U = Word<T>::kUnit;
  const int n0 = tb.g[0].nitem;
  const int n1 = n0 + (ng > 1 ? tb.g[1].nitem : 0);
  const uint32_t* rows = reinterpret_cast<const uint32_t*>(rawb);
  const int row_words = row_slot * (int)sizeof(T) / 4;
  for (int k = warp; k < n1; k += kWarps) {
    const int gi = k >= n0 ? 1 : 0;
    const GroupTab& gt = tb.g[gi];
    const uint32_t itw = gt.item[k - (gi ? n0 : 0)];
    const ClsEntry& e = gt.cls[itw >> 8];
    int col[kG];
#pragma unroll
    for (int q = 0; q < kG; ++q) col[q] = e.rel[q] + phase[kG * gi + q];
    const RowItem it = row_item<Word<T>::kEPW>(rows, row_words, gi, col);
    const int pu = (int)(itw & 255) * 32 + lane;  // unit pair: units 2pu, 2pu + 1
    if (2 * pu * U < e.zlen) Word<T>::build2(it, pu, (2 * pu + 1) * U < e.zlen, Zs + e.zoff);
  }
}

template <typename T, int TT>
__global__ void __launch_bounds__(kThreads, 1) k_dedisp_tiled(const TiledArgs a) {
  constexpr int KT = TT / 32;
  extern __shared__ __align__(16) unsigned char smem[];
  const SmemLayout SL = smem_layout(sizeof(T), 4, a.row_slot, a.zcap);
  T* raw = reinterpret_cast<T*>(smem + SL.raw);
  uint32_t* Zbuf = reinterpret_cast<uint32_t*>(smem + SL.z);
  StageTab* tab = reinterpret_cast<StageTab*>(smem + SL.tab);
  int32_t* phase = reinterpret_cast<int32_t*>(smem + SL.phase);
  unsigned long long* mbar = reinterpret_cast<unsigned long long*>(smem + SL.mbar);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int trial0 = blockIdx.x * kTileTrials;
  const int ntr = min(kTileTrials, a.n_trials - trial0);
  const int64_t j0 = (int64_t)blockIdx.y * TT;
  const int ngroups = a.cpad / kG;
  const int nstages = (ngroups + kNG - 1) / kNG;
  const size_t stage_elems = (size_t)kRows * a.row_slot;

  if (tid == 0) {
    for (int s = 0; s < kNStage; ++s) mbar_init(&mbar[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  // stages whose copies have been issued: kNStage in the prologue, then one per iteration s >= 1
  // (the same count in every thread)
  int issued = min(kNStage, nstages);
  if (warp == kWarps - 1) {
    for (int s = 0; s < kNStage && s < nstages; ++s)
      issue_stage<T, TT>(a, s, nstages, raw + (size_t)s * stage_elems, &tab[s],
                         phase + s * kRows, &mbar[s], trial0, ntr, j0, lane);
  }
  bool ok0 = mbar_wait_bounded(&mbar[0], 0);
  if (ok0) build_stage<T>(tab[0], min(kNG, ngroups), raw, phase, a.row_slot, Zbuf, warp, lane);
  bool aborted = __syncthreads_or(!ok0);
  int s_abort = 0;  // first stage whose copies may still be in flight

  uint32_t acc[kTPW][KT];
#pragma unroll
  for (int q = 0; q < kTPW; ++q)
#pragma unroll
    for (int k = 0; k < KT; ++k) acc[q][k] = 0;

  for (int s = 0; s < nstages && !aborted; ++s) {
    const int ng = min(kNG, ngroups - s * kNG);
    // (1) TMA for stage s + kNStage - 1 into the buffers stage s - 1 used (its words were built
    //     during stage s - 2 and its table last read by the accumulation of stage s - 1)
    if (s >= 1 && s + kNStage - 1 < nstages) {
      const int s2 = s + kNStage - 1;
      const int b2 = s2 % kNStage;
      if (warp == kWarps - 1)
        issue_stage<T, TT>(a, s2, nstages, raw + (size_t)b2 * stage_elems, &tab[b2],
                           phase + b2 * kRows, &mbar[b2], trial0, ntr, j0, lane);
      issued = s2 + 1;
    }
    // (2) pattern words of stage s + 1
    bool ok = true;
    if (s + 1 < nstages) {
      const int b1 = (s + 1) % kNStage;
      ok = mbar_wait_bounded(&mbar[b1], (uint32_t)(((s + 1) / kNStage) & 1));
      if (ok)
        build_stage<T>(tab[b1], min(kNG, ngroups - (s + 1) * kNG), raw + (size_t)b1 * stage_elems,
                       phase + b1 * kRows, a.row_slot, Zbuf + (size_t)((s + 1) & 1) * a.zcap,
                       warp, lane);
    }
    // (3) accumulate stage s
    {
      const StageTab& tc = tab[s % kNStage];
      const uint32_t* Zs = Zbuf + (size_t)(s & 1) * a.zcap + lane;
#pragma unroll
      for (int g = 0; g < kNG; ++g) {
        if (g < ng) {  // uniform; only the last stage may hold fewer groups
          const uint32_t* zp[kTPW];
#pragma unroll
          for (int q = 0; q < kTPW; ++q) zp[q] = Zs + tc.g[g].zstart[warp + kWarps * q];
#pragma unroll
          for (int k = 0; k < KT; ++k)
#pragma unroll
            for (int q = 0; q < kTPW; ++q) acc[q][k] = dot(zp[q][32 * k], acc[q][k]);
        }
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
        mbar_wait_bounded(&mbar[s % kNStage], (uint32_t)((s / kNStage) & 1));
    }
    return;
  }

  // ---- epilogue: series + exact moments
#pragma unroll
  for (int q = 0; q < kTPW; ++q) {
    const int t = warp + kWarps * q;
    if (t < ntr) {
      int32_t* yr = a.y + (int64_t)(trial0 + t) * a.y_stride;
      unsigned long long s1 = 0, lo = 0, hi = 0;
#pragma unroll
      for (int k = 0; k < KT; ++k) {
        const int64_t j = j0 + lane + 32 * k;
        if (j < a.nout) {
          const uint32_t v = acc[q][k];
          yr[j] = (int32_t)v;
          s1 += v;
          const unsigned long long sq = (unsigned long long)v * v;
          lo += sq;
          hi += (lo < sq) ? 1ull : 0ull;
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
}

template <typename T, int TT>
cudaError_t launch_tiled_t(const TiledArgs& a, cudaStream_t st) {
  const SmemLayout SL = smem_layout(sizeof(T), 4, a.row_slot, a.zcap);
  dim3 grid((unsigned)((a.n_trials + kTileTrials - 1) / kTileTrials),
            (unsigned)((a.nout + TT - 1) / TT));
  k_dedisp_tiled<T, TT><<<grid, kThreads, SL.total, st>>>(a);
  return cudaGetLastError();
}

// Ranges sharing an instance need different amounts of shared memory, so the instance is
// allowed the device's opt-in maximum once (a launch still only reserves what it asks for).
template <typename T, int TT>
cudaError_t prepare_t(size_t smem) {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  if (smem > (size_t)optin) return cudaErrorInvalidValue;
  return cudaFuncSetAttribute(k_dedisp_tiled<T, TT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              optin);
}

}  // namespace

int tiled_tile_samples(int is_u16, int choice) {
  // preferred time tile first, a smaller one when the first does not fit shared memory
  if (!is_u16) return choice == 0 ? 512 : 256;
  return choice == 0 ? 256 : 128;
}

// Host: delay classes of every (trial tile, stage) of one range, as the kernel reads them.
// Classes are numbered in order of their first trial; a class's words start at a multiple of 4
// within the stage, groups one after another. Fails (ok = false) where the kernel's limits do
// not hold: a 16-bit lane sums four channels of values up to 255 x decimation, so decimation
// must stay at or below 64; delays must be monotone in the trial within a channel; classes,
// items and the staged rows must fit their fixed-size tables and shared memory.
TiledPlan tiled_plan(const int32_t* tab, int ntr, int cpad, int decimation, int tt) {
  TiledPlan P;
  P.ok = false;
  const bool u16 = decimation > 1;
  if (decimation < 1 || 4 * 255 * decimation > 65535 || cpad % kG) return P;
  const int D = kTileTrials, NG = kNG, U = u16 ? 2 : 4;
  const int ngroups = cpad / kG, nstages = (ngroups + NG - 1) / NG;
  const int ntiles = (ntr + D - 1) / D;
  int64_t spread = 0, zcap = 0;
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
      int words = 0;
      for (int gl = 0; gl < NG && s * NG + gl < ngroups; ++gl) {
        const int g = s * NG + gl;
        GroupTab& gt = st.g[gl];
        const int32_t* first = tab + (int64_t)t0 * cpad + kG * g;
        int b[kTileTrials], cls_of[kTileTrials];
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
        int nitem = 0;
        int zoff[kMaxCls];
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
          // one item = 32 lanes x 2 units
          const int nseg = (zlen / U + 63) / 64;
          for (int q = 0; q < nseg; ++q) {
            if (nitem >= kMaxItems) return P;
            gt.item[nitem++] = (uint16_t)((p << 8) | q);
          }
          words += zlen;
          if (words > 32767) return P;
        }
        for (int i = 0; i < n; ++i)
          gt.zstart[i] = (int16_t)(zoff[cls_of[i]] + b[i] - cmin[cls_of[i]]);
        gt.ncls = ncls;
        gt.nitem = nitem;
      }
      zcap = std::max<int64_t>(zcap, words);
    }
  }
  if (spread > 65536) return P;
  const int A = u16 ? 8 : 16;
  P.tt = tt;
  // staged row: up to A-1 elements of alignment in front, 16-byte rounding behind, and 16
  // elements the word-wise build may read past the last word it uses
  P.row_slot = (int)(((tt + spread + 2 * A + 16) + A - 1) / A * A);
  P.zcap = (int)((std::max<int64_t>(zcap, 4) + 3) / 4 * 4);
  P.smem = smem_layout(u16 ? 2 : 1, 4, P.row_slot, P.zcap).total;
  P.tab_bytes = out.size() * sizeof(StageTab);
  P.tabs.resize(P.tab_bytes);
  std::memcpy(P.tabs.data(), out.data(), P.tab_bytes);
  P.ok = P.smem <= 200 * 1024;
  return P;
}

cudaError_t prepare_tiled(int is_u16, int tt, size_t smem) {
  if (!is_u16 && tt == 512) return prepare_t<uint8_t, 512>(smem);
  if (!is_u16 && tt == 256) return prepare_t<uint8_t, 256>(smem);
  if (is_u16 && tt == 256) return prepare_t<uint16_t, 256>(smem);
  if (is_u16 && tt == 128) return prepare_t<uint16_t, 128>(smem);
  return cudaErrorInvalidValue;
}

cudaError_t launch_tiled(const TiledArgs& a, int is_u16, int tt, cudaStream_t st) {
  if (a.nout <= 0 || a.n_trials <= 0) return cudaSuccess;
  if (!is_u16 && tt == 512) return launch_tiled_t<uint8_t, 512>(a, st);
  if (!is_u16 && tt == 256) return launch_tiled_t<uint8_t, 256>(a, st);
  if (is_u16 && tt == 256) return launch_tiled_t<uint16_t, 256>(a, st);
  if (is_u16 && tt == 128) return launch_tiled_t<uint16_t, 128>(a, st);
  return cudaErrorInvalidValue;
}

}  // namespace ddk
