// Tiled brute-force dedispersion for sm_103a (Sec. 2.1 "dedispersion of data"; the sum is the
// plain definition y[i][j] = sum_c x_d[c][j + s[i][c]], computed exactly in integers).
//
// One CTA (16 warps) owns a tile of kTileTrials consecutive DM trials x TT output samples of one
// range and walks the channels in stages of kNG groups of four channels.
//
//   * TMA (cp.async.bulk) stages the 16 channel rows of a stage into shared memory, kNStage
//     stages ahead; completion is tracked by mbarriers with bounded waits.
//   * For each 4-channel group the tile's trials fall into a few classes by the relative delays
//     (r0, r1, r2, r3) of the four channels (found with __match_any_sync). A class shares one
//     "pattern word" sequence
//        Z_p[u] = x[c0][a + u + r0] | x[c1][a + u + r1] << 8 | x[c2][..] << 16 | x[c3][..] << 24
//     that each of its trials reads at its own base offset b.
//   * The main loop adds one pattern word per (trial, sample): DP4A for uint8 data, two DP2A
//     for uint16 (decimated) data -- one shared-memory load per four channel-adds.
//
// Software pipeline, one __syncthreads per stage s:
//     issue TMA for stage s+kNStage-1 | find classes of stage s+2 | build words of stage s+1 |
//     accumulate stage s
// The words are built four (uint8) or two (uint16) at a time from aligned 32-bit loads,
// funnel shifts and a byte transpose. Exact moments (S1, 128-bit S2) of every series are added
// in the epilogue with integer atomics, so the search needs no second statistics pass.
#include <climits>

#include "dd_internal.h"

namespace ddk {

namespace {

constexpr int kTileTrials = 64;
constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;
constexpr int kTPW = kTileTrials / kWarps;  // trials per warp
constexpr int kNG = 4;                      // 4-channel groups per stage
constexpr int kRows = 4 * kNG;              // channel rows per stage
constexpr int kNStage = 4;                  // raw staging buffers
constexpr int kNTab = 3;                    // class tables in flight (stages s, s+1, s+2)
constexpr int kMaxItems = 128;              // build items (32 units of one class) per group

struct PatEntry {
  int32_t col[4];  // staged element of each channel row for word u = 0
  int32_t zoff;    // first word of the class within its group (multiple of 4)
  int32_t zlen;    // words of the class (multiple of 4)
};

struct StageTab {
  int32_t zstart[kNG][kTileTrials];  // word offset of each trial's sequence within its group
  PatEntry pat[kNG][kTileTrials];
  uint16_t item[kNG][kMaxItems];     // build items: class << 8 | segment of 32 units
  int32_t gtot[kNG];                 // words of each group
  int32_t npat[kNG];
  int32_t nitem[kNG];
};

__host__ __device__ constexpr size_t align16(size_t v) { return (v + 15) & ~size_t(15); }

struct SmemLayout {
  size_t raw, z, tab, mbar, total;
};

__host__ __device__ inline SmemLayout smem_layout(int es, int zes, int row_slot, int zcap) {
  SmemLayout L;
  size_t off = 0;
  L.raw = off;
  off = align16(off + (size_t)kNStage * kRows * row_slot * es);
  L.z = off;
  off = align16(off + (size_t)2 * zcap * zes);
  L.tab = off;
  off = align16(off + sizeof(StageTab) * kNTab);
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

// Delays bounding one stage's channel rows for this tile: lane k < kRows loads the first and the
// last trial's delay of channel stage*kRows + k (delays are non-decreasing in the trial index).
__device__ __forceinline__ void stage_bounds(const TiledArgs& a, int stage, int lane, int trial0,
                                             int ntr, int& smin, int& smax) {
  const int c = stage * kRows + lane;
  smin = smax = 0;
  if (lane < kRows && c < a.c4) {
    smin = __ldg(a.shifts + (int64_t)trial0 * a.c4 + c);
    smax = __ldg(a.shifts + (int64_t)(trial0 + ntr - 1) * a.c4 + c);
  }
}

// Warp-cooperative issue of one stage: lane k copies channel row k with one bulk (TMA) copy of
// whole 16-byte units covering [m0 + j0 + smin, m0 + j0 + smax + TT); lane 0 first arms the
// stage's mbarrier with the total byte count.
template <typename T, int TT>
__device__ void issue_stage(const TiledArgs& a, int stage, T* raw_buf, unsigned long long* bar,
                            int64_t j0, int lane, int smin, int smax) {
  constexpr int A = 16 / (int)sizeof(T);  // elements per 16 bytes
  const int c = stage * kRows + lane;
  const bool mine = lane < kRows && c < a.c4;
  int64_t a0 = 0;
  uint32_t nb = 0;
  if (mine) {
    const int64_t start = a.m0 + j0 + smin;
    a0 = start & ~(int64_t)(A - 1);
    const int64_t end = a.m0 + j0 + smax + TT;
    nb = (uint32_t)(((end - a0) * (int64_t)sizeof(T) + 15) & ~int64_t(15));
  }
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
}

// Classes of one 4-channel group (one warp; lane l holds trials l and l + 32 of the tile).
// `s4[h]` are the delays of the group's four channels for trial l + 32h, `f4` those of the
// tile's first trial. Classes are peeled off one at a time (a handful per group), each loop
// iteration a few warp-wide votes and reductions.
template <typename T, int TT>
__device__ __forceinline__ void find_classes(const TiledArgs& a, StageTab& tb, int g, int lane,
                                             int ntr, int64_t j0, const int4 (&s4)[2], int4 f4) {
  constexpr int A = 16 / (int)sizeof(T);
  unsigned long long key[2];
  int b[2];
  uint32_t rem[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    b[h] = min(min(s4[h].x, s4[h].y), min(s4[h].z, s4[h].w));
    key[h] = (unsigned long long)(uint32_t)(s4[h].x - b[h]) |
             ((unsigned long long)(uint32_t)(s4[h].y - b[h]) << 16) |
             ((unsigned long long)(uint32_t)(s4[h].z - b[h]) << 32) |
             ((unsigned long long)(uint32_t)(s4[h].w - b[h]) << 48);
    rem[h] = __ballot_sync(0xffffffffu, lane + 32 * h < ntr);
  }
#pragma unroll
  for (int h = 0; h < 2; ++h)
    if (lane + 32 * h >= ntr) tb.zstart[g][lane + 32 * h] = 0;  // absent trial: a valid dummy
  constexpr int U = 16 / (int)sizeof(T) / 4;  // pattern words per build unit: 4 (u8), 2 (u16)
  int npat = 0, zoff = 0, nitem = 0;
  while (rem[0] | rem[1]) {
    const int hl = rem[0] ? 0 : 1;
    const int L = __ffs(hl ? rem[1] : rem[0]) - 1;
    const unsigned long long kk = __shfl_sync(0xffffffffu, hl ? key[1] : key[0], L);
    bool in[2];
    int lo = INT_MAX, hi = INT_MIN;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      in[h] = ((rem[h] >> lane) & 1u) && key[h] == kk;
      rem[h] &= ~__ballot_sync(0xffffffffu, in[h]);
      if (in[h]) {
        lo = min(lo, b[h]);
        hi = max(hi, b[h]);
      }
    }
    const int bmin = __reduce_min_sync(0xffffffffu, lo);
    const int bmax = __reduce_max_sync(0xffffffffu, hi);
    const int zlen = (TT + bmax - bmin + 3) & ~3;
#pragma unroll
    for (int h = 0; h < 2; ++h)
      if (in[h]) tb.zstart[g][lane + 32 * h] = zoff + (b[h] - bmin);
    if (lane == 0) {
      const int64_t base = a.m0 + j0 + bmin;
      PatEntry e;
      e.col[0] = (int32_t)(base + (int)(kk & 0xFFFF) - ((a.m0 + j0 + f4.x) & ~(int64_t)(A - 1)));
      e.col[1] = (int32_t)(base + (int)((kk >> 16) & 0xFFFF) -
                           ((a.m0 + j0 + f4.y) & ~(int64_t)(A - 1)));
      e.col[2] = (int32_t)(base + (int)((kk >> 32) & 0xFFFF) -
                           ((a.m0 + j0 + f4.z) & ~(int64_t)(A - 1)));
      e.col[3] = (int32_t)(base + (int)(kk >> 48) - ((a.m0 + j0 + f4.w) & ~(int64_t)(A - 1)));
      e.zoff = zoff;
      e.zlen = zlen;
      tb.pat[g][npat] = e;
    }
    const int nseg = (zlen / U + 31) >> 5;
    for (int q = lane; q < nseg; q += 32)
      if (nitem + q < kMaxItems) tb.item[g][nitem + q] = (uint16_t)((npat << 8) | q);
    nitem += nseg;
    zoff += zlen;
    ++npat;
  }
  if (lane == 0) {
    tb.gtot[g] = zoff;
    tb.npat[g] = npat;
    tb.nitem[g] = nitem;
  }
}

// Delays of one group's four channels for trials lane and lane + 32 of the tile.
__device__ __forceinline__ void load_group_delays(const TiledArgs& a, int trial0, int ntr,
                                                  int gabs, int lane, int4 (&s4)[2]) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    s4[h] = make_int4(0, 0, 0, 0);
    if (lane + 32 * h < ntr)
      s4[h] = __ldg(reinterpret_cast<const int4*>(a.shifts + (int64_t)(trial0 + lane + 32 * h) *
                                                                 a.c4 + 4 * gabs));
  }
}

__device__ __forceinline__ int4 first_trial(int4 s4) {
  return make_int4(__shfl_sync(0xffffffffu, s4.x, 0), __shfl_sync(0xffffffffu, s4.y, 0),
                   __shfl_sync(0xffffffffu, s4.z, 0), __shfl_sync(0xffffffffu, s4.w, 0));
}

template <typename T>
struct Word;

// uint8 data: a unit is four consecutive pattern words. Because a unit starts on a multiple of
// four samples, each channel row is read at a fixed byte phase per class: the row pointer and
// the funnel-shift amount are set once per item.
template <>
struct Word<uint8_t> {
  using Z = uint32_t;
  static constexpr int kUnit = 4;
  struct Item {
    const uint32_t* rp[4];  // row word holding the class's sample 0 of channel k
    uint32_t sh[4];         // bit phase of that sample in the word
  };
  static __device__ __forceinline__ Item item(const uint8_t* rawb, int row_slot, int g,
                                              const PatEntry& e) {
    Item it;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      it.rp[k] = reinterpret_cast<const uint32_t*>(rawb + (size_t)(4 * g + k) * row_slot) +
                 (e.col[k] >> 2);
      it.sh[k] = (uint32_t)(e.col[k] & 3) * 8u;
    }
    return it;
  }
  // unit m = pattern words 4m .. 4m + 3
  static __device__ __forceinline__ void build(const Item& it, int m, Z* dst) {
    uint32_t v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = __funnelshift_r(it.rp[k][m], it.rp[k][m + 1], it.sh[k]);
    // 4x4 byte transpose: word t gets byte t of every channel
    const uint32_t a0 = __byte_perm(v[0], v[1], 0x5140), a1 = __byte_perm(v[0], v[1], 0x7362);
    const uint32_t a2 = __byte_perm(v[2], v[3], 0x5140), a3 = __byte_perm(v[2], v[3], 0x7362);
    uint4 o;
    o.x = __byte_perm(a0, a2, 0x5410);
    o.y = __byte_perm(a0, a2, 0x7632);
    o.z = __byte_perm(a1, a3, 0x5410);
    o.w = __byte_perm(a1, a3, 0x7632);
    reinterpret_cast<uint4*>(dst)[m] = o;
  }
  static __device__ __forceinline__ uint32_t dot(uint32_t z, uint32_t acc) {
    return __dp4a(z, 0x01010101u, acc);
  }
};

// uint16 data: a pattern word is 4 x 16 bits (uint2); a unit is two consecutive words.
template <>
struct Word<uint16_t> {
  using Z = uint2;
  static constexpr int kUnit = 2;
  struct Item {
    const uint32_t* rp[4];
    uint32_t sh[4];
  };
  static __device__ __forceinline__ Item item(const uint16_t* rawb, int row_slot, int g,
                                              const PatEntry& e) {
    Item it;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      it.rp[k] = reinterpret_cast<const uint32_t*>(rawb + (size_t)(4 * g + k) * row_slot) +
                 (e.col[k] >> 1);
      it.sh[k] = (uint32_t)(e.col[k] & 1) * 16u;
    }
    return it;
  }
  // unit m = pattern words 2m, 2m + 1
  static __device__ __forceinline__ void build(const Item& it, int m, Z* dst) {
    uint32_t v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = __funnelshift_r(it.rp[k][m], it.rp[k][m + 1], it.sh[k]);
    uint4 o;
    o.x = __byte_perm(v[0], v[1], 0x5410);  // word 2m:   channels 0,1
    o.y = __byte_perm(v[2], v[3], 0x5410);  //            channels 2,3
    o.z = __byte_perm(v[0], v[1], 0x7632);  // word 2m+1: channels 0,1
    o.w = __byte_perm(v[2], v[3], 0x7632);  //            channels 2,3
    reinterpret_cast<uint4*>(dst)[m] = o;
  }
  static __device__ __forceinline__ uint32_t dot(uint2 z, uint32_t acc) {
    return __dp2a_lo(z.y, 0x0101u, __dp2a_lo(z.x, 0x0101u, acc));
  }
};

// Build every pattern word of one stage. The work is cut into items of 32 units of one class
// (listed by the class search); warps w0 .. kWarps-1 take the items round-robin and each lane
// builds one unit of an item.
template <typename T>
__device__ __forceinline__ void build_stage(const StageTab& tb, int ng, const T* rawb,
                                            int row_slot, typename Word<T>::Z* Zs, int warp,
                                            int lane, int w0) {
  constexpr int U = Word<T>::kUnit;
  if (warp < w0) return;
  int ibeg[kNG + 1], wbeg[kNG];
  ibeg[0] = 0;
  int words = 0;
#pragma unroll
  for (int g = 0; g < kNG; ++g) {
    wbeg[g] = words;
    ibeg[g + 1] = ibeg[g] + (g < ng ? tb.nitem[g] : 0);
    words += (g < ng ? tb.gtot[g] : 0);
  }
  for (int k = warp - w0; k < ibeg[kNG]; k += kWarps - w0) {
    const int gi = (k >= ibeg[1]) + (k >= ibeg[2]) + (k >= ibeg[3]);
    const int kb = gi == 0 ? ibeg[0] : gi == 1 ? ibeg[1] : gi == 2 ? ibeg[2] : ibeg[3];
    const int zb = gi == 0 ? wbeg[0] : gi == 1 ? wbeg[1] : gi == 2 ? wbeg[2] : wbeg[3];
    const uint32_t itw = tb.item[gi][k - kb];
    const PatEntry& e = tb.pat[gi][itw >> 8];
    const typename Word<T>::Item it = Word<T>::item(rawb, row_slot, gi, e);
    const int m = (int)(itw & 255) * 32 + lane;
    if (m * U < e.zlen) Word<T>::build(it, m, Zs + zb + e.zoff);
  }
}

__device__ __forceinline__ int stage_words(const StageTab& tb, int ng) {
  int tot = 0;
#pragma unroll
  for (int g = 0; g < kNG; ++g)
    if (g < ng) tot += tb.gtot[g];
  return tot;
}

template <typename T, int TT>
__global__ void __launch_bounds__(kThreads, 1) k_dedisp_tiled(const TiledArgs a) {
  using ZT = typename Word<T>::Z;
  constexpr int KT = TT / 32;
  extern __shared__ __align__(16) unsigned char smem[];
  const SmemLayout SL = smem_layout(sizeof(T), sizeof(ZT), a.row_slot, a.zcap);
  T* raw = reinterpret_cast<T*>(smem + SL.raw);
  ZT* Zbuf = reinterpret_cast<ZT*>(smem + SL.z);
  StageTab* tab = reinterpret_cast<StageTab*>(smem + SL.tab);
  unsigned long long* mbar = reinterpret_cast<unsigned long long*>(smem + SL.mbar);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int trial0 = blockIdx.x * kTileTrials;
  const int ntr = min(kTileTrials, a.n_trials - trial0);
  const int64_t j0 = (int64_t)blockIdx.y * TT;
  const int ngroups = a.c4 / 4;
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
  if (warp == 0) {
    for (int s = 0; s < kNStage && s < nstages; ++s) {
      int smin, smax;
      stage_bounds(a, s, lane, trial0, ntr, smin, smax);
      issue_stage<T, TT>(a, s, raw + (size_t)s * stage_elems, &mbar[s], j0, lane, smin, smax);
    }
  }
  // classes of stages 0 and 1 (warps 0..kNG-1 and kNG..2kNG-1)
  {
    const int st = warp / kNG, g = warp % kNG;
    if (st < 2 && st < nstages && st * kNG + g < ngroups) {
      int4 s4[2];
      load_group_delays(a, trial0, ntr, st * kNG + g, lane, s4);
      find_classes<T, TT>(a, tab[st], g, lane, ntr, j0, s4, first_trial(s4[0]));
    }
  }
  // delays of the group this warp classifies next (stage 2), loaded one stage ahead
  int4 pre[2] = {make_int4(0, 0, 0, 0), make_int4(0, 0, 0, 0)};
  if (warp < kNG && 2 < nstages && 2 * kNG + warp < ngroups)
    load_group_delays(a, trial0, ntr, 2 * kNG + warp, lane, pre);
  __syncthreads();
  bool ok0 = stage_words(tab[0], min(kNG, ngroups)) <= a.zcap && mbar_wait_bounded(&mbar[0], 0);
  if (ok0) build_stage<T>(tab[0], min(kNG, ngroups), raw, a.row_slot, Zbuf, warp, lane, 0);
  bool aborted = __syncthreads_or(!ok0);
  int s_abort = 0;  // first stage whose copies may still be in flight

  uint32_t acc[kTPW][KT];
#pragma unroll
  for (int q = 0; q < kTPW; ++q)
#pragma unroll
    for (int k = 0; k < KT; ++k) acc[q][k] = 0;

  for (int s = 0; s < nstages && !aborted; ++s) {
    const int ng = min(kNG, ngroups - s * kNG);
    // (1) TMA for stage s + kNStage - 1 into the buffer stage s - 1 used (built during s - 2)
    if (s >= 1 && s + kNStage - 1 < nstages) {
      const int s2 = s + kNStage - 1;
      if (warp == kWarps - 1) {
        int smin, smax;
        stage_bounds(a, s2, lane, trial0, ntr, smin, smax);
        issue_stage<T, TT>(a, s2, raw + (size_t)(s2 % kNStage) * stage_elems,
                           &mbar[s2 % kNStage], j0, lane, smin, smax);
      }
      issued = s2 + 1;
    }
    // (2) classes of stage s + 2
    if (warp < kNG && s + 2 < nstages && (s + 2) * kNG + warp < ngroups) {
      find_classes<T, TT>(a, tab[(s + 2) % kNTab], warp, lane, ntr, j0, pre, first_trial(pre[0]));
      pre[0] = pre[1] = make_int4(0, 0, 0, 0);
      if (s + 3 < nstages && (s + 3) * kNG + warp < ngroups)
        load_group_delays(a, trial0, ntr, (s + 3) * kNG + warp, lane, pre);
    }
    // (3) pattern words of stage s + 1
    bool ok = true;
    if (s + 1 < nstages) {
      const StageTab& tn = tab[(s + 1) % kNTab];
      const int ng1 = min(kNG, ngroups - (s + 1) * kNG);
      ok = stage_words(tn, ng1) <= a.zcap &&
           mbar_wait_bounded(&mbar[(s + 1) % kNStage], (uint32_t)(((s + 1) / kNStage) & 1));
      if (ok)
        build_stage<T>(tn, ng1, raw + (size_t)((s + 1) % kNStage) * stage_elems, a.row_slot,
                       Zbuf + (size_t)((s + 1) & 1) * a.zcap, warp, lane,
                       s + 2 < nstages ? kNG : 0);  // classifying warps sit out
    }
    // (4) accumulate stage s
    {
      const StageTab& tc = tab[s % kNTab];
      const ZT* Zs = Zbuf + (size_t)(s & 1) * a.zcap + lane;
      int gb = 0;
#pragma unroll
      for (int g = 0; g < kNG; ++g) {
        if (g < ng) {  // uniform; only the last stage may hold fewer groups
          const ZT* zp[kTPW];
#pragma unroll
          for (int q = 0; q < kTPW; ++q) zp[q] = Zs + gb + tc.zstart[g][warp + kWarps * q];
#pragma unroll
          for (int k = 0; k < KT; ++k)
#pragma unroll
            for (int q = 0; q < kTPW; ++q) acc[q][k] = Word<T>::dot(zp[q][32 * k], acc[q][k]);
          gb += tc.gtot[g];
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
  using ZT = typename Word<T>::Z;
  const SmemLayout SL = smem_layout(sizeof(T), sizeof(ZT), a.row_slot, a.zcap);
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

int tiled_trials_per_tile() { return kTileTrials; }
int tiled_groups_per_stage() { return kNG; }

size_t tiled_smem_bytes(int is_u16, int row_slot, int zcap) {
  return smem_layout(is_u16 ? 2 : 1, is_u16 ? 8 : 4, row_slot, zcap).total;
}

int tiled_tile_samples(int is_u16, int choice) {
  // preferred time tile first, a smaller one when the first does not fit shared memory
  if (!is_u16) return choice == 0 ? 512 : 256;
  return choice == 0 ? 256 : 128;
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
