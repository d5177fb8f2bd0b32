// Tiled brute-force dedispersion for sm_103a (Sec. 2.1 "dedispersion of data"; the sum is the
// plain definition y[i][j] = sum_c x_d[c][j + s[i][c]], computed exactly in integers).
//
// One CTA owns a tile of kTileTrials consecutive DM trials x TT output samples of one range and
// walks the channels in stages of kNG groups of four channels:
//   1. TMA (cp.async.bulk) stages the 16 channel rows the tile needs into shared memory,
//      kNStage stages deep, completion tracked by mbarriers (bounded waits);
//   2. one warp per 4-channel group finds the distinct relative-delay patterns among the tile's
//      trials (__match_any_sync): trials whose four delays differ from their minimum b by the
//      same (r0, r1, r2, r3) read the same "pattern word" sequence
//        Z_p[u] = x[c0][a + u + r0] | x[c1][a + u + r1] << 8 | x[c2][..] << 16 | x[c3][..] << 24,
//      each at its own offset b;
//   3. all threads build the pattern words of the stage in shared memory;
//   4. the main loop adds one 4-channel pattern word per (trial, sample) with DP4A (uint8 data)
//      or two DP2A (uint16 decimated data): one shared-memory load per 4 channel-adds.
// Exact moments of every series (S1, 128-bit S2) are accumulated in the epilogue with integer
// atomics, so the search needs no second pass for statistics.
#include <type_traits>

#include "dd_internal.h"

namespace ddk {

namespace {

constexpr int kTileTrials = 32;
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kTPW = kTileTrials / kWarps;  // trials per warp
constexpr int kNG = 4;                      // 4-channel groups per stage
constexpr int kRows = 4 * kNG;              // channel rows per stage
constexpr int kNStage = 3;                  // raw staging buffers

struct PatEntry {
  int32_t col[4];  // first staged element of each channel's row for u = 0
  int32_t zoff;    // pattern's first Z entry within its group
  int32_t zlen;    // Z entries of the pattern
};

__host__ __device__ constexpr size_t align16(size_t v) { return (v + 15) & ~size_t(15); }

struct SmemLayout {
  size_t raw, z, zstart, pat, gtot, npat, mbar, total;
};

__host__ __device__ inline SmemLayout smem_layout(int es, int zes, int row_slot, int zcap) {
  SmemLayout L;
  size_t off = 0;
  L.raw = off;
  off = align16(off + (size_t)kNStage * kRows * row_slot * es);
  L.z = off;
  off = align16(off + (size_t)zcap * zes);
  L.zstart = off;
  off = align16(off + sizeof(int32_t) * 2 * kNG * 32);
  L.pat = off;
  off = align16(off + sizeof(PatEntry) * 2 * kNG * 32);
  L.gtot = off;
  off = align16(off + sizeof(int32_t) * 2 * kNG);
  L.npat = off;
  off = align16(off + sizeof(int32_t) * 2 * kNG);
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

template <typename T>
struct ZWord;
template <>
struct ZWord<uint8_t> {
  using type = uint32_t;
  static __device__ __forceinline__ uint32_t pack(const uint8_t* r0, const uint8_t* r1,
                                                  const uint8_t* r2, const uint8_t* r3, int u) {
    return (uint32_t)r0[u] | ((uint32_t)r1[u] << 8) | ((uint32_t)r2[u] << 16) |
           ((uint32_t)r3[u] << 24);
  }
  static __device__ __forceinline__ uint32_t dot(uint32_t z, uint32_t acc) {
    return __dp4a(z, 0x01010101u, acc);
  }
};
template <>
struct ZWord<uint16_t> {
  using type = uint2;
  static __device__ __forceinline__ uint2 pack(const uint16_t* r0, const uint16_t* r1,
                                               const uint16_t* r2, const uint16_t* r3, int u) {
    return make_uint2((uint32_t)r0[u] | ((uint32_t)r1[u] << 16),
                      (uint32_t)r2[u] | ((uint32_t)r3[u] << 16));
  }
  static __device__ __forceinline__ uint32_t dot(uint2 z, uint32_t acc) {
    return __dp2a_lo(z.y, 0x0101u, __dp2a_lo(z.x, 0x0101u, acc));
  }
};

template <typename T, int TT>
__global__ void __launch_bounds__(kThreads, 1) k_dedisp_tiled(const TiledArgs a) {
  using ZT = typename ZWord<T>::type;
  constexpr int KT = TT / 32;
  extern __shared__ __align__(16) unsigned char smem[];
  const SmemLayout SL = smem_layout(sizeof(T), sizeof(ZT), a.row_slot, a.zcap);
  T* raw = reinterpret_cast<T*>(smem + SL.raw);
  ZT* Z = reinterpret_cast<ZT*>(smem + SL.z);
  int32_t* zstart = reinterpret_cast<int32_t*>(smem + SL.zstart);
  PatEntry* pat = reinterpret_cast<PatEntry*>(smem + SL.pat);
  int32_t* gtot = reinterpret_cast<int32_t*>(smem + SL.gtot);
  int32_t* npat = reinterpret_cast<int32_t*>(smem + SL.npat);
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
  // warp 0 issues stages 0 .. kNStage-2 now and stage s + kNStage - 1 during stage s, using
  // delays it loaded one stage earlier (so the loads' latency overlaps the previous stage)
  int issued = 0;
  int nx_min = 0, nx_max = 0;  // bounds of the next stage to issue (warp 0)
  if (warp == 0) {
    for (int s = 0; s < kNStage - 1 && s < nstages; ++s) {
      int smin, smax;
      stage_bounds(a, s, lane, trial0, ntr, smin, smax);
      issue_stage<T, TT>(a, s, raw + (size_t)s * stage_elems, &mbar[s], j0, lane, smin, smax);
      ++issued;
    }
    if (kNStage - 1 < nstages) stage_bounds(a, kNStage - 1, lane, trial0, ntr, nx_min, nx_max);
  }

  uint32_t acc[kTPW][KT];
#pragma unroll
  for (int q = 0; q < kTPW; ++q)
#pragma unroll
    for (int k = 0; k < KT; ++k) acc[q][k] = 0;

  bool aborted = false;
  int s_abort = 0;
  for (int s = 0; s < nstages; ++s) {
    const int buf = s % kNStage;
    const int db = s & 1;
    const int ng = min(kNG, ngroups - s * kNG);
    if (warp == 0 && s + kNStage - 1 < nstages) {
      const int s2 = s + kNStage - 1;
      issue_stage<T, TT>(a, s2, raw + (size_t)(s2 % kNStage) * stage_elems, &mbar[s2 % kNStage],
                         j0, lane, nx_min, nx_max);
      ++issued;
      if (s2 + 1 < nstages) stage_bounds(a, s2 + 1, lane, trial0, ntr, nx_min, nx_max);
    }
    // ---- relative-delay patterns of each 4-channel group (one warp per group)
    if (warp < ng) {
      const int g = warp;
      const int gabs = s * kNG + g;
      const bool act = lane < ntr;
      int4 s4 = make_int4(0, 0, 0, 0);
      if (act)
        s4 = *reinterpret_cast<const int4*>(a.shifts + (int64_t)(trial0 + lane) * a.c4 + 4 * gabs);
      const int b = min(min(s4.x, s4.y), min(s4.z, s4.w));
      const uint32_t r0 = s4.x - b, r1 = s4.y - b, r2 = s4.z - b, r3 = s4.w - b;
      const unsigned long long key = (unsigned long long)r0 | ((unsigned long long)r1 << 16) |
                                     ((unsigned long long)r2 << 32) |
                                     ((unsigned long long)r3 << 48);
      const uint32_t actmask = __ballot_sync(0xffffffffu, act);
      uint32_t mask = 0;
      int bmin = 0, bmax = 0;
      if (act) {
        mask = __match_any_sync(actmask, key);
        bmin = __reduce_min_sync(mask, b);
        bmax = __reduce_max_sync(mask, b);
      }
      const int leader = act ? __ffs(mask) - 1 : 0;
      const bool is_leader = act && leader == lane;
      const uint32_t leaders = __ballot_sync(0xffffffffu, is_leader);
      const int zlen = is_leader ? (TT + bmax - bmin) : 0;
      int incl = zlen;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += t;
      }
      const int zoff_l = incl - zlen;
      const int myzoff = __shfl_sync(0xffffffffu, zoff_l, leader);
      // first staged element of each channel row (matches issue_stage)
      const int s_first0 = __shfl_sync(0xffffffffu, s4.x, 0);
      const int s_first1 = __shfl_sync(0xffffffffu, s4.y, 0);
      const int s_first2 = __shfl_sync(0xffffffffu, s4.z, 0);
      const int s_first3 = __shfl_sync(0xffffffffu, s4.w, 0);
      if (act) zstart[(db * kNG + g) * 32 + lane] = myzoff + (b - bmin);
      if (is_leader) {
        constexpr int A = 16 / (int)sizeof(T);
        const int pid = __popc(leaders & ((1u << lane) - 1));
        PatEntry e;
        const int64_t base = a.m0 + j0 + bmin;
        const int64_t st0 = a.m0 + j0 + s_first0, st1 = a.m0 + j0 + s_first1;
        const int64_t st2 = a.m0 + j0 + s_first2, st3 = a.m0 + j0 + s_first3;
        e.col[0] = (int32_t)(base + r0 - (st0 & ~(int64_t)(A - 1)));
        e.col[1] = (int32_t)(base + r1 - (st1 & ~(int64_t)(A - 1)));
        e.col[2] = (int32_t)(base + r2 - (st2 & ~(int64_t)(A - 1)));
        e.col[3] = (int32_t)(base + r3 - (st3 & ~(int64_t)(A - 1)));
        e.zoff = zoff_l;
        e.zlen = zlen;
        pat[(db * kNG + g) * 32 + pid] = e;
      }
      if (lane == 31) gtot[db * kNG + g] = incl;
      if (lane == 0) npat[db * kNG + g] = __popc(leaders);
    }
    // ---- wait for the stage's channel rows
    bool ok = true;
    if (!aborted) ok = mbar_wait_bounded(&mbar[buf], (uint32_t)((s / kNStage) & 1));
    if (__syncthreads_or(!ok)) {
      aborted = true;
      s_abort = s;
      break;
    }
    // ---- build the pattern words
    int gbase[kNG];
    int ztotal = 0;
#pragma unroll
    for (int g = 0; g < kNG; ++g) {
      gbase[g] = ztotal;
      if (g < ng) ztotal += gtot[db * kNG + g];
    }
    if (ztotal > a.zcap) {  // cannot happen for a table the host sized; refuse, never overflow
      if (tid == 0) atomicOr(a.err, 2);
      aborted = true;
      s_abort = s + 1;  // this stage's copies have landed
      break;
    }
    const T* rawb = raw + (size_t)buf * stage_elems;
#pragma unroll
    for (int g = 0; g < kNG; ++g) {
      if (g < ng) {
        const int np = npat[db * kNG + g];
        for (int p = 0; p < np; ++p) {
          const PatEntry e = pat[(db * kNG + g) * 32 + p];
          const T* q0 = rawb + (size_t)(4 * g + 0) * a.row_slot + e.col[0];
          const T* q1 = rawb + (size_t)(4 * g + 1) * a.row_slot + e.col[1];
          const T* q2 = rawb + (size_t)(4 * g + 2) * a.row_slot + e.col[2];
          const T* q3 = rawb + (size_t)(4 * g + 3) * a.row_slot + e.col[3];
          ZT* zd = Z + gbase[g] + e.zoff;
          for (int u = tid; u < e.zlen; u += kThreads) zd[u] = ZWord<T>::pack(q0, q1, q2, q3, u);
        }
      }
    }
    __syncthreads();
    // ---- accumulate: one pattern word = four channel-adds per (trial, sample)
#pragma unroll
    for (int g = 0; g < kNG; ++g) {
      if (g < ng) {
        const ZT* zg = Z + gbase[g] + lane;
#pragma unroll
        for (int q = 0; q < kTPW; ++q) {
          const int t = warp + kWarps * q;
          if (t < ntr) {
            const ZT* zp = zg + zstart[(db * kNG + g) * 32 + t];
#pragma unroll
            for (int k = 0; k < KT; ++k) acc[q][k] = ZWord<T>::dot(zp[32 * k], acc[q][k]);
          }
        }
      }
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
  using ZT = typename ZWord<T>::type;
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
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
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

cudaError_t prepare_tiled(int is_u16, int tt, size_t smem) {
  if (!is_u16 && tt == 1024) return prepare_t<uint8_t, 1024>(smem);
  if (!is_u16 && tt == 512) return prepare_t<uint8_t, 512>(smem);
  if (is_u16 && tt == 512) return prepare_t<uint16_t, 512>(smem);
  if (is_u16 && tt == 256) return prepare_t<uint16_t, 256>(smem);
  return cudaErrorInvalidValue;
}

cudaError_t launch_tiled(const TiledArgs& a, int is_u16, int tt, cudaStream_t st) {
  if (a.nout <= 0 || a.n_trials <= 0) return cudaSuccess;
  if (!is_u16 && tt == 1024) return launch_tiled_t<uint8_t, 1024>(a, st);
  if (!is_u16 && tt == 512) return launch_tiled_t<uint8_t, 512>(a, st);
  if (is_u16 && tt == 512) return launch_tiled_t<uint16_t, 512>(a, st);
  if (is_u16 && tt == 256) return launch_tiled_t<uint16_t, 256>(a, st);
  return cudaErrorInvalidValue;
}

}  // namespace ddk
