// Kernels of the dedispersion + single-pulse-search path (sm_103a), except the tiled
// dedispersion kernel (dd_dedisp.cu).
//
//   k_shift_table : FP64 delay table, one IEEE operation at a time (Sec. 3 DM plan)
//   k_corner_turn : time-major uint8 spectra -> channel-major ring (Sec. 1 time chunks)
//   k_decimate    : exact x2 time decimation, uint8/uint16 -> uint16
//   k_dedisp_naive: one thread per output sample (reference-shaped; testing aid)
//   k_moments     : exact S1 / 128-bit S2 of each series window (Sec. 2.2)
//   k_sps         : boxcar SNR over prefix sums + block peak finding (Sec. 2.2)
#include <math.h>

#include <algorithm>

#include "dd_internal.h"

namespace ddk {

// ------------------------------------------------------------------ delay table

__constant__ ShiftRange c_ranges[kMaxRanges];

__global__ void k_shift_table(const double* __restrict__ freqs, int32_t nchans, int32_t cpad,
                              double fref, double tsamp, int32_t nranges, int32_t total_rows,
                              int32_t* __restrict__ shifts, int32_t* __restrict__ err) {
  const int64_t total = (int64_t)total_rows * cpad;
  // k_DM = 4.148808e3 s MHz^2 pc^-1 cm^3 (textbook cold-plasma constant).
  const double kdm = 4.148808e3;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t row = (int32_t)(e / cpad);
    const int32_t c = (int32_t)(e - (int64_t)row * cpad);
    int r = 0;
    while (r + 1 < nranges && row >= c_ranges[r + 1].row0) ++r;
    const ShiftRange R = c_ranges[r];
    int32_t s = 0;
    {
      // Padding channels (c >= nchans, all-zero data) repeat the last channel's delay, so they
      // add no delay classes of their own to the last channel group.
      const int32_t cc = c < nchans ? c : nchans - 1;
      // dm = start + i*step; a = 1/(f*f); b = 1/(fref*fref); tau = (k*dm)*(a-b);
      // x = tau/(tsamp*d) + 0.5; s = floor(x).  Explicit round-to-nearest intrinsics: no FMA.
      const double dm = __dadd_rn(R.dm_start, __dmul_rn((double)(row - R.row0), R.dm_step));
      const double f = freqs[cc];
      const double a = __ddiv_rn(1.0, __dmul_rn(f, f));
      const double b = __ddiv_rn(1.0, __dmul_rn(fref, fref));
      const double tau = __dmul_rn(__dmul_rn(kdm, dm), __dsub_rn(a, b));
      const double x = __dadd_rn(__ddiv_rn(tau, __dmul_rn(tsamp, (double)R.decimation)), 0.5);
      const double fl = floor(x);
      if (!(fl >= 0.0 && fl <= 2147483647.0)) {
        atomicOr(err, 1);
        s = 0;
      } else {
        s = (int32_t)fl;
      }
    }
    shifts[e] = s;
  }
}

cudaError_t launch_shift_table(const double* freqs, int32_t nchans, int32_t cpad, double fref,
                               double tsamp, const ShiftRange* ranges, int32_t nranges,
                               int32_t total_rows, int32_t* shifts, int32_t* err,
                               cudaStream_t st) {
  cudaError_t e = cudaMemcpyToSymbolAsync(c_ranges, ranges, sizeof(ShiftRange) * nranges, 0,
                                          cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return e;
  const int64_t total = (int64_t)total_rows * cpad;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 152 * 64) blocks = 152 * 64;
  if (blocks < 1) blocks = 1;
  k_shift_table<<<(unsigned)blocks, 256, 0, st>>>(freqs, nchans, cpad, fref, tsamp, nranges,
                                                  total_rows, shifts, err);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ corner turn

// 64 samples x 64 channels per CTA. 16-byte loads of spectra into shared memory, a 4x4 byte
// transpose in registers (PRMT), 4-byte stores of channel rows.
__global__ void __launch_bounds__(256) k_corner_turn16(const uint8_t* __restrict__ in, int64_t n,
                                                       int32_t nchans, uint8_t* __restrict__ ring,
                                                       int64_t stride, int64_t col0) {
  __shared__ uint32_t S[64][17];
  const int tid = threadIdx.x;
  const int64_t t0 = (int64_t)blockIdx.x * 64;
  const int32_t c0 = blockIdx.y * 64;
  {
    const int r = tid >> 2, q = tid & 3;
    const int64_t t = t0 + r;
    const int32_t c = c0 + 16 * q;
    uint4 v = make_uint4(0, 0, 0, 0);
    if (t < n && c < nchans) v = __ldg(reinterpret_cast<const uint4*>(in + t * nchans + c));
    S[r][4 * q + 0] = v.x;
    S[r][4 * q + 1] = v.y;
    S[r][4 * q + 2] = v.z;
    S[r][4 * q + 3] = v.w;
  }
  __syncthreads();
  const int tb = tid & 15, cw = tid >> 4;
  const uint32_t w0 = S[4 * tb + 0][cw], w1 = S[4 * tb + 1][cw];
  const uint32_t w2 = S[4 * tb + 2][cw], w3 = S[4 * tb + 3][cw];
  const uint32_t a0 = __byte_perm(w0, w1, 0x5140), a1 = __byte_perm(w0, w1, 0x7362);
  const uint32_t a2 = __byte_perm(w2, w3, 0x5140), a3 = __byte_perm(w2, w3, 0x7362);
  uint32_t o[4];
  o[0] = __byte_perm(a0, a2, 0x5410);
  o[1] = __byte_perm(a0, a2, 0x7632);
  o[2] = __byte_perm(a1, a3, 0x5410);
  o[3] = __byte_perm(a1, a3, 0x7632);
  const int64_t t = t0 + 4 * tb;
  if (t >= n) return;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int32_t c = c0 + 4 * cw + j;
    if (c < nchans)
      *reinterpret_cast<uint32_t*>(ring + (int64_t)c * stride + col0 + t) = o[j];
  }
}

// Any channel count / alignment: one byte per thread.
__global__ void k_corner_turn1(const uint8_t* __restrict__ in, int64_t n, int32_t nchans,
                               uint8_t* __restrict__ ring, int64_t stride, int64_t col0) {
  const int64_t total = n * nchans;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = e / nchans;
    const int32_t c = (int32_t)(e - t * nchans);
    ring[(int64_t)c * stride + col0 + t] = in[e];
  }
}

cudaError_t launch_corner_turn(const uint8_t* in, int64_t n, int32_t nchans, uint8_t* ring,
                               int64_t ring_stride, int64_t col0, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const bool fast = (nchans % 16 == 0) && (((uintptr_t)in & 15) == 0) && (ring_stride % 4 == 0) &&
                    (col0 % 4 == 0) && (((uintptr_t)ring & 3) == 0);
  if (fast) {
    dim3 grid((unsigned)((n + 63) / 64), (unsigned)((nchans + 63) / 64));
    k_corner_turn16<<<grid, 256, 0, st>>>(in, n, nchans, ring, ring_stride, col0);
  } else {
    int64_t blocks = (n * nchans + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    k_corner_turn1<<<(unsigned)blocks, 256, 0, st>>>(in, n, nchans, ring, ring_stride, col0);
  }
  return cudaGetLastError();
}

// ------------------------------------------------------------------ decimation

// out[c][m] = in[c][2m] + in[c][2m+1], four outputs per thread. Channels c = blockIdx.y,
// blockIdx.y + gridDim.y, ... (a grid dimension holds at most 65535 of them).
__global__ void k_decimate_u8(const uint8_t* __restrict__ in, int64_t in_stride,
                              uint16_t* __restrict__ out, int64_t out_stride, int64_t n_out,
                              int32_t cpad) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (4 * k >= n_out) return;
  for (int64_t c = blockIdx.y; c < cpad; c += gridDim.y) {
    const uint2 v = __ldg(reinterpret_cast<const uint2*>(in + c * in_stride + 8 * k));
    const uint32_t lo = (v.x & 0xFFu) + ((v.x >> 8) & 0xFFu);
    const uint32_t hi = ((v.x >> 16) & 0xFFu) + (v.x >> 24);
    const uint32_t lo2 = (v.y & 0xFFu) + ((v.y >> 8) & 0xFFu);
    const uint32_t hi2 = ((v.y >> 16) & 0xFFu) + (v.y >> 24);
    uint2 o;
    o.x = lo | (hi << 16);
    o.y = lo2 | (hi2 << 16);
    *reinterpret_cast<uint2*>(out + c * out_stride + 4 * k) = o;
  }
}

__global__ void k_decimate_u16(const uint16_t* __restrict__ in, int64_t in_stride,
                               uint16_t* __restrict__ out, int64_t out_stride, int64_t n_out,
                               int32_t cpad) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (4 * k >= n_out) return;
  for (int64_t c = blockIdx.y; c < cpad; c += gridDim.y) {
    const uint4 v = __ldg(reinterpret_cast<const uint4*>(in + c * in_stride + 8 * k));
    const uint32_t s0 = (v.x & 0xFFFFu) + (v.x >> 16), s1 = (v.y & 0xFFFFu) + (v.y >> 16);
    const uint32_t s2 = (v.z & 0xFFFFu) + (v.z >> 16), s3 = (v.w & 0xFFFFu) + (v.w >> 16);
    uint2 o;
    o.x = s0 | (s1 << 16);
    o.y = s2 | (s3 << 16);
    *reinterpret_cast<uint2*>(out + c * out_stride + 4 * k) = o;
  }
}

cudaError_t launch_decimate(const void* in, int in_is_u16, int64_t in_stride, uint16_t* out,
                            int64_t out_stride, int32_t cpad, int64_t n_out, cudaStream_t st) {
  if (n_out <= 0) return cudaSuccess;
  dim3 grid((unsigned)(((n_out + 3) / 4 + 255) / 256), (unsigned)std::min(cpad, 65535));
  if (in_is_u16)
    k_decimate_u16<<<grid, 256, 0, st>>>(static_cast<const uint16_t*>(in), in_stride, out,
                                         out_stride, n_out, cpad);
  else
    k_decimate_u8<<<grid, 256, 0, st>>>(static_cast<const uint8_t*>(in), in_stride, out,
                                        out_stride, n_out, cpad);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ naive dedispersion

template <typename T>
__global__ void k_dedisp_naive(const T* __restrict__ xd, int64_t stride, int32_t cpad, int64_t m0,
                               int64_t nout, const int32_t* __restrict__ shifts,
                               int32_t* __restrict__ y, int64_t y_stride) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int32_t i = blockIdx.y;
  if (j >= nout) return;
  const int32_t* s = shifts + (int64_t)i * cpad;
  int32_t acc = 0;
  for (int32_t c = 0; c < cpad; ++c) acc += (int32_t)xd[(int64_t)c * stride + m0 + j + s[c]];
  y[(int64_t)i * y_stride + j] = acc;
}

cudaError_t launch_dedisp_naive(const DedispRange& r, int32_t cpad, cudaStream_t st) {
  if (r.nout <= 0 || r.n_trials <= 0) return cudaSuccess;
  dim3 grid((unsigned)((r.nout + 255) / 256), (unsigned)r.n_trials);
  if (r.is_u16)
    k_dedisp_naive<uint16_t><<<grid, 256, 0, st>>>(static_cast<const uint16_t*>(r.xd), r.xd_stride,
                                                   cpad, r.m0, r.nout, r.shifts, r.y, r.y_stride);
  else
    k_dedisp_naive<uint8_t><<<grid, 256, 0, st>>>(static_cast<const uint8_t*>(r.xd), r.xd_stride,
                                                  cpad, r.m0, r.nout, r.shifts, r.y, r.y_stride);
  return cudaGetLastError();
}

// Direct kernel: the fallback for ranges the tiled kernel cannot take (delay classes beyond
// its tables, as with coarse channels, or decimation above x16). A CTA of 8 warps owns 16
// consecutive trials x 512 outputs; a warp takes 2 trials, lane l the 4-sample groups
// 4l + 128g (g = 0..3) of both. Per channel a lane reads, through the read-only cache, the two
// aligned 32-bit words holding its 4 samples and funnel-shifts them into place (the shift is
// the same in every lane of the warp: it depends only on m0 + delay). uint8 samples are added
// in 16-bit SWAR lanes (even / odd samples), flushed to 32-bit sums every 256 channels
// (256 x 255 < 2^16); uint16 samples (up to 255 x 256) are added to 32-bit sums directly.
constexpr int kDirectTrials = 16;
constexpr int kDirectTile = 512;

template <typename T>
__global__ void __launch_bounds__(256) k_dedisp_direct(const T* __restrict__ xd, int64_t stride,
                                                       int32_t cpad, int64_t m0, int64_t nout,
                                                       int32_t n_trials,
                                                       const int32_t* __restrict__ shifts,
                                                       int32_t* __restrict__ y, int64_t y_stride) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int32_t tbase = blockIdx.x * kDirectTrials + 2 * warp;
  if (tbase >= n_trials) return;  // whole warp
  const int ntr = min(2, n_trials - tbase);
  const int64_t j0 = (int64_t)blockIdx.y * kDirectTile;
  uint32_t acc[2][4][4];  // [trial][group g][sample e]
#pragma unroll
  for (int q = 0; q < 2; ++q)
#pragma unroll
    for (int g = 0; g < 4; ++g)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[q][g][e] = 0;
  const char* base = reinterpret_cast<const char*>(xd);
  const int64_t row_bytes = stride * (int64_t)sizeof(T);
  for (int32_t c0 = 0; c0 < cpad; c0 += 256) {
    uint32_t ev[2][4], od[2][4];  // uint8 path: packed 16-bit sums of samples (0,2) and (1,3)
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
      for (int g = 0; g < 4; ++g) ev[q][g] = od[q][g] = 0;
    const int32_t c1 = min(cpad, c0 + 256);
    for (int32_t c = c0; c < c1; ++c) {
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        if (q < ntr) {
          const int64_t s = __ldg(shifts + (int64_t)(tbase + q) * cpad + c);
          // byte address of this lane's first sample of group 0
          const int64_t b = (int64_t)c * row_bytes + (m0 + j0 + s + 4 * lane) * (int64_t)sizeof(T);
          const uint32_t sh = (uint32_t)(b & 3) * 8u;
          const uint32_t* wp = reinterpret_cast<const uint32_t*>(base + (b & ~(int64_t)3));
#pragma unroll
          for (int g = 0; g < 4; ++g) {
            if (sizeof(T) == 1) {
              const uint32_t* p = wp + 32 * g;  // 128 samples further per group
              const uint32_t v = __funnelshift_r(__ldg(p), __ldg(p + 1), sh);
              ev[q][g] += v & 0x00FF00FFu;
              od[q][g] += __byte_perm(v, 0, 0x4341);
            } else {
              const uint32_t* p = wp + 64 * g;
              const uint32_t w0 = __ldg(p), w1 = __ldg(p + 1), w2 = __ldg(p + 2);
              const uint32_t v0 = __funnelshift_r(w0, w1, sh), v1 = __funnelshift_r(w1, w2, sh);
              acc[q][g][0] += v0 & 0xFFFFu;
              acc[q][g][1] += v0 >> 16;
              acc[q][g][2] += v1 & 0xFFFFu;
              acc[q][g][3] += v1 >> 16;
            }
          }
        }
      }
    }
    if (sizeof(T) == 1) {
#pragma unroll
      for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int g = 0; g < 4; ++g) {
          acc[q][g][0] += ev[q][g] & 0xFFFFu;
          acc[q][g][2] += ev[q][g] >> 16;
          acc[q][g][1] += od[q][g] & 0xFFFFu;
          acc[q][g][3] += od[q][g] >> 16;
        }
    }
  }
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    if (q < ntr) {
      int32_t* yr = y + (int64_t)(tbase + q) * y_stride;
#pragma unroll
      for (int g = 0; g < 4; ++g)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int64_t j = j0 + 128 * g + 4 * lane + e;
          if (j < nout) yr[j] = (int32_t)acc[q][g][e];
        }
    }
  }
}

cudaError_t launch_dedisp_direct(const DedispRange& r, int32_t cpad, cudaStream_t st) {
  if (r.nout <= 0 || r.n_trials <= 0) return cudaSuccess;
  dim3 grid((unsigned)((r.n_trials + kDirectTrials - 1) / kDirectTrials),
            (unsigned)((r.nout + kDirectTile - 1) / kDirectTile));
  if (r.is_u16)
    k_dedisp_direct<uint16_t><<<grid, 256, 0, st>>>(static_cast<const uint16_t*>(r.xd),
                                                    r.xd_stride, cpad, r.m0, r.nout, r.n_trials,
                                                    r.shifts, r.y, r.y_stride);
  else
    k_dedisp_direct<uint8_t><<<grid, 256, 0, st>>>(static_cast<const uint8_t*>(r.xd), r.xd_stride,
                                                   cpad, r.m0, r.nout, r.n_trials, r.shifts, r.y,
                                                   r.y_stride);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ moments

struct U128 {
  unsigned long long lo, hi;
};

__device__ __forceinline__ U128 add128(U128 a, U128 b) {
  U128 r;
  r.lo = a.lo + b.lo;
  r.hi = a.hi + b.hi + (r.lo < a.lo ? 1ull : 0ull);
  return r;
}

__global__ void __launch_bounds__(256) k_moments(const int32_t* __restrict__ y, int64_t n,
                                                 int64_t stride, Moments* __restrict__ mom) {
  const int32_t i = blockIdx.x;
  const int32_t* yi = y + (int64_t)i * stride;
  unsigned long long s1 = 0;
  U128 s2 = {0, 0};
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
    const int64_t v = yi[j];
    s1 += (unsigned long long)v;
    s2 = add128(s2, U128{(unsigned long long)(v * v), 0});
  }
  __shared__ unsigned long long sh[3][8];
  for (int off = 16; off > 0; off >>= 1) {
    s1 += __shfl_xor_sync(0xffffffffu, s1, off);
    U128 o;
    o.lo = __shfl_xor_sync(0xffffffffu, s2.lo, off);
    o.hi = __shfl_xor_sync(0xffffffffu, s2.hi, off);
    s2 = add128(s2, o);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    sh[0][w] = s1;
    sh[1][w] = s2.lo;
    sh[2][w] = s2.hi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long a = 0;
    U128 b = {0, 0};
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
      a += sh[0][k];
      b = add128(b, U128{sh[1][k], sh[2][k]});
    }
    mom[i].s1 = a;
    mom[i].s2lo = b.lo;
    mom[i].s2hi = b.hi;
    mom[i].pad = 0;
  }
}

cudaError_t launch_moments(const int32_t* y, int32_t ntr, int64_t n, int64_t stride, Moments* mom,
                           cudaStream_t st) {
  if (ntr <= 0) return cudaSuccess;
  k_moments<<<ntr, 256, 0, st>>>(y, n, stride, mom);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ single pulse search

// Correctly rounded unsigned 128-bit -> double: the top 64 significant bits with a sticky bit
// for everything below, converted with round-to-nearest-even, then scaled by a power of two.
__device__ __forceinline__ double u128_to_f64(unsigned long long hi, unsigned long long lo) {
  if (hi == 0) return __ull2double_rn(lo);
  const int lz = __clzll((long long)hi);
  const int sh = 64 - lz;  // 1..64
  unsigned long long top, sticky;
  if (sh == 64) {
    top = hi;
    sticky = lo != 0;
  } else {
    top = (hi << lz) | (lo >> sh);
    sticky = (lo << lz) != 0;
  }
  return ldexp(__ull2double_rn(top | sticky), sh);
}

// sqrt(n*S2 - S1^2) of a window's moments, V = n*S2 - S1^2 formed exactly in 128 bits (S1 >= 0
// because every series value is a sum of non-negative samples) and rounded once to FP64; 0 for a
// constant series.
__device__ __forceinline__ double window_sqrt_var(const Moments& m, long long n) {
  const unsigned long long un = (unsigned long long)n, us1 = m.s1;
  const unsigned long long p_lo = un * m.s2lo;
  const unsigned long long p_hi = __umul64hi(un, m.s2lo) + un * m.s2hi;
  const unsigned long long q_lo = us1 * us1, q_hi = __umul64hi(us1, us1);
  const unsigned long long v_lo = p_lo - q_lo;
  const unsigned long long v_hi = p_hi - q_hi - (p_lo < q_lo ? 1ull : 0ull);
  if (v_lo == 0 && v_hi == 0) return 0.0;
  return sqrt(u128_to_f64(v_hi, v_lo));
}

// SNR >= thr  <=>  B >= (w*S1 + thr*den) / n. The bound keeps a margin of 2 + 1e-9 relative so
// that rounding in this estimate can never reject a boxcar sum the exact test accepts; as a
// uint32 bound on boxcar sums (< 2^31): at or below 0 every sum passes, above 2^32 - 1 none.
__device__ __forceinline__ uint32_t window_bound(int w, long long s1, double thr, double den,
                                                 long long n) {
  const double t = ((double)w * (double)s1 + thr * den) / (double)n;
  const double tl = t - 2.0 - 1e-9 * fabs(t);
  return tl <= 0.0 ? 0u : (tl >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)floor(tl));
}

constexpr int kSpsThreads = 256;
constexpr int kSpsSeg = kSpsThreads * 16;         // window samples per pass (16 per thread)
constexpr int kSpsPad = 3;                        // aligns P[1 + hist + 4k] to 16 bytes

// Exact argmax over the block: largest v among valid lanes, ties to the lowest lane. Returns
// -1 when the block has no valid lane; `off` = lane offset within the block.
__device__ __forceinline__ int block_argmax(uint32_t v, bool valid, int B, int lane, int& off) {
  unsigned long long key =
      valid ? (((unsigned long long)v << 32) | (0xFFFFFFFFu - (uint32_t)(lane & (B - 1)))) : 0ull;
  for (int o = B >> 1; o > 0; o >>= 1) {
    const unsigned long long t = __shfl_xor_sync(0xffffffffu, key, o);
    key = t > key ? t : key;
  }
  off = key ? (int)(0xFFFFFFFFu - (uint32_t)(key & 0xFFFFFFFFu)) : 0;
  return key ? (int)(key >> 32) : -1;
}

// Prefix sums through window samples q - w .. q + 3 - w of the pass, i.e. entries
// P[idx - w .. idx - w + 3] with idx 16-byte aligned: one aligned 16-byte load when w is a
// multiple of 4, else two, from which the four entries are picked (w is the same in every lane,
// so the pick is a uniform branch). Lanes take consecutive 16-byte units: no bank conflicts.
__device__ __forceinline__ uint4 prefix4(const uint32_t* P, int idx, int w) {
  const int m = (-w) & 3;
  const uint4* q = reinterpret_cast<const uint4*>(P + idx - w - m);
  const uint4 a = q[0];
  if (m == 0) return a;
  const uint4 b = q[1];
  if (m == 1) return make_uint4(a.y, a.z, a.w, b.x);
  if (m == 2) return make_uint4(a.z, a.w, b.x, b.y);
  return make_uint4(a.w, b.x, b.y, b.z);
}

// One pass of the search kernels over window samples seg0 .. seg0 + kSpsSeg - 1 of series yi
// (zero past n): this lane's four 4-sample chunks (samples seg0 + q0 + 128 g + e) are loaded and
// turned into uint32 prefix sums continuing from P[H] (the sum through the sample before the
// pass), returned in v and stored to P[1 + H + q]. Two CTA barriers; P[0 .. H] must be in place.
__device__ __forceinline__ void sps_pass_prefix(const int32_t* __restrict__ yi, bool vec,
                                                long long n, long long seg0, int q0, int lane,
                                                int wid, int H, uint32_t* P, uint32_t* warp_tot,
                                                uint32_t (&v)[4][4]) {
#pragma unroll
  for (int g = 0; g < 4; ++g) {
    const long long j = seg0 + q0 + 128 * g;
    if (vec && j + 4 <= n) {
      const int4 t = __ldg(reinterpret_cast<const int4*>(yi + j));
      v[g][0] = (uint32_t)t.x;
      v[g][1] = (uint32_t)t.y;
      v[g][2] = (uint32_t)t.z;
      v[g][3] = (uint32_t)t.w;
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e) v[g][e] = (j + e < n) ? (uint32_t)__ldg(yi + j + e) : 0u;
    }
  }
  uint32_t run = 0;  // sum of this warp's chunks before the current one (lanes, then g)
#pragma unroll
  for (int g = 0; g < 4; ++g) {
    v[g][1] += v[g][0];
    v[g][2] += v[g][1];
    v[g][3] += v[g][2];
    uint32_t incl = v[g][3];
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t o = __shfl_up_sync(0xffffffffu, incl, off);
      if (lane >= off) incl += o;
    }
    const uint32_t pre = run + incl - v[g][3];
#pragma unroll
    for (int e = 0; e < 4; ++e) v[g][e] += pre;
    run += __shfl_sync(0xffffffffu, incl, 31);
  }
  if (lane == 0) warp_tot[wid] = run;
  __syncthreads();  // warp totals; the history entries P[0 .. H] of this pass
  uint32_t base = P[H];  // sum through the sample before the pass
  for (int k = 0; k < wid; ++k) base += warp_tot[k];
#pragma unroll
  for (int g = 0; g < 4; ++g) {
#pragma unroll
    for (int e = 0; e < 4; ++e) v[g][e] += base;  // now prefix sums through each sample
    *reinterpret_cast<uint4*>(P + 1 + H + q0 + 128 * g) =
        make_uint4(v[g][0], v[g][1], v[g][2], v[g][3]);
  }
  __syncthreads();  // the pass's prefix sums
}

// One CTA per trial; passes of kSpsSeg window samples. Warp v owns pass samples
// 512v .. 512v + 511, lane l the 4-sample chunks 512v + 128g + 4l (g = 0..3). P holds uint32
// prefix sums of the pass and of the H samples before it (entry 1 + H + q = sum through window
// sample seg0 + q; the sums wrap, but every boxcar sum is < 2^31, so the difference of two
// prefixes is exact). The history part is carried over from the previous pass in shared memory.
// Every boxcar sum is compared with an integer bound per width below which the SNR cannot reach
// the threshold; a 32-sample group where one passes is searched exactly by its warp (lane =
// sample): per width the group's largest boxcar sum (earliest sample) per peak block, then the
// FP64 SNRs in the oracle's evaluation order.
__global__ void __launch_bounds__(kSpsThreads) k_sps(const SpsArgs a) {
  extern __shared__ __align__(16) uint32_t Ps[];
  uint32_t* P = Ps + kSpsPad;  // [1 + hist + kSpsSeg]
  __shared__ double den[kMaxWidths];
  __shared__ long long ca[kMaxWidths], cb[kMaxWidths];
  __shared__ uint32_t bthr[kMaxWidths];
  __shared__ uint32_t warp_tot[kSpsThreads / 32];

  const int32_t i = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const long long n = a.n;
  if (n <= 0) return;
  const double thr = (double)a.threshold;
  // Per width k: SNR = (ca[k] * B - cb[k]) / den[k]. Window statistics: ca = n, cb = w * S1,
  // den = sqrt(w) * sqrt(n * S2 - S1^2). Clipped per-width statistics (a.wst): ca = N_k,
  // cb = T1_k, den = sqrt(N_k * T2_k - T1_k^2). A width with den 0 gives no candidates.
  if (a.wst == nullptr) {
    const Moments m = a.mom[i];
    const long long s1 = (long long)m.s1;
    const double sq = window_sqrt_var(m, n);
    if (sq == 0.0) return;  // constant series: no candidates
    if (tid < a.nw) {
      const int w = a.wd[tid];
      den[tid] = sqrt((double)w) * sq;
      ca[tid] = n;
      cb[tid] = (long long)w * s1;
      bthr[tid] = window_bound(w, s1, thr, den[tid], n);
    }
  } else if (tid < a.nw) {
    const WidthStats st = a.wst[(int64_t)i * a.nw + tid];
    const unsigned long long un = (unsigned long long)st.n, ut1 = (unsigned long long)st.t1;
    const unsigned long long p_lo = un * st.t2lo;
    const unsigned long long p_hi = __umul64hi(un, st.t2lo) + un * st.t2hi;
    const unsigned long long q_lo = ut1 * ut1, q_hi = __umul64hi(ut1, ut1);
    const unsigned long long v_lo = p_lo - q_lo;
    const unsigned long long v_hi = p_hi - q_hi - (p_lo < q_lo ? 1ull : 0ull);
    const bool live = st.n > 0 && (v_lo | v_hi) != 0;
    den[tid] = live ? sqrt(u128_to_f64(v_hi, v_lo)) : 0.0;
    ca[tid] = st.n;
    cb[tid] = st.t1;
    // SNR >= thr  <=>  B >= (T1 + thr*den) / N, with the margin above
    const double t = live ? ((double)st.t1 + thr * den[tid]) / (double)st.n : 0.0;
    const double tl = t - 2.0 - 1e-9 * fabs(t);
    bthr[tid] = !live ? 0xFFFFFFFFu
                      : (tl <= 0.0 ? 0u : (tl >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)floor(tl)));
  }
  const int H = a.hist;
  const int nw = a.nw;
  const int wmax = a.wd[nw - 1];
  const int32_t* yi = a.y + (int64_t)i * a.stride;
  const bool vec = (reinterpret_cast<uintptr_t>(yi) & 15) == 0;
  const int B = a.block;
  const int q0 = wid * 512 + 4 * lane;  // pass sample of this lane's chunk g = 0
  // samples before the window are zero: the history of the first pass is all zero
  for (int k = tid; k <= H; k += kSpsThreads) P[k] = 0;

  for (long long seg0 = 0; seg0 < n; seg0 += kSpsSeg) {
    uint32_t v[4][4];
    sps_pass_prefix(yi, vec, n, seg0, q0, lane, wid, H, P, warp_tot, v);

    // ---- filter: every boxcar sum of this lane's samples against the bounds
    const long long wj0 = seg0 + wid * 512;  // the warp's first sample
    const bool interior = wj0 >= wmax - 1 && wj0 + 512 <= n;  // every (sample, width) valid
    unsigned groups = 0;  // 32-sample groups of the warp's 512 samples with a passing sum
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      const int idx = 1 + H + q0 + 128 * g;  // entry of this chunk's first sample
      const long long j = seg0 + q0 + 128 * g;
      bool hot = false;
#pragma unroll
      for (int k = 0; k < kMaxWidths; ++k) {
        if (k >= nw) break;
        const int w = a.wd[k];
        const uint4 st = prefix4(P, idx, w);
        const uint32_t b0 = v[g][0] - st.x, b1 = v[g][1] - st.y;
        const uint32_t b2 = v[g][2] - st.z, b3 = v[g][3] - st.w;
        const uint32_t t = bthr[k];
        if (interior) {
          hot |= (b0 >= t) | (b1 >= t) | (b2 >= t) | (b3 >= t);
        } else {
          hot |= (j < n && j >= w - 1 && b0 >= t) | (j + 1 < n && j + 1 >= w - 1 && b1 >= t) |
                 (j + 2 < n && j + 2 >= w - 1 && b2 >= t) | (j + 3 < n && j + 3 >= w - 1 && b3 >= t);
        }
      }
      // lanes 8c .. 8c + 7 of chunk row g cover the warp's 32-sample group 4g + c
      const unsigned hm = __ballot_sync(0xffffffffu, hot);
#pragma unroll
      for (int c = 0; c < 4; ++c) groups |= ((hm >> (8 * c)) & 0xFFu) ? (1u << (4 * g + c)) : 0u;
    }

    // ---- exact search of the hot groups, lane = sample
    while (groups) {
      const int c = __ffs(groups) - 1;
      groups &= groups - 1;
      const int q = wid * 512 + c * 32 + lane;  // pass sample
      const long long j = seg0 + q;
      const uint32_t pj = P[1 + H + q];
      const bool leader = (lane & (B - 1)) == 0;
      double bs = 0.0;
      long long bj = 0;
      int bwid = 0;
      bool have = false;
      for (int k = 0; k < nw; ++k) {
        const int w = a.wd[k];
        const bool valid = (j < n) && (j >= w - 1) && den[k] != 0.0;
        const uint32_t bw = valid ? pj - P[1 + H + q - w] : 0u;
        int off;
        const int best = block_argmax(bw, valid, B, lane, off);
        if (leader && best >= 0) {
          const long long num = ca[k] * (long long)best - cb[k];
          const double snr = (double)num / den[k];
          const long long jk = j + off;  // the leader holds the block's first sample
          if (!have || snr > bs || (snr == bs && jk < bj)) {
            have = true;
            bs = snr;
            bj = jk;
            bwid = w;
          }
        }
      }
      if (leader && have && bs >= thr) {
        const unsigned long long idx = atomicAdd(a.count, 1ull);
        if ((long long)idx < a.cap) {
          dd_cand_t cd;
          cd.trial = i;
          cd.range = a.range;
          cd.t_start = (a.J0 + bj - bwid + 1) * (long long)a.d;
          cd.width = bwid * a.d;
          cd.pad = 0;
          cd.snr = bs;
          a.cands[idx] = cd;
        }
      }
    }
    __syncthreads();  // every read of this pass's P is done
    // the last H + 1 entries become the next pass's history (P[kSpsSeg] = sum before it)
    for (int k = tid; k <= H; k += kSpsThreads) P[k] = P[kSpsSeg + k];
  }
}

// The search's last step on a range whose block maxima the fused dedispersion kernel recorded:
// one CTA per trial, one thread per peak block. The block's candidate is, over the widths, the
// recorded largest boxcar sum's SNR (the SNR grows with the sum at a fixed width, and the
// recorded sample is the earliest holding it), with k_sps's statistics, evaluation order and
// tie rules, so the candidates are the ones k_sps finds on the same series.
__global__ void __launch_bounds__(kSpsThreads) k_sps_fused(const SpsFusedArgs a) {
  __shared__ double den[kMaxWidths];
  __shared__ long long ca[kMaxWidths], cb[kMaxWidths];
  __shared__ uint32_t kthr[kMaxWidths];
  const int32_t i = blockIdx.x;
  const int tid = threadIdx.x;
  const long long n = a.n;
  if (n <= 0) return;
  const Moments m = a.mom[i];
  const double sq = window_sqrt_var(m, n);
  if (sq == 0.0) return;  // constant series: no candidates
  const double thr = (double)a.threshold;
  if (tid < a.nw) {
    const int w = a.wd[tid];
    den[tid] = sqrt((double)w) * sq;
    ca[tid] = n;
    cb[tid] = (long long)w * (long long)m.s1;
    // a record can reach the threshold only if its sum passes k_sps's integer bound (key =
    // sum + 1, so key > bound); the others are skipped before the FP64 SNR
    kthr[tid] = window_bound(w, (long long)m.s1, thr, den[tid], n);
  }
  __syncthreads();
  const int64_t row = (int64_t)i * a.nw;
  for (int64_t b = tid; b < a.nblk; b += kSpsThreads) {
    double bs = 0.0;
    long long bj = 0;
    int bwid = 0;
    bool have = false;
    for (int k = 0; k < a.nw; ++k) {
      const uint32_t key = a.key[(row + k) * a.nblk + b];
      if (key == 0 || key <= kthr[k]) continue;  // no sample, or below the bound
      const long long best = (long long)(key - 1u);
      const long long jk = b * a.block + a.off[(row + k) * a.nblk + b];
      const long long num = ca[k] * best - cb[k];
      const double snr = (double)num / den[k];
      if (!have || snr > bs || (snr == bs && jk < bj)) {
        have = true;
        bs = snr;
        bj = jk;
        bwid = a.wd[k];
      }
    }
    if (have && bs >= thr) {
      const unsigned long long idx = atomicAdd(a.count, 1ull);
      if ((long long)idx < a.cap) {
        dd_cand_t cd;
        cd.trial = i;
        cd.range = a.range;
        cd.t_start = (a.J0 + bj - bwid + 1) * (long long)a.d;
        cd.width = bwid * a.d;
        cd.pad = 0;
        cd.snr = bs;
        a.cands[idx] = cd;
      }
    }
  }
}

// Clipped statistics of every boxcar series of one trial (one CTA per trial): for each width w,
// the values B_w[j] (window samples j >= w - 1) are summed over the whole window (step 0:
// count, sum, 128-bit sum of squares), then, for up to `iters` steps, again over the values
// within ceil(mu - kappa*sd) .. floor(mu + kappa*sd) of the previous step's mean and population
// deviation (FP64, one rounding per operation, as the oracle). A width whose previous step has no
// values or no variance keeps its statistics. Each step sweeps the series once per group of
// kClipGroup widths, forming the boxcar sums from the carried prefix sums of the search kernel.
constexpr int kClipGroup = 8;

__global__ void __launch_bounds__(kSpsThreads) k_clip_stats(const ClipArgs a) {
  extern __shared__ __align__(16) uint32_t Ps[];
  uint32_t* P = Ps + kSpsPad;  // [1 + hist + kSpsSeg]
  __shared__ uint32_t warp_tot[kSpsThreads / 32];
  __shared__ double lo_b[kMaxWidths], hi_b[kMaxWidths];
  __shared__ int live[kMaxWidths];
  __shared__ WidthStats st[kMaxWidths];
  __shared__ unsigned long long red[kClipGroup][4][kSpsThreads / 32];

  const int32_t i = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const long long n = a.n;
  const int nw = a.nw, H = a.hist;
  const int32_t* yi = a.y + (int64_t)i * a.stride;
  const bool vec = (reinterpret_cast<uintptr_t>(yi) & 15) == 0;
  const int q0 = wid * 512 + 4 * lane;
  if (tid < kMaxWidths) {
    lo_b[tid] = -1.0;  // step 0: every value (all boxcar sums are >= 0)
    hi_b[tid] = 1e300;
    live[tid] = tid < nw ? 1 : 0;
    st[tid] = WidthStats{0, 0, 0, 0};
  }
  __syncthreads();
  for (int step = 0; step <= a.iters; ++step) {
    for (int g0 = 0; g0 < nw; g0 += kClipGroup) {
      bool any = false;
      for (int k = g0; k < min(nw, g0 + kClipGroup); ++k) any |= live[k] != 0;
      if (!any) continue;  // uniform: every thread reads the same flags
      uint32_t cn[kClipGroup];
      unsigned long long c1[kClipGroup], c2l[kClipGroup], c2h[kClipGroup];
#pragma unroll
      for (int kk = 0; kk < kClipGroup; ++kk) cn[kk] = 0, c1[kk] = c2l[kk] = c2h[kk] = 0;
      for (int k = tid; k <= H; k += kSpsThreads) P[k] = 0;  // samples before the window
      for (long long seg0 = 0; seg0 < n; seg0 += kSpsSeg) {
        uint32_t v[4][4];
        sps_pass_prefix(yi, vec, n, seg0, q0, lane, wid, H, P, warp_tot, v);
#pragma unroll
        for (int kk = 0; kk < kClipGroup; ++kk) {
          const int k = g0 + kk;
          const bool on = k < nw && live[min(k, kMaxWidths - 1)];
          const int w = on ? a.wd[k] : 1;
          const double lo = on ? lo_b[k] : 1.0, hi = on ? hi_b[k] : 0.0;  // empty when off
#pragma unroll
          for (int g = 0; g < 4; ++g) {
            const int idx = 1 + H + q0 + 128 * g;
            const uint4 s4 = prefix4(P, idx, w);
            const long long j = seg0 + q0 + 128 * g;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const uint32_t b = v[g][e] - (e == 0 ? s4.x : e == 1 ? s4.y : e == 2 ? s4.z : s4.w);
              const double bd = (double)b;
              if (j + e < n && j + e >= w - 1 && bd >= lo && bd <= hi) {
                const unsigned long long sq = (unsigned long long)b * b;
                cn[kk] += 1;
                c1[kk] += b;
                c2l[kk] += sq;
                c2h[kk] += (c2l[kk] < sq) ? 1ull : 0ull;
              }
            }
          }
        }
        __syncthreads();  // every read of this pass's P is done
        for (int k = tid; k <= H; k += kSpsThreads) P[k] = P[kSpsSeg + k];
      }
      // block sums of the group's widths: warp butterflies, then one lane per width
#pragma unroll
      for (int kk = 0; kk < kClipGroup; ++kk) {
        unsigned long long x0 = cn[kk], x1 = c1[kk], lo = c2l[kk], hi = c2h[kk];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
          x0 += __shfl_xor_sync(0xffffffffu, x0, off);
          x1 += __shfl_xor_sync(0xffffffffu, x1, off);
          const unsigned long long olo = __shfl_xor_sync(0xffffffffu, lo, off);
          const unsigned long long ohi = __shfl_xor_sync(0xffffffffu, hi, off);
          const unsigned long long nlo = lo + olo;
          hi = hi + ohi + (nlo < lo ? 1ull : 0ull);
          lo = nlo;
        }
        if (lane == 0) {
          red[kk][0][wid] = x0;
          red[kk][1][wid] = x1;
          red[kk][2][wid] = lo;
          red[kk][3][wid] = hi;
        }
      }
      __syncthreads();
      if (tid < kClipGroup && g0 + tid < nw && live[g0 + tid]) {
        unsigned long long x0 = 0, x1 = 0, lo = 0, hi = 0;
        for (int q = 0; q < kSpsThreads / 32; ++q) {
          x0 += red[tid][0][q];
          x1 += red[tid][1][q];
          const unsigned long long nlo = lo + red[tid][2][q];
          hi = hi + red[tid][3][q] + (nlo < lo ? 1ull : 0ull);
          lo = nlo;
        }
        st[g0 + tid] = WidthStats{(long long)x0, (long long)x1, lo, hi};
      }
      __syncthreads();
    }
    // bounds of the next step from this step's statistics
    if (step < a.iters && tid < nw && live[tid]) {
      const WidthStats s = st[tid];
      const unsigned long long un = (unsigned long long)s.n, ut1 = (unsigned long long)s.t1;
      const unsigned long long p_lo = un * s.t2lo;
      const unsigned long long p_hi = __umul64hi(un, s.t2lo) + un * s.t2hi;
      const unsigned long long q_lo = ut1 * ut1, q_hi = __umul64hi(ut1, ut1);
      const unsigned long long v_lo = p_lo - q_lo;
      const unsigned long long v_hi = p_hi - q_hi - (p_lo < q_lo ? 1ull : 0ull);
      if (s.n == 0 || (v_lo | v_hi) == 0) {
        live[tid] = 0;
      } else {
        const double dn = __ll2double_rn(s.n);
        const double mu = __ddiv_rn(__ll2double_rn(s.t1), dn);
        const double sd = __ddiv_rn(__dsqrt_rn(u128_to_f64(v_hi, v_lo)), dn);
        const double ks = __dmul_rn(a.kappa, sd);
        lo_b[tid] = ceil(__dsub_rn(mu, ks));
        hi_b[tid] = floor(__dadd_rn(mu, ks));
      }
    }
    __syncthreads();
  }
  if (tid < nw) a.out[(int64_t)i * nw + tid] = st[tid];
}

cudaError_t launch_clip_stats(const ClipArgs& a, cudaStream_t st) {
  if (a.n <= 0 || a.n_trials <= 0 || a.nw <= 0) return cudaSuccess;
  if (a.hist < 0 || a.hist % 4 || a.hist + 1 > kSpsSeg || a.iters < 0 || !(a.kappa > 0))
    return cudaErrorInvalidValue;
  const size_t smem = sizeof(uint32_t) * (size_t)(kSpsPad + 1 + a.hist + kSpsSeg);
  k_clip_stats<<<a.n_trials, kSpsThreads, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_sps(const SpsArgs& a, cudaStream_t st) {
  if (a.n <= 0 || a.n_trials <= 0 || a.nw <= 0) return cudaSuccess;
  if (a.hist < 0 || a.hist % 4 || a.hist + 1 > kSpsSeg || a.block < 1 || a.block > 32)
    return cudaErrorInvalidValue;
  const size_t smem = sizeof(uint32_t) * (size_t)(kSpsPad + 1 + a.hist + kSpsSeg);
  k_sps<<<a.n_trials, kSpsThreads, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_sps_fused(const SpsFusedArgs& a, cudaStream_t st) {
  if (a.n <= 0 || a.n_trials <= 0 || a.nw <= 0) return cudaSuccess;
  if (a.block < 1 || a.block > 32 || a.nblk != (a.n + a.block - 1) / a.block)
    return cudaErrorInvalidValue;
  k_sps_fused<<<a.n_trials, kSpsThreads, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace ddk
