// Micro-benchmarks of the issue rates that bound the dedispersion kernels on this GPU: integer
// lane-instructions of the ALU pipe (LOP3), of the dot-product pipe (DP2A), of both interleaved,
// plain 32-bit adds, and warp-wide conflict-free 32-bit shared-memory loads (one wavefront each).
// They are the measured denominators of the dedispersion roofline; nothing on the hot path calls
// them.
//
// Every kernel runs two CTAs of 16 warps per SM. Each CTA records, from its first thread, the SM
// it ran on and its start and end in SM cycles (clock64) and in nanoseconds (globaltimer). The
// rate of an SM is the operations of the CTAs it ran divided by the cycles from their earliest
// start to their latest end (one SM's cycle counter is consistent with itself); the result is
// the mean over SMs. The clock is the CTAs' summed cycles over their summed nanoseconds.
#include <algorithm>
#include <vector>

#include "dd_internal.h"

namespace {

constexpr int kPeakThreads = 512;
constexpr int kPeakCtasPerSm = 2;
constexpr int kPeakIters = 2048;
constexpr int kChains = 8;          // independent dependency chains per thread
constexpr int kLdsWords = 4096;     // shared-memory words the load test reads (128 rows of 32)

struct CtaTime {
  unsigned long long c0, c1, t0, t1;
  uint32_t smid, pad;
};

enum Kind { kLop3 = 0, kDp2a = 1, kMix = 2, kAdd = 3, kLds = 4, kKinds = 5 };

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t lop3_xor(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm volatile("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}

__device__ __forceinline__ uint32_t dp2a(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm volatile("dp2a.lo.u32.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}

__device__ __forceinline__ uint32_t add32(uint32_t a, uint32_t b) {
  uint32_t d;
  asm volatile("add.u32 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
  return d;
}

template <int OFF>
__device__ __forceinline__ uint32_t lds_at(uint32_t addr) {
  uint32_t v;
  asm volatile("ld.shared.u32 %0, [%1+%2];" : "=r"(v) : "r"(addr), "n"(OFF));
  return v;
}

// acc += the 32-bit words at base + 128 j, j = J .. 0 (immediate offsets).
template <int J>
__device__ __forceinline__ void lds_rows(uint32_t base, uint32_t& acc) {
  acc += lds_at<128 * J>(base);
  lds_rows<J - 1>(base, acc);
}
template <>
__device__ __forceinline__ void lds_rows<-1>(uint32_t, uint32_t&) {}

// Operations per thread of one kernel (each inner step is kChains operations).
constexpr int kStepsPerIter = 8;
constexpr long long kOpsPerThread = (long long)kPeakIters * kStepsPerIter * kChains;

template <int KIND>
__global__ void __launch_bounds__(kPeakThreads, kPeakCtasPerSm)
    k_peak(uint32_t seed, uint32_t* sink, CtaTime* times) {
  __shared__ uint32_t buf[kLdsWords];
  const int tid = threadIdx.x;
  uint32_t a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = seed * (uint32_t)(2 * i + 1) + (uint32_t)tid;
  const uint32_t b = seed ^ 0x00010001u;
  if (KIND == kLds) {
    for (int k = tid; k < kLdsWords; k += kPeakThreads) buf[k] = seed + (uint32_t)k;
  }
  __syncthreads();
  CtaTime ct;
  if (tid == 0) {
    ct.c0 = clock64();
    ct.t0 = gtimer();
  }
  __syncthreads();
  if (KIND == kLds) {
    // lane l of a warp reads word l of a 128-byte row: 32 consecutive words, one wavefront per
    // load. The kStepsPerIter * kChains loads of an iteration read distinct consecutive rows at
    // immediate offsets from one base (no address arithmetic per load, and no two loads alike),
    // and the base moves from one iteration to the next.
    const uint32_t base0 = (uint32_t)__cvta_generic_to_shared(buf) + 4u * (uint32_t)(tid & 31);
    uint32_t acc = a[0];
    for (int it = 0; it < kPeakIters; ++it) {
      const uint32_t base = base0 + 128u * ((uint32_t)(it * 7 + (tid >> 5)) & 63u);
      lds_rows<kStepsPerIter * kChains - 1>(base, acc);
    }
    a[0] = acc;
  } else {
    for (int it = 0; it < kPeakIters; ++it) {
#pragma unroll
      for (int s = 0; s < kStepsPerIter; ++s) {
#pragma unroll
        for (int i = 0; i < kChains; ++i) {
          const uint32_t x = a[(i + 1) % kChains], y = a[(i + 2) % kChains];
          if (KIND == kLop3) a[i] = lop3_xor(a[i], x, y);
          if (KIND == kDp2a) a[i] = dp2a(x, b, a[i]);
          if (KIND == kMix) a[i] = (i & 1) ? dp2a(x, b, a[i]) : lop3_xor(a[i], x, y);
          if (KIND == kAdd) a[i] = add32(a[i], x);
        }
      }
    }
  }
  __syncthreads();
  if (tid == 0) {
    ct.c1 = clock64();
    ct.t1 = gtimer();
    uint32_t sm;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(sm));
    ct.smid = sm;
    ct.pad = 0;
    times[blockIdx.x] = ct;
  }
  uint32_t r = 0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) r ^= a[i];
  if (r == 0x9E3779B9u) atomicAdd(sink, 1u);  // keeps every chain live
}

template <int KIND>
cudaError_t run_peak(int grid, uint32_t seed, uint32_t* sink, CtaTime* times) {
  k_peak<KIND><<<grid, kPeakThreads>>>(seed, sink, times);
  return cudaGetLastError();
}

}  // namespace

extern "C" {

int dd_measure_peaks(int32_t device, dd_peaks_t* out) {
  if (!out) return ddk::report_error(DD_ERR_ARG, "dd_measure_peaks: out is NULL");
  if (cudaSetDevice(device) != cudaSuccess)
    return ddk::report_error(DD_ERR_ARG, "dd_measure_peaks: no such device");
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      sms < 1)
    return ddk::report_error(DD_ERR_CUDA, "dd_measure_peaks: no multiprocessor count");
  const int grid = sms * kPeakCtasPerSm;
  uint32_t* sink = nullptr;
  CtaTime* d_times = nullptr;
  if (cudaMalloc(&sink, sizeof(uint32_t)) != cudaSuccess ||
      cudaMalloc(&d_times, sizeof(CtaTime) * grid) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(sink);
    return ddk::report_error(DD_ERR_NOMEM, "dd_measure_peaks: device buffers");
  }
  std::vector<CtaTime> h(grid);
  double rate[kKinds] = {};
  double cyc_sum = 0, ns_sum = 0;
  cudaError_t e = cudaMemset(sink, 0, sizeof(uint32_t));
  for (int kind = 0; kind < kKinds && e == cudaSuccess; ++kind) {
    // one untimed warm-up launch per kind, then the measured one
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
      switch (kind) {
        case kLop3: e = run_peak<kLop3>(grid, 12345u + rep, sink, d_times); break;
        case kDp2a: e = run_peak<kDp2a>(grid, 12345u + rep, sink, d_times); break;
        case kMix: e = run_peak<kMix>(grid, 12345u + rep, sink, d_times); break;
        case kAdd: e = run_peak<kAdd>(grid, 12345u + rep, sink, d_times); break;
        default: e = run_peak<kLds>(grid, 12345u + rep, sink, d_times); break;
      }
      if (e == cudaSuccess) e = cudaDeviceSynchronize();
    }
    if (e == cudaSuccess)
      e = cudaMemcpy(h.data(), d_times, sizeof(CtaTime) * grid, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) break;
    // per SM: operations of its CTAs over the cycles from the first start to the last end
    std::vector<unsigned long long> lo(1024, ~0ull), hi(1024, 0);
    std::vector<int> n(1024, 0);
    for (const auto& t : h) {
      if (t.smid >= 1024) continue;
      lo[t.smid] = std::min(lo[t.smid], t.c0);
      hi[t.smid] = std::max(hi[t.smid], t.c1);
      n[t.smid] += 1;
      cyc_sum += (double)(t.c1 - t.c0);
      ns_sum += (double)(t.t1 - t.t0);
    }
    // lane-operations per CTA (the load test counts wavefronts: one per warp-wide load)
    const double per_cta = kind == kLds ? (double)(kPeakThreads / 32) * kPeakIters *
                                              kStepsPerIter * kChains
                                        : (double)kPeakThreads * (double)kOpsPerThread;
    double acc = 0;
    int used = 0;
    for (int s = 0; s < 1024; ++s)
      if (n[s] > 0 && hi[s] > lo[s]) {
        acc += per_cta * n[s] / (double)(hi[s] - lo[s]);
        ++used;
      }
    rate[kind] = used ? acc / used : 0;
  }
  cudaFree(sink);
  cudaFree(d_times);
  if (e != cudaSuccess)
    return ddk::report_error(DD_ERR_CUDA, cudaGetErrorString(e));
  out->sms = sms;
  out->pad = 0;
  out->sm_mhz = ns_sum > 0 ? 1e3 * cyc_sum / ns_sum : 0;
  out->alu_lanes_per_clk = rate[kLop3];
  out->dp_lanes_per_clk = rate[kDp2a];
  out->int_lanes_per_clk = rate[kMix];
  out->add_per_clk = rate[kAdd];
  out->lds_wavefronts_per_clk = rate[kLds];
  return DD_OK;
}

}  // extern "C"
