// C ABI of the library: planning, the chunk/stream scheduler and the search driver.
//
// Scheduler (Sec. 1 and Sec. 2 of the paper: time chunks, stream IDs, pinned memory,
// asynchronous copies, no allocation or implicit synchronisation in the compute loop):
//   chunk k runs on slot k mod n_streams, each slot owning a CUDA stream and its own device
//   buffers (staging, channel-major ring, decimated rings, series, moments, candidates).
//   The history a chunk needs (the last H >= O samples of the stream so far) lives on the
//   device in `hist`; chunk k loads it after chunk k-1 saved it (one event per plan), so the
//   only cross-stream dependency is this short device-to-device copy.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <functional>
#include <mutex>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "dd_internal.h"

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

#define DD_CK(call)                                                                      \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail(DD_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));          \
  } while (0)

int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }

int ilog2(int64_t v) {
  int l = 0;
  while ((int64_t(1) << l) < v) ++l;
  return l;
}

// Bounded wait on an event (no spin on the GPU side; host polls with a deadline).
int wait_event(cudaEvent_t ev, int64_t timeout_ms) {
  if (timeout_ms <= 0) timeout_ms = 600000;
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    const cudaError_t e = cudaEventQuery(ev);
    if (e == cudaSuccess) return DD_OK;
    if (e != cudaErrorNotReady)
      return fail(DD_ERR_CUDA, "event wait failed: %s", cudaGetErrorString(e));
    const auto dt = std::chrono::steady_clock::now() - t0;
    if (std::chrono::duration_cast<std::chrono::milliseconds>(dt).count() > timeout_ms)
      return fail(DD_ERR_TIMEOUT, "GPU work did not finish within %lld ms",
                  (long long)timeout_ms);
    std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
}

// Host threads that split one host-to-host copy (pageable chunk -> pinned staging buffer)
// between them (Sec. 2.1: CPU threads filling small pinned buffers). copy() returns when every
// part is done.
class StagingPool {
 public:
  explicit StagingPool(int n) : n_(n) {
    for (int i = 0; i < n; ++i) threads_.emplace_back([this, i] { run(i); });
  }
  ~StagingPool() {
    {
      std::lock_guard<std::mutex> l(mu_);
      stop_ = true;
    }
    cv_.notify_all();
    for (auto& t : threads_) t.join();
  }
  void copy(uint8_t* dst, const uint8_t* src, size_t bytes) {
    std::unique_lock<std::mutex> l(mu_);
    dst_ = dst;
    src_ = src;
    bytes_ = bytes;
    pending_ = n_;
    ++gen_;
    cv_.notify_all();
    done_cv_.wait(l, [this] { return pending_ == 0; });
  }

 private:
  void run(int i) {
    uint64_t seen = 0;
    for (;;) {
      uint8_t* dst;
      const uint8_t* src;
      size_t bytes;
      {
        std::unique_lock<std::mutex> l(mu_);
        cv_.wait(l, [&] { return stop_ || gen_ != seen; });
        if (stop_) return;
        seen = gen_;
        dst = dst_;
        src = src_;
        bytes = bytes_;
      }
      const size_t n = (size_t)n_;  // workers never touch threads_ (filled while they start)
      const size_t part = (bytes + n - 1) / n;
      const size_t b0 = std::min(bytes, part * (size_t)i), b1 = std::min(bytes, b0 + part);
      if (b1 > b0) std::memcpy(dst + b0, src + b0, b1 - b0);
      {
        std::lock_guard<std::mutex> l(mu_);
        if (--pending_ == 0) done_cv_.notify_all();
      }
    }
  }
  const int n_;
  std::vector<std::thread> threads_;
  std::mutex mu_;
  std::condition_variable cv_, done_cv_;
  bool stop_ = false;
  uint64_t gen_ = 0;
  int pending_ = 0;
  uint8_t* dst_ = nullptr;
  const uint8_t* src_ = nullptr;
  size_t bytes_ = 0;
};

struct Slot {
  cudaStream_t stream = nullptr;
  cudaStream_t used = nullptr;  // stream the current chunk was enqueued on
  uint8_t* staging = nullptr;   // [chunk_len][nchans] host-input landing buffer
  uint8_t* ring1 = nullptr;     // [Cp][R1] channel-major, column 0 = global sample T - H
  uint16_t* ringd[9] = {};      // level l >= 1 (decimation 2^l): [Cp][Rd[l]]
  int32_t* series = nullptr;    // every range, at series_off[r]
  ddk::Moments* mom = nullptr;  // [total trials]
  ddk::WidthStats* wst = nullptr;  // [total trials][kMaxWidths] clipped statistics
  dd_cand_t* cands = nullptr;   // [max_cands]
  unsigned long long* d_count = nullptr;  // [0] candidates, [1] kernel error bits
  unsigned long long* h_count = nullptr;  // pinned copy of d_count
  cudaEvent_t ev_free = nullptr;          // last work enqueued for this slot
  cudaEvent_t ev_sps = nullptr;           // search + count readback done
  uint8_t* h_stage = nullptr;             // pinned staging buffer (staging_threads > 0)
  cudaEvent_t ev_staged = nullptr;        // copy out of h_stage finished
  uint8_t* fused = nullptr;               // fused-search records of every fused range
  int64_t seq = -1, T = 0, n = 0, lo = 0, hi = 0;
  bool searched = false;
};

}  // namespace

// How one range is dedispersed: the tiled delay-class kernel (with its tile shape, staging
// buffers and shared-memory sizes) or, when the plan does not fit it, the direct kernel (the
// one-thread-per-output kernel with DD_FLAG_NAIVE).
struct RangeKernel {
  bool tiled = false;
  int tt = 0;
  int trials = 0;             // trials per tile
  int threads = 0;            // threads per CTA
  int ctas = 0;               // CTAs per SM of the tile shape
  int nseg = 0;
  int nstage = 0;
  int row_slot = 0;
  int zcap = 0;
  size_t smem = 0;
  uint8_t* d_tabs = nullptr;  // device copy of the delay-class tables
  int64_t lsu_wavefronts = 0; // shared-memory work of one row of time tiles (TiledPlan)
  int64_t copy_bytes = 0;
  // search fused into the kernel (dd_fuse_search): decimated widths, the largest (hist),
  // shared-memory arrangement, most segments, and the offsets of the range's block records
  // (keys, offsets) and segment edges in the slot's fused arena
  bool fused = false;
  int nw = 0;
  int wd[ddk::kMaxWidths] = {};
  int hist = 0, hp = 0;
  int32_t e_off = 0;
  size_t fsmem = 0;
  int smax = 0;
  size_t key_off = 0, off_off = 0, edge_off = 0;
};

struct dd_plan_s {
  int device = 0;
  int32_t C = 0, Cp = 0;
  double tsamp = 0;
  std::vector<dd_range_t> ranges;
  dd_opts_t opts{};
  std::vector<int32_t> row0;       // first shift-table row of each range
  int32_t total_rows = 0;
  std::vector<int32_t> h_shifts;   // [total_rows][C] (plan_info view)
  int32_t* d_shifts = nullptr;     // [total_rows][Cp]
  int64_t O = 0, H = 0, L = 0;
  int dmax = 1, levels = 0;
  int64_t R1 = 0;
  int64_t Rd[9] = {};
  std::vector<int64_t> series_off, series_stride;
  int64_t series_elems = 0;
  std::vector<RangeKernel> rk;
  uint8_t* hist = nullptr;         // [Cp][H] device history
  cudaEvent_t ev_hist = nullptr;
  std::vector<Slot> slots;
  cudaStream_t io = nullptr;
  cudaEvent_t ev_io = nullptr;
  dd_cand_t* h_cands = nullptr;    // pinned [max_cands]
  int64_t next_seq = 0, T_total = 0;
  int64_t launches = 0;
  StagingPool* pool = nullptr;     // staging_threads > 0
  int32_t* err_word = nullptr;     // if set, kernel error bits go here instead of the slot's
  cudaEvent_t gate = nullptr;      // if set, the next chunk's dedispersion waits for it (once)
  std::vector<int32_t> fused_widths;  // dd_fuse_search's widths (original samples); empty: none
  bool fused_series = false;       // fused ranges also write their series
  int sms = 0;
  // dedispersion timing (DD_FLAG_TIMING): every launch is bracketed by an event pair; the pairs
  // are turned into [start, end) intervals against a common reference event and merged, so that
  // launches of different chunks running at the same time on different streams count once
  std::vector<cudaEvent_t> tev;
  std::vector<int32_t> tev_range;  // range of each recorded launch
  int64_t tev_used = 0;
  cudaEvent_t tref = nullptr;
  bool tref_set = false;
  std::vector<std::pair<double, double>> intervals;
  std::vector<int32_t> interval_range;
  double dedisp_ms = 0;
  int64_t dedisp_launches = 0;
};

namespace {

void free_plan(dd_plan_s* p) {
  if (!p) return;
  cudaSetDevice(p->device);
  for (auto& s : p->slots) {
    if (s.stream) cudaStreamSynchronize(s.stream);
  }
  if (p->io) cudaStreamSynchronize(p->io);
  delete p->pool;
  for (auto& s : p->slots) {
    cudaFreeHost(s.h_stage);
    if (s.ev_staged) cudaEventDestroy(s.ev_staged);
    cudaFree(s.staging);
    cudaFree(s.ring1);
    for (auto* r : s.ringd) cudaFree(r);
    cudaFree(s.series);
    cudaFree(s.fused);
    cudaFree(s.mom);
    cudaFree(s.wst);
    cudaFree(s.cands);
    cudaFree(s.d_count);
    cudaFreeHost(s.h_count);
    if (s.ev_free) cudaEventDestroy(s.ev_free);
    if (s.ev_sps) cudaEventDestroy(s.ev_sps);
    if (s.stream) cudaStreamDestroy(s.stream);
  }
  for (auto e : p->tev) cudaEventDestroy(e);
  if (p->tref) cudaEventDestroy(p->tref);
  for (auto& k : p->rk) cudaFree(k.d_tabs);
  cudaFree(p->d_shifts);
  cudaFree(p->hist);
  cudaFreeHost(p->h_cands);
  if (p->ev_hist) cudaEventDestroy(p->ev_hist);
  if (p->ev_io) cudaEventDestroy(p->ev_io);
  if (p->io) cudaStreamDestroy(p->io);
  delete p;
}

template <typename T>
int dalloc(T** ptr, size_t bytes, const char* what) {
  if (bytes == 0) bytes = 16;
  if (cudaMalloc((void**)ptr, bytes) != cudaSuccess) {
    cudaGetLastError();
    *ptr = nullptr;
    return fail(DD_ERR_NOMEM, "device allocation of %zu bytes for %s failed", bytes, what);
  }
  return DD_OK;
}

// Plan one range on the tiled kernel with one tile shape (tt outputs x trials trials): the
// delay-class tables on the device and the kernel instance's shared-memory attribute. *ok =
// false (and nothing allocated) when the shape does not fit the range.
int plan_tiled_shape(const int32_t* tab, int ntr, int cpad, int d, int tt, int trials,
                     int threads, RangeKernel* k, bool* ok) {
  *ok = false;
  ddk::TiledPlan tp = ddk::tiled_plan(tab, ntr, cpad, d, tt, trials, threads);
  if (!tp.ok) return DD_OK;
  RangeKernel r;
  if (dalloc(&r.d_tabs, tp.tab_bytes, "delay-class tables")) return DD_ERR_NOMEM;
  cudaError_t e = cudaMemcpy(r.d_tabs, tp.tabs.data(), tp.tab_bytes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = ddk::prepare_tiled(d > 1, tt, tp.nstage, trials, threads, tp.smem);
  if (e != cudaSuccess) {
    cudaFree(r.d_tabs);
    return fail(DD_ERR_CUDA, "tiled kernel set-up: %s", cudaGetErrorString(e));
  }
  r.tiled = true;
  r.tt = tt;
  r.trials = trials;
  r.threads = threads;
  r.ctas = tp.ctas;
  r.nseg = tp.nseg;
  r.nstage = tp.nstage;
  r.row_slot = tp.row_slot;
  r.zcap = tp.zcap;
  r.smem = tp.smem;
  r.lsu_wavefronts = tp.lsu_wavefronts;
  r.copy_bytes = tp.copy_bytes;
  *k = r;
  *ok = true;
  return DD_OK;
}

// Tile shapes (outputs, trials, threads per CTA) in the order a plan tries them.
constexpr int kShapes[4][3] = {{512, 64, 512}, {512, 64, 1024}, {256, 64, 512}, {256, 32, 512}};

// Turn recorded event pairs into intervals relative to the reference event.
int harvest_timing(dd_plan_s* p) {
  for (int64_t k = 0; k < p->tev_used; ++k) {
    cudaEvent_t a = p->tev[2 * k], b = p->tev[2 * k + 1];
    DD_CK(cudaEventSynchronize(b));
    float t0 = 0, t1 = 0;
    DD_CK(cudaEventElapsedTime(&t0, p->tref, a));
    DD_CK(cudaEventElapsedTime(&t1, p->tref, b));
    p->intervals.emplace_back(t0, t1);
    p->interval_range.push_back(p->tev_range[k]);
    p->dedisp_launches += 1;
  }
  p->tev_used = 0;
  return DD_OK;
}

// Length of the union of the harvested intervals (ms).
double union_ms(std::vector<std::pair<double, double>> v) {
  std::sort(v.begin(), v.end());
  double total = 0, cs = 0, ce = -1e300;
  for (auto& iv : v) {
    if (iv.first > ce) {
      if (ce > cs) total += ce - cs;
      cs = iv.first;
      ce = iv.second;
    } else if (iv.second > ce) {
      ce = iv.second;
    }
  }
  if (ce > cs) total += ce - cs;
  return total;
}

int timing_begin(dd_plan_s* p, cudaStream_t st, int32_t range, int64_t* slot) {
  *slot = -1;
  if (!(p->opts.flags & DD_FLAG_TIMING)) return DD_OK;
  if (!p->tref_set) {
    DD_CK(cudaEventRecord(p->tref, st));
    p->tref_set = true;
  }
  if (2 * (p->tev_used + 1) > (int64_t)p->tev.size()) {
    int rc = harvest_timing(p);
    if (rc) return rc;
  }
  *slot = p->tev_used++;
  p->tev_range[*slot] = range;
  DD_CK(cudaEventRecord(p->tev[2 * *slot], st));
  return DD_OK;
}

int timing_end(dd_plan_s* p, cudaStream_t st, int64_t slot) {
  if (slot < 0) return DD_OK;
  DD_CK(cudaEventRecord(p->tev[2 * slot + 1], st));
  return DD_OK;
}

}  // namespace

namespace ddk {
int report_error(int code, const char* msg) { return fail(code, "%s", msg); }

int plan_reset(dd_plan_s* p) {
  DD_CK(cudaSetDevice(p->device));
  for (auto& s : p->slots) {
    DD_CK(cudaStreamSynchronize(s.stream));
    if (s.used && s.used != s.stream) DD_CK(cudaStreamSynchronize(s.used));
    s.seq = -1;
    s.searched = false;
    s.used = nullptr;
  }
  p->next_seq = 0;
  p->T_total = 0;
  return DD_OK;
}

void plan_streams(dd_plan_s* p, std::vector<cudaStream_t>* out) {
  for (auto& s : p->slots) out->push_back(s.stream);
}

int64_t plan_outputs(dd_plan_s* p, int64_t nsamp) {
  int64_t n = 0;
  const int64_t hi = std::max<int64_t>(0, nsamp - p->O);
  for (auto& r : p->ranges) n += (int64_t)r.n_trials * (hi / r.decimation);
  return n;
}

int sps_enqueue(dd_plan_s* p, const int32_t* widths, int32_t nwidths, float threshold,
                dd_cand_t* cands, unsigned long long* count, int64_t cap) {
  if (p->next_seq == 0) return fail(DD_ERR_STATE, "no chunk has been run");
  Slot& s = p->slots[(p->next_seq - 1) % p->slots.size()];
  if (s.searched) return fail(DD_ERR_STATE, "the latest chunk was already searched");
  for (const auto& k : p->rk)
    if (k.fused) return fail(DD_ERR_STATE, "a fused plan's search runs through sps_run");
  cudaStream_t st = s.used;
  DD_CK(cudaMemsetAsync(count, 0, sizeof(unsigned long long), st));
  for (size_t r = 0; r < p->ranges.size(); ++r) {
    const int d = p->ranges[r].decimation;
    ddk::SpsArgs a;
    std::memset(&a, 0, sizeof a);
    for (int k = 0; k < nwidths; ++k)
      if (widths[k] >= d && widths[k] % d == 0) a.wd[a.nw++] = widths[k] / d;
    a.n = (s.hi - s.lo) / d;
    if (a.nw == 0 || a.n <= 0) continue;
    a.y = s.series + p->series_off[r];
    a.stride = p->series_stride[r];
    a.mom = s.mom + p->row0[r];
    a.n_trials = p->ranges[r].n_trials;
    a.range = (int32_t)r;
    a.d = d;
    a.block = p->opts.peak_block;
    a.J0 = s.lo / d;
    a.hist = (int32_t)round_up(std::max(a.wd[a.nw - 1] - 1, 0), 256);
    a.threshold = threshold;
    a.cands = cands;
    a.count = count;
    a.cap = cap;
    DD_CK(ddk::launch_sps(a, st));
    p->launches += 1;
  }
  DD_CK(cudaEventRecord(s.ev_free, st));
  s.searched = true;
  return DD_OK;
}

// Time the tiled kernel of every range at each of its candidate tile sizes on the plan's own
// buffers (contents irrelevant) and keep the fastest; the plan must be idle.
int plan_autotune(dd_plan_s* p) {
  DD_CK(cudaSetDevice(p->device));
  Slot& s = p->slots[0];
  cudaEvent_t e0, e1;
  DD_CK(cudaEventCreate(&e0));
  DD_CK(cudaEventCreate(&e1));
  int rc = DD_OK;
  for (size_t r = 0; r < p->ranges.size() && rc == DD_OK; ++r) {
    RangeKernel& cur = p->rk[r];
    if (!cur.tiled) continue;
    const int d = p->ranges[r].decimation;
    const bool u16 = d > 1;
    const int l = ilog2(d);
    std::vector<int32_t> tab((size_t)p->ranges[r].n_trials * p->Cp);
    if (cudaMemcpy(tab.data(), p->d_shifts + (int64_t)p->row0[r] * p->Cp,
                   sizeof(int32_t) * tab.size(), cudaMemcpyDeviceToHost) != cudaSuccess) {
      rc = fail(DD_ERR_CUDA, "autotune: reading the delay table failed");
      break;
    }
    float best_ms = 1e30f;
    RangeKernel best = cur;
    for (int shape = 0; shape < 4; ++shape) {
      const int tt = kShapes[shape][0], trials = kShapes[shape][1], nt = kShapes[shape][2];
      RangeKernel k = cur;
      if (tt != cur.tt || trials != cur.trials || nt != cur.threads) {
        bool ok = false;
        rc = plan_tiled_shape(tab.data(), p->ranges[r].n_trials, p->Cp, d, tt, trials, nt, &k,
                              &ok);
        if (rc) break;
        if (!ok) continue;
      }
      ddk::TiledArgs A;
      A.xd = (l == 0) ? (const void*)s.ring1 : (const void*)s.ringd[l];
      A.xd_stride = (l == 0) ? p->R1 : p->Rd[l];
      if (ddk::make_ring_map(&A.rows, A.xd, u16, A.xd_stride, p->Cp, k.nseg) != cudaSuccess) {
        if (k.d_tabs != cur.d_tabs) cudaFree(k.d_tabs);
        rc = fail(DD_ERR_CUDA, "autotune: tensor map of the ring could not be made");
        break;
      }
      A.m0 = 0;
      A.nout = std::max<int64_t>(1, (p->L - p->O + p->H) / d);
      A.nout = std::min<int64_t>(A.nout, p->L / d);
      A.y = s.series + p->series_off[r];
      A.y_stride = p->series_stride[r];
      A.mom = s.mom + p->row0[r];
      A.shifts = p->d_shifts + (int64_t)p->row0[r] * p->Cp;
      A.n_trials = p->ranges[r].n_trials;
      A.cpad = p->Cp;
      A.row_slot = k.row_slot;
      A.zcap = k.zcap;
      A.nstage = k.nstage;
      A.tabs = k.d_tabs;
      A.err = reinterpret_cast<int32_t*>(s.d_count + 1);
      // one warm-up launch, then the better of two timed ones
      float ms = 1e30f;
      cudaError_t e = ddk::launch_tiled(A, u16, k.tt, k.trials, k.threads, s.stream);
      for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
        float t = 0;
        e = cudaEventRecord(e0, s.stream);
        if (e == cudaSuccess) e = ddk::launch_tiled(A, u16, k.tt, k.trials, k.threads, s.stream);
        if (e == cudaSuccess) e = cudaEventRecord(e1, s.stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
        ms = std::min(ms, t);
      }
      if (e != cudaSuccess) {
        if (k.d_tabs != cur.d_tabs) cudaFree(k.d_tabs);
        rc = fail(DD_ERR_CUDA, "autotune: timing launch failed: %s", cudaGetErrorString(e));
        break;
      }
      if (ms < best_ms) {
        if (best.d_tabs != cur.d_tabs) cudaFree(best.d_tabs);
        best_ms = ms;
        best = k;
      } else if (k.d_tabs != cur.d_tabs) {
        cudaFree(k.d_tabs);
      }
    }
    if (rc != DD_OK) break;
    if (best.d_tabs != cur.d_tabs) {
      cudaFree(cur.d_tabs);
      cur = best;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  DD_CK(cudaMemsetAsync(s.d_count, 0, 2 * sizeof(unsigned long long), s.stream));
  DD_CK(cudaStreamSynchronize(s.stream));
  return rc;
}

int range_tile(dd_plan_s* p, int r) { return p->rk[r].tiled ? p->rk[r].tt : 0; }

void plan_gate_next(dd_plan_s* p, cudaEvent_t ev) { p->gate = ev; }

cudaEvent_t chunk_done_event(dd_plan_s* p, int64_t seq) {
  const int64_t S = (int64_t)p->slots.size();
  if (seq < 0 || seq >= p->next_seq || seq < p->next_seq - S) return nullptr;
  Slot& s = p->slots[seq % S];
  return (s.seq == seq && s.searched) ? s.ev_sps : nullptr;
}

void plan_redirect_errors(dd_plan_s* p, int32_t* err) { p->err_word = err; }

int chunk_state(dd_plan_s* p, int64_t seq) {
  const int64_t S = (int64_t)p->slots.size();
  if (seq < 0 || seq >= p->next_seq || seq < p->next_seq - S) return DD_ERR_STATE;
  Slot& s = p->slots[seq % S];
  if (s.seq != seq || !s.searched) return DD_ERR_STATE;
  const cudaError_t e = cudaEventQuery(s.ev_sps);
  if (e == cudaSuccess) return 1;
  if (e == cudaErrorNotReady) return 0;
  return fail(DD_ERR_CUDA, "chunk state: %s", cudaGetErrorString(e));
}
}  // namespace ddk

extern "C" {

const char* dd_last_error(void) { return g_err.c_str(); }

int dd_plan(const double* freqs_mhz, int32_t nchans, double tsamp_s, const dd_range_t* ranges,
            int32_t nranges, const dd_opts_t* opts, dd_plan_t* out) {
  if (!out) return fail(DD_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!freqs_mhz || !ranges || !opts) return fail(DD_ERR_ARG, "NULL argument");
  if (nchans < 1 || nchans > 65532) return fail(DD_ERR_ARG, "nchans %d outside 1..65532", nchans);
  if (!(tsamp_s > 0) || !std::isfinite(tsamp_s)) return fail(DD_ERR_ARG, "tsamp must be > 0");
  if (nranges < 1 || nranges > ddk::kMaxRanges)
    return fail(DD_ERR_ARG, "nranges %d outside 1..%d", nranges, ddk::kMaxRanges);
  for (int c = 0; c < nchans; ++c)
    if (!(freqs_mhz[c] > 0) || !std::isfinite(freqs_mhz[c]))
      return fail(DD_ERR_ARG, "frequency %d is not a positive finite number", c);
  int dmax = 1;
  int64_t total_rows = 0;
  for (int r = 0; r < nranges; ++r) {
    const dd_range_t& R = ranges[r];
    if (R.n_trials < 1 || R.n_trials > 65535)
      return fail(DD_ERR_ARG, "range %d: n_trials %d outside 1..65535", r, R.n_trials);
    if (!is_pow2(R.decimation) || R.decimation > 256)
      return fail(DD_ERR_ARG, "range %d: decimation %d is not a power of two <= 256", r,
                  R.decimation);
    if (!(R.dm_start >= 0) || !(R.dm_step >= 0) || !std::isfinite(R.dm_start) ||
        !std::isfinite(R.dm_step))
      return fail(DD_ERR_ARG, "range %d: dm_start and dm_step must be finite and >= 0", r);
    dmax = std::max(dmax, R.decimation);
    total_rows += R.n_trials;
  }
  if (total_rows > (1 << 24)) return fail(DD_ERR_ARG, "too many trials");
  const dd_opts_t& o = *opts;
  // launch grids: time tiles of >= 256 outputs and one row per trial in a 65535-wide dimension
  if (o.chunk_len < 256 || o.chunk_len % 256 != 0 || o.chunk_len > int64_t(65535) * 256)
    return fail(DD_ERR_ARG, "chunk_len %lld must be a multiple of 256 in 256..16776960",
                (long long)o.chunk_len);
  if (o.n_streams < 1 || o.n_streams > 16)
    return fail(DD_ERR_ARG, "n_streams %d outside 1..16", o.n_streams);
  if (o.max_width < 1 || o.max_width > 1024)
    return fail(DD_ERR_ARG, "max_width %d outside 1..1024", o.max_width);
  if (!is_pow2(o.peak_block) || o.peak_block > 32)
    return fail(DD_ERR_ARG, "peak_block %d must be a power of two <= 32", o.peak_block);
  if ((int64_t)nchans * 255 * std::max(dmax, o.max_width) >= (int64_t(1) << 31))
    return fail(DD_ERR_ARG, "nchans*255*max(width, decimation) must be < 2^31 (int32 sums)");
  if (o.max_cands < 0) return fail(DD_ERR_ARG, "max_cands < 0");
  if (o.staging_threads < 0 || o.staging_threads > 64)
    return fail(DD_ERR_ARG, "staging_threads %d outside 0..64", o.staging_threads);

  int ndev = 0;
  DD_CK(cudaGetDeviceCount(&ndev));
  if (o.device < 0 || o.device >= ndev)
    return fail(DD_ERR_ARG, "device %d not present (%d devices)", o.device, ndev);
  DD_CK(cudaSetDevice(o.device));

  dd_plan_s* p = new dd_plan_s();
  p->device = o.device;
  p->C = nchans;
  p->Cp = (int32_t)round_up(nchans, 8);
  p->tsamp = tsamp_s;
  p->ranges.assign(ranges, ranges + nranges);
  p->opts = o;
  if (p->opts.max_cands == 0) p->opts.max_cands = int64_t(1) << 20;
  p->total_rows = (int32_t)total_rows;
  p->dmax = dmax;
  p->levels = ilog2(dmax);
  p->L = o.chunk_len;
  int rc = DD_OK;
#define DD_TRY(x)          \
  do {                     \
    rc = (x);              \
    if (rc) {              \
      free_plan(p);        \
      return rc;           \
    }                      \
  } while (0)
#define DD_TRYCK(call)                                                             \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      free_plan(p);                                                                \
      return fail(DD_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));    \
    }                                                                              \
  } while (0)

  // ---- delay table on the GPU (plan phase: one-off)
  std::vector<ddk::ShiftRange> sr(nranges);
  p->row0.resize(nranges);
  int32_t row = 0;
  for (int r = 0; r < nranges; ++r) {
    sr[r] = {ranges[r].dm_start, ranges[r].dm_step, ranges[r].n_trials, ranges[r].decimation,
             row, 0};
    p->row0[r] = row;
    row += ranges[r].n_trials;
  }
  double fref = freqs_mhz[0];
  for (int c = 1; c < nchans; ++c) fref = std::max(fref, freqs_mhz[c]);
  double* d_freqs = nullptr;
  int32_t* d_err = nullptr;
  DD_TRY(dalloc(&p->d_shifts, sizeof(int32_t) * (size_t)total_rows * p->Cp, "delay table"));
  DD_TRY(dalloc(&d_freqs, sizeof(double) * nchans, "frequencies"));
  if (dalloc(&d_err, sizeof(int32_t), "flag")) {
    cudaFree(d_freqs);
    free_plan(p);
    return DD_ERR_NOMEM;
  }
  {
    cudaError_t e = cudaMemcpy(d_freqs, freqs_mhz, sizeof(double) * nchans, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(d_err, 0, sizeof(int32_t));
    if (e == cudaSuccess)
      e = ddk::launch_shift_table(d_freqs, nchans, p->Cp, fref, tsamp_s, sr.data(), nranges,
                                  (int32_t)total_rows, p->d_shifts, d_err, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    int32_t herr = 0;
    std::vector<int32_t> full((size_t)total_rows * p->Cp);
    if (e == cudaSuccess) e = cudaMemcpy(&herr, d_err, sizeof herr, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess)
      e = cudaMemcpy(full.data(), p->d_shifts, sizeof(int32_t) * full.size(),
                     cudaMemcpyDeviceToHost);
    cudaFree(d_freqs);
    cudaFree(d_err);
    if (e != cudaSuccess) {
      free_plan(p);
      return fail(DD_ERR_CUDA, "delay table: %s", cudaGetErrorString(e));
    }
    p->launches += 1;
    if (herr) {
      free_plan(p);
      return fail(DD_ERR_ARG, "a delay does not fit a non-negative int32 sample count");
    }
    p->h_shifts.resize((size_t)total_rows * nchans);
    for (int64_t rr = 0; rr < total_rows; ++rr)
      std::memcpy(&p->h_shifts[rr * nchans], &full[rr * p->Cp], sizeof(int32_t) * nchans);
    // overlap O = d_max * ceil(max_r(d_r * max s_r) / d_max)
    int64_t need = 0;
    for (int r = 0; r < nranges; ++r) {
      int64_t smax = 0;
      for (int64_t rr = p->row0[r]; rr < p->row0[r] + ranges[r].n_trials; ++rr)
        for (int c = 0; c < nchans; ++c) smax = std::max<int64_t>(smax, p->h_shifts[rr * nchans + c]);
      need = std::max<int64_t>(need, smax * ranges[r].decimation);
    }
    p->O = round_up(need, dmax);
    p->rk.resize(nranges);
    if (!(o.flags & DD_FLAG_NAIVE)) {
      for (int r = 0; r < nranges; ++r) {
        // the first shape that fits, in kShapes order; testing aids force the 256-output tile
        // (DD_FLAG_TILE256) or the 32-trial tile (DD_FLAG_TRIALS32)
        for (int shape = 0; shape < 4 && !p->rk[r].tiled; ++shape) {
          const int tt = kShapes[shape][0], trials = kShapes[shape][1], nt = kShapes[shape][2];
          if ((o.flags & DD_FLAG_TILE256) && tt != 256) continue;
          if ((o.flags & DD_FLAG_TRIALS32) && trials != 32) continue;
          if ((o.flags & DD_FLAG_WARPS32) != 0 && nt != 1024) continue;
          bool ok = false;
          const int rc2 = plan_tiled_shape(&full[(size_t)p->row0[r] * p->Cp], ranges[r].n_trials,
                                           p->Cp, ranges[r].decimation, tt, trials, nt,
                                           &p->rk[r], &ok);
          if (rc2) {
            free_plan(p);
            return rc2;
          }
        }
      }
    }
  }
  // history kept on the device: O rounded up so every ring row starts 256-byte aligned
  p->H = round_up(p->O, 256);
  const int64_t span = p->H + p->L;
  // rows carry slack past the data so a ragged last time tile may stage (and ignore) a full tile
  p->R1 = round_up(span, 256) + 2048;
  for (int l = 1; l <= p->levels; ++l) p->Rd[l] = round_up(span >> l, 128) + 2048;
  p->series_off.resize(nranges);
  p->series_stride.resize(nranges);
  int64_t off = 0;
  for (int r = 0; r < nranges; ++r) {
    const int64_t st = round_up(p->L / ranges[r].decimation, 32);
    p->series_off[r] = off;
    p->series_stride[r] = st;
    off += st * ranges[r].n_trials;
  }
  p->series_elems = off;

  // ---- buffers (all allocation happens here)
  DD_TRY(dalloc(&p->hist, (size_t)p->Cp * std::max<int64_t>(p->H, 1), "history"));
  DD_TRYCK(cudaMemset(p->hist, 0, (size_t)p->Cp * std::max<int64_t>(p->H, 1)));
  DD_TRYCK(cudaEventCreateWithFlags(&p->ev_hist, cudaEventDisableTiming));
  DD_TRYCK(cudaStreamCreateWithFlags(&p->io, cudaStreamNonBlocking));
  DD_TRYCK(cudaEventCreateWithFlags(&p->ev_io, cudaEventDisableTiming));
  if (cudaMallocHost((void**)&p->h_cands, sizeof(dd_cand_t) * p->opts.max_cands) != cudaSuccess) {
    cudaGetLastError();
    p->h_cands = nullptr;
    free_plan(p);
    return fail(DD_ERR_NOMEM, "pinned candidate buffer");
  }
  p->slots.resize(o.n_streams);
  for (auto& s : p->slots) {
    DD_TRYCK(cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking));
    DD_TRYCK(cudaEventCreateWithFlags(&s.ev_free, cudaEventDisableTiming));
    DD_TRYCK(cudaEventCreateWithFlags(&s.ev_sps, cudaEventDisableTiming));
    if (!(o.flags & DD_FLAG_DEVICE_INPUT))
      DD_TRY(dalloc(&s.staging, (size_t)p->L * nchans, "staging"));
    DD_TRY(dalloc(&s.ring1, (size_t)p->Cp * p->R1, "ring"));
    DD_TRYCK(cudaMemset(s.ring1, 0, (size_t)p->Cp * p->R1));
    for (int l = 1; l <= p->levels; ++l) {
      DD_TRY(dalloc(&s.ringd[l], sizeof(uint16_t) * (size_t)p->Cp * p->Rd[l], "decimated ring"));
      DD_TRYCK(cudaMemset(s.ringd[l], 0, sizeof(uint16_t) * (size_t)p->Cp * p->Rd[l]));
    }
    DD_TRY(dalloc(&s.series, sizeof(int32_t) * (size_t)p->series_elems, "series"));
    DD_TRY(dalloc(&s.mom, sizeof(ddk::Moments) * (size_t)total_rows, "moments"));
    DD_TRY(dalloc(&s.wst, sizeof(ddk::WidthStats) * (size_t)total_rows * ddk::kMaxWidths,
                  "clipped statistics"));
    DD_TRY(dalloc(&s.cands, sizeof(dd_cand_t) * (size_t)p->opts.max_cands, "candidates"));
    DD_TRY(dalloc(&s.d_count, 2 * sizeof(unsigned long long), "count"));
    DD_TRYCK(cudaMemset(s.d_count, 0, 2 * sizeof(unsigned long long)));
    if (o.staging_threads > 0) {
      if (cudaMallocHost((void**)&s.h_stage, (size_t)p->L * nchans) != cudaSuccess) {
        cudaGetLastError();
        s.h_stage = nullptr;
        free_plan(p);
        return fail(DD_ERR_NOMEM, "pinned staging buffer");
      }
      DD_TRYCK(cudaEventCreateWithFlags(&s.ev_staged, cudaEventDisableTiming));
    }
    if (cudaMallocHost((void**)&s.h_count, 2 * sizeof(unsigned long long)) != cudaSuccess) {
      cudaGetLastError();
      s.h_count = nullptr;
      free_plan(p);
      return fail(DD_ERR_NOMEM, "pinned count");
    }
  }
  if (o.staging_threads > 0) p->pool = new StagingPool(o.staging_threads);
  if (o.flags & DD_FLAG_TIMING) {
    p->tev.resize(2 * 1024);
    p->tev_range.resize(1024);
    for (auto& e : p->tev) DD_TRYCK(cudaEventCreate(&e));
    DD_TRYCK(cudaEventCreate(&p->tref));
    p->intervals.reserve(1 << 16);
  }
  DD_TRYCK(cudaDeviceSynchronize());
  if (o.flags & DD_FLAG_AUTOTUNE) DD_TRY(ddk::plan_autotune(p));
#undef DD_TRY
#undef DD_TRYCK
  *out = p;
  return DD_OK;
}

int dd_plan_info(dd_plan_t p, int64_t* overlap, int32_t* ntrials, const int32_t** shifts) {
  if (!p) return fail(DD_ERR_ARG, "plan is NULL");
  if (overlap) *overlap = p->O;
  if (ntrials) *ntrials = p->total_rows;
  if (shifts) *shifts = p->h_shifts.data();
  return DD_OK;
}

int dd_plan_kernel(dd_plan_t p, int32_t range, int32_t* kind, int32_t* tile_samples) {
  if (!p) return fail(DD_ERR_ARG, "plan is NULL");
  if (range < 0 || range >= (int32_t)p->rk.size())
    return fail(DD_ERR_ARG, "range %d out of bounds", (int)range);
  const bool tiled = p->rk[range].tiled;
  if (kind)
    *kind = tiled ? DD_KERNEL_TILED
                  : ((p->opts.flags & DD_FLAG_NAIVE) ? DD_KERNEL_PER_OUTPUT : DD_KERNEL_DIRECT);
  if (tile_samples) *tile_samples = tiled ? p->rk[range].tt : 0;
  return DD_OK;
}

int dd_plan_model(dd_plan_t p, int32_t range, int64_t nout, dd_launch_model_t* out) {
  if (!p || !out) return fail(DD_ERR_ARG, "NULL argument");
  if (range < 0 || range >= (int32_t)p->rk.size() || nout < 0)
    return fail(DD_ERR_ARG, "range out of bounds or nout < 0");
  const RangeKernel& k = p->rk[range];
  const dd_range_t& R = p->ranges[range];
  std::memset(out, 0, sizeof *out);
  out->kind = k.tiled ? DD_KERNEL_TILED
                      : ((p->opts.flags & DD_FLAG_NAIVE) ? DD_KERNEL_PER_OUTPUT : DD_KERNEL_DIRECT);
  out->tile_samples = k.tiled ? k.tt : 0;
  out->tile_trials = k.tiled ? k.trials : 0;
  out->cta_threads = k.tiled ? k.threads : 0;
  out->ctas_per_sm = k.tiled ? k.ctas : 0;
  out->outputs = (int64_t)R.n_trials * nout;
  out->adds = (double)out->outputs * p->C;
  int64_t smax = 0;
  for (int64_t rr = p->row0[range]; rr < p->row0[range] + R.n_trials; ++rr)
    for (int c = 0; c < p->C; ++c) smax = std::max<int64_t>(smax, p->h_shifts[rr * p->C + c]);
  const int es = R.decimation > 1 ? 2 : 1;
  // written per output: the int32 series, or, fused, a 4-byte sum and a 1-byte sample per
  // (width, peak block) (and the series if kept)
  double out_bytes = 4.0 * out->outputs;
  if (k.fused) {
    const double blocks = (double)R.n_trials * (double)((nout + p->opts.peak_block - 1) /
                                                        p->opts.peak_block);
    out_bytes = 5.0 * k.nw * blocks + (p->fused_series ? out_bytes : 0.0);
    out->fused = 1;
  }
  out->dram_bytes = nout > 0 ? (double)p->C * (double)(nout + smax) * es + out_bytes : 0;
  if (k.tiled && nout > 0) {
    const double rows = (double)((nout + k.tt - 1) / k.tt);
    out->smem_wavefronts = rows * (double)k.lsu_wavefronts;
    out->copy_bytes = rows * (double)k.copy_bytes;
  }
  return DD_OK;
}

int dd_fuse_search(dd_plan_t p, const int32_t* widths, int32_t nwidths, uint32_t fuse_flags,
                   int32_t* nfused) {
  if (!p) return fail(DD_ERR_ARG, "plan is NULL");
  if (!widths || nwidths < 1 || nwidths > ddk::kMaxWidths)
    return fail(DD_ERR_ARG, "nwidths must be 1..%d", ddk::kMaxWidths);
  for (int k = 0; k < nwidths; ++k) {
    if (widths[k] < 1 || widths[k] > p->opts.max_width)
      return fail(DD_ERR_ARG, "width %d outside 1..max_width", widths[k]);
    if (k > 0 && widths[k] <= widths[k - 1])
      return fail(DD_ERR_ARG, "widths must be strictly increasing");
  }
  if (fuse_flags & ~DD_FUSE_KEEP_SERIES) return fail(DD_ERR_ARG, "unknown fuse flags");
  if (p->next_seq != 0)
    return fail(DD_ERR_STATE, "dd_fuse_search must come before the plan's first dd_run");
  if (!p->fused_widths.empty()) return fail(DD_ERR_STATE, "the plan's search is already fused");
  DD_CK(cudaSetDevice(p->device));
  DD_CK(cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, p->device));
  const bool keep = (fuse_flags & DD_FUSE_KEEP_SERIES) != 0;
  const int nr = (int)p->ranges.size();
  std::vector<int32_t> full;  // the delay table at the padded stride, for re-planning a range
  std::vector<RangeKernel> nk = p->rk;
  std::vector<bool> replanned(nr, false);
  size_t arena = 0;
  int count = 0;
  int rc = DD_OK;
  for (int r = 0; r < nr && rc == DD_OK && !(p->opts.flags & DD_FLAG_NAIVE); ++r) {
    const int d = p->ranges[r].decimation, ntr = p->ranges[r].n_trials;
    int wd[ddk::kMaxWidths], nw = 0;
    for (int k = 0; k < nwidths; ++k)
      if (widths[k] >= d && widths[k] % d == 0) wd[nw++] = widths[k] / d;
    if (nw == 0 || wd[nw - 1] > 512 || !nk[r].tiled) continue;
    RangeKernel& K = nk[r];
    if (!(K.tt == 512 && K.trials == 64 && K.threads == 512)) {
      // the fused form exists for the 64 x 512 x 512 shape: plan the range on it
      if (full.empty()) {
        full.resize((size_t)p->total_rows * p->Cp);
        const cudaError_t e = cudaMemcpy(full.data(), p->d_shifts, sizeof(int32_t) * full.size(),
                                         cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
          rc = fail(DD_ERR_CUDA, "delay table: %s", cudaGetErrorString(e));
          break;
        }
      }
      RangeKernel k2;
      bool ok = false;
      rc = plan_tiled_shape(&full[(size_t)p->row0[r] * p->Cp], ntr, p->Cp, d, 512, 64, 512, &k2,
                            &ok);
      if (rc || !ok) continue;
      K = k2;
      replanned[r] = true;
    }
    const int hp = (int)round_up(wd[nw - 1], 32);
    int32_t e_off = 0;
    size_t fsmem = 0;
    if (!ddk::fused_smem(d > 1, K.row_slot, K.zcap, K.nstage, hp, &e_off, &fsmem)) {
      if (replanned[r]) {  // keep the range as it was planned
        cudaFree(K.d_tabs);
        K = p->rk[r];
        replanned[r] = false;
      }
      continue;
    }
    const cudaError_t e = ddk::prepare_fused(d > 1, K.nstage, fsmem);
    if (e != cudaSuccess) {
      rc = fail(DD_ERR_CUDA, "fused kernel set-up: %s", cudaGetErrorString(e));
      break;
    }
    K.fused = true;
    K.nw = nw;
    for (int k = 0; k < nw; ++k) K.wd[k] = wd[k];
    K.hist = wd[nw - 1];
    K.hp = hp;
    K.e_off = e_off;
    K.fsmem = fsmem;
    // record sizes for the longest window (L / d outputs)
    const int64_t nmax = p->L / d;
    const int ntx = (ntr + 63) / 64, ntt = (int)((nmax + 511) / 512);
    K.smax = ddk::fused_segments(ntx, ntt, p->sms, ntt);
    const int64_t nblk = (nmax + p->opts.peak_block - 1) / p->opts.peak_block;
    const size_t recs = (size_t)ntr * nw * (size_t)nblk;
    K.key_off = arena;
    arena = (size_t)round_up((int64_t)(arena + 4 * recs), 256);
    K.off_off = arena;
    arena = (size_t)round_up((int64_t)(arena + recs), 256);
    K.edge_off = arena;
    arena = (size_t)round_up(
        (int64_t)(arena + (size_t)K.smax * ntx * 2 * 64 * (size_t)K.hist * 4), 256);
    ++count;
  }
  // series: fused ranges keep none unless asked to
  std::vector<int64_t> off(nr, 0);
  int64_t elems = 0;
  for (int r = 0; r < nr; ++r) {
    if (nk[r].fused && !keep) continue;
    off[r] = elems;
    elems += p->series_stride[r] * p->ranges[r].n_trials;
  }
  std::vector<int32_t*> series(p->slots.size(), nullptr);
  std::vector<uint8_t*> fused(p->slots.size(), nullptr);
  for (size_t i = 0; i < p->slots.size() && rc == DD_OK && count > 0; ++i) {
    rc = dalloc(&series[i], sizeof(int32_t) * (size_t)elems, "series");
    if (rc == DD_OK) rc = dalloc(&fused[i], arena, "fused search records");
  }
  if (rc != DD_OK) {
    for (size_t i = 0; i < series.size(); ++i) {
      cudaFree(series[i]);
      cudaFree(fused[i]);
    }
    for (int r = 0; r < nr; ++r)
      if (replanned[r]) cudaFree(nk[r].d_tabs);
    return rc;
  }
  p->fused_widths.assign(widths, widths + nwidths);
  p->fused_series = keep;
  if (count > 0) {
    for (int r = 0; r < nr; ++r)
      if (replanned[r]) cudaFree(p->rk[r].d_tabs);
    p->rk = nk;
    p->series_off = off;
    p->series_elems = elems;
    for (size_t i = 0; i < p->slots.size(); ++i) {
      cudaFree(p->slots[i].series);
      p->slots[i].series = series[i];
      p->slots[i].fused = fused[i];
    }
  }
  if (nfused) *nfused = count;
  return DD_OK;
}

// dd_run's work; with `defer`, the tiled launches of the 64 x 512 x 512 shape are not made but
// handed back (argument block and instance) for a persistent launch the caller makes later on
// the same stream.
static int run_impl(dd_plan_t p, const uint8_t* chunk, int64_t nsamp, void* cuda_stream,
                    std::vector<ddk::DeferredTile>* defer) {
  if (!p) return fail(DD_ERR_ARG, "plan is NULL");
  if (!chunk) return fail(DD_ERR_ARG, "chunk is NULL");
  if (nsamp <= 0 || nsamp > p->L || nsamp % p->dmax != 0)
    return fail(DD_ERR_ARG, "nsamp %lld must be in 1..chunk_len and a multiple of %d",
                (long long)nsamp, p->dmax);
  DD_CK(cudaSetDevice(p->device));
  const int64_t seq = p->next_seq;
  Slot& s = p->slots[seq % p->slots.size()];
  cudaStream_t st = cuda_stream ? (cudaStream_t)cuda_stream : s.stream;
  // the slot's previous chunk (possibly on another stream) must be finished with its buffers;
  // the wait for the previous chunk's history comes after the copy of this chunk's samples, so
  // that the copy does not queue behind the history chain
  if (s.seq >= 0) DD_CK(cudaStreamWaitEvent(st, s.ev_free, 0));

  cudaPointerAttributes attr;
  DD_CK(cudaPointerGetAttributes(&attr, chunk));
  if ((p->opts.flags & DD_FLAG_DEVICE_INPUT) && attr.type != cudaMemoryTypeDevice &&
      attr.type != cudaMemoryTypeManaged)
    return fail(DD_ERR_ARG, "the plan takes device chunks only (DD_FLAG_DEVICE_INPUT)");
  const uint8_t* src = chunk;
  if (attr.type == cudaMemoryTypeUnregistered && p->pool) {
    // pageable chunk: host threads copy it into the slot's pinned buffer (once the previous
    // copy out of that buffer has finished), then it goes to the device asynchronously
    int rc = wait_event(s.ev_staged, 0);
    if (rc) return rc;
    p->pool->copy(s.h_stage, chunk, (size_t)nsamp * p->C);
    DD_CK(cudaMemcpyAsync(s.staging, s.h_stage, (size_t)nsamp * p->C, cudaMemcpyHostToDevice, st));
    DD_CK(cudaEventRecord(s.ev_staged, st));
    src = s.staging;
  } else if (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged) {
    DD_CK(cudaMemcpyAsync(s.staging, chunk, (size_t)nsamp * p->C, cudaMemcpyHostToDevice, st));
    src = s.staging;
  }
  // the slot's kernel error bits describe this chunk only
  if (!p->err_word) DD_CK(cudaMemsetAsync(s.d_count + 1, 0, sizeof(unsigned long long), st));
  const int64_t H = p->H;
  if (seq > 0) DD_CK(cudaStreamWaitEvent(st, p->ev_hist, 0));
  if (seq > 0 && H > 0)
    DD_CK(cudaMemcpy2DAsync(s.ring1, p->R1, p->hist, H, H, p->Cp, cudaMemcpyDeviceToDevice, st));
  DD_CK(ddk::launch_corner_turn(src, nsamp, p->C, s.ring1, p->R1, H, st));
  p->launches += 1;
  if (H > 0) {
    DD_CK(cudaMemcpy2DAsync(p->hist, H, s.ring1 + nsamp, p->R1, H, p->Cp,
                            cudaMemcpyDeviceToDevice, st));
    DD_CK(cudaEventRecord(p->ev_hist, st));
  }
  // hierarchical x2 decimation of the whole ring (history + new samples)
  for (int l = 1; l <= p->levels; ++l) {
    const void* in = (l == 1) ? (const void*)s.ring1 : (const void*)s.ringd[l - 1];
    const int64_t in_stride = (l == 1) ? p->R1 : p->Rd[l - 1];
    DD_CK(ddk::launch_decimate(in, l > 1, in_stride, s.ringd[l], p->Rd[l], p->Cp,
                               (H + nsamp) >> l, st));
    p->launches += 1;
  }
  // an external ordering point (serving: another beam's chunk must finish first); the copy,
  // corner turn and decimation above still overlap that chunk's work
  if (p->gate) {
    DD_CK(cudaStreamWaitEvent(st, p->gate, 0));
    p->gate = nullptr;
  }
  const int64_t T = p->T_total;
  const int64_t lo = std::max<int64_t>(0, T - p->O), hi = std::max<int64_t>(0, T + nsamp - p->O);
  if (hi > lo) DD_CK(cudaMemsetAsync(s.mom, 0, sizeof(ddk::Moments) * p->total_rows, st));
  for (size_t r = 0; r < p->ranges.size(); ++r) {
    const int d = p->ranges[r].decimation;
    const int l = ilog2(d);
    ddk::DedispRange R;
    R.xd = (l == 0) ? (const void*)s.ring1 : (const void*)s.ringd[l];
    R.xd_stride = (l == 0) ? p->R1 : p->Rd[l];
    R.m0 = (lo - (T - H)) / d;
    R.nout = (hi - lo) / d;
    R.y = s.series + p->series_off[r];
    R.y_stride = p->series_stride[r];
    R.mom = s.mom + p->row0[r];
    R.shifts = p->d_shifts + (int64_t)p->row0[r] * p->Cp;
    R.n_trials = p->ranges[r].n_trials;
    R.is_u16 = l > 0;
    if (R.nout <= 0) continue;
    int64_t ts;
    int rc = timing_begin(p, st, (int32_t)r, &ts);
    if (rc) return rc;
    const RangeKernel& K = p->rk[r];
    if (K.tiled) {
      ddk::TiledArgs A;
      A.xd = R.xd;
      A.xd_stride = R.xd_stride;
      if (ddk::make_ring_map(&A.rows, A.xd, R.is_u16, A.xd_stride, p->Cp, K.nseg) != cudaSuccess)
        return fail(DD_ERR_CUDA, "tensor map of the ring could not be made");
      A.m0 = R.m0;
      A.nout = R.nout;
      A.y = R.y;
      A.y_stride = R.y_stride;
      A.mom = R.mom;
      A.shifts = R.shifts;
      A.n_trials = R.n_trials;
      A.cpad = p->Cp;
      A.row_slot = K.row_slot;
      A.zcap = K.zcap;
      A.nstage = K.nstage;
      A.tabs = K.d_tabs;
      A.err = p->err_word ? p->err_word : reinterpret_cast<int32_t*>(s.d_count + 1);
      if (K.fused) {
        ddk::FusedArgs F;
        std::memset(&F, 0, sizeof F);
        F.key = reinterpret_cast<uint32_t*>(s.fused + K.key_off);
        F.off = s.fused + K.off_off;
        F.edge = reinterpret_cast<uint32_t*>(s.fused + K.edge_off);
        F.block = p->opts.peak_block;
        F.nblk = (R.nout + F.block - 1) / F.block;
        F.nw = K.nw;
        for (int k = 0; k < K.nw; ++k) F.wd[k] = K.wd[k];
        F.hist = K.hist;
        F.hp = K.hp;
        const int ntx = (R.n_trials + 63) / 64, ntt = (int)((R.nout + 511) / 512);
        F.nsegs = ddk::fused_segments(ntx, ntt, p->sms, K.smax);
        F.seg_tiles = (ntt + F.nsegs - 1) / F.nsegs;
        F.keep_series = p->fused_series ? 1 : 0;
        F.e_off = K.e_off;
        if (!p->fused_series) {
          A.y = nullptr;
          A.y_stride = 0;
        }
        DD_CK(ddk::launch_fused(A, F, R.is_u16, K.fsmem, st));
        p->launches += F.nsegs > 1 ? 2 : 1;
      } else if (defer && K.tt == 512 && K.trials == 64 && K.threads == 512) {
        ddk::DeferredTile dt;
        dt.args = A;
        dt.is_u16 = R.is_u16;
        dt.nstage = K.nstage;
        dt.smem = K.smem;
        defer->push_back(dt);
      } else {
        DD_CK(ddk::launch_tiled(A, R.is_u16, K.tt, K.trials, K.threads, st));
        p->launches += 1;
      }
    } else if (p->opts.flags & DD_FLAG_NAIVE) {
      DD_CK(ddk::launch_dedisp_naive(R, p->Cp, st));
    } else {
      DD_CK(ddk::launch_dedisp_direct(R, p->Cp, st));
    }
    rc = timing_end(p, st, ts);
    if (rc) return rc;
    if (!K.tiled) {
      DD_CK(ddk::launch_moments(R.y, R.n_trials, R.nout, R.y_stride, R.mom, st));
      p->launches += 2;
    }
  }
  DD_CK(cudaEventRecord(s.ev_free, st));
  s.used = st;
  s.seq = seq;
  s.T = T;
  s.n = nsamp;
  s.lo = lo;
  s.hi = hi;
  s.searched = false;
  p->T_total += nsamp;
  p->next_seq += 1;
  return DD_OK;
}

int dd_run(dd_plan_t p, const uint8_t* chunk, int64_t nsamp, void* cuda_stream) {
  return run_impl(p, chunk, nsamp, cuda_stream, nullptr);
}

int dd_series(dd_plan_t p, int32_t range, const int32_t** dev_ptr, int64_t* len, int64_t* stride,
              int64_t* j0) {
  if (!p) return fail(DD_ERR_ARG, "plan is NULL");
  if (range < 0 || range >= (int32_t)p->ranges.size()) return fail(DD_ERR_ARG, "bad range");
  if (p->next_seq == 0) return fail(DD_ERR_STATE, "no chunk has been run");
  if (p->rk[range].fused && !p->fused_series)
    return fail(DD_ERR_STATE, "range %d's search is fused: its series are not kept", (int)range);
  const Slot& s = p->slots[(p->next_seq - 1) % p->slots.size()];
  const int d = p->ranges[range].decimation;
  if (dev_ptr) *dev_ptr = s.series + p->series_off[range];
  if (len) *len = (s.hi - s.lo) / d;
  if (stride) *stride = p->series_stride[range];
  if (j0) *j0 = s.lo / d;
  return DD_OK;
}

int dd_moments(dd_plan_t p, int32_t range, const dd_moments_t** dev_ptr, int64_t* n) {
  if (!p) return fail(DD_ERR_ARG, "plan is NULL");
  if (range < 0 || range >= (int32_t)p->ranges.size()) return fail(DD_ERR_ARG, "bad range");
  if (p->next_seq == 0) return fail(DD_ERR_STATE, "no chunk has been run");
  const Slot& s = p->slots[(p->next_seq - 1) % p->slots.size()];
  const int d = p->ranges[range].decimation;
  if (dev_ptr) *dev_ptr = reinterpret_cast<const dd_moments_t*>(s.mom + p->row0[range]);
  if (n) *n = (s.hi - s.lo) / d;
  return DD_OK;
}

int sps_run_ex(dd_plan_t p, const int32_t* widths, int32_t nwidths, float threshold,
               const dd_sps_opts_t* how) {
  if (!p) return fail(DD_ERR_ARG, "plan is NULL");
  if (!widths || nwidths < 1 || nwidths > ddk::kMaxWidths)
    return fail(DD_ERR_ARG, "nwidths must be 1..%d", ddk::kMaxWidths);
  for (int k = 0; k < nwidths; ++k) {
    if (widths[k] < 1 || widths[k] > p->opts.max_width)
      return fail(DD_ERR_ARG, "width %d outside 1..max_width", widths[k]);
    if (k > 0 && widths[k] <= widths[k - 1])
      return fail(DD_ERR_ARG, "widths must be strictly increasing");
  }
  if (!std::isfinite(threshold)) return fail(DD_ERR_ARG, "threshold must be finite");
  const bool clipped = how && how->estimator == DD_EST_CLIPPED;
  if (how && how->estimator != DD_EST_WINDOW && !clipped)
    return fail(DD_ERR_ARG, "unknown estimator %d", how->estimator);
  if (clipped && (how->clip_iters < 0 || how->clip_iters > 16 || !(how->clip_kappa > 0) ||
                  !std::isfinite(how->clip_kappa)))
    return fail(DD_ERR_ARG, "clipping needs 0 <= clip_iters <= 16 and a finite clip_kappa > 0");
  if (p->next_seq == 0) return fail(DD_ERR_STATE, "no chunk has been run");
  Slot& s = p->slots[(p->next_seq - 1) % p->slots.size()];
  if (s.searched) return fail(DD_ERR_STATE, "the latest chunk was already searched");
  bool any_fused = false;
  for (const auto& k : p->rk) any_fused |= k.fused;
  if (any_fused) {
    if (p->fused_widths != std::vector<int32_t>(widths, widths + nwidths))
      return fail(DD_ERR_ARG, "the plan's search is fused with other widths (dd_fuse_search)");
    if (clipped && !p->fused_series)
      return fail(DD_ERR_STATE, "clipped statistics need the series, which a fused plan does not "
                                "keep (DD_FUSE_KEEP_SERIES)");
  }
  DD_CK(cudaSetDevice(p->device));
  cudaStream_t st = s.used;
  DD_CK(cudaMemsetAsync(s.d_count, 0, sizeof(unsigned long long), st));
  for (size_t r = 0; r < p->ranges.size(); ++r) {
    const int d = p->ranges[r].decimation;
    ddk::SpsArgs a;
    std::memset(&a, 0, sizeof a);
    a.nw = 0;
    for (int k = 0; k < nwidths; ++k)
      if (widths[k] >= d && widths[k] % d == 0) a.wd[a.nw++] = widths[k] / d;
    a.n = (s.hi - s.lo) / d;
    if (a.nw == 0 || a.n <= 0) continue;
    const RangeKernel& K = p->rk[r];
    if (K.fused && !clipped) {
      ddk::SpsFusedArgs f;
      std::memset(&f, 0, sizeof f);
      f.key = reinterpret_cast<const uint32_t*>(s.fused + K.key_off);
      f.off = s.fused + K.off_off;
      f.block = p->opts.peak_block;
      f.n = a.n;
      f.nblk = (a.n + f.block - 1) / f.block;
      f.mom = s.mom + p->row0[r];
      f.n_trials = p->ranges[r].n_trials;
      f.range = (int32_t)r;
      f.d = d;
      f.J0 = s.lo / d;
      f.nw = a.nw;
      for (int k = 0; k < a.nw; ++k) f.wd[k] = a.wd[k];
      f.threshold = threshold;
      f.cands = s.cands;
      f.count = s.d_count;
      f.cap = p->opts.max_cands;
      DD_CK(ddk::launch_sps_fused(f, st));
      p->launches += 1;
      continue;
    }
    a.y = s.series + p->series_off[r];
    a.stride = p->series_stride[r];
    a.mom = s.mom + p->row0[r];
    a.n_trials = p->ranges[r].n_trials;
    a.range = (int32_t)r;
    a.d = d;
    a.block = p->opts.peak_block;
    a.J0 = s.lo / d;
    a.hist = (int32_t)round_up(std::max(a.wd[a.nw - 1] - 1, 0), 256);
    a.threshold = threshold;
    a.cands = s.cands;
    a.count = s.d_count;
    a.cap = p->opts.max_cands;
    if (clipped) {
      ddk::ClipArgs c;
      std::memset(&c, 0, sizeof c);
      c.y = a.y;
      c.stride = a.stride;
      c.n = a.n;
      c.n_trials = a.n_trials;
      c.nw = a.nw;
      for (int k = 0; k < a.nw; ++k) c.wd[k] = a.wd[k];
      c.hist = a.hist;
      c.iters = how->clip_iters;
      c.kappa = how->clip_kappa;
      c.out = s.wst + (int64_t)p->row0[r] * ddk::kMaxWidths;
      DD_CK(ddk::launch_clip_stats(c, st));
      p->launches += 1;
      a.wst = c.out;
    }
    DD_CK(ddk::launch_sps(a, st));
    p->launches += 1;
  }
  DD_CK(cudaMemcpyAsync(s.h_count, s.d_count, 2 * sizeof(unsigned long long),
                        cudaMemcpyDeviceToHost, st));
  DD_CK(cudaEventRecord(s.ev_sps, st));
  DD_CK(cudaEventRecord(s.ev_free, st));
  s.searched = true;
  return DD_OK;
}

int sps_run(dd_plan_t p, const int32_t* widths, int32_t nwidths, float threshold) {
  return sps_run_ex(p, widths, nwidths, threshold, nullptr);
}

int dd_candidates(dd_plan_t p, int64_t seq, dd_cand_t* out, int64_t cap, int64_t* ncands,
                  int64_t timeout_ms) {
  if (!p) return fail(DD_ERR_ARG, "plan is NULL");
  if (!ncands || (cap > 0 && !out) || cap < 0) return fail(DD_ERR_ARG, "bad output arguments");
  const int64_t S = (int64_t)p->slots.size();
  if (seq < 0 || seq >= p->next_seq || seq < p->next_seq - S)
    return fail(DD_ERR_STATE, "chunk %lld is not among the last %lld chunks", (long long)seq,
                (long long)S);
  Slot& s = p->slots[seq % S];
  if (s.seq != seq || !s.searched) return fail(DD_ERR_STATE, "chunk %lld was not searched",
                                               (long long)seq);
  DD_CK(cudaSetDevice(p->device));
  int rc = wait_event(s.ev_sps, timeout_ms);
  if (rc) return rc;
  if (s.h_count[1] != 0)
    return fail(DD_ERR_TIMEOUT, "a dedispersion kernel stopped early (error bits %llu)",
                (unsigned long long)s.h_count[1]);
  const int64_t count = (int64_t)s.h_count[0];
  const int64_t kept = std::min<int64_t>(count, p->opts.max_cands);
  if (kept > 0) {
    DD_CK(cudaStreamWaitEvent(p->io, s.ev_sps, 0));
    DD_CK(cudaMemcpyAsync(p->h_cands, s.cands, sizeof(dd_cand_t) * kept, cudaMemcpyDeviceToHost,
                          p->io));
    DD_CK(cudaEventRecord(p->ev_io, p->io));
    rc = wait_event(p->ev_io, timeout_ms);
    if (rc) return rc;
    std::sort(p->h_cands, p->h_cands + kept, [](const dd_cand_t& a, const dd_cand_t& b) {
      if (a.range != b.range) return a.range < b.range;
      if (a.trial != b.trial) return a.trial < b.trial;
      if (a.t_start != b.t_start) return a.t_start < b.t_start;
      return a.width < b.width;
    });
    std::memcpy(out, p->h_cands, sizeof(dd_cand_t) * std::min(kept, cap));
  }
  *ncands = count;
  if (count > cap || count > p->opts.max_cands)
    return fail(DD_ERR_CAP, "%lld candidates exceed the buffer (cap %lld, max_cands %lld)",
                (long long)count, (long long)cap, (long long)p->opts.max_cands);
  return DD_OK;
}

int dd_tiled_plan_check(const int32_t* shifts, int32_t n_trials, int32_t cpad,
                        int32_t decimation, int32_t tile_samples, int32_t tile_trials,
                        int32_t* ok, int64_t* violations) {
  if (!shifts || !ok || !violations) return fail(DD_ERR_ARG, "NULL argument");
  if (n_trials < 1 || cpad < 8 || cpad % 8 || (tile_samples != 256 && tile_samples != 512) ||
      (tile_trials != 32 && tile_trials != 64))
    return fail(DD_ERR_ARG, "need n_trials >= 1, cpad a multiple of 8, tile_samples 256 or 512, "
                            "tile_trials 32 or 64");
  int k = 0;
  *violations = ddk::tiled_plan_check(shifts, n_trials, cpad, decimation, tile_samples,
                                      tile_trials, &k);
  *ok = k;
  return DD_OK;
}

int dd_selftest_wait(int32_t device, int32_t* timed_out, double* waited_ms) {
  if (!timed_out) return fail(DD_ERR_ARG, "timed_out is NULL");
  *timed_out = 0;
  DD_CK(cudaSetDevice(device));
  const auto t0 = std::chrono::steady_clock::now();
  int32_t* d_err = nullptr;
  if (cudaMalloc(&d_err, sizeof(int32_t)) != cudaSuccess)
    return fail(DD_ERR_NOMEM, "self-test: no device memory for the status word");
  cudaStream_t st = nullptr;
  int32_t herr = 0;
  cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_err, 0, sizeof(int32_t), st);
  if (e == cudaSuccess) e = ddk::launch_wait_selftest(d_err, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (st) cudaStreamDestroy(st);
  cudaFree(d_err);
  if (e != cudaSuccess) return fail(DD_ERR_CUDA, "self-test: %s", cudaGetErrorString(e));
  *timed_out = (herr & 1) ? 1 : 0;
  if (waited_ms)
    *waited_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0)
                     .count();
  return DD_OK;
}

int dd_sync(dd_plan_t p) {
  if (!p) return fail(DD_ERR_ARG, "plan is NULL");
  DD_CK(cudaSetDevice(p->device));
  for (auto& s : p->slots) {
    DD_CK(cudaStreamSynchronize(s.stream));
    if (s.used && s.used != s.stream) DD_CK(cudaStreamSynchronize(s.used));
  }
  DD_CK(cudaStreamSynchronize(p->io));
  return DD_OK;
}

int dd_stats(dd_plan_t p, int64_t* launches, double* dedisp_ms, int64_t* dedisp_launches,
             int32_t reset) {
  if (!p) return fail(DD_ERR_ARG, "plan is NULL");
  DD_CK(cudaSetDevice(p->device));
  if (p->tref_set) {
    int rc = harvest_timing(p);
    if (rc) return rc;
  }
  if (launches) *launches = p->launches;
  if (dedisp_ms) *dedisp_ms = union_ms(p->intervals);
  if (dedisp_launches) *dedisp_launches = p->dedisp_launches;
  if (reset) {
    p->launches = 0;
    p->intervals.clear();
    p->interval_range.clear();
    p->dedisp_launches = 0;
    p->tref_set = false;  // the next launch records a fresh reference
  }
  return DD_OK;
}

int dd_stats_range(dd_plan_t p, int32_t range, double* dedisp_ms, int64_t* dedisp_launches) {
  if (!p) return fail(DD_ERR_ARG, "plan is NULL");
  if (range < 0 || range >= (int32_t)p->ranges.size()) return fail(DD_ERR_ARG, "bad range");
  DD_CK(cudaSetDevice(p->device));
  if (p->tref_set) {
    int rc = harvest_timing(p);
    if (rc) return rc;
  }
  std::vector<std::pair<double, double>> mine;
  for (size_t k = 0; k < p->intervals.size(); ++k)
    if (p->interval_range[k] == range) mine.push_back(p->intervals[k]);
  if (dedisp_launches) *dedisp_launches = (int64_t)mine.size();
  if (dedisp_ms) *dedisp_ms = union_ms(mine);
  return DD_OK;
}

void dd_plan_destroy(dd_plan_t p) { free_plan(p); }

}  // extern "C"

namespace ddk {
int run_deferred(dd_plan_s* p, const uint8_t* chunk, int64_t nsamp, cudaStream_t st,
                 std::vector<DeferredTile>* out) {
  return run_impl(p, chunk, nsamp, st, out);
}
}  // namespace ddk
