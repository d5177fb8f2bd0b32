// Serving loop: many beams, each a plan of its own, whose chunks arrive at arbitrary times.
//
// A dispatcher thread owns every plan call. Requests wait in per-beam FIFO queues and are
// admitted oldest first across beams as soon as (a) fewer chunks are on the GPU than the
// admission limit below and (b) the request's beam has a free stream slot (its plan keeps
// n_streams chunks in flight: the per-beam cap). So a chunk that arrives while others are
// being processed starts as soon as capacity frees up, and chunks of different beams overlap on
// the device, each beam on its own streams (Sec. 1: work split over CUDA streams; Sec. 2.2: all
// memory allocated when a beam is planned, so admitting a chunk allocates nothing). A beam is
// accepted only if its plan's device memory fits the server's HBM budget. Latency = submission
// -> candidates copied to the caller.
//
// Admission limit. One chunk's dedispersion launches already fill the GPU (thousands of CTAs),
// so chunks sharing the GPU mostly slow each other down; overlap pays only in the gaps between
// launches and at their partial last waves. The limit therefore follows the backlog: with at
// most two requests waiting, two chunks may be on the GPU, and the newer one's dedispersion is
// ordered after the older one's search (its copy, corner turn and decimation still overlap
// it), so chunks complete in arrival order at close to their own service time; with a longer
// backlog, up to as many chunks as are waiting (never more than max_inflight) run unordered, so
// that their launches fill each other's gaps and throughput rises.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "dd_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  int64_t ticket;
  int32_t beam;
  const uint8_t* chunk;
  int64_t nsamp;
  dd_cand_t* out;
  int64_t cap;
  Clock::time_point t_submit, t_admit;
  int64_t seq;
};

struct Beam {
  dd_plan_t plan = nullptr;
  int n_streams = 1;
  std::vector<int32_t> widths;
  float threshold = 0;
  int64_t bytes = 0;
  int64_t next_seq = 0;
  int failed = DD_OK;  // first enqueue error; a failed beam takes no further chunks
  std::deque<Request> queue, inflight;
};

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

}  // namespace

struct dd_server_s {
  int device = 0;
  int max_inflight = 1;
  int64_t budget = 0, used = 0;
  std::vector<Beam*> beams;
  std::mutex mu;
  std::mutex add_mu;  // one dd_serve_add_beam at a time: its memory measurement is a difference
  std::condition_variable work_cv, done_cv;
  std::deque<dd_serve_result_t> done;
  std::thread worker;
  bool stop = false;
  int inflight = 0;
  int64_t next_ticket = 0;
  dd_plan_t last_plan = nullptr;  // the most recently admitted chunk
  int64_t last_seq = -1;

  void run();
};

void dd_server_s::run() {
  cudaSetDevice(device);
  // Only this thread calls into the plans; the lock guards the queues, counters and the beam
  // list, and is released around every plan call so that submitters and pollers never wait
  // for a copy, a launch sequence or a candidate sort.
  std::unique_lock<std::mutex> lk(mu);
  std::vector<std::pair<Beam*, Request>> ready;
  std::vector<int> ready_state;
  while (!stop) {
    bool progress = false;
    // completions: the oldest in-flight chunks of every beam whose search has finished
    ready.clear();
    ready_state.clear();
    for (int b = 0; b < (int)beams.size(); ++b) {
      Beam& bm = *beams[b];
      while (!bm.inflight.empty()) {
        const int st = ddk::chunk_state(bm.plan, bm.inflight.front().seq);
        if (st == 0) break;
        ready.emplace_back(&bm, bm.inflight.front());
        ready_state.push_back(st);
        bm.inflight.pop_front();
      }
    }
    if (!ready.empty()) {
      lk.unlock();
      std::vector<dd_serve_result_t> res(ready.size());
      for (size_t k = 0; k < ready.size(); ++k) {
        const Request& r = ready[k].second;
        int64_t n = 0;
        const int st = ready_state[k];
        res[k].ticket = r.ticket;
        res[k].beam = r.beam;
        res[k].seq = r.seq;
        res[k].status = st < 0 ? st : dd_candidates(ready[k].first->plan, r.seq, r.out, r.cap,
                                                    &n, 0);
        const auto now = Clock::now();
        res[k].ncands = n;
        res[k].queue_ms = ms_between(r.t_submit, r.t_admit);
        res[k].latency_ms = ms_between(r.t_submit, now);
      }
      lk.lock();
      for (auto& x : res) done.push_back(x);
      inflight -= (int)ready.size();
      done_cv.notify_all();
      progress = true;
    }
    // admissions: earliest submitted request whose beam has a free slot, while fewer chunks
    // are on the GPU than the backlog-dependent limit
    for (;;) {
      if (stop) break;
      int64_t queued = 0;
      for (auto* bm : beams) queued += (int64_t)bm->queue.size();
      const int limit = (int)std::min<int64_t>(max_inflight, std::max<int64_t>(2, queued));
      if (inflight >= limit) break;
      const bool ordered = queued <= 2;  // light load: complete in arrival order
      Beam* pick = nullptr;
      for (auto* bm : beams) {
        if (bm->queue.empty() || (int)bm->inflight.size() >= bm->n_streams) continue;
        if (!pick || bm->queue.front().ticket < pick->queue.front().ticket) pick = bm;
      }
      if (!pick) break;
      Request r = pick->queue.front();
      pick->queue.pop_front();
      r.t_admit = Clock::now();
      if (pick->failed != DD_OK) {  // the beam's stream state was lost: refuse its chunks
        dd_serve_result_t res{r.ticket, r.beam, pick->failed, -1, 0, 0.0, 0.0};
        done.push_back(res);
        done_cv.notify_all();
        progress = true;
        continue;
      }
      ++inflight;  // reserved while the chunk is being enqueued
      dd_plan_t prev_plan = last_plan;
      const int64_t prev_seq = last_seq;
      lk.unlock();
      if (ordered && prev_plan && inflight > 1) {
        cudaEvent_t ev = ddk::chunk_done_event(prev_plan, prev_seq);
        if (ev) ddk::plan_gate_next(pick->plan, ev);
      }
      int rc = dd_run(pick->plan, r.chunk, r.nsamp, nullptr);
      bool ran = false;
      if (rc == DD_OK) {
        ran = true;
        r.seq = pick->next_seq++;
        rc = sps_run(pick->plan, pick->widths.data(), (int32_t)pick->widths.size(),
                     pick->threshold);
      }
      if (rc != DD_OK && ran) {
        // the chunk is on the plan's slot but unsearched: finish the beam's work so the plan's
        // slots and this beam's bookkeeping cannot disagree later
        ddk::plan_reset(pick->plan);
      }
      lk.lock();
      if (rc != DD_OK) {
        --inflight;
        if (ran) {
          pick->failed = rc;
          // chunks of this beam already on the GPU finished with the reset; report them too
          for (auto& q : pick->inflight) {
            dd_serve_result_t res{q.ticket, q.beam, rc, q.seq, 0, 0.0, 0.0};
            done.push_back(res);
            --inflight;
          }
          pick->inflight.clear();
        }
        dd_serve_result_t res{r.ticket, r.beam, rc, -1, 0, 0.0, 0.0};
        done.push_back(res);
        done_cv.notify_all();
        progress = true;
        continue;
      }
      pick->inflight.push_back(r);
      last_plan = pick->plan;
      last_seq = r.seq;
      progress = true;
    }
    if (!progress) work_cv.wait_for(lk, std::chrono::microseconds(inflight ? 50 : 2000));
  }
}

extern "C" {

int dd_serve_create(int32_t max_inflight, int64_t hbm_budget_bytes, int32_t device,
                    dd_server_t* out) {
  if (!out) return ddk::report_error(DD_ERR_ARG, "dd_serve_create: out is NULL");
  *out = nullptr;
  if (max_inflight < 1 || max_inflight > 1024)
    return ddk::report_error(DD_ERR_ARG, "dd_serve_create: max_inflight must be 1..1024");
  if (hbm_budget_bytes <= 0)
    return ddk::report_error(DD_ERR_ARG, "dd_serve_create: hbm_budget_bytes must be > 0");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
    return ddk::report_error(DD_ERR_ARG, "dd_serve_create: no such device");
  dd_server_s* s = new dd_server_s();
  s->device = device;
  s->max_inflight = max_inflight;
  s->budget = hbm_budget_bytes;
  s->worker = std::thread([s] { s->run(); });
  *out = s;
  return DD_OK;
}

int dd_serve_add_beam(dd_server_t s, const double* freqs_mhz, int32_t nchans, double tsamp_s,
                      const dd_range_t* ranges, int32_t nranges, const dd_opts_t* opts,
                      const int32_t* widths, int32_t nwidths, float threshold, int32_t* beam) {
  if (!s || !beam || !opts || !widths || nwidths < 1 || nwidths > ddk::kMaxWidths)
    return ddk::report_error(DD_ERR_ARG, "dd_serve_add_beam: bad argument");
  // the search parameters are checked here, as sps_run would check them, so that a beam's
  // chunks cannot fail their search after their dedispersion was enqueued
  for (int k = 0; k < nwidths; ++k)
    if (widths[k] < 1 || widths[k] > opts->max_width || (k > 0 && widths[k] <= widths[k - 1]))
      return ddk::report_error(DD_ERR_ARG, "dd_serve_add_beam: widths must be strictly "
                                           "increasing within 1..max_width");
  if (!std::isfinite(threshold))
    return ddk::report_error(DD_ERR_ARG, "dd_serve_add_beam: threshold must be finite");
  if (cudaSetDevice(s->device) != cudaSuccess)
    return ddk::report_error(DD_ERR_CUDA, "dd_serve_add_beam: cudaSetDevice failed");
  dd_opts_t o = *opts;
  o.device = s->device;
  std::lock_guard<std::mutex> add_lk(s->add_mu);
  size_t free0 = 0, free1 = 0, total = 0;
  cudaMemGetInfo(&free0, &total);
  dd_plan_t plan = nullptr;
  int rc = dd_plan(freqs_mhz, nchans, tsamp_s, ranges, nranges, &o, &plan);
  if (rc) return rc;
  cudaMemGetInfo(&free1, &total);
  const int64_t bytes = free0 > free1 ? (int64_t)(free0 - free1) : 0;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->used + bytes > s->budget) {
    dd_plan_destroy(plan);
    return ddk::report_error(DD_ERR_NOMEM, "dd_serve_add_beam: the beam's plan exceeds the "
                                           "server's HBM budget");
  }
  Beam* b = new Beam();
  b->plan = plan;
  b->n_streams = o.n_streams;
  b->widths.assign(widths, widths + nwidths);
  b->threshold = threshold;
  b->bytes = bytes;
  s->used += bytes;
  s->beams.push_back(b);
  *beam = (int32_t)s->beams.size() - 1;
  return DD_OK;
}

int dd_serve_submit(dd_server_t s, int32_t beam, const uint8_t* chunk, int64_t nsamp,
                    dd_cand_t* out, int64_t cap, int64_t* ticket) {
  if (!s || !chunk || (!out && cap > 0) || cap < 0)
    return ddk::report_error(DD_ERR_ARG, "dd_serve_submit: bad argument");
  const auto t_submit = Clock::now();  // before the lock: time spent waiting for it counts
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (beam < 0 || beam >= (int32_t)s->beams.size())
      return ddk::report_error(DD_ERR_ARG, "dd_serve_submit: unknown beam");
    Request r;
    r.ticket = s->next_ticket++;
    r.beam = beam;
    r.chunk = chunk;
    r.nsamp = nsamp;
    r.out = out;
    r.cap = cap;
    r.t_submit = t_submit;
    r.t_admit = t_submit;
    r.seq = -1;
    s->beams[beam]->queue.push_back(r);
    if (ticket) *ticket = r.ticket;
  }
  s->work_cv.notify_all();
  return DD_OK;
}

int dd_serve_poll(dd_server_t s, dd_serve_result_t* out, int32_t max, int32_t* n,
                  int64_t timeout_ms) {
  if (!s || !out || !n || max < 1) return ddk::report_error(DD_ERR_ARG, "dd_serve_poll: bad argument");
  std::unique_lock<std::mutex> lk(s->mu);
  if (s->done.empty() && timeout_ms > 0)
    s->done_cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), [s] { return !s->done.empty(); });
  int32_t k = 0;
  while (k < max && !s->done.empty()) {
    out[k++] = s->done.front();
    s->done.pop_front();
  }
  *n = k;
  return DD_OK;
}

int dd_serve_pending(dd_server_t s, int64_t* queued, int32_t* inflight) {
  if (!s) return ddk::report_error(DD_ERR_ARG, "dd_serve_pending: server is NULL");
  std::lock_guard<std::mutex> lk(s->mu);
  int64_t q = 0;
  for (auto* b : s->beams) q += (int64_t)b->queue.size();
  if (queued) *queued = q;
  if (inflight) *inflight = s->inflight;
  return DD_OK;
}

void dd_serve_destroy(dd_server_t s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->work_cv.notify_all();
  s->worker.join();
  for (auto* b : s->beams) {
    dd_plan_destroy(b->plan);
    delete b;
  }
  delete s;
}

}  // extern "C"
