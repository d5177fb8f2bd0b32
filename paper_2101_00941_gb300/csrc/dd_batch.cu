// Batched execution: many beams of uneven length and channel count, each with a plan of its
// own, processed from their first sample in one enqueued step (Sec. 1: time chunks over CUDA
// streams, applied across beams). Every (beam, chunk) has its own candidate buffer, so one step
// keeps every result. Two ways to run a step:
//   streams    : chunks are enqueued round-robin over the beams, each beam on its own streams,
//                so different beams' launches overlap on the device;
//   persistent : (DD_BATCH_PERSISTENT) round c takes chunk c of every beam that has one, on one
//                stream: the beams' copies, corner turns and decimations, then ONE persistent
//                dedispersion launch per instance (uint8 / uint16 data, staging buffers) whose
//                CTAs, one per SM, take (beam, range, trial tile, time tile) items from a device
//                work list until it is empty, then every beam's search.
// Optionally the whole step is captured once as a CUDA graph and replayed (the beams' inputs
// stay at the same device addresses; each step starts again at sample 0; the persistent work
// lists are copied from pinned host memory written when the step was captured), and every
// plan's tile shapes are chosen by timing the candidates.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <thread>
#include <vector>

#include "dd_internal.h"

struct dd_batch_s {
  int device = 0;
  uint32_t flags = 0;
  int64_t chunk_len = 0, cap = 0;
  std::vector<dd_plan_t> plans;
  std::vector<const uint8_t*> inputs;
  std::vector<int64_t> nsamp, nchunks, first;  // first: index of the beam's chunk 0 in buffers
  std::vector<int32_t> nchans;
  std::vector<int32_t> widths;
  float threshold = 0;
  int64_t total_chunks = 0;
  dd_cand_t* d_cands = nullptr;             // [total_chunks][cap]
  // [total_chunks] candidate counts, then one word of dedispersion-kernel error bits (every
  // plan's tiled kernels report into it; cleared at the start of each step)
  unsigned long long* d_counts = nullptr;   // [total_chunks + 1]
  unsigned long long* h_counts = nullptr;   // pinned [total_chunks + 1]
  dd_cand_t* h_cands = nullptr;             // pinned [cap]
  cudaStream_t root = nullptr;
  std::vector<cudaStream_t> streams;        // every plan's streams
  std::vector<cudaEvent_t> join;            // one per plan stream
  cudaEvent_t fork = nullptr, done = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool counts_ready = false;
  // persistent mode: per round, the deferred tiled launches' argument blocks and the work-list
  // segments of each instance, in pinned host memory and on the device
  int64_t rounds = 0, max_descs = 0;
  ddk::TiledArgs* h_descs = nullptr;   // [rounds][max_descs]
  ddk::TiledArgs* d_descs = nullptr;
  int32_t* h_segd = nullptr;           // [rounds][max_descs] descriptor of each segment
  int32_t* d_segd = nullptr;
  int64_t* h_segf = nullptr;           // [rounds][max_descs + 4] segment firsts per instance
  int64_t* d_segf = nullptr;
  unsigned long long* d_counters = nullptr;  // [rounds][4]
  int sms = 0;
};

namespace {

void free_batch(dd_batch_s* b) {
  if (!b) return;
  cudaSetDevice(b->device);
  if (b->root) cudaStreamSynchronize(b->root);
  for (auto p : b->plans) dd_plan_destroy(p);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (auto e : b->join) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->done) cudaEventDestroy(b->done);
  if (b->root) cudaStreamDestroy(b->root);
  cudaFree(b->d_cands);
  cudaFree(b->d_counts);
  cudaFreeHost(b->h_descs);
  cudaFree(b->d_descs);
  cudaFreeHost(b->h_segd);
  cudaFree(b->d_segd);
  cudaFreeHost(b->h_segf);
  cudaFree(b->d_segf);
  cudaFree(b->d_counters);
  cudaFreeHost(b->h_counts);
  cudaFreeHost(b->h_cands);
  delete b;
}

int ck(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return DD_OK;
  char buf[256];
  snprintf(buf, sizeof buf, "dd_batch: %s: %s", what, cudaGetErrorString(e));
  return ddk::report_error(DD_ERR_CUDA, buf);
}

// Enqueue one whole step on the beams' own streams, forked from and joined back to `root`.
int enqueue_step(dd_batch_s* b) {
  int rc = ck(cudaMemsetAsync(b->d_counts + b->total_chunks, 0, sizeof(unsigned long long),
                              b->root),
              "error word");
  if (rc == DD_OK) rc = ck(cudaEventRecord(b->fork, b->root), "fork");
  for (size_t k = 0; rc == DD_OK && k < b->streams.size(); ++k)
    rc = ck(cudaStreamWaitEvent(b->streams[k], b->fork, 0), "fork wait");
  const int64_t L = b->chunk_len;
  int64_t maxc = 0;
  for (auto n : b->nchunks) maxc = std::max(maxc, n);
  for (int64_t c = 0; rc == DD_OK && c < maxc; ++c) {
    for (size_t i = 0; rc == DD_OK && i < b->plans.size(); ++i) {
      if (c >= b->nchunks[i]) continue;
      const int64_t n = std::min(L, b->nsamp[i] - c * L);
      rc = dd_run(b->plans[i], b->inputs[i] + (size_t)(c * L) * b->nchans[i], n, nullptr);
      if (rc == DD_OK) {
        const int64_t slot = b->first[i] + c;
        rc = ddk::sps_enqueue(b->plans[i], b->widths.data(), (int32_t)b->widths.size(),
                              b->threshold, b->d_cands + slot * b->cap, b->d_counts + slot,
                              b->cap);
      }
    }
  }
  for (size_t k = 0; rc == DD_OK && k < b->streams.size(); ++k) {
    rc = ck(cudaEventRecord(b->join[k], b->streams[k]), "join");
    if (rc == DD_OK) rc = ck(cudaStreamWaitEvent(b->root, b->join[k], 0), "join wait");
  }
  if (rc == DD_OK)
    rc = ck(cudaMemcpyAsync(b->h_counts, b->d_counts,
                            sizeof(unsigned long long) * (b->total_chunks + 1),
                            cudaMemcpyDeviceToHost, b->root),
            "count readback");
  return rc;
}

// One step in persistent mode, every launch on the root stream (see the file comment).
int enqueue_step_persistent(dd_batch_s* b) {
  int rc = ck(cudaMemsetAsync(b->d_counts + b->total_chunks, 0, sizeof(unsigned long long),
                              b->root),
              "error word");
  const int64_t L = b->chunk_len;
  std::vector<ddk::DeferredTile> defs;
  for (int64_t c = 0; rc == DD_OK && c < b->rounds; ++c) {
    defs.clear();
    for (size_t i = 0; rc == DD_OK && i < b->plans.size(); ++i) {
      if (c >= b->nchunks[i]) continue;
      const int64_t n = std::min(L, b->nsamp[i] - c * L);
      rc = ddk::run_deferred(b->plans[i], b->inputs[i] + (size_t)(c * L) * b->nchans[i], n,
                             b->root, &defs);
    }
    if (rc) break;
    if ((int64_t)defs.size() > b->max_descs)
      return ddk::report_error(DD_ERR_STATE, "dd_batch: more deferred launches than planned");
    // the round's work lists: one per instance (uint8/uint16 x 3/4 staging buffers), each a run
    // of segments (one per deferred launch: all its tiles)
    ddk::TiledArgs* hd = b->h_descs + c * b->max_descs;
    int32_t* hs = b->h_segd + c * b->max_descs;
    int64_t* hf = b->h_segf + c * (b->max_descs + 4);
    for (size_t k = 0; k < defs.size(); ++k) hd[k] = defs[k].args;
    int nseg_total = 0;
    int64_t fpos = 0;
    struct Inst {
      int is_u16, nstage, nseg, seg0;
      int64_t f0;
      size_t smem;
    };
    std::vector<Inst> insts;
    for (int u16 = 0; u16 < 2; ++u16)
      for (int ns = 3; ns <= 4; ++ns) {
        Inst in{u16, ns, 0, nseg_total, fpos, 0};
        int64_t first = 0;
        for (size_t k = 0; k < defs.size(); ++k) {
          if (defs[k].is_u16 != u16 || defs[k].nstage != ns) continue;
          const ddk::TiledArgs& a = defs[k].args;
          const int64_t tiles = (int64_t)((a.n_trials + 63) / 64) * ((a.nout + 511) / 512);
          hs[nseg_total + in.nseg] = (int32_t)k;
          hf[fpos + in.nseg] = first;
          first += tiles;
          in.smem = std::max(in.smem, defs[k].smem);
          in.nseg += 1;
        }
        if (in.nseg == 0) continue;
        hf[fpos + in.nseg] = first;
        nseg_total += in.nseg;
        fpos += in.nseg + 1;
        insts.push_back(in);
      }
    ddk::TiledArgs* dd_ = b->d_descs + c * b->max_descs;
    int32_t* ds = b->d_segd + c * b->max_descs;
    int64_t* df = b->d_segf + c * (b->max_descs + 4);
    // (a round whose ranges all run on the direct kernel has no work list, only searches)
    if (!defs.empty()) {
      rc = ck(cudaMemcpyAsync(dd_, hd, sizeof(ddk::TiledArgs) * defs.size(),
                              cudaMemcpyHostToDevice, b->root),
              "work list");
      if (rc == DD_OK)
        rc = ck(cudaMemcpyAsync(ds, hs, sizeof(int32_t) * nseg_total, cudaMemcpyHostToDevice,
                                b->root),
                "work list");
      if (rc == DD_OK)
        rc = ck(cudaMemcpyAsync(df, hf, sizeof(int64_t) * fpos, cudaMemcpyHostToDevice, b->root),
                "work list");
      if (rc == DD_OK)
        rc = ck(cudaMemsetAsync(b->d_counters + 4 * c, 0, 4 * sizeof(unsigned long long),
                                b->root),
                "counters");
    }
    for (size_t g = 0; rc == DD_OK && g < insts.size(); ++g) {
      const Inst& in = insts[g];
      ddk::PersistArgs pa;
      pa.descs = dd_;
      pa.seg_desc = ds + in.seg0;
      pa.seg_first = df + in.f0;
      pa.nseg = in.nseg;
      pa.pad = 0;
      pa.counter = b->d_counters + 4 * c + g;
      rc = ck(ddk::launch_tiled_persistent(pa, in.is_u16, 512, in.nstage, 64, 512, in.smem,
                                           b->sms, b->root),
              "persistent dedispersion");
    }
    for (size_t i = 0; rc == DD_OK && i < b->plans.size(); ++i) {
      if (c >= b->nchunks[i]) continue;
      const int64_t slot = b->first[i] + c;
      rc = ddk::sps_enqueue(b->plans[i], b->widths.data(), (int32_t)b->widths.size(),
                            b->threshold, b->d_cands + slot * b->cap, b->d_counts + slot,
                            b->cap);
    }
  }
  if (rc == DD_OK)
    rc = ck(cudaMemcpyAsync(b->h_counts, b->d_counts,
                            sizeof(unsigned long long) * (b->total_chunks + 1),
                            cudaMemcpyDeviceToHost, b->root),
            "count readback");
  return rc;
}

int step(dd_batch_s* b) {
  return (b->flags & DD_BATCH_PERSISTENT) ? enqueue_step_persistent(b) : enqueue_step(b);
}

int reset_all(dd_batch_s* b) {
  for (auto p : b->plans) {
    const int rc = ddk::plan_reset(p);
    if (rc) return rc;
  }
  return DD_OK;
}

}  // namespace

extern "C" {

int dd_batch_create(int32_t nbeams, const dd_batch_beam_t* beams, const dd_range_t* ranges,
                    int32_t nranges, const dd_opts_t* opts, const int32_t* widths,
                    int32_t nwidths, float threshold, int64_t cap_per_chunk, uint32_t flags,
                    dd_batch_t* out) {
  if (!out) return ddk::report_error(DD_ERR_ARG, "dd_batch_create: out is NULL");
  *out = nullptr;
  if (nbeams < 1 || !beams || !opts || !widths || nwidths < 1 || cap_per_chunk < 1)
    return ddk::report_error(DD_ERR_ARG, "dd_batch_create: bad argument");
  if (opts->flags & DD_FLAG_TIMING)
    return ddk::report_error(DD_ERR_ARG, "dd_batch_create: DD_FLAG_TIMING is not supported");
  dd_batch_s* b = new dd_batch_s();
  b->device = opts->device;
  b->flags = flags;
  b->chunk_len = opts->chunk_len;
  b->cap = cap_per_chunk;
  b->widths.assign(widths, widths + nwidths);
  b->threshold = threshold;
  int rc = DD_OK;
  for (int32_t i = 0; i < nbeams && rc == DD_OK; ++i) {
    const dd_batch_beam_t& bm = beams[i];
    if (!bm.input || bm.nsamp < 1) {
      rc = ddk::report_error(DD_ERR_ARG, "dd_batch_create: a beam has no input");
      break;
    }
    dd_plan_t p = nullptr;
    rc = dd_plan(bm.freqs_mhz, bm.nchans, bm.tsamp_s, ranges, nranges, opts, &p);
    if (rc) break;
    b->plans.push_back(p);
    b->inputs.push_back(bm.input);
    b->nsamp.push_back(bm.nsamp);
    b->nchans.push_back(bm.nchans);
    const int64_t nc = (bm.nsamp + b->chunk_len - 1) / b->chunk_len;
    b->nchunks.push_back(nc);
    b->first.push_back(b->total_chunks);
    b->total_chunks += nc;
    ddk::plan_streams(p, &b->streams);
  }
  if (rc == DD_OK) rc = ck(cudaSetDevice(b->device), "set device");
  if (rc == DD_OK && (flags & DD_BATCH_AUTOTUNE)) {
    for (auto p : b->plans) {
      rc = ddk::plan_autotune(p);
      if (rc) break;
    }
  }
  if (rc == DD_OK) rc = ck(cudaStreamCreateWithFlags(&b->root, cudaStreamNonBlocking), "stream");
  if (rc == DD_OK) rc = ck(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming), "event");
  if (rc == DD_OK) rc = ck(cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming), "event");
  b->join.resize(b->streams.size(), nullptr);
  for (auto& e : b->join)
    if (rc == DD_OK) rc = ck(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event");
  if (rc == DD_OK &&
      cudaMalloc(&b->d_cands, sizeof(dd_cand_t) * (size_t)(b->total_chunks * b->cap)) !=
          cudaSuccess) {
    cudaGetLastError();
    rc = ddk::report_error(DD_ERR_NOMEM, "dd_batch_create: candidate buffers");
  }
  if (rc == DD_OK &&
      cudaMalloc(&b->d_counts, sizeof(unsigned long long) * (b->total_chunks + 1)) !=
          cudaSuccess) {
    cudaGetLastError();
    rc = ddk::report_error(DD_ERR_NOMEM, "dd_batch_create: counts");
  }
  if (rc == DD_OK &&
      (cudaMallocHost(&b->h_counts, sizeof(unsigned long long) * (b->total_chunks + 1)) !=
           cudaSuccess ||
       cudaMallocHost(&b->h_cands, sizeof(dd_cand_t) * b->cap) != cudaSuccess)) {
    cudaGetLastError();
    rc = ddk::report_error(DD_ERR_NOMEM, "dd_batch_create: pinned buffers");
  }
  if (rc == DD_OK && (flags & DD_BATCH_PERSISTENT)) {
    for (auto n : b->nchunks) b->rounds = std::max(b->rounds, n);
    b->max_descs = (int64_t)b->plans.size() * nranges;
    const size_t nd = (size_t)(b->rounds * b->max_descs);
    const size_t nf = (size_t)(b->rounds * (b->max_descs + 4));
    if (cudaMallocHost(&b->h_descs, sizeof(ddk::TiledArgs) * std::max<size_t>(nd, 1)) !=
            cudaSuccess ||
        cudaMallocHost(&b->h_segd, sizeof(int32_t) * std::max<size_t>(nd, 1)) != cudaSuccess ||
        cudaMallocHost(&b->h_segf, sizeof(int64_t) * std::max<size_t>(nf, 1)) != cudaSuccess ||
        cudaMalloc(&b->d_descs, sizeof(ddk::TiledArgs) * std::max<size_t>(nd, 1)) !=
            cudaSuccess ||
        cudaMalloc(&b->d_segd, sizeof(int32_t) * std::max<size_t>(nd, 1)) != cudaSuccess ||
        cudaMalloc(&b->d_segf, sizeof(int64_t) * std::max<size_t>(nf, 1)) != cudaSuccess ||
        cudaMalloc(&b->d_counters, sizeof(unsigned long long) * 4 *
                                       std::max<size_t>((size_t)b->rounds, 1)) != cudaSuccess) {
      cudaGetLastError();
      rc = ddk::report_error(DD_ERR_NOMEM, "dd_batch_create: persistent work lists");
    }
    if (rc == DD_OK)
      rc = ck(cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device),
              "multiprocessor count");
  }
  if (rc == DD_OK)
    for (auto p : b->plans)
      ddk::plan_redirect_errors(p, reinterpret_cast<int32_t*>(b->d_counts + b->total_chunks));
  if (rc == DD_OK && (flags & DD_BATCH_GRAPH)) {
    // capture one whole step; every plan starts at sample 0, so the graph replays correctly
    rc = reset_all(b);
    if (rc == DD_OK)
      rc = ck(cudaStreamBeginCapture(b->root, cudaStreamCaptureModeRelaxed), "begin capture");
    if (rc == DD_OK) {
      rc = step(b);
      cudaGraph_t g = nullptr;
      const cudaError_t e = cudaStreamEndCapture(b->root, &g);
      if (rc == DD_OK) rc = ck(e, "end capture");
      b->graph = g;
    }
    if (rc == DD_OK) rc = ck(cudaGraphInstantiate(&b->exec, b->graph, 0), "instantiate");
  }
  if (rc) {
    free_batch(b);
    return rc;
  }
  *out = b;
  return DD_OK;
}

int dd_batch_run(dd_batch_t b) {
  if (!b) return ddk::report_error(DD_ERR_ARG, "dd_batch_run: batch is NULL");
  int rc = ck(cudaSetDevice(b->device), "set device");
  b->counts_ready = false;
  if (rc == DD_OK && b->exec) {
    rc = ck(cudaGraphLaunch(b->exec, b->root), "graph launch");
  } else if (rc == DD_OK) {
    rc = reset_all(b);
    if (rc == DD_OK) rc = step(b);
  }
  if (rc == DD_OK) rc = ck(cudaEventRecord(b->done, b->root), "record");
  return rc;
}

int dd_batch_wait(dd_batch_t b, int64_t timeout_ms) {
  if (!b) return ddk::report_error(DD_ERR_ARG, "dd_batch_wait: batch is NULL");
  if (timeout_ms <= 0) timeout_ms = 600000;
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    const cudaError_t e = cudaEventQuery(b->done);
    if (e == cudaSuccess) break;
    if (e != cudaErrorNotReady) return ck(e, "wait");
    if (std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0)
            .count() > timeout_ms)
      return ddk::report_error(DD_ERR_TIMEOUT, "dd_batch_wait: the step did not finish in time");
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
  if (b->h_counts[b->total_chunks] != 0)
    return ddk::report_error(DD_ERR_TIMEOUT,
                             "dd_batch_wait: a dedispersion kernel stopped early; the step's "
                             "results are not valid");
  b->counts_ready = true;
  return DD_OK;
}

int dd_batch_info(dd_batch_t b, int32_t beam, int64_t* nchunks, int64_t* outputs,
                  int32_t* tile_samples) {
  if (!b || beam < 0 || beam >= (int32_t)b->plans.size())
    return ddk::report_error(DD_ERR_ARG, "dd_batch_info: bad beam");
  if (nchunks) *nchunks = b->nchunks[beam];
  if (outputs) *outputs = ddk::plan_outputs(b->plans[beam], b->nsamp[beam]);
  if (tile_samples) *tile_samples = ddk::range_tile(b->plans[beam], 0);
  return DD_OK;
}

int dd_batch_candidates(dd_batch_t b, int32_t beam, int64_t chunk, dd_cand_t* out, int64_t cap,
                        int64_t* ncands) {
  if (!b || !ncands || (cap > 0 && !out) || beam < 0 || beam >= (int32_t)b->plans.size() ||
      chunk < 0 || chunk >= b->nchunks[beam])
    return ddk::report_error(DD_ERR_ARG, "dd_batch_candidates: bad argument");
  if (!b->counts_ready)
    return ddk::report_error(DD_ERR_STATE, "dd_batch_candidates: call dd_batch_wait first");
  const int64_t slot = b->first[beam] + chunk;
  const int64_t count = (int64_t)b->h_counts[slot];
  const int64_t kept = std::min(count, b->cap);
  if (kept > 0) {
    int rc = ck(cudaMemcpy(b->h_cands, b->d_cands + slot * b->cap, sizeof(dd_cand_t) * kept,
                           cudaMemcpyDeviceToHost),
                "candidate readback");
    if (rc) return rc;
    std::sort(b->h_cands, b->h_cands + kept, [](const dd_cand_t& x, const dd_cand_t& y) {
      if (x.range != y.range) return x.range < y.range;
      if (x.trial != y.trial) return x.trial < y.trial;
      if (x.t_start != y.t_start) return x.t_start < y.t_start;
      return x.width < y.width;
    });
    std::memcpy(out, b->h_cands, sizeof(dd_cand_t) * std::min(kept, cap));
  }
  *ncands = count;
  if (count > cap || count > b->cap)
    return ddk::report_error(DD_ERR_CAP, "dd_batch_candidates: more candidates than the buffer");
  return DD_OK;
}

void dd_batch_destroy(dd_batch_t b) { free_batch(b); }

}  // extern "C"
