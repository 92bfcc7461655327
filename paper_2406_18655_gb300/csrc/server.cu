// Serving runtime: continuous batching of single-shot decode requests over several codes.
//
// Requests (code, syndrome pointer, correction pointer, status pointer) arrive from any
// thread through lsd_server_submit (or from the built-in Poisson generator).  One scheduler
// thread owns the GPU side: per code it keeps `slots` in-flight batches, each slot a decoder
// of its own with its own stream, so a batch launches as soon as a slot is idle and the
// memory budget admits it, while earlier batches are still on the device.  A batch is a list
// of request pointers written to pinned memory; a gather kernel pulls the syndromes into the
// slot's device buffer (host memory is read directly by the GPU), the decoder runs BP + LSD,
// and a scatter kernel writes each correction and status back to its request's buffer.  The
// host does O(1) work per request.  Completion is detected by polling the slot's event.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <random>
#include <thread>
#include <vector>

#include "lsd_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

inline int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(Clock::now().time_since_epoch())
      .count();
}

struct Request {
  int32_t code;
  const uint8_t* syn;
  uint8_t* corr;
  uint8_t* status;
  int64_t arrival_ns;
  int64_t id;
};

// Per-shot pointers of one batch (pinned host memory, read by the gather/scatter kernels).
struct BatchDesc {
  const uint8_t** syn;
  uint8_t** corr;
  uint8_t** status;
};

__global__ void gather_kernel(const long long* count, int m, const uint8_t* const* syn,
                              uint8_t* out) {
  const int lane = threadIdx.x & 31;
  const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (w >= *count) return;
  const uint8_t* src = syn[w];
  uint8_t* dst = out + (size_t)w * m;
  for (int i = lane; i < m; i += 32) dst[i] = src[i];
}

__global__ void scatter_kernel(const long long* count, int n, const uint8_t* corr,
                               const uint8_t* status, uint8_t* const* corr_out,
                               uint8_t* const* status_out) {
  const int lane = threadIdx.x & 31;
  const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (w >= *count) return;
  uint8_t* dst = corr_out[w];
  if (dst) {
    const uint8_t* src = corr + (size_t)w * n;
    for (int i = lane; i < n; i += 32) dst[i] = src[i];
  }
  if (lane == 0 && status_out[w]) *status_out[w] = status[w];
}

struct Slot {
  lsd_decoder* dec = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t done = nullptr;
  uint8_t* d_syn = nullptr;
  uint8_t* d_corr = nullptr;
  uint8_t* d_status = nullptr;
  BatchDesc desc{};            // pinned
  long long* count = nullptr;  // pinned, read by the kernels: shots of the batch
  cudaGraphExec_t graph = nullptr;  // gather -> BP -> LSD -> scatter, captured once
  std::vector<Request> reqs;   // requests of the batch in flight
  size_t reserved = 0;         // admitted bytes
  bool busy = false;
};

struct Code {
  int m = 0, n = 0;
  size_t bytes_per_shot = 0;   // device bytes one in-flight shot holds
  std::vector<Slot> slots;
  std::deque<Request> pending;
};

struct Report {
  int64_t submitted = 0, completed = 0, batches = 0, batched_shots = 0, admission_waits = 0;
  int64_t first_arrival = 0, last_completion = 0;
  size_t peak_bytes = 0;
  std::vector<int64_t> latency_ns;
};

}  // namespace

struct lsd_server {
  std::vector<Code> codes;
  lsd_server_options opt{};
  std::mutex mu;                       // guards pending queues and the report
  std::condition_variable cv_work;     // scheduler wake-up
  std::condition_variable cv_done;     // completion of all requests
  std::atomic<bool> stop{false};
  std::atomic<int64_t> outstanding{0};
  std::atomic<int64_t> next_id{0};
  std::thread sched;
  size_t reserved = 0;                 // scheduler thread only
  Report rep;                          // guarded by mu
  int error = LSD_OK;
};

namespace {

int cuda_rc(cudaError_t e) {
  if (e == cudaSuccess) return LSD_OK;
  lsdgb::record_cuda_error(e);
  return e == cudaErrorMemoryAllocation ? LSD_ERR_OOM : LSD_ERR_CUDA;
}

// The GPU reads request buffers directly: they must be page-locked host memory or device
// (or managed) memory.
bool gpu_accessible(const void* p) {
  if (!p) return true;
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeDevice ||
         a.type == cudaMemoryTypeManaged;
}

void enqueue(lsd_server* sv, const Request* r, size_t count);

// Enqueues the slot's pipeline for *s.count shots: gather, BP + LSD, scatter.
int enqueue_pipeline(Code& c, Slot& s, int max_batch) {
  const int blocks = (max_batch + 7) / 8;
  gather_kernel<<<blocks, 256, 0, s.st>>>(s.count, c.m, s.desc.syn, s.d_syn);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_rc(e);
  int rc = lsdgb::decode_batch_counted(s.dec, max_batch, s.count, s.d_syn, s.d_corr, s.d_status);
  if (rc) return rc;
  scatter_kernel<<<blocks, 256, 0, s.st>>>(s.count, c.n, s.d_corr, s.d_status, s.desc.corr,
                                           s.desc.status);
  return cuda_rc(cudaGetLastError());
}

// Launches one batch of code c on slot s (scheduler thread): one graph launch.
int launch_batch(lsd_server* sv, Code& c, Slot& s) {
  const int b = (int)s.reqs.size();
  for (int k = 0; k < b; ++k) {
    s.desc.syn[k] = s.reqs[k].syn;
    s.desc.corr[k] = s.reqs[k].corr;
    s.desc.status[k] = s.reqs[k].status;
  }
  *s.count = b;
  cudaError_t e;
  if (s.graph) {
    e = cudaGraphLaunch(s.graph, s.st);
    if (e != cudaSuccess) return cuda_rc(e);
  } else {
    const int rc = enqueue_pipeline(c, s, sv->opt.max_batch);
    if (rc) return rc;
  }
  e = cudaEventRecord(s.done, s.st);
  return cuda_rc(e);
}

void scheduler(lsd_server* sv) {
  const int64_t wait_ns = (int64_t)sv->opt.max_wait_us * 1000;
  const size_t budget = sv->opt.mem_budget;
  std::vector<Request> done;
  while (true) {
    bool progressed = false;
    // ---- completions ----
    for (auto& c : sv->codes) {
      for (auto& s : c.slots) {
        if (!s.busy || cudaEventQuery(s.done) != cudaSuccess) continue;
        const int64_t t = now_ns();
        {
          std::lock_guard<std::mutex> lk(sv->mu);
          for (auto& r : s.reqs) sv->rep.latency_ns.push_back(t - r.arrival_ns);
          sv->rep.completed += (int64_t)s.reqs.size();
          sv->rep.last_completion = t;
        }
        sv->outstanding -= (int64_t)s.reqs.size();
        sv->reserved -= s.reserved;
        s.reserved = 0;
        s.reqs.clear();
        s.busy = false;
        progressed = true;
        sv->cv_done.notify_all();
      }
    }
    // ---- launches: every idle slot takes the code's pending requests ----
    for (auto& c : sv->codes) {
      for (auto& s : c.slots) {
        if (s.busy) continue;
        std::unique_lock<std::mutex> lk(sv->mu);
        if (c.pending.empty()) break;
        const int64_t age = now_ns() - c.pending.front().arrival_ns;
        const size_t want = std::min<size_t>(c.pending.size(), (size_t)sv->opt.max_batch);
        if ((int)want < sv->opt.max_batch && age < wait_ns && !sv->stop) break;
        size_t take = want;
        if (budget) {  // admission by memory: shrink the batch to what the budget still holds
          const size_t room = budget > sv->reserved ? budget - sv->reserved : 0;
          take = std::min(take, room / c.bytes_per_shot);
          if (take == 0) {
            sv->rep.admission_waits++;
            break;
          }
        }
        for (size_t k = 0; k < take; ++k) {
          s.reqs.push_back(c.pending.front());
          c.pending.pop_front();
        }
        sv->rep.batches++;
        sv->rep.batched_shots += (int64_t)take;
        lk.unlock();
        s.reserved = take * c.bytes_per_shot;
        sv->reserved += s.reserved;
        {
          std::lock_guard<std::mutex> lk2(sv->mu);
          if (sv->reserved > sv->rep.peak_bytes) sv->rep.peak_bytes = sv->reserved;
        }
        s.busy = true;
        const int rc = launch_batch(sv, c, s);
        if (rc) {
          std::lock_guard<std::mutex> lk2(sv->mu);
          sv->error = rc;
        }
        progressed = true;
      }
    }
    if (sv->stop && sv->outstanding.load() == 0) break;
    if (!progressed) {
      bool any_busy = false;
      for (auto& c : sv->codes)
        for (auto& s : c.slots) any_busy = any_busy || s.busy;
      std::unique_lock<std::mutex> lk(sv->mu);
      bool any_pending = false;
      for (auto& c : sv->codes) any_pending = any_pending || !c.pending.empty();
      if (!any_busy && !any_pending && !sv->stop)
        sv->cv_work.wait_for(lk, std::chrono::microseconds(200));
      else if (!any_busy)
        sv->cv_work.wait_for(lk, std::chrono::microseconds(std::max(1, sv->opt.max_wait_us / 4)));
      // with batches in flight: spin on their events
    }
  }
}

void enqueue(lsd_server* sv, const Request* r, size_t count) {
  if (!count) return;
  sv->outstanding += (int64_t)count;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->rep.submitted == 0) sv->rep.first_arrival = r[0].arrival_ns;
    sv->rep.submitted += (int64_t)count;
    for (size_t k = 0; k < count; ++k) sv->codes[r[k].code].pending.push_back(r[k]);
  }
  sv->cv_work.notify_one();
}

void free_server(lsd_server* sv) {
  for (auto& c : sv->codes)
    for (auto& s : c.slots) {
      if (s.st) cudaStreamSynchronize(s.st);
      if (s.dec) lsd_destroy(s.dec);
      if (s.d_syn) cudaFree(s.d_syn);
      if (s.d_corr) cudaFree(s.d_corr);
      if (s.d_status) cudaFree(s.d_status);
      if (s.desc.syn) cudaFreeHost(s.desc.syn);
      if (s.desc.corr) cudaFreeHost(s.desc.corr);
      if (s.desc.status) cudaFreeHost(s.desc.status);
      if (s.count) cudaFreeHost(s.count);
      if (s.graph) cudaGraphExecDestroy(s.graph);
      if (s.done) cudaEventDestroy(s.done);
      if (s.st) cudaStreamDestroy(s.st);
    }
  cudaGetLastError();
  delete sv;
}

int64_t percentile(std::vector<int64_t>& v, double q) {
  if (v.empty()) return 0;
  const size_t k = (size_t)(q * (double)(v.size() - 1) + 0.5);
  std::nth_element(v.begin(), v.begin() + k, v.end());
  return v[k];
}

}  // namespace

extern "C" {

int lsd_server_create(lsd_server** out, int32_t n_codes, const lsd_server_code* codes,
                      const lsd_server_options* opt) {
  if (!out || n_codes < 1 || !codes) return LSD_ERR_INVALID_ARG;
  *out = nullptr;
  lsd_server_options o{};
  if (opt) o = *opt;
  if (o.slots_per_code == 0) o.slots_per_code = 3;
  if (o.max_batch == 0) o.max_batch = 8192;
  if (o.max_wait_us == 0) o.max_wait_us = 50;
  if (o.slots_per_code < 1 || o.slots_per_code > 16 || o.max_batch < 1 || o.max_wait_us < 0 ||
      o.use_graphs < -1 || o.use_graphs > 0)
    return LSD_ERR_INVALID_ARG;
  lsd_server* sv = new (std::nothrow) lsd_server();
  if (!sv) return LSD_ERR_OOM;
  sv->opt = o;
  sv->codes.resize(n_codes);
  int rc = LSD_OK;
  for (int ci = 0; ci < n_codes && !rc; ++ci) {
    const lsd_server_code& cd = codes[ci];
    Code& c = sv->codes[ci];
    c.m = cd.m;
    c.n = cd.n;
    c.bytes_per_shot = (size_t)cd.m + 2 * (size_t)cd.n + 2 + 4 * ((size_t)cd.n + 1);
    if (o.mem_budget && c.bytes_per_shot > o.mem_budget) rc = LSD_ERR_ADMISSION;
    c.slots.resize(o.slots_per_code);
    for (auto& s : c.slots) {
      if (rc) break;
      cudaError_t e = cudaStreamCreateWithFlags(&s.st, cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming);
      const size_t B = (size_t)o.max_batch;
      if (e == cudaSuccess) e = cudaMalloc(&s.d_syn, B * cd.m);
      if (e == cudaSuccess) e = cudaMalloc(&s.d_corr, B * cd.n);
      if (e == cudaSuccess) e = cudaMalloc(&s.d_status, B);
      if (e == cudaSuccess) e = cudaHostAlloc(&s.desc.syn, B * sizeof(void*), cudaHostAllocMapped);
      if (e == cudaSuccess) e = cudaHostAlloc(&s.desc.corr, B * sizeof(void*), cudaHostAllocMapped);
      if (e == cudaSuccess) e = cudaHostAlloc(&s.desc.status, B * sizeof(void*), cudaHostAllocMapped);
      if (e == cudaSuccess) e = cudaHostAlloc(&s.count, sizeof(long long), cudaHostAllocMapped);
      if (e != cudaSuccess) {
        rc = cuda_rc(e);
        break;
      }
      lsd_options dopt{};
      dopt.stream = s.st;
      rc = lsd_create(&s.dec, cd.m, cd.n, cd.nnz, cd.rows, cd.cols, cd.channel_probs, cd.bp_iters,
                      cd.lsd_order, &dopt);
      // size the decoder's workspace for a full batch now, so serving never allocates
      if (!rc) e = cudaMemsetAsync(s.d_syn, 0, B * cd.m, s.st);
      if (!rc && e != cudaSuccess) rc = cuda_rc(e);
      if (!rc) rc = lsd_decode_batch(s.dec, (int64_t)B, s.d_syn, s.d_corr, s.d_status, nullptr, nullptr);
      if (!rc) rc = cuda_rc(cudaStreamSynchronize(s.st));
      // capture the per-batch pipeline once; every batch is then one graph launch
      if (!rc && o.use_graphs >= 0) {
        *s.count = 0;
        for (size_t k = 0; k < B; ++k) {
          s.desc.syn[k] = nullptr;
          s.desc.corr[k] = nullptr;
          s.desc.status[k] = nullptr;
        }
        cudaGraph_t g = nullptr;
        e = cudaStreamBeginCapture(s.st, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
          const int rc2 = enqueue_pipeline(c, s, o.max_batch);
          e = cudaStreamEndCapture(s.st, &g);
          if (rc2) rc = rc2;
        }
        if (!rc && e == cudaSuccess) e = cudaGraphInstantiate(&s.graph, g, 0);
        if (g) cudaGraphDestroy(g);
        if (!rc && e != cudaSuccess) rc = cuda_rc(e);
      }
      s.reqs.reserve(o.max_batch);
    }
  }
  if (rc) {
    free_server(sv);
    return rc;
  }
  sv->sched = std::thread(scheduler, sv);
  *out = sv;
  return LSD_OK;
}

int lsd_server_submit(lsd_server* sv, int32_t code, const uint8_t* syndrome, uint8_t* correction,
                      uint8_t* status, int64_t* id) {
  if (!sv || code < 0 || code >= (int32_t)sv->codes.size() || !syndrome) return LSD_ERR_INVALID_ARG;
  if (!gpu_accessible(syndrome) || !gpu_accessible(correction) || !gpu_accessible(status))
    return LSD_ERR_INVALID_ARG;
  Request r{code, syndrome, correction, status, now_ns(), sv->next_id++};
  enqueue(sv, &r, 1);
  if (id) *id = r.id;
  return LSD_OK;
}

int lsd_server_wait_all(lsd_server* sv) {
  if (!sv) return LSD_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(sv->mu);
  sv->cv_work.notify_one();
  while (sv->outstanding.load() > 0) {
    sv->cv_done.wait_for(lk, std::chrono::milliseconds(1));
    if (sv->error) break;
  }
  return sv->error;
}

int lsd_server_get_report(lsd_server* sv, lsd_server_report* out, int32_t reset) {
  if (!sv || !out) return LSD_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(sv->mu);
  Report& r = sv->rep;
  std::memset(out, 0, sizeof(*out));
  out->submitted = r.submitted;
  out->completed = r.completed;
  out->batches = r.batches;
  out->mean_batch = r.batches ? (double)r.batched_shots / (double)r.batches : 0.0;
  out->admission_waits = r.admission_waits;
  out->peak_inflight_bytes = (int64_t)r.peak_bytes;
  out->seconds = r.completed ? (double)(r.last_completion - r.first_arrival) * 1e-9 : 0.0;
  out->shots_per_s = out->seconds > 0 ? (double)r.completed / out->seconds : 0.0;
  if (!r.latency_ns.empty()) {
    std::vector<int64_t> v = r.latency_ns;
    double sum = 0;
    int64_t mx = 0;
    for (int64_t x : v) {
      sum += (double)x;
      mx = std::max(mx, x);
    }
    out->mean_us = sum / (double)v.size() * 1e-3;
    out->max_us = (double)mx * 1e-3;
    out->p50_us = (double)percentile(v, 0.50) * 1e-3;
    out->p99_us = (double)percentile(v, 0.99) * 1e-3;
  }
  if (reset) r = Report{};
  return sv->error;
}

int lsd_server_run_poisson(lsd_server* sv, double rate, double seconds, const double* mix,
                           const uint8_t* const* pools, const int64_t* pool_sizes, uint64_t seed,
                           lsd_server_report* out) {
  if (!sv || !(rate > 0) || !(seconds > 0) || !mix || !pools || !pool_sizes || !out)
    return LSD_ERR_INVALID_ARG;
  const int nc = (int)sv->codes.size();
  std::vector<double> cdf(nc);
  double acc = 0;
  for (int c = 0; c < nc; ++c) {
    if (mix[c] < 0 || (mix[c] > 0 && (!pools[c] || pool_sizes[c] < 1))) return LSD_ERR_INVALID_ARG;
    acc += mix[c];
    cdf[c] = acc;
  }
  if (!(acc > 0)) return LSD_ERR_INVALID_ARG;
  for (int c = 0; c < nc; ++c)
    if (mix[c] > 0 && !gpu_accessible(pools[c])) return LSD_ERR_INVALID_ARG;
  lsd_server_report dummy;
  lsd_server_get_report(sv, &dummy, 1);
  std::mt19937_64 rng(seed);
  std::exponential_distribution<double> gap(rate);
  std::uniform_real_distribution<double> uni(0.0, acc);
  std::vector<int64_t> cursor(nc, 0);
  std::vector<Request> burst;
  burst.reserve(4096);
  const int64_t t0 = now_ns();
  const int64_t t_end = t0 + (int64_t)(seconds * 1e9);
  double t_next = (double)t0 + gap(rng) * 1e9;
  int64_t generated = 0;
  // every request whose scheduled arrival has passed is enqueued at once, stamped with its
  // scheduled arrival time (the model's arrival), so the generator keeps up at high rates
  while ((int64_t)t_next < t_end) {
    const int64_t now = now_ns();
    while ((int64_t)t_next <= now && (int64_t)t_next < t_end && burst.size() < 4096) {
      const double u = uni(rng);
      int c = 0;
      while (c < nc - 1 && u >= cdf[c]) ++c;
      const uint8_t* syn = pools[c] + (size_t)(cursor[c] % pool_sizes[c]) * sv->codes[c].m;
      cursor[c]++;
      burst.push_back(Request{c, syn, nullptr, nullptr, (int64_t)t_next, sv->next_id++});
      t_next += gap(rng) * 1e9;
    }
    generated += (int64_t)burst.size();
    enqueue(sv, burst.data(), burst.size());
    burst.clear();
  }
  const int rc = lsd_server_wait_all(sv);
  lsd_server_get_report(sv, out, 1);
  out->offered_rate = rate;
  out->generated = generated;
  return rc;
}

int lsd_server_destroy(lsd_server* sv) {
  if (!sv) return LSD_OK;
  sv->stop = true;
  sv->cv_work.notify_all();
  if (sv->sched.joinable()) sv->sched.join();
  free_server(sv);
  return LSD_OK;
}

}  // extern "C"
