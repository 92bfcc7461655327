// Serving runtime: continuous batching of decode requests over several codes.
//
// Two kinds of requests share one scheduler, one memory budget and the GPU:
//   * shots: one syndrome of a code's check matrix, decoded whole (lsd_server_submit);
//   * rounds: one detector block of a stream of repeated syndrome rounds, decoded in (w, c)
//     overlapping windows (Methods 4.3; lsd_server_submit_round).  The server keeps every
//     stream's blocks and the measurement faults of its last committed round; a block that
//     completes a window turns into a window job, decoded like a shot on the window's matrix
//     (every inner window of a code has the same matrix; the final window has its own).
// Per internal code (a shot code, or a window code's inner / final window matrix) the
// scheduler keeps `slots` in-flight batches, each slot a decoder of its own with its own
// stream, so a batch launches as soon as a slot is idle and the memory budget admits it,
// while earlier batches are still on the device.  A batch is a list of request pointers
// written to pinned memory; a gather kernel pulls the syndromes (or a window's blocks) into
// the slot's device buffer, the decoder runs BP, a scatter (commit) kernel writes back the
// rows BP solved, then LSD runs on the others and a second scatter writes them back.  A
// request completes when its own row is written back: the shots BP solves do not wait for
// the rare shot of their batch that needs a long LSD.  Each slot's pipeline is captured
// once as two CUDA graphs (before and after the event that marks the first write-back).
// The host does O(1) work per request (O(m) for a block, which it copies into the stream's
// history).  Completion is detected by polling events.
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
  int32_t code;          // internal code
  const uint8_t* syn;    // shots: the syndrome; window jobs: unused (blocks are in the history)
  uint8_t* corr;
  uint8_t* status;
  int64_t arrival_ns;
  int64_t id;
  int32_t stream = -1;   // window jobs: stream, first round of the window, history half
  int32_t t = 0, half = 0;
  int64_t enqueue_ns = 0;  // when the server took it (arrival_ns may be a scheduled time)
  int64_t launch_ns = 0;   // when its batch was launched
  bool done = false;       // completed (a shot BP solved completes before its batch's LSD)
};

// Per-shot pointers and window-job fields of one batch (pinned host memory, read by the
// gather / scatter kernels).
struct BatchDesc {
  const uint8_t** syn;
  uint8_t** corr;
  uint8_t** status;
  int32_t* job;          // window jobs: stream, t, half (3 ints per job)
};

// Copies `bytes` bytes, one warp: 16-byte words where source and destination share their
// alignment, bytes elsewhere.
__device__ __forceinline__ void warp_copy(uint8_t* dst, const uint8_t* src, int bytes, int lane) {
  const int mis = (int)((reinterpret_cast<uintptr_t>(dst) ^ reinterpret_cast<uintptr_t>(src)) & 15);
  int head = 0;
  if (!mis) {
    head = (int)((16 - (reinterpret_cast<uintptr_t>(dst) & 15)) & 15);
    if (head > bytes) head = bytes;
    const int words = (bytes - head) >> 4;
    const uint4* s4 = reinterpret_cast<const uint4*>(src + head);
    uint4* d4 = reinterpret_cast<uint4*>(dst + head);
    for (int i = lane; i < words; i += 32) d4[i] = s4[i];
    for (int i = head + (words << 4) + lane; i < bytes; i += 32) dst[i] = src[i];
    if (lane < head) dst[lane] = src[lane];
    return;
  }
  for (int i = lane; i < bytes; i += 32) dst[i] = src[i];
}

__global__ void gather_kernel(const long long* count, int m, const uint8_t* const* syn,
                              uint8_t* out) {
  const int lane = threadIdx.x & 31;
  const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (w >= *count) return;
  warp_copy(out + (size_t)w * m, syn[w], m, lane);
}

// Which rows a scatter (commit) writes: every row, only the rows BP solved (written right
// after BP, with every row's status also copied to the slot's early flags), or the rest.
enum { kAllRows = 0, kBpRows = 1, kLsdRows = 2 };

__device__ __forceinline__ bool row_in_phase(int phase, uint8_t st) {
  return phase == kAllRows || ((st == LSD_SHOT_OK_BP) == (phase == kBpRows));
}

__global__ void scatter_kernel(const long long* count, int n, const uint8_t* corr,
                               const uint8_t* status, uint8_t* const* corr_out,
                               uint8_t* const* status_out, int phase, uint8_t* early) {
  const int lane = threadIdx.x & 31;
  const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (w >= *count) return;
  const uint8_t st = status[w];
  if (phase == kBpRows && lane == 0) early[w] = st;
  if (!row_in_phase(phase, st)) return;
  if (corr_out[w]) warp_copy(corr_out[w], corr + (size_t)w * n, n, lane);
  if (lane == 0 && status_out[w]) *status_out[w] = status[w];
}

// Window job k: blocks t..t+bn-1 of its stream's history half -> the window's syndrome; the
// first block takes the measurement faults of the stream's last committed round (t > 0).
__global__ void window_gather_kernel(const long long* count, int m, int bn, int hist_row,
                                     const uint8_t* hist, const uint8_t* carry,
                                     const int32_t* job, uint8_t* out) {
  const int lane = threadIdx.x & 31;
  const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (w >= *count) return;
  const int s = job[3 * w], t = job[3 * w + 1], half = job[3 * w + 2];
  const uint8_t* src = hist + ((size_t)s * 2 + half) * hist_row + (size_t)t * m;
  uint8_t* dst = out + (size_t)w * bn * m;
  warp_copy(dst, src, bn * m, lane);
  if (t > 0) {
    __syncwarp();
    const uint8_t* cs = carry + (size_t)s * m;
    for (int i = lane; i < m; i += 32) dst[i] ^= cs[i];
  }
}

// Window job k: rounds 0..commit-1 of the decoded window -> the request's correction; the
// measurement faults of round commit-1 -> the stream's carry (they flip the first block of
// the stream's next window).
__global__ void window_commit_kernel(const long long* count, int n, int m, int wrow, int commit,
                                     const uint8_t* corr, const uint8_t* status,
                                     const int32_t* job, uint8_t* carry,
                                     uint8_t* const* corr_out, uint8_t* const* status_out,
                                     int phase, uint8_t* early) {
  const int lane = threadIdx.x & 31;
  const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (w >= *count) return;
  const uint8_t st0 = status[w];
  if (phase == kBpRows && lane == 0) early[w] = st0;
  if (!row_in_phase(phase, st0)) return;
  const uint8_t* row = corr + (size_t)w * wrow;
  if (corr_out[w]) warp_copy(corr_out[w], row, commit * (n + m), lane);
  const uint8_t* meas = row + (size_t)(commit - 1) * (n + m) + n;
  uint8_t* cs = carry + (size_t)job[3 * w] * m;
  for (int i = lane; i < m; i += 32) cs[i] = meas[i];
  if (lane == 0 && status_out[w]) *status_out[w] = status[w];
}

struct Slot {
  lsd_decoder* dec = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t done = nullptr;
  cudaEvent_t start = nullptr;  // recorded before the batch: its GPU time is start -> done
  cudaEvent_t bp_done = nullptr;  // recorded once the rows BP solved are written back
  uint8_t* early = nullptr;    // pinned: every row's status after BP (read once bp_done is)
  bool early_seen = false;     // the batch's BP-solved requests have been completed
  uint8_t* d_syn = nullptr;
  uint8_t* d_corr = nullptr;
  uint8_t* d_status = nullptr;
  BatchDesc desc{};            // pinned
  long long* count = nullptr;  // pinned: shots of the batch, written by the scheduler
  long long* d_count = nullptr;  // device copy, made at the start of every batch and read by
                                 // its kernels (one host read per batch, not one per warp)
  cudaGraphExec_t graph[2] = {nullptr, nullptr};  // the pipeline's two parts, captured once
  std::vector<Request> reqs;   // requests of the batch in flight
  int64_t launch_call_ns = 0;  // host time its launch calls took
  size_t reserved = 0;         // admitted bytes
  bool busy = false;
};

struct WindowCode;

struct Code {
  int m = 0, n = 0;            // of the matrix decoded (a window's, for window codes)
  int user = 0;                // the code id callers see
  WindowCode* win = nullptr;   // window codes: the stream state shared by inner and final
  int blocks = 0, commit = 0;  // window codes: detector blocks gathered, rounds committed
  size_t bytes_per_shot = 0;   // device bytes one in-flight shot holds
  std::vector<Slot> slots;
  std::deque<Request> pending;
  int64_t npending = 0;        // pending.size(), written under the mutex, read without it
};

// Appends to a code's pending queue (the server mutex is held).
void push_pending(Code& c, const Request& r) {
  c.pending.push_back(r);
  __atomic_store_n(&c.npending, (int64_t)c.pending.size(), __ATOMIC_RELEASE);
}

struct Stream {
  int next_block = 0;          // blocks received in the current sequence
  int seq = 0;                 // sequences started (its parity is the history half)
  int t_next = 0;              // first round of the sequence's next window
  bool busy = false;           // one of its windows is pending or on the GPU
  std::deque<Request> waiting; // windows formed while another was busy
  int outstanding[2] = {0, 0}; // windows not yet completed, per history half
};

struct WindowCode {
  int m = 0, n = 0, d = 0, w = 0, c = 0, t_final = 0;
  int inner = -1, fin = -1;    // internal codes of the two window matrices
  uint8_t* hist = nullptr;     // pinned host [streams][2][(d+1) m]: blocks of two sequences
  uint8_t* carry = nullptr;    // device [streams][m]
  std::vector<Stream> streams;
};

struct Stats {
  int64_t submitted = 0, completed = 0;
  std::vector<int64_t> latency_ns;
  // the latency's parts: scheduled arrival to submission (a load generator's lag),
  // submission to batch launch (queueing), launch to completion observed (service)
  std::vector<int64_t> lag_ns, queue_ns, service_ns;
  std::vector<int64_t> batch_gpu_ns;  // per batch: GPU time from its start to its done event
  std::vector<int64_t> launch_call_ns;  // per batch: host time of the launch calls
  int64_t batches = 0, batched = 0;
};

struct Report {
  int64_t submitted = 0, completed = 0, batches = 0, batched_shots = 0, admission_waits = 0;
  int64_t first_arrival = 0, last_completion = 0;
  size_t peak_bytes = 0;
  std::vector<int64_t> latency_ns;
  std::vector<Stats> by_code;  // per user code
};

}  // namespace

struct lsd_server {
  std::vector<Code> codes;             // internal codes
  std::vector<WindowCode> wins;        // window codes (user ids n_shot .. n_shot + size - 1)
  int n_shot = 0;                      // user codes 0 .. n_shot-1 are shot codes
  lsd_server_options opt{};
  std::mutex mu;                       // guards pending queues, streams and the report
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

// The scatter (or commit) of a phase's rows of the slot's batch.
int write_back(Code& c, Slot& s, int max_batch, int phase) {
  const int blocks = (max_batch + 7) / 8;
  WindowCode* W = c.win;
  if (W)
    window_commit_kernel<<<blocks, 256, 0, s.st>>>(s.d_count, W->n, W->m, c.n, c.commit, s.d_corr,
                                                   s.d_status, s.desc.job, W->carry, s.desc.corr,
                                                   s.desc.status, phase, s.early);
  else
    scatter_kernel<<<blocks, 256, 0, s.st>>>(s.d_count, c.n, s.d_corr, s.d_status, s.desc.corr,
                                             s.desc.status, phase, s.early);
  return cuda_rc(cudaGetLastError());
}

// The slot's pipeline for *s.count shots in two parts (one graph each): part 0 = gather,
// BP and the scatter (or commit) of the rows BP solved; part 1 = LSD and the scatter of the
// other rows.  The host records bp_done between them.
int enqueue_part(Code& c, Slot& s, int max_batch, int part) {
  if (part == 1) {
    const int rc = lsdgb::lsd_batch_counted(s.dec, max_batch, s.d_syn, s.d_corr, s.d_status);
    return rc ? rc : write_back(c, s, max_batch, kLsdRows);
  }
  const int blocks = (max_batch + 7) / 8;
  WindowCode* W = c.win;
  cudaError_t e0 = cudaMemcpyAsync(s.d_count, s.count, sizeof(long long), cudaMemcpyHostToDevice,
                                   s.st);
  if (e0 != cudaSuccess) return cuda_rc(e0);
  if (W)
    window_gather_kernel<<<blocks, 256, 0, s.st>>>(s.d_count, W->m, c.blocks, (W->d + 1) * W->m,
                                                   W->hist, W->carry, s.desc.job, s.d_syn);
  else
    gather_kernel<<<blocks, 256, 0, s.st>>>(s.d_count, c.m, s.desc.syn, s.d_syn);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_rc(e);
  // statuses start at 0, so a row that BP leaves unsolved never reads as LSD_SHOT_OK_BP
  e = cudaMemsetAsync(s.d_status, 0, (size_t)max_batch, s.st);
  if (e != cudaSuccess) return cuda_rc(e);
  const int rc = lsdgb::bp_batch_counted(s.dec, max_batch, s.d_count, s.d_syn, s.d_corr, s.d_status);
  return rc ? rc : write_back(c, s, max_batch, kBpRows);
}

// Launches one batch of code c on slot s (scheduler thread): one graph launch.
int launch_batch(lsd_server* sv, Code& c, Slot& s) {
  const int b = (int)s.reqs.size();
  const int64_t t_launch = now_ns();
  for (int k = 0; k < b; ++k) {
    Request& r = s.reqs[k];
    r.launch_ns = t_launch;
    s.desc.syn[k] = r.syn;
    s.desc.corr[k] = r.corr;
    s.desc.status[k] = r.status;
    s.desc.job[3 * k] = r.stream;
    s.desc.job[3 * k + 1] = r.t;
    s.desc.job[3 * k + 2] = r.half;
  }
  *s.count = b;
  s.early_seen = false;
  cudaError_t e = cudaEventRecord(s.start, s.st);
  if (e != cudaSuccess) return cuda_rc(e);
  for (int part = 0; part < 2; ++part) {
    if (s.graph[part]) {
      e = cudaGraphLaunch(s.graph[part], s.st);
      if (e != cudaSuccess) return cuda_rc(e);
    } else {
      const int rc = enqueue_part(c, s, sv->opt.max_batch, part);
      if (rc) return rc;
    }
    if (part == 0) {
      e = cudaEventRecord(s.bp_done, s.st);
      if (e != cudaSuccess) return cuda_rc(e);
    }
  }
  e = cudaEventRecord(s.done, s.st);
  s.launch_call_ns = now_ns() - t_launch;
  return cuda_rc(e);
}

// A window job left the GPU (mu held): the stream's next formed window, if any, becomes
// pending (windows of one stream run one at a time, in order: each reads the carry the
// previous one wrote).
void window_done(lsd_server* sv, WindowCode& W, const Request& r) {
  Stream& S = W.streams[r.stream];
  S.outstanding[r.half]--;
  S.busy = false;
  if (!S.waiting.empty()) {
    Request nx = S.waiting.front();
    S.waiting.pop_front();
    S.busy = true;
    push_pending(sv->codes[nx.code], nx);
  }
}

// Records a request's completion at time t (mu held).
void complete_request(lsd_server* sv, Code& c, Stats& cs, Request& r, int64_t t) {
  sv->rep.latency_ns.push_back(t - r.arrival_ns);
  cs.latency_ns.push_back(t - r.arrival_ns);
  cs.lag_ns.push_back(r.enqueue_ns - r.arrival_ns);
  cs.queue_ns.push_back(r.launch_ns - r.enqueue_ns);
  cs.service_ns.push_back(t - r.launch_ns);
  if (c.win) window_done(sv, *c.win, r);
  sv->rep.completed++;
  cs.completed++;
  r.done = true;
}

void scheduler(lsd_server* sv) {
  const int64_t wait_ns = (int64_t)sv->opt.max_wait_us * 1000;
  const size_t budget = sv->opt.mem_budget;
  while (true) {
    bool progressed = false;
    // ---- completions ----
    // A request whose shot BP solved completes once its batch's first part is done (its row
    // is written back before bp_done); the others when the whole batch is.
    for (auto& c : sv->codes) {
      for (auto& s : c.slots) {
        if (!s.busy) continue;
        if (!s.early_seen && cudaEventQuery(s.bp_done) == cudaSuccess) {
          s.early_seen = true;
          const int64_t t = now_ns();
          int64_t k_done = 0;
          {
            std::lock_guard<std::mutex> lk(sv->mu);
            Stats& cs = sv->rep.by_code[c.user];
            for (size_t k = 0; k < s.reqs.size(); ++k) {
              if (s.early[k] != LSD_SHOT_OK_BP) continue;
              complete_request(sv, c, cs, s.reqs[k], t);
              ++k_done;
            }
            if (k_done) sv->rep.last_completion = t;
          }
          if (k_done) {
            sv->outstanding -= k_done;
            progressed = true;
            sv->cv_done.notify_all();
          }
        }
        if (cudaEventQuery(s.done) != cudaSuccess) continue;
        const int64_t t = now_ns();
        float gpu_ms = 0.f;
        if (cudaEventElapsedTime(&gpu_ms, s.start, s.done) != cudaSuccess) cudaGetLastError();
        int64_t k_done = 0;
        {
          std::lock_guard<std::mutex> lk(sv->mu);
          Stats& cs = sv->rep.by_code[c.user];
          cs.batch_gpu_ns.push_back((int64_t)(gpu_ms * 1e6));
          cs.launch_call_ns.push_back(s.launch_call_ns);
          cs.batches++;
          cs.batched += (int64_t)s.reqs.size();
          for (auto& r : s.reqs) {
            if (r.done) continue;
            complete_request(sv, c, cs, r, t);
            ++k_done;
          }
          sv->rep.last_completion = t;
        }
        sv->outstanding -= k_done;
        sv->reserved -= s.reserved;
        s.reserved = 0;
        s.reqs.clear();
        s.busy = false;
        progressed = true;
        sv->cv_done.notify_all();
      }
    }
    // ---- launches: every idle slot takes the code's pending requests ----
    // (the mutex is taken only for codes with pending requests, so a scheduler spinning on
    // batches in flight does not hold up the threads that submit)
    for (auto& c : sv->codes) {
      if (__atomic_load_n(&c.npending, __ATOMIC_ACQUIRE) == 0) continue;
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
        __atomic_store_n(&c.npending, (int64_t)c.pending.size(), __ATOMIC_RELEASE);
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
      // idle: sleep until a submission wakes us (the timeout only bounds a missed wake-up);
      // requests waiting for a fuller batch: sleep a fraction of max_wait_us; batches in
      // flight: spin on their events
      if (!any_busy && !any_pending && !sv->stop)
        sv->cv_work.wait_for(lk, std::chrono::microseconds(200));
      else if (!any_busy)
        sv->cv_work.wait_for(lk, std::chrono::microseconds(std::max(1, sv->opt.max_wait_us / 4)));
    }
  }
}

// Requests of shot codes (r[k].code internal = user id).
void enqueue(lsd_server* sv, const Request* r, size_t count) {
  if (!count) return;
  sv->outstanding += (int64_t)count;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->rep.submitted == 0) sv->rep.first_arrival = r[0].arrival_ns;
    sv->rep.submitted += (int64_t)count;
    const int64_t t = now_ns();
    for (size_t k = 0; k < count; ++k) {
      sv->rep.by_code[sv->codes[r[k].code].user].submitted++;
      Request q = r[k];
      q.enqueue_ns = t;
      push_pending(sv->codes[q.code], q);
    }
  }
  sv->cv_work.notify_one();
}

// One detector block of a stream (mu held).  Stores it; when it completes a window, forms
// the window job.  Returns LSD_ERR_ADMISSION when the block would overwrite history that a
// window two sequences back still needs.
int submit_round_locked(lsd_server* sv, int user, WindowCode& W, int stream,
                        const uint8_t* block, uint8_t* corr, uint8_t* status, int64_t arrival,
                        int64_t id, int32_t* first_round, int32_t* rounds, bool* formed) {
  Stream& S = W.streams[stream];
  const int half = S.seq & 1;
  const int b = S.next_block;
  *formed = false;
  if (b == 0 && S.outstanding[half] > 0) return LSD_ERR_ADMISSION;
  std::memcpy(W.hist + ((size_t)stream * 2 + half) * (size_t)(W.d + 1) * W.m + (size_t)b * W.m,
              block, (size_t)W.m);
  S.next_block = b + 1;
  const int t = S.t_next;
  const bool final = t == W.t_final;
  if (b != (final ? W.d : t + W.w - 1)) return LSD_OK;
  Request r{final ? W.fin : W.inner, nullptr, corr, status, arrival, id, stream, t, half,
            now_ns()};
  if (first_round) *first_round = t;
  if (rounds) *rounds = final ? W.d - t : W.c;
  S.outstanding[half]++;
  if (final) {  // the sequence is complete: the stream's next block starts a new one
    S.next_block = 0;
    S.t_next = 0;
    S.seq++;
  } else {
    S.t_next = t + W.c;
  }
  if (sv->rep.submitted == 0) sv->rep.first_arrival = arrival;
  sv->rep.submitted++;
  sv->rep.by_code[user].submitted++;
  sv->outstanding++;
  if (S.busy) {
    S.waiting.push_back(r);
  } else {
    S.busy = true;
    push_pending(sv->codes[r.code], r);
  }
  *formed = true;
  return LSD_OK;
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
      if (s.desc.job) cudaFreeHost(s.desc.job);
      if (s.count) cudaFreeHost(s.count);
      if (s.d_count) cudaFree(s.d_count);
      for (auto& gx : s.graph)
        if (gx) cudaGraphExecDestroy(gx);
      if (s.done) cudaEventDestroy(s.done);
      if (s.start) cudaEventDestroy(s.start);
      if (s.bp_done) cudaEventDestroy(s.bp_done);
      if (s.early) cudaFreeHost(s.early);
      if (s.st) cudaStreamDestroy(s.st);
    }
  for (auto& W : sv->wins) {
    if (W.hist) cudaFreeHost(W.hist);
    if (W.carry) cudaFree(W.carry);
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

// p99 of the latency parts of the given codes' requests.
void fill_parts(const std::vector<const Stats*>& codes, lsd_server_report* out) {
  std::vector<int64_t> lag, queue, service;
  for (const Stats* st : codes) {
    lag.insert(lag.end(), st->lag_ns.begin(), st->lag_ns.end());
    queue.insert(queue.end(), st->queue_ns.begin(), st->queue_ns.end());
    service.insert(service.end(), st->service_ns.begin(), st->service_ns.end());
  }
  out->p99_lag_us = (double)percentile(lag, 0.99) * 1e-3;
  out->p99_queue_us = (double)percentile(queue, 0.99) * 1e-3;
  out->p99_service_us = (double)percentile(service, 0.99) * 1e-3;
}

void fill_latency(std::vector<int64_t> v, lsd_server_report* out) {
  if (v.empty()) return;
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

// Slots of one internal code: decoders created by make_dec, buffers for max_batch shots of
// the matrix c.m x c.n, the decoder's workspace sized now (serving never allocates), and
// the pipeline captured as a graph.
template <class MakeDec>
int make_slots(lsd_server* sv, Code& c, MakeDec&& make_dec) {
  const lsd_server_options& o = sv->opt;
  c.bytes_per_shot = (size_t)c.m + 2 * (size_t)c.n + 2 + 4 * ((size_t)c.n + 1);
  if (o.mem_budget && c.bytes_per_shot > o.mem_budget) return LSD_ERR_ADMISSION;
  c.slots.resize(o.slots_per_code);
  const size_t B = (size_t)o.max_batch;
  for (auto& s : c.slots) {
    cudaError_t e = cudaStreamCreateWithFlags(&s.st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&s.done);
    if (e == cudaSuccess) e = cudaEventCreate(&s.start);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.bp_done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaHostAlloc(&s.early, B, cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaMalloc(&s.d_syn, B * c.m);
    if (e == cudaSuccess) e = cudaMalloc(&s.d_corr, B * c.n);
    if (e == cudaSuccess) e = cudaMalloc(&s.d_status, B);
    if (e == cudaSuccess) e = cudaHostAlloc(&s.desc.syn, B * sizeof(void*), cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostAlloc(&s.desc.corr, B * sizeof(void*), cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostAlloc(&s.desc.status, B * sizeof(void*), cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostAlloc(&s.desc.job, B * 3 * sizeof(int32_t), cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostAlloc(&s.count, sizeof(long long), cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaMalloc(&s.d_count, sizeof(long long));
    if (e != cudaSuccess) return cuda_rc(e);
    lsd_options dopt{};
    dopt.stream = s.st;
    dopt.bp_kernel = 3;  // batches are small at low load: the shortest per-shot BP latency
    int rc = make_dec(&s.dec, &dopt);
    if (!rc) rc = cuda_rc(cudaMemsetAsync(s.d_syn, 0, B * c.m, s.st));
    if (!rc) rc = lsd_decode_batch(s.dec, (int64_t)B, s.d_syn, s.d_corr, s.d_status, nullptr, nullptr);
    if (!rc) rc = cuda_rc(cudaStreamSynchronize(s.st));
    if (rc) return rc;
    *s.count = 0;
    for (size_t k = 0; k < B; ++k) {
      s.desc.syn[k] = nullptr;
      s.desc.corr[k] = nullptr;
      s.desc.status[k] = nullptr;
    }
    std::memset(s.desc.job, 0, B * 3 * sizeof(int32_t));
    for (int part = 0; part < 2 && o.use_graphs >= 0; ++part) {  // a batch: two graph launches
      cudaGraph_t g = nullptr;
      e = cudaStreamBeginCapture(s.st, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        const int rc2 = enqueue_part(c, s, o.max_batch, part);
        e = cudaStreamEndCapture(s.st, &g);
        if (rc2) rc = rc2;
      }
      if (!rc && e == cudaSuccess) e = cudaGraphInstantiate(&s.graph[part], g, 0);
      if (g) cudaGraphDestroy(g);
      if (!rc && e != cudaSuccess) rc = cuda_rc(e);
      if (rc) return rc;
    }
    s.reqs.reserve(o.max_batch);
  }
  return LSD_OK;
}

}  // namespace

extern "C" {

int lsd_server_create_with_windows(lsd_server** out, int32_t n_codes, const lsd_server_code* codes,
                                   int32_t n_window_codes, const lsd_server_window_code* wcodes,
                                   const lsd_server_options* opt) {
  if (!out || n_codes < 0 || n_window_codes < 0 || n_codes + n_window_codes < 1 ||
      (n_codes && !codes) || (n_window_codes && !wcodes))
    return LSD_ERR_INVALID_ARG;
  *out = nullptr;
  lsd_server_options o{};
  if (opt) o = *opt;
  if (o.slots_per_code == 0) o.slots_per_code = 3;
  if (o.max_batch == 0) o.max_batch = 8192;
  if (o.slots_per_code < 1 || o.slots_per_code > 16 || o.max_batch < 1 || o.max_wait_us < 0 ||
      o.use_graphs < -1 || o.use_graphs > 0)
    return LSD_ERR_INVALID_ARG;
  for (int k = 0; k < n_window_codes; ++k) {
    const lsd_server_window_code& wc = wcodes[k];
    if (wc.m < 1 || wc.n < 1 || wc.nnz < 0 || (wc.nnz > 0 && (!wc.rows || !wc.cols)) ||
        !wc.p_data || !wc.q_meas || wc.rounds < 1 || wc.window < 1 || wc.commit < 1 ||
        wc.commit > wc.window || wc.streams < 1 || wc.streams > (1 << 24))
      return LSD_ERR_INVALID_ARG;
    for (int64_t e = 0; e < wc.nnz; ++e)
      if (wc.rows[e] < 0 || wc.rows[e] >= wc.m || wc.cols[e] < 0 || wc.cols[e] >= wc.n)
        return LSD_ERR_INVALID_ARG;
  }
  lsd_server* sv = new (std::nothrow) lsd_server();
  if (!sv) return LSD_ERR_OOM;
  sv->opt = o;
  sv->n_shot = n_codes;
  sv->wins.resize(n_window_codes);
  sv->rep.by_code.resize(n_codes + n_window_codes);
  int n_internal = n_codes;
  for (int k = 0; k < n_window_codes; ++k) {
    const lsd_server_window_code& wc = wcodes[k];
    WindowCode& W = sv->wins[k];
    W.m = wc.m;
    W.n = wc.n;
    W.d = wc.rounds;
    W.w = wc.window;
    W.c = wc.commit;
    W.t_final = lsdgb::window_final_round(W.d, W.w, W.c);
    W.inner = W.t_final > 0 ? n_internal++ : -1;
    W.fin = n_internal++;
  }
  sv->codes.resize(n_internal);
  int rc = LSD_OK;
  for (int ci = 0; ci < n_codes && !rc; ++ci) {
    const lsd_server_code& cd = codes[ci];
    Code& c = sv->codes[ci];
    c.m = cd.m;
    c.n = cd.n;
    c.user = ci;
    rc = make_slots(sv, c, [&](lsd_decoder** dec, const lsd_options* dopt) {
      return lsd_create(dec, cd.m, cd.n, cd.nnz, cd.rows, cd.cols, cd.channel_probs,
                        cd.bp_iters, cd.lsd_order, dopt);
    });
  }
  for (int k = 0; k < n_window_codes && !rc; ++k) {
    const lsd_server_window_code& wc = wcodes[k];
    WindowCode& W = sv->wins[k];
    std::vector<std::pair<int, int>> h((size_t)wc.nnz);
    for (int64_t e = 0; e < wc.nnz; ++e) h[(size_t)e] = {wc.rows[e], wc.cols[e]};
    W.streams.resize(wc.streams);
    const size_t hist = (size_t)wc.streams * 2 * (W.d + 1) * W.m;
    cudaError_t e = cudaHostAlloc(&W.hist, hist, cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaMalloc(&W.carry, (size_t)wc.streams * W.m);
    if (e == cudaSuccess) e = cudaMemset(W.carry, 0, (size_t)wc.streams * W.m);
    if (e != cudaSuccess) {
      rc = cuda_rc(e);
      break;
    }
    std::memset(W.hist, 0, hist);
    for (int part = 0; part < 2 && !rc; ++part) {
      const bool final = part == 1;
      if (!final && W.inner < 0) continue;
      Code& c = sv->codes[final ? W.fin : W.inner];
      const int rounds = final ? W.d - W.t_final : W.w;
      c.blocks = final ? rounds + 1 : W.w;
      c.commit = final ? rounds : W.c;
      c.m = c.blocks * W.m;
      c.n = rounds * (W.n + W.m);
      c.user = n_codes + k;
      c.win = &W;
      rc = make_slots(sv, c, [&](lsd_decoder** dec, const lsd_options* dopt) {
        return lsdgb::window_decoder(dec, W.m, W.n, h, wc.p_data, wc.q_meas, rounds, c.blocks,
                                     wc.bp_iters, wc.lsd_order, dopt);
      });
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

int lsd_server_create(lsd_server** out, int32_t n_codes, const lsd_server_code* codes,
                      const lsd_server_options* opt) {
  if (n_codes < 1) return LSD_ERR_INVALID_ARG;
  return lsd_server_create_with_windows(out, n_codes, codes, 0, nullptr, opt);
}

int lsd_server_submit(lsd_server* sv, int32_t code, const uint8_t* syndrome, uint8_t* correction,
                      uint8_t* status, int64_t* id) {
  if (!sv || code < 0 || code >= sv->n_shot || !syndrome) return LSD_ERR_INVALID_ARG;
  if (!gpu_accessible(syndrome) || !gpu_accessible(correction) || !gpu_accessible(status))
    return LSD_ERR_INVALID_ARG;
  Request r{code, syndrome, correction, status, now_ns(), sv->next_id++};
  enqueue(sv, &r, 1);
  if (id) *id = r.id;
  return LSD_OK;
}

int lsd_server_submit_round(lsd_server* sv, int32_t code, int32_t stream, const uint8_t* block,
                            uint8_t* correction, uint8_t* status, int32_t* first_round,
                            int32_t* rounds, int64_t* id) {
  if (first_round) *first_round = -1;
  if (rounds) *rounds = 0;
  if (!sv || code < sv->n_shot || code >= sv->n_shot + (int32_t)sv->wins.size() || !block)
    return LSD_ERR_INVALID_ARG;
  WindowCode& W = sv->wins[code - sv->n_shot];
  if (stream < 0 || stream >= (int32_t)W.streams.size()) return LSD_ERR_INVALID_ARG;
  if (!gpu_accessible(correction) || !gpu_accessible(status)) return LSD_ERR_INVALID_ARG;
  const int64_t rid = sv->next_id++;
  bool formed = false;
  int rc;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    rc = submit_round_locked(sv, code, W, stream, block, correction, status, now_ns(), rid,
                             first_round, rounds, &formed);
  }
  if (formed) sv->cv_work.notify_one();
  if (id) *id = rid;
  return rc;
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
  fill_latency(r.latency_ns, out);
  {
    std::vector<const Stats*> all;
    for (const Stats& st : r.by_code) all.push_back(&st);
    fill_parts(all, out);
  }
  if (reset) {
    const size_t nc = r.by_code.size();
    r = Report{};
    r.by_code.resize(nc);
  }
  return sv->error;
}

int lsd_server_get_code_report(lsd_server* sv, int32_t code, lsd_server_report* out) {
  if (!sv || !out || code < 0 || code >= (int32_t)sv->rep.by_code.size())
    return LSD_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(sv->mu);
  const Stats& s = sv->rep.by_code[code];
  std::memset(out, 0, sizeof(*out));
  out->submitted = s.submitted;
  out->completed = s.completed;
  const Report& r = sv->rep;
  out->seconds = r.completed ? (double)(r.last_completion - r.first_arrival) * 1e-9 : 0.0;
  out->shots_per_s = out->seconds > 0 ? (double)s.completed / out->seconds : 0.0;
  fill_latency(s.latency_ns, out);
  fill_parts({&s}, out);
  {
    std::vector<int64_t> g = s.batch_gpu_ns;
    out->p99_batch_gpu_us = (double)percentile(g, 0.99) * 1e-3;
    std::vector<int64_t> lc = s.launch_call_ns;
    out->p99_launch_call_us = (double)percentile(lc, 0.99) * 1e-3;
    out->batches = s.batches;
    out->mean_batch = s.batches ? (double)s.batched / (double)s.batches : 0.0;
  }
  return sv->error;
}

int lsd_server_run_poisson(lsd_server* sv, double rate, double seconds, const double* mix,
                           const uint8_t* const* pools, const int64_t* pool_sizes, uint64_t seed,
                           lsd_server_report* out) {
  if (!sv || !(rate > 0) || !(seconds > 0) || !mix || !pools || !pool_sizes || !out)
    return LSD_ERR_INVALID_ARG;
  const int nc = sv->n_shot + (int)sv->wins.size();
  std::vector<double> cdf(nc);
  double acc = 0;
  for (int c = 0; c < nc; ++c) {
    if (mix[c] < 0 || (mix[c] > 0 && (!pools[c] || pool_sizes[c] < 1))) return LSD_ERR_INVALID_ARG;
    acc += mix[c];
    cdf[c] = acc;
  }
  if (!(acc > 0)) return LSD_ERR_INVALID_ARG;
  for (int c = 0; c < sv->n_shot; ++c)
    if (mix[c] > 0 && !gpu_accessible(pools[c])) return LSD_ERR_INVALID_ARG;
  lsd_server_report dummy;
  lsd_server_get_report(sv, &dummy, 1);
  std::mt19937_64 rng(seed);
  std::exponential_distribution<double> gap(rate);
  std::uniform_real_distribution<double> uni(0.0, acc);
  std::vector<int64_t> cursor(nc, 0);
  // window codes: arrivals go to the streams in turn; stream s plays the pool's sequences
  // s, s + S, s + 2S, ... block by block, continuing from the stream's place in the server
  // (its sequence count and next block), so that successive runs extend the same sequences
  std::vector<Request> burst;
  burst.reserve(4096);
  const int64_t t0 = now_ns();
  const int64_t t_end = t0 + (int64_t)(seconds * 1e9);
  double t_next = (double)t0 + gap(rng) * 1e9;
  int64_t generated = 0, refused = 0;
  // every request whose scheduled arrival has passed is enqueued at once, stamped with its
  // scheduled arrival time (the model's arrival), so the generator keeps up at high rates
  while ((int64_t)t_next < t_end) {
    const int64_t now = now_ns();
    bool woke = false;
    {
      std::unique_lock<std::mutex> lk(sv->mu, std::defer_lock);
      int blocks_held = 0;  // window blocks submitted under this hold of the mutex
      while ((int64_t)t_next <= now && (int64_t)t_next < t_end && burst.size() < 4096 &&
             blocks_held < 256) {
        const double u = uni(rng);
        int c = 0;
        while (c < nc - 1 && u >= cdf[c]) ++c;
        if (c < sv->n_shot) {
          const uint8_t* syn = pools[c] + (size_t)(cursor[c] % pool_sizes[c]) * sv->codes[c].m;
          cursor[c]++;
          burst.push_back(Request{c, syn, nullptr, nullptr, (int64_t)t_next, sv->next_id++});
        } else {
          const int k = c - sv->n_shot;
          WindowCode& W = sv->wins[k];
          const int s = (int)(cursor[c]++ % (int64_t)W.streams.size());
          bool formed = false;
          if (!lk.owns_lock()) lk.lock();
          ++blocks_held;
          const Stream& S = W.streams[s];
          const size_t row = (size_t)(((int64_t)s + (int64_t)S.seq * (int64_t)W.streams.size()) %
                                      pool_sizes[c]);
          const uint8_t* blk = pools[c] + (row * (W.d + 1) + (size_t)S.next_block) * W.m;
          const int rc = submit_round_locked(sv, c, W, s, blk, nullptr, nullptr,
                                             (int64_t)t_next, sv->next_id++, nullptr, nullptr,
                                             &formed);
          if (rc == LSD_OK) {
            ++generated;
            woke = woke || formed;
          } else {
            ++refused;  // the stream's history is still needed: this block is dropped
          }
        }
        t_next += gap(rng) * 1e9;
      }
    }
    if (woke) sv->cv_work.notify_one();
    generated += (int64_t)burst.size();
    enqueue(sv, burst.data(), burst.size());
    burst.clear();
  }
  const int rc = lsd_server_wait_all(sv);
  lsd_server_get_report(sv, out, 0);
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    out->admission_waits += refused;
  }
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
