// (w, c) overlapping-window decoding of repeated syndrome rounds (Methods 4.3) on top of the
// batch decoder: the host walks the windows; every window is one lsd_decode_batch over all
// shots on the window's matrix, followed by one kernel that commits the window's first c
// rounds into the shots' corrections and gathers the next window's syndromes.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <new>
#include <utility>
#include <vector>

#include "lsd_internal.cuh"

using namespace lsdgb;

struct lsd_window {
  int m = 0, n = 0, d = 0, w = 0, c = 0;
  int t_final = 0;  // first round of the final window
  lsd_decoder* inner = nullptr;
  lsd_decoder* fin = nullptr;
  cudaStream_t st = nullptr;
  int sms = 0;
  // workspace: window syndromes [cap][bmax m] (bmax = w, or w + 1 when c = w and the final
  // window also holds the noiseless block), window corrections [cap][w (n+m)], status [cap]
  int bmax = 0;
  uint8_t* ws = nullptr;
  uint8_t* wc = nullptr;
  uint8_t* wst = nullptr;
  size_t cap = 0;
  int64_t launches = 0;
  // streaming state: syndrome history [scap][(d+1) m] of `sshots` streams, blocks received,
  // the next window's first round, and the last decoded window (rounds, committed rounds)
  uint8_t* hist = nullptr;
  size_t scap = 0;
  int64_t sshots = -1;
  int received = 0, t_next = 0, prev_t = -1, prev_wr = 0, prev_commit = 0;
};

namespace {

int wfail(cudaError_t e) {
  record_cuda_error(e);
  return e == cudaErrorMemoryAllocation ? LSD_ERR_OOM : LSD_ERR_CUDA;
}

// One window transition, one warp per shot (rows are tens of words: a warp covers one in a
// couple of coalesced passes).  Sizes in units of T (bytes, or 4-byte words when every row
// and block size is a multiple of 4):
//   F = n + m (one fault round), M = m (one detector block), N = n.
// Commit (t >= 0 and do_commit): rounds 0..commit-1 of the decoded window (row wc_row) ->
// rounds t..t+commit-1 of the correction (row c_row); status = max over windows.  Gather
// (t_next >= 0): blocks t_next..t_next+bn-1 of the syndrome (row s_row) -> the next window's
// syndrome; when t >= 0 its first block also takes the measurement faults of round
// commit-1 of the window at t (the last committed round).
template <class T>
__global__ void __launch_bounds__(256) window_step_kernel(
    long long shots, int F, int M, int N, int s_row, int c_row, const T* __restrict__ syn,
    const T* __restrict__ wc, int wc_row, const uint8_t* __restrict__ wst, int t, int commit,
    int do_commit, T* __restrict__ out, uint8_t* __restrict__ status, int t_next, int bn,
    T* __restrict__ ws) {
  const int lane = threadIdx.x & 31;
  const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long k = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); k < shots;
       k += warps) {
    const T* wrow = wc + k * wc_row;
    if (t >= 0 && do_commit) {
      T* orow = out + k * c_row + (long long)t * F;
      for (int j = lane; j < commit * F; j += 32) orow[j] = wrow[j];
      if (lane == 0 && status) {
        const uint8_t now = wst[k];
        status[k] = (t == 0 || now > status[k]) ? now : status[k];
      }
    }
    if (t_next >= 0) {
      const T* srow = syn + k * s_row + (long long)t_next * M;
      T* dst = ws + k * (long long)bn * M;
      const T* meas = t >= 0 ? wrow + (long long)(commit - 1) * F + N : nullptr;
      for (int j = lane; j < bn * M; j += 32) {
        T v = srow[j];
        if (meas && j < M) v ^= meas[j];
        dst[j] = v;
      }
    }
  }
}

// Streaming: detector block b of every stream ([shots][m]) into the history [shots][(d+1) m].
__global__ void __launch_bounds__(256) block_store_kernel(long long shots, int m, int s_row, int b,
                                                         const uint8_t* __restrict__ block,
                                                         uint8_t* __restrict__ hist) {
  const long long total = shots * m;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long k = i / m;
    hist[k * s_row + (long long)b * m + (i - k * m)] = block[i];
  }
}

int ensure(lsd_window* W, int64_t shots) {
  if ((size_t)shots <= W->cap) return LSD_OK;
  cudaError_t e = cudaStreamSynchronize(W->st);
  if (e != cudaSuccess) return wfail(e);
  cudaFree(W->ws);
  cudaFree(W->wc);
  cudaFree(W->wst);
  W->ws = W->wc = W->wst = nullptr;
  W->cap = 0;
  const size_t S = (size_t)shots;
  e = cudaMalloc(&W->ws, S * W->bmax * W->m);
  if (e == cudaSuccess) e = cudaMalloc(&W->wc, S * W->w * (W->n + W->m));
  if (e == cudaSuccess) e = cudaMalloc(&W->wst, S);
  if (e != cudaSuccess) {
    cudaFree(W->ws);
    cudaFree(W->wc);
    cudaFree(W->wst);
    W->ws = W->wc = W->wst = nullptr;
    return wfail(e);
  }
  W->cap = S;
  return LSD_OK;
}

int launch_step(lsd_window* W, int64_t shots, const uint8_t* syn, int wr, int t, int commit,
                bool do_commit, uint8_t* out, uint8_t* status, int t_next, int bn) {
  const int m = W->m, n = W->n, F = n + m, d = W->d;
  const bool words = m % 4 == 0 && n % 4 == 0 && ((uintptr_t)syn & 3) == 0 &&
                     ((uintptr_t)out & 3) == 0;
  const long long blocks = std::min<long long>((shots + 7) / 8, (long long)W->sms * 16);
  const int grid = (int)std::max<long long>(blocks, 1);
  if (words) {
    window_step_kernel<uint32_t><<<grid, 256, 0, W->st>>>(
        shots, F / 4, m / 4, n / 4, (d + 1) * m / 4, d * F / 4,
        reinterpret_cast<const uint32_t*>(syn), reinterpret_cast<const uint32_t*>(W->wc),
        wr * F / 4, W->wst, t, commit, do_commit ? 1 : 0, reinterpret_cast<uint32_t*>(out),
        status, t_next, bn, reinterpret_cast<uint32_t*>(W->ws));
  } else {
    window_step_kernel<uint8_t><<<grid, 256, 0, W->st>>>(
        shots, F, m, n, (d + 1) * m, d * F, syn, W->wc, wr * F, W->wst, t, commit,
        do_commit ? 1 : 0, out, status, t_next, bn, W->ws);
  }
  W->launches++;
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LSD_OK : wfail(e);
}

}  // namespace

namespace lsdgb {

// COO of a window: detector blocks 0..blocks-1, fault rounds 0..rounds-1.
static void window_coo(int m, int n, const std::vector<std::pair<int, int>>& h, int rounds,
                       int blocks, std::vector<int32_t>& rows, std::vector<int32_t>& cols) {
  rows.clear();
  cols.clear();
  const int F = n + m;
  for (int r = 0; r < rounds; ++r) {
    for (const auto& e : h) {
      rows.push_back(r * m + e.first);
      cols.push_back(r * F + e.second);
    }
    for (int i = 0; i < m; ++i) {
      rows.push_back(r * m + i);
      cols.push_back(r * F + n + i);
      if (r + 1 < blocks) {
        rows.push_back((r + 1) * m + i);
        cols.push_back(r * F + n + i);
      }
    }
  }
}

int window_decoder(lsd_decoder** out, int m, int n, const std::vector<std::pair<int, int>>& h,
                   const float* p, const float* q, int rounds, int blocks, int bp_iters,
                   int order, const lsd_options* opt) {
  std::vector<int32_t> rows, cols;
  window_coo(m, n, h, rounds, blocks, rows, cols);
  std::vector<float> probs;
  probs.reserve((size_t)rounds * (n + m));
  for (int r = 0; r < rounds; ++r) {
    probs.insert(probs.end(), p, p + n);
    probs.insert(probs.end(), q, q + m);
  }
  return lsd_create(out, blocks * m, rounds * (n + m), (int64_t)rows.size(), rows.data(),
                    cols.data(), probs.data(), bp_iters, order, opt);
}

int window_final_round(int d, int w, int c) {
  int t = 0;
  while (t + w - 1 < d && t + c < d) t += c;
  return t;
}

}  // namespace lsdgb

extern "C" {

int lsd_window_create(lsd_window** out, int32_t m, int32_t n, int64_t nnz, const int32_t* rows,
                      const int32_t* cols, const float* p_data, const float* q_meas,
                      int32_t rounds, int32_t window, int32_t commit, int32_t bp_iters,
                      int32_t lsd_order, const lsd_options* opt) {
  if (!out) return LSD_ERR_INVALID_ARG;
  *out = nullptr;
  if (m < 1 || n < 1 || nnz < 0 || (nnz > 0 && (!rows || !cols)) || !p_data || !q_meas ||
      rounds < 1 || window < 1 || commit < 1 || commit > window)
    return LSD_ERR_INVALID_ARG;
  std::vector<std::pair<int, int>> h((size_t)nnz);
  for (int64_t k = 0; k < nnz; ++k) {
    if (rows[k] < 0 || rows[k] >= m || cols[k] < 0 || cols[k] >= n) return LSD_ERR_INVALID_ARG;
    h[(size_t)k] = {rows[k], cols[k]};
  }
  lsd_window* W = new (std::nothrow) lsd_window();
  if (!W) return LSD_ERR_OOM;
  W->m = m;
  W->n = n;
  W->d = rounds;
  W->w = window;
  W->c = commit;
  W->st = opt ? static_cast<cudaStream_t>(opt->stream) : nullptr;
  const int t = window_final_round(rounds, window, commit);
  W->t_final = t;
  W->bmax = std::max(window, rounds - t + 1);
  int rc = LSD_OK;
  if (t > 0)
    rc = window_decoder(&W->inner, m, n, h, p_data, q_meas, window, window, bp_iters, lsd_order,
                      opt);
  if (rc == LSD_OK)
    rc = window_decoder(&W->fin, m, n, h, p_data, q_meas, rounds - t, rounds - t + 1, bp_iters,
                      lsd_order, opt);
  if (rc == LSD_OK) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&W->sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) rc = wfail(e);
  }
  if (rc != LSD_OK) {
    lsd_window_destroy(W);
    return rc;
  }
  *out = W;
  return LSD_OK;
}

int lsd_window_decode(lsd_window* W, int64_t shots, const uint8_t* syndromes,
                      uint8_t* corrections, uint8_t* status, lsd_stats* stats) {
  if (!W || shots < 0 || shots > INT32_MAX) return LSD_ERR_INVALID_ARG;
  if (stats) std::memset(stats, 0, sizeof(*stats));
  if (shots == 0) return LSD_OK;
  if (!syndromes || !corrections) return LSD_ERR_INVALID_ARG;
  int rc = ensure(W, shots);
  if (rc) return rc;
  const int d = W->d, w = W->w, c = W->c;
  auto blocks_of = [&](int t) { return t == W->t_final ? d - t + 1 : w; };
  // the first window's syndromes
  rc = launch_step(W, shots, syndromes, 0, -1, 0, false, corrections, status, 0, blocks_of(0));
  if (rc) return rc;
  for (int t = 0;; t += c) {
    const bool final = t == W->t_final;
    lsd_stats one{};
    rc = lsd_decode_batch(final ? W->fin : W->inner, shots, W->ws, W->wc, W->wst, nullptr,
                          stats ? &one : nullptr);
    if (rc) return rc;
    if (stats) {
      stats->shots += one.shots;
      stats->bp_converged += one.bp_converged;
      stats->lsd_shots += one.lsd_shots;
      stats->unsolvable += one.unsolvable;
      stats->bp_iterations += one.bp_iterations;
      stats->lsd_steps += one.lsd_steps;
      stats->kappa_max = std::max(stats->kappa_max, one.kappa_max);
      stats->nu_max = std::max(stats->nu_max, one.nu_max);
      stats->ms_bp += one.ms_bp;
      stats->ms_lsd += one.ms_lsd;
      stats->lsd_spilled += one.lsd_spilled;
    }
    const int wr = final ? d - t : w;
    const int commit = final ? d - t : c;
    const int t_next = final ? -1 : t + c;
    rc = launch_step(W, shots, syndromes, wr, t, commit, true, corrections, status, t_next,
                     final ? 0 : blocks_of(t_next));
    if (rc) return rc;
    if (final) break;
  }
  if (stats) {
    cudaError_t e = cudaStreamSynchronize(W->st);
    if (e != cudaSuccess) return wfail(e);
  }
  return LSD_OK;
}

int lsd_window_stream_reset(lsd_window* W, int64_t shots) {
  if (!W || shots < 1 || shots > INT32_MAX) return LSD_ERR_INVALID_ARG;
  int rc = ensure(W, shots);
  if (rc) return rc;
  const size_t need = (size_t)shots * (W->d + 1) * W->m;
  if (need > W->scap) {
    cudaError_t e = cudaStreamSynchronize(W->st);
    if (e != cudaSuccess) return wfail(e);
    cudaFree(W->hist);
    W->hist = nullptr;
    W->scap = 0;
    e = cudaMalloc(&W->hist, need);
    if (e != cudaSuccess) return wfail(e);
    W->scap = need;
  }
  W->sshots = shots;
  W->received = 0;
  W->t_next = 0;
  W->prev_t = -1;
  W->prev_wr = W->prev_commit = 0;
  return LSD_OK;
}

int lsd_window_stream_push(lsd_window* W, const uint8_t* block, uint8_t* corrections,
                           uint8_t* status, int32_t* first_round, int32_t* rounds_committed) {
  if (!W || !block || !corrections || W->sshots < 1 || W->received > W->d)
    return LSD_ERR_INVALID_ARG;
  if (first_round) *first_round = 0;
  if (rounds_committed) *rounds_committed = 0;
  const int64_t shots = W->sshots;
  const int d = W->d, m = W->m;
  {
    const long long total = (long long)shots * m;
    const int grid = (int)std::max<long long>(
        1, std::min<long long>((total + 255) / 256, (long long)W->sms * 8));
    block_store_kernel<<<grid, 256, 0, W->st>>>(shots, m, (d + 1) * m, W->received, block,
                                                 W->hist);
    W->launches++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return wfail(e);
  }
  const int last = W->received++;
  const int t = W->t_next;
  if (t > d) return LSD_OK;  // every round already committed
  const bool final = t == W->t_final;
  const int need = final ? d : t + W->w - 1;
  if (last < need) return LSD_OK;
  const int blocks = final ? d - t + 1 : W->w;
  // gather the window (its first block takes the last committed round's measurement faults)
  int rc = launch_step(W, shots, W->hist, W->prev_wr, W->prev_t, W->prev_commit, false,
                       corrections, status, t, blocks);
  if (rc) return rc;
  rc = lsd_decode_batch(final ? W->fin : W->inner, shots, W->ws, W->wc, W->wst, nullptr,
                        nullptr);
  if (rc) return rc;
  const int wr = final ? d - t : W->w;
  const int commit = final ? d - t : W->c;
  rc = launch_step(W, shots, W->hist, wr, t, commit, true, corrections, status, -1, 0);
  if (rc) return rc;
  W->prev_t = t;
  W->prev_wr = wr;
  W->prev_commit = commit;
  W->t_next = final ? d + 1 : t + W->c;
  if (first_round) *first_round = t;
  if (rounds_committed) *rounds_committed = commit;
  return LSD_OK;
}

int lsd_window_kernel_launches(const lsd_window* W, int64_t* count) {
  if (!W || !count) return LSD_ERR_INVALID_ARG;
  int64_t a = 0, b = 0;
  if (W->inner) lsd_kernel_launches(W->inner, &a);
  if (W->fin) lsd_kernel_launches(W->fin, &b);
  *count = W->launches + a + b;
  return LSD_OK;
}

int lsd_window_destroy(lsd_window* W) {
  if (!W) return LSD_OK;
  if (W->st || W->cap || W->scap) cudaStreamSynchronize(W->st);
  cudaFree(W->ws);
  cudaFree(W->wc);
  cudaFree(W->wst);
  cudaFree(W->hist);
  lsd_destroy(W->inner);
  lsd_destroy(W->fin);
  delete W;
  return LSD_OK;
}

}  // extern "C"
