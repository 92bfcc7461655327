// Internal declarations shared by the kernels and the host API of liblsd.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>
#include <vector>

#include "../../include/lsd.h"

namespace lsdgb {

// Device copy of the Tanner graph of H.
//   Edges are numbered in check-major order: edge e = (chk_ptr[i] + k) is the k-th
//   one of row i, columns ascending.  var_edge lists, for each column j, its edges in
//   ascending row order; var_chk the matching rows.
struct DevGraph {
  int32_t m, n, E;
  int32_t max_row_deg, max_col_deg;
  int32_t min_row_deg, min_col_deg;
  const int32_t* chk_ptr;   // [m+1]
  const uint16_t* chk_var;  // [E]  column of edge e
  const int32_t* var_ptr;   // [n+1]
  const uint16_t* var_edge; // [E]  edges of column j (ascending row)
  const uint16_t* var_chk;  // [E]  rows of column j (ascending)
  const float* prior;       // [n]  lambda_j (float32)
  const long long* wfix;    // [n]  2^-32 fixed point of lambda_j, LSD-mu costs
};

// Counters accumulated by the kernels of one call (reset per call).
struct DevCounters {
  unsigned long long next_shot;     // BP work queue head
  unsigned long long lsd_count;     // unconverged shots appended by BP
  unsigned long long lsd_next;      // LSD work queue head
  unsigned long long bp_converged;
  unsigned long long bp_iterations;
  unsigned long long unsolvable;
  unsigned long long lsd_steps;
  int kappa_max;
  int nu_max;
  int timeout_flag;
  int pad;
  unsigned long long spill_count;   // shots the small sparse LSD instance handed on
};

struct BPArgs {
  DevGraph g;
  long long shots;
  const long long* shots_dev; // if set, the shot count is read from here at kernel start
  const uint8_t* syndromes;  // [shots][m] bytes, or packed: [shots][ceil(m/32)] words
  int packed;                // 1: syndromes and corrections bit-packed (see syn_bit)
  int iters;
  float alpha;
  int method;                // 0 min-sum, 1 sum-product
  int early_exit;
  // decode mode outputs
  uint8_t* corrections;      // [shots][n] nullable (written for converged shots)
  uint8_t* status;           // [shots] nullable
  float* posteriors;         // [shots][n] nullable
  uint8_t* converged_out;    // [shots] nullable
  int32_t* iters_out;        // [shots] nullable
  int32_t* queue;            // [shots] unconverged shot ids, nullable (BP-only mode)
  float* queue_llr;          // [shots][n] LLRs of queued shots (row = queue slot)
  DevCounters* ctr;
};

struct LSDArgs {
  DevGraph g;
  long long count;            // number of work items when count_from_ctr == 0
  int count_from_ctr;         // 1: work items = ctr->lsd_count (appended by BP)
  const int32_t* queue;       // work item -> shot id; NULL = identity
  const float* llr;           // [items or shots][n]
  int llr_by_item;            // 1: LLR row = work item, 0: LLR row = shot id
  const uint8_t* syndromes;   // [shots][m] bytes, or packed: [shots][ceil(m/32)] words
  uint8_t* corrections;       // [shots][n] bytes, or packed: [shots][ceil(n/32)] words
  int packed;
  uint8_t* status;            // [shots] nullable
  int32_t* shot_info;         // [shots][3] nullable
  int order;                  // LSD-mu: extra growth steps per cluster
  int osd_cs;                 // LSD-mu reprocessing: -1 = OSD-E of order `order`, w >= 0 = OSD-CS-w
  int single_cluster;
  DevCounters* ctr;
};

// Launch helpers (return a cudaError_t).
cudaError_t launch_priors(const float* probs, float* prior, long long* wfix, int n,
                          cudaStream_t st);
// BP launch variants: `variant` in/out (-1 = choose); kind 0 auto, 1 generic, 2 register.
cudaError_t launch_bp(const BPArgs& a, int variant, int grid, int block, size_t smem,
                      cudaStream_t st);
cudaError_t bp_config(const DevGraph& g, int lanes, int method, int kind, int* variant,
                      int* grid, int* block, size_t* smem);
int bp_num_variants();
const char* bp_variant_name(int variant);  // nullptr for an unknown id
cudaError_t launch_lsd(const LSDArgs& a, int warps, int grid, size_t smem, cudaStream_t st);
cudaError_t lsd_config(const DevGraph& g, int order, int warps, int* warps_out, int* grid,
                       size_t* smem, int* words);

// Lets `fn` use all the shared memory a block may opt into (the dynamic limit is a property
// of the function, shared by every decoder; it excludes the function's static allocation).
// Records the CUDA error behind an LSD_ERR_CUDA / LSD_ERR_OOM return for lsd_last_error()
// (per host thread).
void record_cuda_error(cudaError_t e);

inline cudaError_t allow_max_dynamic_smem(const void* fn, int max_smem) {
  cudaFuncAttributes at{};
  cudaError_t e = cudaFuncGetAttributes(&at, fn);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              max_smem - (int)at.sharedSizeBytes);
}

// Learned prior (prior.cu).
int prior_num_params();
size_t prior_smem(int m, int n, int E, bool train);
size_t prior_scratch_floats(int m, int n, int rounds, int grid);
cudaError_t prior_config(int m, int n, int E, bool train, int* grid);
cudaError_t launch_prior(bool train, int grid, const DevGraph& g, int rounds, const float* params,
                         long long shots, const uint8_t* syndromes, const uint8_t* errors,
                         float* llr_out, float* scratch, float* grads, double* loss,
                         cudaStream_t st);
cudaError_t launch_adam(float* p, const float* g, float* m, float* v, int count, float lr,
                        int step, cudaStream_t st);
cudaError_t launch_sample(const DevGraph& g, const float* probs, unsigned long long seed,
                          long long first, long long shots, uint8_t* errors, uint8_t* syndromes,
                          cudaStream_t st);
// Inference of the learned prior: LLRs into llr_out, or (llr_out null) decode mode, where the
// kernel takes the hard decision itself and queues the shots it does not solve for LSD.
cudaError_t launch_prior_decode(int grid, const DevGraph& g, int rounds, const float* params,
                                long long shots, const uint8_t* syndromes, float* llr_out,
                                uint8_t* corrections, uint8_t* status, int32_t* queue,
                                float* queue_llr, DevCounters* ctr, cudaStream_t st);
constexpr int kPriorMaxRounds = 8;
// Inference of the learned prior on tcgen05 tensor cores with TMEM-resident projections
// (prior_tc.cu): graphs of at most 8 tiles of 128 node rows; same outputs as
// launch_prior_decode; a completion wait that runs out sets *timeout_flag (nullable).
cudaError_t prior_tc_config(const DevGraph& g, int* grid);
cudaError_t launch_prior_tc(int grid, const DevGraph& g, int rounds, const float* params,
                            long long shots, const uint8_t* syndromes, float* llr_out,
                            uint8_t* corrections, uint8_t* status, int32_t* queue,
                            float* queue_llr, DevCounters* ctr, int* timeout_flag,
                            cudaStream_t st);

// Decode whose shot count is read from device-visible memory at run time, so that one
// captured CUDA graph serves every batch size up to max_shots (api.cu; used by the server).
int decode_batch_counted(lsd_decoder* dec, int64_t max_shots, const long long* shots_dev,
                         const uint8_t* syndromes, uint8_t* corrections, uint8_t* status);
// Its two halves, so that work can be enqueued between them: BP (statuses of the shots BP
// solves become LSD_SHOT_OK_BP, the others are queued), then LSD on the queued shots.
int bp_batch_counted(lsd_decoder* dec, int64_t max_shots, const long long* shots_dev,
                     const uint8_t* syndromes, uint8_t* corrections, uint8_t* status);
int lsd_batch_counted(lsd_decoder* dec, int64_t max_shots, const uint8_t* syndromes,
                      uint8_t* corrections, uint8_t* status);

// Bit-packed batch I/O: element i of a row of k elements is bit (i & 31) of 32-bit word
// i >> 5 of a row of ceil(k/32) words.
__device__ __forceinline__ int packed_words(int k) { return (k + 31) >> 5; }
// Syndrome bit i of `shot` (bytes or packed words).
__device__ __forceinline__ unsigned syn_bit(const uint8_t* syn, int packed, long long shot,
                                            int m, int i) {
  if (packed) {
    const uint32_t* w = reinterpret_cast<const uint32_t*>(syn) + shot * packed_words(m);
    return (w[i >> 5] >> (i & 31)) & 1u;
  }
  return syn[shot * m + i] ? 1u : 0u;
}
// Hard decision [L_j < 0] of n posteriors (shared memory) into word `w` of a packed row.
__device__ __forceinline__ uint32_t sign_word(const float* L, int n, int w) {
  uint32_t x = 0;
  const int j0 = w << 5, j1 = j0 + 32 < n ? j0 + 32 : n;
  for (int j = j0; j < j1; ++j) x |= (L[j] < 0.f ? 1u : 0u) << (j - j0);
  return x;
}
// The hard decision of a converged shot as packed words, `nt` threads from `t` (out of line:
// the byte path of the BP kernels keeps its own register allocation).
static __device__ __noinline__ void write_packed_decision(uint8_t* corrections, long long shot, int n,
                                                   const float* Lam, int t, int nt) {
  uint32_t* co = reinterpret_cast<uint32_t*>(corrections) + shot * packed_words(n);
  for (int w = t; w < packed_words(n); w += nt) co[w] = sign_word(Lam, n, w);
}
// G flags of a group of G lanes (G = 8, 16 or 32, aligned within its warp, every lane of the
// group present) as the low G bits of one word, lane 0's flag in bit 0.
template <int G>
__device__ __forceinline__ uint32_t group_bits(bool b, unsigned gmask) {
  const unsigned x = __ballot_sync(gmask, b);
  if constexpr (G == 32) {
    return x;
  } else {
    return (x >> ((threadIdx.x & 31) & ~(G - 1))) & ((1u << G) - 1u);
  }
}
// The hard decision [Lam_j < 0] of a converged shot as packed words, written by a group of G
// lanes in which lane `lane` owns the variables lane + G v (v < VPL, G VPL >= n): one ballot
// per G variables, lane 0 stores each finished word.
template <int G, int VPL>
__device__ __forceinline__ void group_packed_decision(uint8_t* corrections, long long shot, int n,
                                                      const float* Lam, int lane, unsigned gmask) {
  uint32_t* co = reinterpret_cast<uint32_t*>(corrections) + shot * packed_words(n);
  uint32_t word = 0;
#pragma unroll
  for (int v = 0; v < VPL; ++v) {
    const int j = lane + G * v;
    word |= group_bits<G>(j < n && Lam[j] < 0.f, gmask) << ((G * v) & 31);
    if (((G * (v + 1)) & 31) == 0 || v == VPL - 1) {
      if (lane == 0 && ((G * v) & ~31) < n) co[(G * v) >> 5] = word;
      word = 0;
    }
  }
}
// The same for a CTA of NT threads (whole warps) in which thread `tid` owns the variables
// tid + NT v: the 32 variables of a warp's ballot are exactly one word.
template <int NT, int VPL>
__device__ __forceinline__ void cta_packed_decision(uint8_t* corrections, long long shot, int n,
                                                    const float* Lam, int tid) {
  static_assert(NT % 32 == 0, "whole warps");
  uint32_t* co = reinterpret_cast<uint32_t*>(corrections) + shot * packed_words(n);
#pragma unroll
  for (int v = 0; v < VPL; ++v) {
    const int j = tid + NT * v;
    const unsigned b = __ballot_sync(0xffffffffu, j < n && Lam[j] < 0.f);
    if ((tid & 31) == 0 && j < n) co[j >> 5] = b;
  }
}
// The hard decision of a converged shot: bytes or packed words, `nt` threads from `t`.
__device__ __forceinline__ void write_hard_decision(uint8_t* corrections, int packed,
                                                    long long shot, int n, const float* Lam,
                                                    int t, int nt) {
  if (packed) {
    write_packed_decision(corrections, shot, n, Lam, t, nt);
  } else {
    uint8_t* co = corrections + shot * n;
    for (int j = t; j < n; j += nt) co[j] = (Lam[j] < 0.f) ? 1 : 0;
  }
}

// Decoder of one window of phenomenological rounds of H (window.cu; used by the server):
// detector blocks 0..blocks-1 by fault rounds 0..rounds-1, [n data | m measurement] faults
// per round with probabilities p (n) and q (m); h holds the (row, column) pairs of H.
int window_decoder(lsd_decoder** out, int m, int n, const std::vector<std::pair<int, int>>& h,
                   const float* p, const float* q, int rounds, int blocks, int bp_iters,
                   int order, const lsd_options* opt);
// First round of the final window of d rounds in (w, c) windows.
int window_final_round(int d, int w, int c);

// LSD for large matrices (lsd_sparse.cu).
size_t sparse_scratch_ints(int m, int n, bool big, bool mu);
cudaError_t sparse_config(const DevGraph& g, int order, int* grid_small, int* grid_big);
int sparse_warps_small();
cudaError_t launch_sparse(const LSDArgs& a, bool big, int grid, int* scratch, size_t stride,
                          int* spill, unsigned long long* spill_count, const int* items,
                          const unsigned long long* item_count, cudaStream_t st);

// Limits of this build's kernels.
constexpr int kMaxLsdWords = 16;    // LSD: m <= 32 * kMaxLsdWords detectors per shot
constexpr int kMaxRowDeg = 32;      // BP: check degree (sign bits in one word)
constexpr int kMaxOrder = 12;       // LSD-mu order with OSD-E (2^mu patterns per cluster)
constexpr int kMaxCsGrowth = 65535; // LSD-mu growth steps with OSD-CS
constexpr int kMaxCsOrder = 8;      // w of OSD-CS-w

}  // namespace lsdgb
