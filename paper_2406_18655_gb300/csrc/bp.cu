// Priors and belief propagation kernels.
//
// Priors (Sec. 4.1, LLR form): lambda_j = ln((1 - p_j) / p_j), evaluated in double and
// rounded to float32.  BP (Sec. 4.3): min-sum with scaling alpha on the whole check
// message, flooding ("parallel") schedule, a shot stops as soon as its hard decision
// [Lambda < 0] satisfies H e = s (App. C.4), otherwise after `iters` iterations.
//
// Layout.  A group of G lanes (G = 8, 16 or 32) owns one shot at a time; the grid is
// persistent and groups pull shots from a global counter, so early-exiting shots free
// their lanes at once.  The shot's whole message state lives in shared memory:
//   r[E]    check -> variable messages, edges in check-major order,
//   Lam[n]  posteriors of the last variable update,
// and q = Lam - r is recomputed in the check phase instead of being stored.  The
// Tanner graph (CSR + CSC as uint16 indices) and the priors are staged once per CTA.
// Check phase: lane <- check, running (min1, min2, argmin, sign parity) over its edges.
// Variable phase: lane <- variable, Lam_j = lambda_j + sum of incoming r in ascending
// check order.  The parity test of Lam^(t) is fused into check phase t+1.
// Every float operation on the min-sum path is an explicit round-to-nearest intrinsic
// (no contraction), so results do not depend on compiler fusion.
#include "lsd_internal.cuh"

namespace lsdgb {

namespace {

constexpr float kBig = 0x1p100f;  // minimum over an empty set (a degree-1 check)

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

__host__ __device__ inline size_t bp_graph_bytes(int m, int n, int E) {
  return align16((size_t)(m + 1 + n + 1 + n) * 4 + (size_t)E * 4);
}
__host__ __device__ inline size_t bp_group_bytes(int m, int n, int E) {
  return align16((size_t)E * 4 + (size_t)n * 4 + (size_t)m);
}

__global__ void priors_kernel(const float* __restrict__ probs, float* __restrict__ prior,
                              long long* __restrict__ wfix, int n) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double p = (double)probs[j];
  const float lf = (float)log((1.0 - p) / p);
  prior[j] = lf;
  // LSD-mu costs: the float prior in 2^-32 fixed point (exact for |lambda| >= 2^-9)
  wfix[j] = __double2ll_rn((double)lf * 4294967296.0);
}

template <int G>
__device__ __forceinline__ unsigned group_mask() {
  if constexpr (G == 32) {
    return 0xffffffffu;
  } else {
    return ((1u << G) - 1u) << ((threadIdx.x & 31) & ~(G - 1));
  }
}

// METHOD 0: min-sum; 1: sum-product.
template <int G, int METHOD>
__global__ void __launch_bounds__(256) bp_kernel(BPArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int m = a.g.m, n = a.g.n, E = a.g.E;
  int32_t* s_chk_ptr = reinterpret_cast<int32_t*>(smem);
  int32_t* s_var_ptr = s_chk_ptr + (m + 1);
  float* s_prior = reinterpret_cast<float*>(s_var_ptr + (n + 1));
  uint16_t* s_chk_var = reinterpret_cast<uint16_t*>(s_prior + n);
  uint16_t* s_var_edge = s_chk_var + E;
  for (int i = threadIdx.x; i <= m; i += blockDim.x) s_chk_ptr[i] = a.g.chk_ptr[i];
  for (int j = threadIdx.x; j <= n; j += blockDim.x) s_var_ptr[j] = a.g.var_ptr[j];
  for (int j = threadIdx.x; j < n; j += blockDim.x) s_prior[j] = a.g.prior[j];
  for (int e = threadIdx.x; e < E; e += blockDim.x) {
    s_chk_var[e] = a.g.chk_var[e];
    s_var_edge[e] = a.g.var_edge[e];
  }
  __syncthreads();

  const int lane = threadIdx.x & (G - 1);
  const int group = threadIdx.x / G;
  const unsigned gmask = group_mask<G>();
  const int leader = (threadIdx.x & 31) & ~(G - 1);
  unsigned char* gbase = smem + bp_graph_bytes(m, n, E) + (size_t)group * bp_group_bytes(m, n, E);
  float* r = reinterpret_cast<float*>(gbase);
  float* Lam = r + E;
  uint8_t* syn = reinterpret_cast<uint8_t*>(Lam + n);
  const float alpha = a.alpha;

  unsigned long long my_iters = 0, my_conv = 0;
  for (;;) {
    unsigned long long shot_u = 0;
    if (lane == 0) shot_u = atomicAdd(&a.ctr->next_shot, 1ULL);
    shot_u = __shfl_sync(gmask, shot_u, leader);
    if (shot_u >= (unsigned long long)a.shots) break;
    const long long shot = (long long)shot_u;

    const uint8_t* sp = a.syndromes + shot * m;
    for (int i = lane; i < m; i += G) syn[i] = sp[i] ? 1 : 0;
    for (int e = lane; e < E; e += G) r[e] = 0.f;
    for (int j = lane; j < n; j += G) Lam[j] = s_prior[j];
    __syncwarp(gmask);

    int t = 0;
    bool conv = false;
    for (;;) {
      const bool msgs = t < a.iters;
      unsigned unsat = 0;
      // ---- check phase: parity of [Lam^(t) < 0] and messages r^(t+1) ----
      for (int i = lane; i < m; i += G) {
        const int b = s_chk_ptr[i], e1 = s_chk_ptr[i + 1];
        const unsigned si = syn[i];
        unsigned hp = si;
        if constexpr (METHOD == 0) {
          float min1 = kBig, min2 = kBig;
          int idx = 0;
          unsigned negs = 0, sgn = si;
          for (int e = b; e < e1; ++e) {
            const float L = Lam[s_chk_var[e]];
            hp ^= (L < 0.f) ? 1u : 0u;
            if (msgs) {
              const float q = __fsub_rn(L, r[e]);
              const float aq = fabsf(q);
              const unsigned ng = (q < 0.f) ? 1u : 0u;
              sgn ^= ng;
              negs |= ng << (e - b);
              if (aq < min1) {
                min2 = min1;
                min1 = aq;
                idx = e - b;
              } else if (aq < min2) {
                min2 = aq;
              }
            }
          }
          if (msgs) {
            const float m1 = __fmul_rn(alpha, min1), m2 = __fmul_rn(alpha, min2);
            for (int e = b; e < e1; ++e) {
              const int k = e - b;
              const float mag = (k == idx) ? m2 : m1;
              r[e] = ((sgn ^ (negs >> k)) & 1u) ? -mag : mag;
            }
          }
        } else {
          // sum-product: r = (-1)^s 2 atanh(prod of tanh(q/2) over the other edges)
          float qv[kMaxRowDeg];
          for (int e = b; e < e1; ++e) {
            const float L = Lam[s_chk_var[e]];
            hp ^= (L < 0.f) ? 1u : 0u;
            qv[e - b] = __fsub_rn(L, r[e]);
          }
          if (msgs) {
            for (int e = b; e < e1; ++e) {
              float prod = 1.f;
              for (int e2 = b; e2 < e1; ++e2)
                if (e2 != e) prod = prod * tanhf(0.5f * qv[e2 - b]);
              const float lim = 0.99999994f;
              prod = fminf(fmaxf(prod, -lim), lim);
              const float v = 2.f * atanhf(prod);
              r[e] = si ? -v : v;
            }
          }
        }
        unsat |= hp;
      }
      if (t > 0) {
        conv = !__any_sync(gmask, unsat != 0);
        if (conv && a.early_exit) break;
      }
      if (!msgs) break;
      __syncwarp(gmask);
      // ---- variable phase: Lam^(t+1) ----
      for (int j = lane; j < n; j += G) {
        float L = s_prior[j];
        const int v1 = s_var_ptr[j + 1];
        for (int k = s_var_ptr[j]; k < v1; ++k) L = __fadd_rn(L, r[s_var_edge[k]]);
        Lam[j] = L;
      }
      __syncwarp(gmask);
      ++t;
    }

    // ---- outputs ----
    if (a.posteriors) {
      float* po = a.posteriors + shot * n;
      for (int j = lane; j < n; j += G) po[j] = Lam[j];
    }
    if (lane == 0) {
      if (a.converged_out) a.converged_out[shot] = conv ? 1 : 0;
      if (a.iters_out) a.iters_out[shot] = t;
    }
    my_iters += (lane == 0) ? (unsigned long long)t : 0ull;
    my_conv += (lane == 0 && conv) ? 1ull : 0ull;
    if (a.queue) {
      if (conv) {
        uint8_t* co = a.corrections + shot * n;
        for (int j = lane; j < n; j += G) co[j] = (Lam[j] < 0.f) ? 1 : 0;
        if (lane == 0 && a.status) a.status[shot] = LSD_SHOT_OK_BP;
      } else {
        unsigned long long slot = 0;
        if (lane == 0) slot = atomicAdd(&a.ctr->lsd_count, 1ULL);
        slot = __shfl_sync(gmask, slot, leader);
        if (lane == 0) a.queue[slot] = (int32_t)shot;
        float* lo = a.queue_llr + (long long)slot * n;
        for (int j = lane; j < n; j += G) lo[j] = Lam[j];
      }
    }
    __syncwarp(gmask);
  }
  // one atomic per warp for the batch counters
  for (int off = 16; off > 0; off >>= 1) {
    my_iters += __shfl_down_sync(0xffffffffu, my_iters, off);
    my_conv += __shfl_down_sync(0xffffffffu, my_conv, off);
  }
  if ((threadIdx.x & 31) == 0) {
    if (my_iters) atomicAdd(&a.ctr->bp_iterations, my_iters);
    if (my_conv) atomicAdd(&a.ctr->bp_converged, my_conv);
  }
}

}  // namespace

cudaError_t launch_priors(const float* probs, float* prior, long long* wfix, int n,
                          cudaStream_t st) {
  priors_kernel<<<(n + 255) / 256, 256, 0, st>>>(probs, prior, wfix, n);
  return cudaGetLastError();
}

cudaError_t bp_config(const DevGraph& g, int lanes, int method, int* grid, int* block,
                      size_t* smem) {
  int dev = 0, sms = 0, max_smem = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const size_t gb = bp_graph_bytes(g.m, g.n, g.E), grp = bp_group_bytes(g.m, g.n, g.E);
  int b = 256;
  while (b > lanes && gb + (size_t)(b / lanes) * grp > (size_t)max_smem) b /= 2;
  if (gb + (size_t)(b / lanes) * grp > (size_t)max_smem) return cudaErrorInvalidValue;
  *block = b;
  *smem = gb + (size_t)(b / lanes) * grp;
  int per_sm = 0;
  const void* fns[6] = {(const void*)bp_kernel<8, 0>,  (const void*)bp_kernel<16, 0>,
                        (const void*)bp_kernel<32, 0>, (const void*)bp_kernel<8, 1>,
                        (const void*)bp_kernel<16, 1>, (const void*)bp_kernel<32, 1>};
  // the limit is a property of the function, shared by every decoder: allow the maximum
  for (const void* f : fns) {
    err = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
    if (err != cudaSuccess) return err;
  }
  const void* fn = fns[(lanes == 8 ? 0 : lanes == 16 ? 1 : 2) + (method ? 3 : 0)];
  err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, b, *smem);
  if (err != cudaSuccess) return err;
  if (per_sm < 1) return cudaErrorInvalidValue;
  *grid = per_sm * sms;
  return cudaSuccess;
}

cudaError_t launch_bp(const BPArgs& a, int lanes, int grid, int block, size_t smem,
                      cudaStream_t st) {
  const int sel = (lanes == 8 ? 0 : lanes == 16 ? 1 : 2) + (a.method ? 3 : 0);
  switch (sel) {
    case 0: bp_kernel<8, 0><<<grid, block, smem, st>>>(a); break;
    case 1: bp_kernel<16, 0><<<grid, block, smem, st>>>(a); break;
    case 2: bp_kernel<32, 0><<<grid, block, smem, st>>>(a); break;
    case 3: bp_kernel<8, 1><<<grid, block, smem, st>>>(a); break;
    case 4: bp_kernel<16, 1><<<grid, block, smem, st>>>(a); break;
    default: bp_kernel<32, 1><<<grid, block, smem, st>>>(a); break;
  }
  return cudaGetLastError();
}

}  // namespace lsdgb
