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
#include "bp_shot.cuh"
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
__host__ __device__ inline size_t bp_reg_group_bytes(int n, int E) {
  return align16((size_t)E * 4 + (size_t)n * 4);
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
  const long long shots = a.shots_dev ? *a.shots_dev : a.shots;
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
    if (shot_u >= (unsigned long long)shots) break;
    const long long shot = (long long)shot_u;

    for (int i = lane; i < m; i += G) syn[i] = (uint8_t)syn_bit(a.syndromes, a.packed, shot, m, i);
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
        write_hard_decision(a.corrections, a.packed, shot, n, Lam, lane, G);
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

// Min-sum on a regular Tanner graph (every check of degree DC, every variable of degree
// DV) with the per-lane graph tables in registers.  A group of G lanes owns a shot; lane l
// owns checks l, l+G, ... (at most CPL) and variables l, l+G, ... (at most VPL).  Check i's
// edges are i*DC .. i*DC+DC-1 (CSR order), so only the column indices of the lane's checks
// and the edge slots of its variables are kept, two 16-bit indices per register.  Loops
// are unrolled over the compile-time degrees; r[E], Lam[n] and the priors live in shared
// memory as the exchange between the two phases.  Same operations in the same order as
// bp_kernel<G, 0>, so the results are identical.
template <int G, int CPL, int DC, int VPL, int DV, bool PK>
__global__ void __launch_bounds__(256) bp_reg_kernel(BPArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int m = a.g.m, n = a.g.n, E = a.g.E;
  const long long shots = a.shots_dev ? *a.shots_dev : a.shots;
  const int lane = threadIdx.x & (G - 1);
  const int group = threadIdx.x / G;
  const unsigned gmask = group_mask<G>();
  const int leader = (threadIdx.x & 31) & ~(G - 1);
  float* s_prior = reinterpret_cast<float*>(smem);
  for (int j = threadIdx.x; j < n; j += blockDim.x) s_prior[j] = a.g.prior[j];
  __syncthreads();
  float* r = reinterpret_cast<float*>(smem + align16((size_t)n * 4) +
                                      (size_t)group * bp_reg_group_bytes(n, E));
  float* Lam = r + E;
  bpreg::Tables<CPL, DC, VPL, DV> T;
  bpreg::load_tables<G>(a.g, lane, T);
  (void)m;

  unsigned long long my_iters = 0, my_conv = 0;
  for (;;) {
    unsigned long long shot_u = 0;
    if (lane == 0) shot_u = atomicAdd(&a.ctr->next_shot, 1ULL);
    shot_u = __shfl_sync(gmask, shot_u, leader);
    if (shot_u >= (unsigned long long)shots) break;
    const long long shot = (long long)shot_u;
    bool conv = false;
    const int t = bpreg::shot_bp<G, CPL, DC, VPL, DV, PK>(a, T, shot, r, Lam, s_prior, lane, gmask, conv);

    // ---- outputs (each lane writes its own variables) ----
    if (a.posteriors) {
      float* po = a.posteriors + shot * n;
#pragma unroll
      for (int v = 0; v < VPL; ++v) {
        const int j = lane + G * v;
        if (j < n) po[j] = Lam[j];
      }
    }
    if (lane == 0) {
      if (a.converged_out) a.converged_out[shot] = conv ? 1 : 0;
      if (a.iters_out) a.iters_out[shot] = t;
    }
    my_iters += (lane == 0) ? (unsigned long long)t : 0ull;
    my_conv += (lane == 0 && conv) ? 1ull : 0ull;
    if (a.queue) {
      if (conv) {
        if constexpr (PK) {
          group_packed_decision<G, VPL>(a.corrections, shot, n, Lam, lane, gmask);
        } else {
          uint8_t* co = a.corrections + shot * n;
#pragma unroll
          for (int v = 0; v < VPL; ++v) {
            const int j = lane + G * v;
            if (j < n) co[j] = (Lam[j] < 0.f) ? 1 : 0;
          }
        }
        if (lane == 0 && a.status) a.status[shot] = LSD_SHOT_OK_BP;
      } else {
        unsigned long long slot = 0;
        if (lane == 0) slot = atomicAdd(&a.ctr->lsd_count, 1ULL);
        slot = __shfl_sync(gmask, slot, leader);
        if (lane == 0) a.queue[slot] = (int32_t)shot;
        float* lo = a.queue_llr + (long long)slot * n;
#pragma unroll
        for (int v = 0; v < VPL; ++v) {
          const int j = lane + G * v;
          if (j < n) lo[j] = Lam[j];
        }
      }
    }
    __syncwarp(gmask);
  }
  for (int off = 16; off > 0; off >>= 1) {
    my_iters += __shfl_down_sync(0xffffffffu, my_iters, off);
    my_conv += __shfl_down_sync(0xffffffffu, my_conv, off);
  }
  if ((threadIdx.x & 31) == 0) {
    if (my_iters) atomicAdd(&a.ctr->bp_iterations, my_iters);
    if (my_conv) atomicAdd(&a.ctr->bp_converged, my_conv);
  }
}

// BP for graphs whose state does not fit a warp group: one CTA owns one shot, the Tanner
// graph is read through the read-only cache, and r[E], Lam[n], s[m] live in the CTA's
// shared memory.  Same operations in the same order as bp_kernel.
template <int METHOD>
__global__ void __launch_bounds__(512) bp_cta_kernel(BPArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned long long s_shot;
  __shared__ unsigned long long s_slot;
  const int m = a.g.m, n = a.g.n, E = a.g.E;
  const long long shots = a.shots_dev ? *a.shots_dev : a.shots;
  const int tid = threadIdx.x, nt = blockDim.x;
  float* r = reinterpret_cast<float*>(smem);
  float* Lam = r + E;
  uint8_t* syn = reinterpret_cast<uint8_t*>(Lam + n);
  const int32_t* __restrict__ chk_ptr = a.g.chk_ptr;
  const uint16_t* __restrict__ chk_var = a.g.chk_var;
  const int32_t* __restrict__ var_ptr = a.g.var_ptr;
  const uint16_t* __restrict__ var_edge = a.g.var_edge;
  const float* __restrict__ prior = a.g.prior;
  const float alpha = a.alpha;
  unsigned long long my_iters = 0, my_conv = 0;
  for (;;) {
    if (tid == 0) s_shot = atomicAdd(&a.ctr->next_shot, 1ULL);
    __syncthreads();
    const unsigned long long shot_u = s_shot;
    if (shot_u >= (unsigned long long)shots) break;
    const long long shot = (long long)shot_u;
    for (int i = tid; i < m; i += nt) syn[i] = (uint8_t)syn_bit(a.syndromes, a.packed, shot, m, i);
    for (int e = tid; e < E; e += nt) r[e] = 0.f;
    for (int j = tid; j < n; j += nt) Lam[j] = __ldg(prior + j);
    __syncthreads();
    int t = 0;
    bool conv = false;
    for (;;) {
      const bool msgs = t < a.iters;
      int unsat = 0;
      for (int i = tid; i < m; i += nt) {
        const int b = __ldg(chk_ptr + i), e1 = __ldg(chk_ptr + i + 1);
        const unsigned si = syn[i];
        unsigned hp = si;
        if constexpr (METHOD == 0) {
          float min1 = kBig, min2 = kBig;
          int idx = 0;
          unsigned negs = 0, sgn = si;
          for (int e = b; e < e1; ++e) {
            const float L = Lam[__ldg(chk_var + e)];
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
          float qv[kMaxRowDeg];
          for (int e = b; e < e1; ++e) {
            const float L = Lam[__ldg(chk_var + e)];
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
        unsat |= (int)hp;
      }
      const int any_unsat = __syncthreads_or(unsat);
      if (t > 0) {
        conv = !any_unsat;
        if (conv && a.early_exit) break;
      }
      if (!msgs) break;
      for (int j = tid; j < n; j += nt) {
        float L = __ldg(prior + j);
        const int v1 = __ldg(var_ptr + j + 1);
        for (int k = __ldg(var_ptr + j); k < v1; ++k) L = __fadd_rn(L, r[__ldg(var_edge + k)]);
        Lam[j] = L;
      }
      __syncthreads();
      ++t;
    }
    if (a.posteriors) {
      float* po = a.posteriors + shot * n;
      for (int j = tid; j < n; j += nt) po[j] = Lam[j];
    }
    if (tid == 0) {
      if (a.converged_out) a.converged_out[shot] = conv ? 1 : 0;
      if (a.iters_out) a.iters_out[shot] = t;
      my_iters += (unsigned long long)t;
      my_conv += conv ? 1ull : 0ull;
    }
    if (a.queue) {
      if (conv) {
        write_hard_decision(a.corrections, a.packed, shot, n, Lam, tid, nt);
        if (tid == 0 && a.status) a.status[shot] = LSD_SHOT_OK_BP;
      } else {
        if (tid == 0) {
          s_slot = atomicAdd(&a.ctr->lsd_count, 1ULL);
          a.queue[s_slot] = (int32_t)shot;
        }
        __syncthreads();
        float* lo = a.queue_llr + (long long)s_slot * n;
        for (int j = tid; j < n; j += nt) lo[j] = Lam[j];
      }
    }
    __syncthreads();
  }
  if (tid == 0) {
    if (my_iters) atomicAdd(&a.ctr->bp_iterations, my_iters);
    if (my_conv) atomicAdd(&a.ctr->bp_converged, my_conv);
  }
}

// BP for large graphs with register-resident tables: one CTA of NT threads owns one shot;
// like bp_reg_kernel, thread t keeps the column indices of checks t, t + NT, ... and the
// message slots of variables t, t + NT, ... in registers (two 16-bit indices per register),
// so no graph table is read while iterating.  Messages r live in shared memory row-major
// with DC slots per check (slot i * DC + k for the k-th edge of check i) plus a slot Z = m DC
// that stays zero; columns of degree < DV are padded with Z, added last, which leaves Lambda
// unchanged.  PAD: checks of degree < DC are padded with a dummy column n whose Lambda stays
// 2^100 (kBig) and whose slots are read as zero and never written.  kBig is also where the
// two running minima of a check start, so a padded edge changes neither minimum, sign nor
// hard-decision parity: the update equals the unpadded one bit for bit.  Same operations in
// the same order as bp_kernel<G, 0>.
template <int NT, int CPL, int DC, int VPL, int DV, bool PAD, int MINB, bool PK>
__global__ void __launch_bounds__(NT, MINB) bp_regcta_kernel(BPArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned long long s_shot;
  __shared__ unsigned long long s_slot;
  const int m = a.g.m, n = a.g.n;
  const int Z = m * DC;
  const long long shots = a.shots_dev ? *a.shots_dev : a.shots;
  const int tid = threadIdx.x;
  float* r = reinterpret_cast<float*>(smem);           // [m DC + 1], r[Z] == 0
  float* Lam = r + align16((size_t)(Z + 1) * 4) / 4;   // [n + 1], Lam[n] == kBig
  float* s_prior = Lam + align16((size_t)(n + 1) * 4) / 4;  // [n]
  const float alpha = a.alpha;
  uint32_t cv[CPL][(DC + 1) / 2];
#pragma unroll
  for (int c = 0; c < CPL; ++c) {
    const int i = tid + NT * c;
#pragma unroll
    for (int k = 0; k < (DC + 1) / 2; ++k) cv[c][k] = 0;
    if (i < m) {
      // row-regular graphs (PAD false): chk_ptr[i] = i DC
      const int p0 = PAD ? a.g.chk_ptr[i] : i * DC;
      const int deg = PAD ? a.g.chk_ptr[i + 1] - p0 : DC;
#pragma unroll
      for (int k = 0; k < DC; ++k) {
        const uint32_t j = k < deg ? (uint32_t)a.g.chk_var[p0 + k] : (uint32_t)n;
        cv[c][k >> 1] |= j << (16 * (k & 1));
      }
    }
  }
  uint32_t ve[VPL][(DV + 1) / 2];
#pragma unroll
  for (int v = 0; v < VPL; ++v) {
    const int j = tid + NT * v;
#pragma unroll
    for (int k = 0; k < (DV + 1) / 2; ++k) ve[v][k] = 0;
    if (j < n) {
      const int q0 = a.g.var_ptr[j], deg = a.g.var_ptr[j + 1] - q0;
#pragma unroll
      for (int k = 0; k < DV; ++k) {
        uint32_t e = (uint32_t)Z;
        if (k < deg) {
          if constexpr (PAD) {
            const int i = a.g.var_chk[q0 + k];
            e = (uint32_t)(i * DC + (a.g.var_edge[q0 + k] - a.g.chk_ptr[i]));
          } else {
            e = (uint32_t)a.g.var_edge[q0 + k];  // = i DC + k when every row has DC edges
          }
        }
        ve[v][k >> 1] |= e << (16 * (k & 1));
      }
      s_prior[j] = a.g.prior[j];
    }
  }
  if (tid == 0) {
    r[Z] = 0.f;
    Lam[n] = kBig;
  }
  unsigned long long my_iters = 0, my_conv = 0;
  for (;;) {
    if (tid == 0) s_shot = atomicAdd(&a.ctr->next_shot, 1ULL);
    __syncthreads();
    const unsigned long long shot_u = s_shot;
    if (shot_u >= (unsigned long long)shots) break;
    const long long shot = (long long)shot_u;
    const uint8_t* sp = a.syndromes + shot * m;
    unsigned sbits = 0;
#pragma unroll
    for (int c = 0; c < CPL; ++c) {
      const int i = tid + NT * c;
      if (i < m) {
        if constexpr (PK) {
          const uint32_t* spw = reinterpret_cast<const uint32_t*>(a.syndromes) + shot * packed_words(m);
          if ((spw[i >> 5] >> (i & 31)) & 1u) sbits |= 1u << c;
        } else {
          if (sp[i]) sbits |= 1u << c;
        }
#pragma unroll
        for (int k = 0; k < DC; ++k) r[i * DC + k] = 0.f;
      }
    }
#pragma unroll
    for (int v = 0; v < VPL; ++v) {
      const int j = tid + NT * v;
      if (j < n) Lam[j] = s_prior[j];
    }
    __syncthreads();
    int t = 0;
    bool conv = false;
    for (;;) {
      const bool msgs = t < a.iters;
      unsigned unsat = 0;
      // ---- check phase (the update of bp_reg_kernel) ----
#pragma unroll
      for (int c = 0; c < CPL; ++c) {
        const int i = tid + NT * c;
        if (i >= m) continue;
        uint32_t hp = (sbits >> c) << 31;
        uint32_t sx = hp;
        float min1 = kBig, min2 = kBig;
        float aq[DC];
        uint32_t qb[DC];
        float* rc = r + i * DC;
#pragma unroll
        for (int k = 0; k < DC; ++k) {
          const int j = (cv[c][k >> 1] >> (16 * (k & 1))) & 0xffff;
          const float L = Lam[j];
          hp ^= __float_as_uint(L);
          const float q = __fsub_rn(L, rc[k]);
          qb[k] = __float_as_uint(q);
          sx ^= qb[k];
          aq[k] = fabsf(q);
          min2 = fminf(min2, fmaxf(min1, aq[k]));
          min1 = fminf(min1, aq[k]);
        }
        unsat |= hp >> 31;
        if (msgs) {
          const float m1 = __fmul_rn(alpha, min1), m2 = __fmul_rn(alpha, min2);
#pragma unroll
          for (int k = 0; k < DC; ++k) {
            const float mag = (aq[k] == min1) ? m2 : m1;
            if (!PAD || ((cv[c][k >> 1] >> (16 * (k & 1))) & 0xffff) != (uint32_t)n)
              rc[k] = __uint_as_float(__float_as_uint(mag) | ((sx ^ qb[k]) & 0x80000000u));
          }
        }
      }
      const int any_unsat = __syncthreads_or((int)unsat);
      if (t > 0) {
        conv = !any_unsat;
        if (conv && a.early_exit) break;
      }
      if (!msgs) break;
      // ---- variable phase ----
#pragma unroll
      for (int v = 0; v < VPL; ++v) {
        const int j = tid + NT * v;
        if (j >= n) continue;
        float L = s_prior[j];
#pragma unroll
        for (int k = 0; k < DV; ++k) L = __fadd_rn(L, r[(ve[v][k >> 1] >> (16 * (k & 1))) & 0xffff]);
        Lam[j] = L;
      }
      __syncthreads();
      ++t;
    }
    // ---- outputs ----
    if (a.posteriors) {
      float* po = a.posteriors + shot * n;
#pragma unroll
      for (int v = 0; v < VPL; ++v) {
        const int j = tid + NT * v;
        if (j < n) po[j] = Lam[j];
      }
    }
    if (tid == 0) {
      if (a.converged_out) a.converged_out[shot] = conv ? 1 : 0;
      if (a.iters_out) a.iters_out[shot] = t;
      my_iters += (unsigned long long)t;
      my_conv += conv ? 1ull : 0ull;
    }
    if (a.queue) {
      if (conv) {
        if constexpr (PK) {
          cta_packed_decision<NT, VPL>(a.corrections, shot, n, Lam, tid);
        } else {
          uint8_t* co = a.corrections + shot * n;
#pragma unroll
          for (int v = 0; v < VPL; ++v) {
            const int j = tid + NT * v;
            if (j < n) co[j] = (Lam[j] < 0.f) ? 1 : 0;
          }
        }
        if (tid == 0 && a.status) a.status[shot] = LSD_SHOT_OK_BP;
      } else {
        if (tid == 0) {
          s_slot = atomicAdd(&a.ctr->lsd_count, 1ULL);
          a.queue[s_slot] = (int32_t)shot;
        }
        __syncthreads();
        float* lo = a.queue_llr + (long long)s_slot * n;
#pragma unroll
        for (int v = 0; v < VPL; ++v) {
          const int j = tid + NT * v;
          if (j < n) lo[j] = Lam[j];
        }
      }
    }
    __syncthreads();
  }
  if (tid == 0) {
    if (my_iters) atomicAdd(&a.ctr->bp_iterations, my_iters);
    if (my_conv) atomicAdd(&a.ctr->bp_converged, my_conv);
  }
}

// Shapes of bp_reg_kernel: (G, CPL, DC, VPL, DV).
struct RegShape {
  int G, cpl, dc, vpl, dv;
  const void* fn;     // byte-per-bit syndromes and corrections
  const void* fn_pk;  // bit-packed
  const char* name;
};

#define LSD_REG_SHAPE(G, C, DCx, V, DVx)                                      \
  {G, C, DCx, V, DVx, (const void*)bp_reg_kernel<G, C, DCx, V, DVx, false>,   \
   (const void*)bp_reg_kernel<G, C, DCx, V, DVx, true>,                       \
   "bp_reg_kernel<" #G "," #C "," #DCx "," #V "," #DVx ">"}
const RegShape kRegShapes[] = {
    LSD_REG_SHAPE(16, 3, 6, 5, 3),   // m <= 48,  n <= 80   (BB [[72,12,6]])
    LSD_REG_SHAPE(32, 3, 6, 5, 3),   // m <= 96,  n <= 160  (BB [[144,12,12]])
    LSD_REG_SHAPE(16, 5, 6, 9, 3),   // m <= 80,  n <= 144  (BB [[144,12,12]])
    LSD_REG_SHAPE(32, 5, 6, 9, 3),   // m <= 160, n <= 288  (BB [[288,12,18]])
    LSD_REG_SHAPE(8, 5, 6, 9, 3),    // m <= 40,  n <= 72   (BB [[72,12,6]])
};
#undef LSD_REG_SHAPE
constexpr int kNumRegShapes = sizeof(kRegShapes) / sizeof(kRegShapes[0]);

bool reg_shape_fits(const RegShape& s, const DevGraph& g) {
  // regular graphs only: every row has degree dc and every column degree dv
  return g.m <= s.G * s.cpl && g.n <= s.G * s.vpl && g.max_row_deg == s.dc &&
         g.min_row_deg == s.dc && g.max_col_deg == s.dv && g.min_col_deg == s.dv;
}

}  // namespace

cudaError_t launch_priors(const float* probs, float* prior, long long* wfix, int n,
                          cudaStream_t st) {
  priors_kernel<<<(n + 255) / 256, 256, 0, st>>>(probs, prior, wfix, n);
  return cudaGetLastError();
}

// Variant ids: 0..2 generic min-sum with G = 8, 16, 32; 3..5 generic sum-product;
// 6 + i register-resident min-sum shape kRegShapes[i].
namespace {
const void* generic_fn(int v) {
  switch (v) {
    case 0: return (const void*)bp_kernel<8, 0>;
    case 1: return (const void*)bp_kernel<16, 0>;
    case 2: return (const void*)bp_kernel<32, 0>;
    case 3: return (const void*)bp_kernel<8, 1>;
    case 4: return (const void*)bp_kernel<16, 1>;
    default: return (const void*)bp_kernel<32, 1>;
  }
}
// Shapes of bp_regcta_kernel: (NT, CPL, DC, VPL, DV, PAD, MINB); rows of degree exactly DC
// (PAD false) or at most DC (PAD true), columns of degree at most DV; MINB CTAs per SM bound
// the registers a thread may take.
struct RegCtaShape {
  int nt, cpl, dc, vpl, dv;
  bool pad;
  const void* fn;
  const void* fn_pk;
  const char* name;
};
#define LSD_REGCTA_SHAPE(NT, C, DCx, V, DVx, P, MB)                                       \
  {NT, C, DCx, V, DVx, P, (const void*)bp_regcta_kernel<NT, C, DCx, V, DVx, P, MB, false>, \
   (const void*)bp_regcta_kernel<NT, C, DCx, V, DVx, P, MB, true>,                         \
   "bp_regcta_kernel<" #NT "," #C "," #DCx "," #V "," #DVx "," #P "," #MB ">"}
const RegCtaShape kRegCtaShapes[] = {
    LSD_REGCTA_SHAPE(768, 4, 7, 9, 4, false, 1),   // m <= 3072, n <= 6912 (HGP of a 48 x 64 (3,4) code)
    LSD_REGCTA_SHAPE(512, 6, 7, 13, 4, false, 1),  // same graphs, fewer threads
    // space-time matrices of BB codes: rows of degree w + 2 (and 1 in the last block),
    // columns of degree <= 3
    LSD_REGCTA_SHAPE(128, 3, 8, 6, 3, true, 6),  // m <= 384, n <= 768 (BB144 (3,1) windows)
    LSD_REGCTA_SHAPE(256, 4, 8, 11, 3, true, 2),  // m <= 1024, n <= 2816 (BB144, d = 12)
    LSD_REGCTA_SHAPE(512, 2, 8, 6, 3, true, 1),  // m <= 1024, n <= 3072
    LSD_REGCTA_SHAPE(512, 6, 8, 16, 3, true, 1),  // m <= 3072, n <= 8192 (BB288, d = 18)
    // ... with mid-round hook faults: rows of degree up to 17
    LSD_REGCTA_SHAPE(256, 2, 17, 9, 3, true, 2),  // m <= 512, n <= 2304 (BB144, d = 6)
    LSD_REGCTA_SHAPE(512, 1, 17, 5, 3, true, 1),  // m <= 512, n <= 2560
    // latency shapes (bp_kernel = 3, small batches): as many threads per shot as a CTA holds
    LSD_REGCTA_SHAPE(1024, 3, 8, 8, 3, true, 1),  // m <= 3072, n <= 8192 (BB288, d = 18)
    LSD_REGCTA_SHAPE(1024, 1, 8, 3, 3, true, 1),  // m <= 1024, n <= 3072 (BB144, d = 12)
    LSD_REGCTA_SHAPE(512, 1, 8, 2, 3, true, 1),   // m <= 512, n <= 1024 (BB72, d = 6)
};
#undef LSD_REGCTA_SHAPE
constexpr int kNumRegCtaShapes = sizeof(kRegCtaShapes) / sizeof(kRegCtaShapes[0]);

size_t regcta_smem(const RegCtaShape& s, const DevGraph& g) {
  return align16(((size_t)g.m * s.dc + 1) * 4) + align16(((size_t)g.n + 1) * 4) +
         align16((size_t)g.n * 4);
}
bool regcta_fits(const RegCtaShape& s, const DevGraph& g) {
  const bool rows = s.pad ? g.max_row_deg <= s.dc : (g.min_row_deg == s.dc && g.max_row_deg == s.dc);
  return rows && g.m <= s.nt * s.cpl && g.n <= s.nt * s.vpl && g.max_col_deg <= s.dv &&
         (long)g.m * s.dc < 65535 && g.n < 65535;
}

constexpr int kCtaBase = 6 + kNumRegShapes;     // + method: one CTA per shot
constexpr int kRegCtaBase = kCtaBase + 2;       // + i: kRegCtaShapes[i]
bool is_cta(int v) { return v >= kCtaBase && v < kRegCtaBase; }
bool is_regcta(int v) { return v >= kRegCtaBase; }
int lanes_of(int variant) {
  if (is_cta(variant) || is_regcta(variant)) return 0;
  if (variant >= 6) return kRegShapes[variant - 6].G;
  return variant % 3 == 0 ? 8 : variant % 3 == 1 ? 16 : 32;
}
// The kernel of a variant; `packed`: the instance with bit-packed syndromes and corrections
// (the generic and cache-read kernels take the layout from their arguments at run time).
const void* variant_fn(int v, bool packed = false) {
  if (is_regcta(v)) return packed ? kRegCtaShapes[v - kRegCtaBase].fn_pk : kRegCtaShapes[v - kRegCtaBase].fn;
  if (is_cta(v)) return v == kCtaBase ? (const void*)bp_cta_kernel<0> : (const void*)bp_cta_kernel<1>;
  if (v >= 6) return packed ? kRegShapes[v - 6].fn_pk : kRegShapes[v - 6].fn;
  return generic_fn(v);
}
}  // namespace

int bp_num_variants() { return kRegCtaBase + kNumRegCtaShapes; }

const char* bp_variant_name(int v) {
  static const char* const generic[6] = {"bp_kernel<8,0>", "bp_kernel<16,0>", "bp_kernel<32,0>",
                                         "bp_kernel<8,1>", "bp_kernel<16,1>", "bp_kernel<32,1>"};
  if (v < 0 || v >= bp_num_variants()) return nullptr;
  if (is_regcta(v)) return kRegCtaShapes[v - kRegCtaBase].name;
  if (is_cta(v)) return v == kCtaBase ? "bp_cta_kernel<0>" : "bp_cta_kernel<1>";
  return v >= 6 ? kRegShapes[v - 6].name : generic[v];
}

cudaError_t bp_config(const DevGraph& g, int lanes, int method, int kind, int* variant,
                      int* grid, int* block, size_t* smem) {
  int dev = 0, sms = 0, max_smem = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  // choose the variant: a register-resident shape for min-sum when one fits (the one that
  // wastes the fewest lane slots), else the generic kernel
  int v = -1;
  if (*variant >= 0) {
    v = *variant;
    if (v >= bp_num_variants()) return cudaErrorInvalidValue;
    if (is_regcta(v)) {
      if (method != 0 || !regcta_fits(kRegCtaShapes[v - kRegCtaBase], g)) return cudaErrorInvalidValue;
    } else if (is_cta(v)) {
      if ((v - kCtaBase) != (method != 0 ? 1 : 0)) return cudaErrorInvalidValue;
    } else if (v >= 6 && (method != 0 || !reg_shape_fits(kRegShapes[v - 6], g))) {
      return cudaErrorInvalidValue;
    } else if (v < 6 && (v >= 3) != (method != 0)) {
      return cudaErrorInvalidValue;
    }
  } else {
    if (method == 0 && kind == 3) {
      // latency: the CTA-per-shot shape with the most threads (the first of equal size) among
      // those with at least one fault per thread
      for (int i = 0; i < kNumRegCtaShapes; ++i) {
        const RegCtaShape& sh = kRegCtaShapes[i];
        if (regcta_fits(sh, g) && g.n >= sh.nt && regcta_smem(sh, g) <= (size_t)max_smem &&
            (v < 0 || sh.nt > kRegCtaShapes[v - kRegCtaBase].nt))
          v = kRegCtaBase + i;
      }
    }
    if (v < 0 && method == 0 && kind != 1) {
      // least work per lane first (fewer registers, shorter per-shot latency), then the
      // fewest idle lane slots
      long best_lane = -1, best_slots = -1;
      for (int i = 0; i < kNumRegShapes; ++i) {
        const RegShape& sh = kRegShapes[i];
        if (!reg_shape_fits(sh, g) || (lanes && sh.G != lanes)) continue;
        const long per_lane = (long)sh.cpl * sh.dc + (long)sh.vpl * sh.dv;
        const long slots = (long)sh.G * per_lane;
        if (best_lane < 0 || per_lane < best_lane || (per_lane == best_lane && slots < best_slots)) {
          best_lane = per_lane;
          best_slots = slots;
          v = 6 + i;
        }
      }
    }
    if (v < 0 && method == 0 && (kind == 0 || kind == 3) && lanes == 0) {
      // irregular or large graphs: one CTA per shot with register tables when a shape fits
      // and the graph has at least one check per thread (no graph table read per edge, and
      // a shot's latency spread over NT threads instead of one warp group)
      for (int i = 0; i < kNumRegCtaShapes; ++i) {
        const RegCtaShape& sh = kRegCtaShapes[i];
        if (regcta_fits(sh, g) && g.m >= sh.nt && regcta_smem(sh, g) <= (size_t)max_smem) {
          v = kRegCtaBase + i;
          break;
        }
      }
    }
    if (v < 0 && kind == 2) {  // register tables requested: a CTA shape, or nothing
      if (method == 0)
        for (int i = 0; i < kNumRegCtaShapes; ++i)
          if (regcta_fits(kRegCtaShapes[i], g) && regcta_smem(kRegCtaShapes[i], g) <= (size_t)max_smem) {
            v = kRegCtaBase + i;
            break;
          }
      if (v < 0) return cudaErrorInvalidValue;
    }
    if (v < 0) {
      const int l = lanes ? lanes : 32;
      v = (l == 8 ? 0 : l == 16 ? 1 : 2) + (method ? 3 : 0);
      // a graph whose warp-group state does not fit next to the staged graph: one CTA per
      // shot, with register tables when a shape fits
      if (bp_graph_bytes(g.m, g.n, g.E) + bp_group_bytes(g.m, g.n, g.E) > (size_t)max_smem) {
        v = kCtaBase + (method ? 1 : 0);
        if (method == 0 && kind != 1)
          for (int i = 0; i < kNumRegCtaShapes; ++i)
            if (regcta_fits(kRegCtaShapes[i], g) && regcta_smem(kRegCtaShapes[i], g) <= (size_t)max_smem) {
              v = kRegCtaBase + i;
              break;
            }
      }
    }
  }
  size_t gb, grp;
  int b;
  if (is_regcta(v)) {
    gb = 0;
    grp = regcta_smem(kRegCtaShapes[v - kRegCtaBase], g);
    if (grp > (size_t)max_smem) return cudaErrorInvalidValue;
    b = kRegCtaShapes[v - kRegCtaBase].nt;
  } else if (is_cta(v)) {
    gb = 0;
    grp = bp_group_bytes(g.m, g.n, g.E);
    if (grp > (size_t)max_smem) return cudaErrorInvalidValue;
    b = g.m >= 2048 ? 512 : 256;
  } else {
    const int G = lanes_of(v);
    if (v >= 6) {
      gb = align16((size_t)g.n * 4);
      grp = bp_reg_group_bytes(g.n, g.E);
    } else {
      gb = bp_graph_bytes(g.m, g.n, g.E);
      grp = bp_group_bytes(g.m, g.n, g.E);
    }
    b = 256;
    while (b > G && gb + (size_t)(b / G) * grp > (size_t)max_smem) b /= 2;
    if (gb + (size_t)(b / G) * grp > (size_t)max_smem) return cudaErrorInvalidValue;
    grp *= (size_t)(b / G);
  }
  *block = b;
  *smem = gb + grp;
  const void* fn = variant_fn(v);
  err = allow_max_dynamic_smem(fn, max_smem);
  if (err == cudaSuccess && variant_fn(v, true) != fn)
    err = allow_max_dynamic_smem(variant_fn(v, true), max_smem);
  if (err != cudaSuccess) return err;
  int per_sm = 0;
  err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, b, *smem);
  if (err != cudaSuccess) return err;
  if (per_sm < 1) return cudaErrorInvalidValue;
  *grid = per_sm * sms;
  *variant = v;
  return cudaSuccess;
}

cudaError_t launch_bp(const BPArgs& a, int variant, int grid, int block, size_t smem,
                      cudaStream_t st) {
  const void* fn = variant_fn(variant, a.packed != 0);
  void* args[] = {const_cast<BPArgs*>(&a)};
  return cudaLaunchKernel(fn, dim3(grid), dim3(block), args, smem, st);
}

}  // namespace lsdgb
