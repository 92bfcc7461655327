// Min-sum BP of one shot by a group of G lanes (G | 32) whose graph tables sit in
// registers: lane l keeps the column indices of checks l, l + G, ... and the edge slots of
// variables l, l + G, ... (two 16-bit indices per register); r[E] and Lam[n] are the shot's
// message state in shared memory.  Used by bp_reg_kernel.
// Same operations in the same order as bp_kernel<G, 0> (the flooding min-sum of Sec. 4.3).
#pragma once

#include "lsd_internal.cuh"

namespace lsdgb {
namespace bpreg {

constexpr float kBig = 0x1p100f;  // minimum over an empty set (a degree-1 check)

template <int CPL, int DC, int VPL, int DV>
struct Tables {
  uint32_t cv[CPL][(DC + 1) / 2];
  uint32_t ve[VPL][(DV + 1) / 2];
};

template <int G, int CPL, int DC, int VPL, int DV>
__device__ __forceinline__ void load_tables(const DevGraph& g, int lane,
                                            Tables<CPL, DC, VPL, DV>& T) {
#pragma unroll
  for (int c = 0; c < CPL; ++c) {
    const int i = lane + G * c;
#pragma unroll
    for (int k = 0; k < (DC + 1) / 2; ++k) T.cv[c][k] = 0;
    if (i < g.m) {
#pragma unroll
      for (int k = 0; k < DC; ++k) T.cv[c][k >> 1] |= (uint32_t)g.chk_var[i * DC + k] << (16 * (k & 1));
    }
  }
#pragma unroll
  for (int v = 0; v < VPL; ++v) {
    const int j = lane + G * v;
#pragma unroll
    for (int k = 0; k < (DV + 1) / 2; ++k) T.ve[v][k] = 0;
    if (j < g.n) {
#pragma unroll
      for (int k = 0; k < DV; ++k) T.ve[v][k >> 1] |= (uint32_t)g.var_edge[j * DV + k] << (16 * (k & 1));
    }
  }
}

// BP on `shot` from the channel priors; returns the iterations run and sets conv (the hard
// decision of the final Lam satisfies the syndrome).  Lam holds the posteriors on return.
template <int G, int CPL, int DC, int VPL, int DV, bool PK = false>
__device__ __forceinline__ int shot_bp(const BPArgs& a, const Tables<CPL, DC, VPL, DV>& T,
                                       long long shot, float* r, float* Lam,
                                       const float* s_prior, int lane, unsigned gmask,
                                       bool& conv) {
  const int m = a.g.m, n = a.g.n;
  const float alpha = a.alpha;
  const uint8_t* sp = a.syndromes + shot * m;
  unsigned sbits = 0;
#pragma unroll
  for (int c = 0; c < CPL; ++c) {
    const int i = lane + G * c;
    if (i < m) {
      if constexpr (PK) {  // bit-packed syndromes (lsd_decode_batch_packed)
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
    const int j = lane + G * v;
    if (j < n) Lam[j] = s_prior[j];
  }
  __syncwarp(gmask);

  int t = 0;
  conv = false;
  for (;;) {
    const bool msgs = t < a.iters;
    unsigned unsat = 0;
    // ---- check phase: parity of [Lam^(t) < 0] and messages r^(t+1) ----
    // Sign bits stand for the comparisons "< 0": the priors are finite and never -0
    // (0 < p < 1), so no Lam and no q = Lam - r is -0 or NaN.  The two smallest
    // magnitudes come from min/max alone; the edge holding the minimum takes the second
    // one (on a tie both are equal, as with a first-index rule).
#pragma unroll
    for (int c = 0; c < CPL; ++c) {
      const int i = lane + G * c;
      if (i >= m) continue;
      uint32_t hp = (sbits >> c) << 31;  // bit 31: syndrome ^ signs of Lam
      uint32_t sx = hp;                   // bit 31: syndrome ^ signs of q
      float min1 = kBig, min2 = kBig;
      float aq[DC];
      uint32_t qb[DC];
      float* rc = r + i * DC;
#pragma unroll
      for (int k = 0; k < DC; ++k) {
        const int j = (T.cv[c][k >> 1] >> (16 * (k & 1))) & 0xffff;
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
          rc[k] = __uint_as_float(__float_as_uint(mag) | ((sx ^ qb[k]) & 0x80000000u));
        }
      }
    }
    if (t > 0) {
      conv = !__any_sync(gmask, unsat != 0);
      if (conv && a.early_exit) break;
    }
    if (!msgs) break;
    __syncwarp(gmask);
    // ---- variable phase: Lam^(t+1) ----
#pragma unroll
    for (int v = 0; v < VPL; ++v) {
      const int j = lane + G * v;
      if (j >= n) continue;
      float L = s_prior[j];
#pragma unroll
      for (int k = 0; k < DV; ++k) L = __fadd_rn(L, r[(T.ve[v][k >> 1] >> (16 * (k & 1))) & 0xffff]);
      Lam[j] = L;
    }
    __syncwarp(gmask);
    ++t;
  }
  return t;
}

}  // namespace bpreg
}  // namespace lsdgb
