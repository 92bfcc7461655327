// LSD for large check matrices (space-time and hypergraph-product codes): the same
// algorithm and results as lsd.cu (Alg. 1 of Sec. 4.1, on-the-fly elimination of Sec. 4.2,
// LSD-mu of App. D), with state sized by what a shot touches instead of by m and n.
//
// One warp owns one shot.
//   * Per-detector and per-fault arrays live in a per-warp global scratch (L1/L2 resident):
//       dlab[m]  cluster of a claimed detector (seed ordinal, flattened to the root; -1 none)
//       slot[m]  elimination row of a claimed detector (claim order; -1 none)
//       fst[n]   fault state: -2 untouched, -1 candidate (next to a claimed detector),
//                >= 0 the seed ordinal of the cluster it joined
//       front[n] the candidate list (Def. 4.3's Lambda over all clusters), compacted per step
//   * Clusters are indexed by seed ordinal (flipped detectors in ascending order, so a root
//     -- the smallest seed of a cluster -- is the same as in lsd.cu), elimination rows by
//     slot: R[slot][W], T[slot][W] over CAP slots, in shared memory, or in global scratch
//     for the spill instance.
//   * A pick is the minimum 64-bit key (order-preserving LLR bits, index) over the candidate
//     list of each growing cluster (atomicMin), so no per-shot sort is needed.
// A shot that needs more than CAP slots (or SC seeds, or CAP dependent columns) stops with
// status LSD_SHOT_SPILL_ and is queued for the global-memory instance.
#include <climits>

#include "lsd_internal.cuh"

namespace lsdgb {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr unsigned long long kNoKey = ~0ull;
constexpr int kSpill = 4;  // internal status: retry with the large-capacity instance
constexpr int kMaskSeeds = 1024;  // spill instance: shots with at most this many seeds use masks

__host__ __device__ constexpr size_t al16(size_t x) { return (x + 15) & ~(size_t)15; }

// Per-warp layout of the parts kept in shared memory (or global for GLOBAL_RT).
template <int CAP, int SC, bool MU>
struct SLay {
  static constexpr int W = CAP / 32;
  static constexpr size_t R = 0;
  static constexpr size_t T = R + (size_t)CAP * W * 4;
  static constexpr size_t pcol = T + (size_t)CAP * W * 4;
  static constexpr size_t dslot = pcol + (size_t)CAP * 4;         // detector of a slot
  static constexpr size_t npN = dslot + (size_t)CAP * 4;          // dependent columns
  static constexpr size_t npk = npN + (MU ? (size_t)CAP * W * 4 : 0);
  static constexpr size_t ext = npk + (MU ? (size_t)CAP * 8 : 0);
  static constexpr size_t rt_total = al16(ext + (MU ? (size_t)CAP * 4 : 0));
  // always in shared memory
  static constexpr size_t best = 0;                               // [SC] u64
  static constexpr size_t newk = best + (size_t)SC * 8;           // [SC] u64
  static constexpr size_t srt = newk + (size_t)SC * 8;            // [SC] u64
  static constexpr size_t seed = srt + (size_t)SC * 8;            // [SC] detector of a seed
  static constexpr size_t parent = seed + (size_t)SC * 4;
  static constexpr size_t mark = parent + (size_t)SC * 4;
  static constexpr size_t inv = mark + (size_t)SC * 4;
  static constexpr size_t mlist = inv + (size_t)SC * 4;
  static constexpr size_t dnew = mlist + (size_t)SC * 4;          // [CAP]
  static constexpr size_t words = dnew + (size_t)CAP * 4;         // syn sred xsol cm [W]
  static constexpr size_t scal = words + (size_t)4 * W * 4;
  static constexpr size_t gflag = scal + 16 * 4;                  // [SC] growing flags
  static constexpr size_t sm_total = al16(gflag + (size_t)SC);
};

struct SGraph {
  const int32_t* chk_ptr;
  const uint16_t* chk_var;
  const int32_t* var_ptr;
  const uint16_t* var_chk;
  int max_col_deg;
};

template <class L>
struct SShot {
  unsigned char* sm;    // shared part
  unsigned char* rt;    // elimination part (shared or global)
  int* dlab;            // [m]  global scratch
  int* slot;            // [m]
  int* fst;             // [n]
  int* front;           // [n]
  uint32_t* cmask;      // spill instance: per seed, its clusters' candidate faults [SC][wn]
  int wn;               // words of a candidate mask (ceil(n / 32)); 0 = no masks
  template <class T>
  __device__ __forceinline__ T* s(size_t off) const { return reinterpret_cast<T*>(sm + off); }
  template <class T>
  __device__ __forceinline__ T* r(size_t off) const { return reinterpret_cast<T*>(rt + off); }
  __device__ __forceinline__ uint32_t* R() const { return r<uint32_t>(L::R); }
  __device__ __forceinline__ uint32_t* T() const { return r<uint32_t>(L::T); }
  __device__ __forceinline__ int* pcol() const { return r<int>(L::pcol); }
  __device__ __forceinline__ int* dslot() const { return r<int>(L::dslot); }
  __device__ __forceinline__ uint32_t* npN() const { return r<uint32_t>(L::npN); }
  __device__ __forceinline__ unsigned long long* npk() const { return r<unsigned long long>(L::npk); }
  __device__ __forceinline__ int* ext() const { return r<int>(L::ext); }
  __device__ __forceinline__ unsigned long long* best() const { return s<unsigned long long>(L::best); }
  __device__ __forceinline__ unsigned long long* newk() const { return s<unsigned long long>(L::newk); }
  __device__ __forceinline__ unsigned long long* srt() const { return s<unsigned long long>(L::srt); }
  __device__ __forceinline__ int* seed() const { return s<int>(L::seed); }
  __device__ __forceinline__ int* parent() const { return s<int>(L::parent); }
  __device__ __forceinline__ unsigned* mark() const { return s<unsigned>(L::mark); }
  __device__ __forceinline__ int* inv() const { return s<int>(L::inv); }
  __device__ __forceinline__ int* mlist() const { return s<int>(L::mlist); }
  __device__ __forceinline__ int* dnew() const { return s<int>(L::dnew); }
  __device__ __forceinline__ uint32_t* syn() const { return s<uint32_t>(L::words); }
  __device__ __forceinline__ uint32_t* sred() const { return s<uint32_t>(L::words + L::W * 4); }
  __device__ __forceinline__ uint32_t* xsol() const { return s<uint32_t>(L::words + 2 * L::W * 4); }
  __device__ __forceinline__ uint32_t* cm() const { return s<uint32_t>(L::words + 3 * L::W * 4); }
  __device__ __forceinline__ int* scal() const { return s<int>(L::scal); }
  __device__ __forceinline__ unsigned char* gflag() const { return s<unsigned char>(L::gflag); }
};

// scal slots
enum { S_NEW = 0, S_NP, S_EXT, S_MERGED, S_DNEW, S_INV, S_SLOTS, S_NSEED, S_NFRONT, S_OVF };

__device__ __forceinline__ unsigned long long llr_key(float x, int j) {
  x = __fadd_rn(x, 0.0f);
  unsigned u = __float_as_uint(x);
  u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
  return ((unsigned long long)u << 32) | (unsigned)j;
}

__device__ __forceinline__ int uf_find(const volatile int* parent, int x) {
  int p = parent[x];
  while (p != x) {
    x = p;
    p = parent[x];
  }
  return x;
}

template <class L>
__device__ __forceinline__ void uf_unite(const SShot<L>& S, int a, int b) {
  int* parent = S.parent();
  const volatile int* vp = parent;
  for (;;) {
    a = uf_find(vp, a);
    b = uf_find(vp, b);
    if (a == b) return;
    if (a < b) {
      const int t = a;
      a = b;
      b = t;
    }
    if (atomicCAS(parent + a, a, b) == a) {
      const int k = atomicAdd(&S.scal()[S_MERGED], 1);
      S.mlist()[k] = a;
      return;
    }
  }
}

__device__ __forceinline__ bool bit_of(const uint32_t* v, int i) {
  return (v[i >> 5] >> (i & 31)) & 1u;
}

// Claims detector d for cluster r (lane-local).  Returns false on slot overflow.
template <class L, int CAP>
__device__ __forceinline__ void claim(const SShot<L>& S, int d, int r) {
  const int o = atomicCAS(&S.dlab[d], -1, r);
  if (o == -1) {
    const int sl = atomicAdd(&S.scal()[S_SLOTS], 1);
    if (sl >= CAP) {
      S.scal()[S_OVF] = 1;
      return;
    }
    S.slot[d] = sl;
    S.dslot()[sl] = d;
    const int k = atomicAdd(&S.scal()[S_DNEW], 1);
    S.dnew()[k] = d;
  } else if (o != r) {
    uf_unite(S, r, o);
  }
}

template <class L>
__device__ int collect_invalid(const SShot<L>& S, int lane) {
  if (lane == 0) S.scal()[S_INV] = 0;
  __syncwarp();
  for (int w = lane; w < L::W; w += 32) {
    uint32_t bits = S.sred()[w];
    while (bits) {
      const int sl = w * 32 + __ffs(bits) - 1;
      bits &= bits - 1;
      const int root = S.dlab[S.dslot()[sl]];
      if (root >= 0 && atomicCAS(&S.mark()[root], 0u, 1u) == 0u) {
        const int k = atomicAdd(&S.scal()[S_INV], 1);
        S.inv()[k] = root;
      }
    }
  }
  __syncwarp();
  const int count = S.scal()[S_INV];
  for (int t = lane; t < count; t += 32) S.mark()[S.inv()[t]] = 0u;
  __syncwarp();
  return count;
}

template <class L>
__device__ int collect_all(const SShot<L>& S, int lane) {
  const int ns = S.scal()[S_NSEED];
  int count = 0;
  for (int b = 0; b < ns; b += 32) {
    const int k = b + lane;
    const bool pred = k < ns && S.parent()[k] == k;
    const unsigned bal = __ballot_sync(kFull, pred);
    if (pred) S.inv()[count + __popc(bal & ((1u << lane) - 1u))] = k;
    count += __popc(bal);
  }
  __syncwarp();
  return count;
}

// Adds fault g (order key `key`) to its cluster's factorization, rows in slot space.  Lane l
// holds words l, l+32, ... of the column being reduced.
// Only the first wc = ceil(slots / 32) words of a row can be nonzero: rows are written in
// full (zeros past the slots in use) when they become pivots, and every later update XORs
// rows that are zero there too.
template <class L, bool MU, int CAP>
__device__ void add_column(const SGraph& G, const SShot<L>& S, int g, unsigned long long key,
                           int lane) {
  constexpr int W = L::W;
  constexpr int WC = (W + 31) / 32;
  const int nsl = min(S.scal()[S_SLOTS], CAP);
  const int wc = (nsl + 31) >> 5;
  uint32_t bw[WC], tw[WC];
#pragma unroll
  for (int c = 0; c < WC; ++c) bw[c] = tw[c] = 0;
  const int v0 = G.var_ptr[g], v1 = G.var_ptr[g + 1];
  for (int q = v0; q < v1; ++q) {
    const int sl = S.slot[G.var_chk[q]];
    const bool piv = S.pcol()[sl] >= 0;
#pragma unroll
    for (int c = 0; c < WC; ++c) {
      const int w = c * 32 + lane;
      if (w < wc) {
        if ((sl >> 5) == w) bw[c] ^= 1u << (sl & 31);
        if (piv) {
          bw[c] ^= S.R()[sl * W + w];
          tw[c] ^= S.T()[sl * W + w];
        }
      }
    }
  }
  int p = -1;
#pragma unroll
  for (int c = 0; c < WC; ++c) {
    const unsigned nz = __ballot_sync(kFull, bw[c] != 0);
    if (p < 0 && nz) {
      const int wl = __ffs(nz) - 1;
      const uint32_t word = __shfl_sync(kFull, bw[c], wl);
      p = (c * 32 + wl) * 32 + __ffs(word) - 1;
    }
  }
  if (p < 0) {
    if constexpr (MU) {
      const int k = __shfl_sync(kFull, S.scal()[S_NP], 0);
      if (k >= CAP) {
        if (lane == 0) S.scal()[S_OVF] = 1;
      } else {
#pragma unroll
        for (int c = 0; c < WC; ++c) {
          const int w = c * 32 + lane;
          if (w < W) S.npN()[k * W + w] = tw[c];
        }
        __syncwarp();
        if (lane == 0) {
          S.npk()[k] = key;
          S.scal()[S_NP] = k + 1;
        }
      }
      __syncwarp();
    }
    return;
  }
  const int pw = p >> 5;
  const uint32_t pb = 1u << (p & 31);
#pragma unroll
  for (int c = 0; c < WC; ++c)
    if (c * 32 + lane == pw) tw[c] ^= pb;
  const bool sflag = (S.sred()[pw] & pb) != 0;
#pragma unroll
  for (int c = 0; c < WC; ++c) {
    const int w = c * 32 + lane;
    if (w < W) {
      S.R()[p * W + w] = bw[c];
      S.T()[p * W + w] = tw[c];
    }
  }
  if (lane == 0) S.pcol()[p] = g;
  __syncwarp();
  // back-elimination: rows holding bit p found by ballot, each XORed by the whole warp
  // (lane = word) with the new pivot row, which the lanes still hold in registers
  for (int d0 = 0; d0 < nsl; d0 += 32) {
    const int d = d0 + lane;
    const bool hit = d < nsl && d != p && S.pcol()[d] >= 0 && (S.R()[d * W + pw] & pb) != 0;
    unsigned bal = __ballot_sync(kFull, hit);
    while (bal) {
      const int dd = d0 + __ffs(bal) - 1;
      bal &= bal - 1;
#pragma unroll
      for (int c = 0; c < WC; ++c) {
        const int w = c * 32 + lane;
        if (w < wc) {
          S.R()[dd * W + w] ^= bw[c];
          S.T()[dd * W + w] ^= tw[c];
        }
      }
    }
  }
  if (sflag) {
#pragma unroll
    for (int c = 0; c < WC; ++c) {
      const int w = c * 32 + lane;
      if (w < W) {
        S.sred()[w] ^= bw[c];
        S.xsol()[w] ^= tw[c];
      }
    }
  }
  __syncwarp();
}

// One synchronous growth step of the k clusters in inv[] (same contract as lsd.cu).
template <class L, bool MU, int CAP>
__device__ int sparse_step(const SGraph& G, const SShot<L>& S, const float* llr, int k,
                           bool strict, int lane) {
  for (int t = lane; t < k; t += 32) {
    const int r = S.inv()[t];
    S.best()[r] = kNoKey;
    S.gflag()[r] = 1;
  }
  __syncwarp();
  // find_candidate.  With few growing clusters (the spill instance's late steps, one huge
  // cluster growing alone), each scans its own candidate mask: the set bits are the free
  // faults next to it, so only their LLRs are read.  Otherwise one pass over the compacted
  // candidate list, 4 entries per lane at a time: the dependent loads (entry, state,
  // column, labels) of the four are issued together.
  if (S.wn > 0 && (long long)k * S.wn < 2LL * S.scal()[S_NFRONT]) {
    for (int t = 0; t < k; ++t) {
      const int r = S.inv()[t];
      const uint32_t* cm = S.cmask + (size_t)r * S.wn;
      unsigned long long best = kNoKey;
      for (int w = lane; w < S.wn; w += 32) {
        uint32_t bits = cm[w];
        while (bits) {
          const int f = w * 32 + __ffs(bits) - 1;
          bits &= bits - 1;
          if (S.fst[f] != -1) continue;  // already in a cluster
          const unsigned long long key = llr_key(llr[f], f);
          if (key < best) best = key;
        }
      }
      for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long o = __shfl_xor_sync(kFull, best, off);
        if (o < best) best = o;
      }
      if (lane == 0) S.best()[r] = best;
    }
    __syncwarp();
  } else {
    const int nf = S.scal()[S_NFRONT];
    const unsigned below = (1u << lane) - 1u;
    int kept = 0;
    for (int b = 0; b < nf; b += 128) {
      int f[4], q0[4], q1[4];
      unsigned long long key[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = b + 32 * u + lane;
        f[u] = i < nf ? S.front[i] : -1;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (f[u] >= 0 && S.fst[f[u]] != -1) f[u] = -1;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        key[u] = kNoKey;
        q0[u] = q1[u] = 0;
        if (f[u] >= 0) {
          key[u] = llr_key(llr[f[u]], f[u]);
          q0[u] = G.var_ptr[f[u]];
          q1[u] = G.var_ptr[f[u] + 1];
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const unsigned bal = __ballot_sync(kFull, f[u] >= 0);
        if (f[u] >= 0) S.front[kept + __popc(bal & below)] = f[u];
        kept += __popc(bal);
      }
      for (int qq = 0; qq < G.max_col_deg; ++qq) {
        int r[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int q = q0[u] + qq;
          r[u] = q < q1[u] ? S.dlab[G.var_chk[q]] : -1;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (r[u] >= 0 && S.gflag()[r[u]]) atomicMin(&S.best()[r[u]], key[u]);
      }
      __syncwarp();
    }
    if (lane == 0) S.scal()[S_NFRONT] = kept;
  }
  __syncwarp();
  bool none = false, some = false;
  for (int t = lane; t < k; t += 32) {
    const int r = S.inv()[t];
    S.gflag()[r] = 0;
    if (S.best()[r] == kNoKey) none = true;
    else some = true;
  }
  none = __any_sync(kFull, none);
  some = __any_sync(kFull, some);
  if ((strict && none) || !some) {
    __syncwarp();
    return (strict && none) ? 1 : 2;
  }
  if (lane == 0) {
    S.scal()[S_NEW] = 0;
    S.scal()[S_MERGED] = 0;
    S.scal()[S_DNEW] = 0;
  }
  __syncwarp();
  // parallel_union
  for (int t = lane; t < k; t += 32) {
    const int r = S.inv()[t];
    const unsigned long long key = S.best()[r];
    if (key == kNoKey) continue;
    const int g = (int)(key & 0xffffffffu);
    const int old = atomicCAS(&S.fst[g], -1, r);
    if (old == -1) {
      const int q = atomicAdd(&S.scal()[S_NEW], 1);
      S.newk()[q] = key;
    } else {
      uf_unite(S, r, old);
    }
    const int v1 = G.var_ptr[g + 1];
    for (int q = G.var_ptr[g]; q < v1; ++q) claim<L, CAP>(S, G.var_chk[q], r);
  }
  __syncwarp();
  if (S.scal()[S_OVF]) return 3;
  // flatten after merges
  if (S.scal()[S_MERGED]) {
    const int ns = S.scal()[S_NSEED];
    for (int x = lane; x < ns; x += 32) S.parent()[x] = uf_find(S.parent(), x);
    __syncwarp();
    const int nsl = S.scal()[S_SLOTS];
    for (int sl = lane; sl < nsl; sl += 32) {
      const int d = S.dslot()[sl];
      S.dlab[d] = S.parent()[S.dlab[d]];
    }
    __syncwarp();
  }
  // candidate masks: the absorbed clusters' masks fold into their roots
  if (S.wn > 0 && S.scal()[S_MERGED]) {
    const int nm = S.scal()[S_MERGED];
    for (int i = 0; i < nm; ++i) {
      const int x = S.mlist()[i];
      const uint32_t* src = S.cmask + (size_t)x * S.wn;
      uint32_t* dst = S.cmask + (size_t)S.parent()[x] * S.wn;
      for (int w = lane; w < S.wn; w += 32) {
        const uint32_t v = src[w];
        if (v) atomicOr(&dst[w], v);
      }
    }
    __syncwarp();
  }
  // candidates next to the newly claimed detectors (and, with masks, in their cluster's mask)
  {
    const int nd = S.scal()[S_DNEW];
    for (int t = lane; t < nd; t += 32) {
      const int d = S.dnew()[t];
      uint32_t* cm = S.wn > 0 ? S.cmask + (size_t)S.dlab[d] * S.wn : nullptr;
      const int c1 = G.chk_ptr[d + 1];
      for (int e = G.chk_ptr[d]; e < c1; ++e) {
        const int f = G.chk_var[e];
        if (atomicCAS(&S.fst[f], -2, -1) == -2) {
          const int q = atomicAdd(&S.scal()[S_NFRONT], 1);
          S.front[q] = f;
        }
        if (cm && S.fst[f] < 0) atomicOr(&cm[f >> 5], 1u << (f & 31));
      }
    }
  }
  __syncwarp();
  // new columns in key order
  const int n_new = S.scal()[S_NEW];
  for (int t = lane; t < n_new; t += 32) {
    const unsigned long long kt = S.newk()[t];
    int pos = 0;
    for (int u = 0; u < n_new; ++u) pos += (S.newk()[u] < kt) ? 1 : 0;
    S.srt()[pos] = kt;
  }
  __syncwarp();
  for (int t = 0; t < n_new; ++t) {
    const unsigned long long key = S.srt()[t];
    add_column<L, MU, CAP>(G, S, (int)(key & 0xffffffffu), key, lane);
  }
  return S.scal()[S_OVF] ? 3 : 0;
}

template <class L>
__device__ void sparse_osd_e(const LSDArgs& a, const SShot<L>& S, int lane) {
  constexpr int W = L::W;
  const long long* wfix = a.g.wfix;
  const int order = a.order;
  const int nroots = collect_all(S, lane);
  const int n_np = S.scal()[S_NP];
  const int nsl = S.scal()[S_SLOTS];
  for (int ci = 0; ci < nroots; ++ci) {
    const int r = S.inv()[ci];
    for (int c = 0; c < W; ++c) {
      const int sl = c * 32 + lane;
      const bool in = sl < nsl && S.dlab[S.dslot()[sl]] == r;
      const unsigned bal = __ballot_sync(kFull, in);
      if (lane == 0) S.cm()[c] = bal;
    }
    __syncwarp();
    int sel[kMaxOrder];
    int nt = 0;
    unsigned long long last = 0;
    for (int it = 0; it < order; ++it) {
      unsigned long long bk = kNoKey;
      int bi = -1;
      for (int u = lane; u < n_np; u += 32) {
        const unsigned long long ku = S.npk()[u];
        if (it > 0 && ku <= last) continue;
        if (S.parent()[S.fst[(int)(ku & 0xffffffffu)]] != r) continue;
        if (ku < bk) {
          bk = ku;
          bi = u;
        }
      }
      for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long ok = __shfl_xor_sync(kFull, bk, off);
        const int oi = __shfl_xor_sync(kFull, bi, off);
        if (ok < bk) {
          bk = ok;
          bi = oi;
        }
      }
      if (bk == kNoKey) break;
      sel[nt++] = bi;
      last = bk;
    }
    if (nt == 0) continue;
    long long bcost = LLONG_MAX;
    int bt = 0;
    for (int t = lane; t < (1 << nt); t += 32) {
      long long cost = 0;
      for (int w = 0; w < W; ++w) {
        uint32_t mw = S.xsol()[w] & S.cm()[w];
        for (int k2 = 0; k2 < nt; ++k2)
          if ((t >> k2) & 1) mw ^= S.npN()[sel[k2] * W + w];
        while (mw) {
          const int b = __ffs(mw) - 1;
          mw &= mw - 1;
          cost += wfix[S.pcol()[w * 32 + b]];
        }
      }
      for (int k2 = 0; k2 < nt; ++k2)
        if ((t >> k2) & 1) cost += wfix[(int)(S.npk()[sel[k2]] & 0xffffffffu)];
      if (cost < bcost) {
        bcost = cost;
        bt = t;
      }
    }
    for (int off = 16; off > 0; off >>= 1) {
      const long long oc = __shfl_xor_sync(kFull, bcost, off);
      const int ot = __shfl_xor_sync(kFull, bt, off);
      if (oc < bcost || (oc == bcost && ot < bt)) {
        bcost = oc;
        bt = ot;
      }
    }
    for (int w = lane; w < W; w += 32) {
      uint32_t delta = 0;
      for (int k2 = 0; k2 < nt; ++k2)
        if ((bt >> k2) & 1) delta ^= S.npN()[sel[k2] * W + w];
      S.xsol()[w] ^= delta;
    }
    if (lane == 0) {
      int ne = S.scal()[S_EXT];
      for (int k2 = 0; k2 < nt; ++k2)
        if ((bt >> k2) & 1) S.ext()[ne++] = (int)(S.npk()[sel[k2]] & 0xffffffffu);
      S.scal()[S_EXT] = ne;
    }
    __syncwarp();
  }
}

// Cost of cluster r's local solution (xsol masked by cm) with the dependent columns of slots
// u1 and u2 flipped (-1 = none).
template <class L>
__device__ __forceinline__ long long sparse_pattern_cost(const LSDArgs& a, const SShot<L>& S,
                                                         int u1, int u2) {
  constexpr int W = L::W;
  const long long* wfix = a.g.wfix;
  long long cost = 0;
  for (int w = 0; w < W; ++w) {
    uint32_t mw = S.xsol()[w] & S.cm()[w];
    if (u1 >= 0) mw ^= S.npN()[u1 * W + w];
    if (u2 >= 0) mw ^= S.npN()[u2 * W + w];
    while (mw) {
      const int b = __ffs(mw) - 1;
      mw &= mw - 1;
      cost += wfix[S.pcol()[w * 32 + b]];
    }
  }
  if (u1 >= 0) cost += wfix[(int)(S.npk()[u1] & 0xffffffffu)];
  if (u2 >= 0) cost += wfix[(int)(S.npk()[u2] & 0xffffffffu)];
  return cost;
}

// OSD-CS-w reprocessing of every cluster (App. D), as osd_cs in lsd.cu: no flip, every
// single dependent column, every pair among the first w in key order; ranked by
// (cost, class, key) with class 0 = no flip, 1 = single (key = the column's 64-bit order
// key), 2 = pair (key = i * 16 + j).
template <class L>
__device__ void sparse_osd_cs(const LSDArgs& a, const SShot<L>& S, int lane) {
  constexpr int W = L::W;
  const int nroots = collect_all(S, lane);
  const int n_np = S.scal()[S_NP];
  const int nsl = S.scal()[S_SLOTS];
  const int w_cs = a.osd_cs;
  for (int ci = 0; ci < nroots; ++ci) {
    const int r = S.inv()[ci];
    for (int c = 0; c < W; ++c) {
      const int sl = c * 32 + lane;
      const bool in = sl < nsl && S.dlab[S.dslot()[sl]] == r;
      const unsigned bal = __ballot_sync(kFull, in);
      if (lane == 0) S.cm()[c] = bal;
    }
    __syncwarp();
    int sel[kMaxCsOrder];
    int nt = 0;
    unsigned long long last = 0;
    for (int it = 0; it < w_cs; ++it) {
      unsigned long long bk = kNoKey;
      int bi = -1;
      for (int u = lane; u < n_np; u += 32) {
        const unsigned long long ku = S.npk()[u];
        if (it > 0 && ku <= last) continue;
        if (S.parent()[S.fst[(int)(ku & 0xffffffffu)]] != r) continue;
        if (ku < bk) {
          bk = ku;
          bi = u;
        }
      }
      for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long ok = __shfl_xor_sync(kFull, bk, off);
        const int oi = __shfl_xor_sync(kFull, bi, off);
        if (ok < bk) {
          bk = ok;
          bi = oi;
        }
      }
      if (bk == kNoKey) break;
      sel[nt++] = bi;
      last = bk;
    }
    long long bc = LLONG_MAX;
    int bcls = 3, b1 = -1, b2 = -1;
    unsigned long long bkey = 0;
    auto consider = [&](long long c, int cls, unsigned long long key, int u1, int u2) {
      if (c < bc || (c == bc && (cls < bcls || (cls == bcls && key < bkey)))) {
        bc = c;
        bcls = cls;
        bkey = key;
        b1 = u1;
        b2 = u2;
      }
    };
    if (lane == 0) consider(sparse_pattern_cost(a, S, -1, -1), 0, 0, -1, -1);
    for (int u = lane; u < n_np; u += 32) {
      const unsigned long long ku = S.npk()[u];
      if (S.parent()[S.fst[(int)(ku & 0xffffffffu)]] != r) continue;
      consider(sparse_pattern_cost(a, S, u, -1), 1, ku, u, -1);
    }
    const int npairs = nt * (nt - 1) / 2;
    for (int t = lane; t < npairs; t += 32) {
      int i = 0, rem = t;
      while (rem >= nt - 1 - i) {
        rem -= nt - 1 - i;
        ++i;
      }
      const int j = i + 1 + rem;
      consider(sparse_pattern_cost(a, S, sel[i], sel[j]), 2, (unsigned long long)(i * 16 + j),
               sel[i], sel[j]);
    }
    for (int off = 16; off > 0; off >>= 1) {
      const long long oc = __shfl_xor_sync(kFull, bc, off);
      const int ocls = __shfl_xor_sync(kFull, bcls, off);
      const unsigned long long okey = __shfl_xor_sync(kFull, bkey, off);
      const int o1 = __shfl_xor_sync(kFull, b1, off);
      const int o2 = __shfl_xor_sync(kFull, b2, off);
      consider(oc, ocls, okey, o1, o2);
    }
    if (b1 < 0) continue;  // no flip: OSD-0's local solution stands
    for (int w = lane; w < W; w += 32) {
      uint32_t delta = S.npN()[b1 * W + w];
      if (b2 >= 0) delta ^= S.npN()[b2 * W + w];
      S.xsol()[w] ^= delta;
    }
    if (lane == 0) {
      int ne = S.scal()[S_EXT];
      S.ext()[ne++] = (int)(S.npk()[b1] & 0xffffffffu);
      if (b2 >= 0) S.ext()[ne++] = (int)(S.npk()[b2] & 0xffffffffu);
      S.scal()[S_EXT] = ne;
    }
    __syncwarp();
  }
}

// Work items come from a.queue / a.count as in lsd.cu.  Shots that overflow the capacity are
// appended to spill[] (spill_count) when spill != nullptr, else reported unsolvable.
template <int CAP, int SC, bool MU, bool GLOBAL_RT>
__global__ void __launch_bounds__(128, 1) lsd_sparse_kernel(LSDArgs a, int* scratch, size_t stride,
                                                         int* spill, unsigned long long* spill_count,
                                                         const int* items, const unsigned long long* item_count) {
  using L = SLay<CAP, SC, MU>;
  constexpr int W = L::W;
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gw = blockIdx.x * (blockDim.x >> 5) + warp;
  const int m = a.g.m, n = a.g.n;
  // the spill instance keeps all of its state in its global scratch (no shared memory), so
  // that many of its warps can be resident per SM
  const size_t per_sm = GLOBAL_RT ? 0 : L::sm_total + L::rt_total;
  SShot<L> S;
  S.sm = smem + (size_t)warp * per_sm;
  int* ws = scratch + (size_t)gw * stride;
  S.dlab = ws;
  S.slot = ws + m;
  S.fst = ws + 2 * m;
  S.front = ws + 2 * m + n;
  S.rt = GLOBAL_RT ? reinterpret_cast<unsigned char*>(ws + 2 * m + 2 * n) : S.sm + L::sm_total;
  if (GLOBAL_RT) S.sm = S.rt + L::rt_total;
  // the spill instance also keeps one candidate mask per seed (up to kMaskSeeds) after its
  // other state
  const int wn_masks = GLOBAL_RT ? (n + 31) / 32 : 0;
  S.wn = 0;
  S.cmask = GLOBAL_RT ? reinterpret_cast<uint32_t*>(S.sm + L::sm_total) : nullptr;
  SGraph G{a.g.chk_ptr, a.g.chk_var, a.g.var_ptr, a.g.var_chk, a.g.max_col_deg};

  long long count;
  if (items) count = (long long)*item_count;
  else count = a.count_from_ctr ? (long long)a.ctr->lsd_count : a.count;
  unsigned long long steps_acc = 0, unsolv = 0;
  int kappa_max = 0, nu_max = 0;
  for (;;) {
    unsigned long long item = 0;
    if (lane == 0) item = atomicAdd(&a.ctr->lsd_next, 1ULL);
    item = __shfl_sync(kFull, item, 0);
    if (item >= (unsigned long long)count) break;
    const long long qi = items ? (long long)items[item] : (long long)item;
    const long long shot = a.queue ? (long long)a.queue[qi] : qi;
    const float* llr = a.llr + (a.llr_by_item ? qi : shot) * n;
    // the shot's correction: bytes, or packed words (set bits with atomicOr: lanes share words)
    uint8_t* co = a.packed ? nullptr : a.corrections + shot * n;
    uint32_t* cw = a.packed ? reinterpret_cast<uint32_t*>(a.corrections) + shot * packed_words(n)
                            : nullptr;

    // ---- init ----
    for (int d = lane; d < m; d += 32) {
      S.dlab[d] = -1;
      S.slot[d] = -1;
    }
    for (int j = lane; j < n; j += 32) S.fst[j] = -2;
    for (int sl = lane; sl < CAP; sl += 32) S.pcol()[sl] = -1;
    for (int w = lane; w < W; w += 32) {
      S.syn()[w] = 0;
      S.xsol()[w] = 0;
    }
    if (lane < 16) S.scal()[lane] = 0;
    __syncwarp();
    int ns = 0;
    for (int b0 = 0; b0 < m; b0 += 32) {
      const int d = b0 + lane;
      const bool f = d < m && syn_bit(a.syndromes, a.packed, shot, m, d) != 0;
      const unsigned bal = __ballot_sync(kFull, f);
      if (f) {
        const int k = ns + __popc(bal & ((1u << lane) - 1u));
        if (k < SC && k < CAP) {
          S.seed()[k] = d;
          S.parent()[k] = k;
          S.mark()[k] = 0u;
          S.gflag()[k] = 0;
          S.dlab[d] = k;
          S.slot[d] = k;
          S.dslot()[k] = d;
          atomicOr(&S.syn()[k >> 5], 1u << (k & 31));
        }
      }
      ns += __popc(bal);
    }
    int status = LSD_SHOT_OK_LSD, steps = 0;
    if (ns > SC || ns > CAP) status = kSpill;
    S.wn = ns <= kMaskSeeds ? wn_masks : 0;
    if (lane == 0) {
      S.scal()[S_NSEED] = min(ns, SC);
      S.scal()[S_SLOTS] = min(ns, CAP);
    }
    __syncwarp();
    for (int w = lane; w < W; w += 32) S.sred()[w] = S.syn()[w];
    // candidates next to the seeds (and each seed's candidate mask)
    if (status == LSD_SHOT_OK_LSD) {
      if (S.wn > 0) {
        for (size_t w = lane; w < (size_t)ns * S.wn; w += 32) S.cmask[w] = 0u;
        __syncwarp();
      }
      for (int k = lane; k < ns; k += 32) {
        const int d = S.seed()[k];
        uint32_t* cm = S.wn > 0 ? S.cmask + (size_t)k * S.wn : nullptr;
        for (int e = G.chk_ptr[d]; e < G.chk_ptr[d + 1]; ++e) {
          const int f = G.chk_var[e];
          if (atomicCAS(&S.fst[f], -2, -1) == -2) {
            const int q = atomicAdd(&S.scal()[S_NFRONT], 1);
            S.front[q] = f;
          }
          if (cm) atomicOr(&cm[f >> 5], 1u << (f & 31));
        }
      }
    }
    __syncwarp();
    int k = status == LSD_SHOT_OK_LSD ? ns : 0;
    if (status == LSD_SHOT_OK_LSD && lane == 0)
      for (int t = 0; t < ns; ++t) S.inv()[t] = t;
    __syncwarp();

    // ---- LSD-0 ----
    while (k > 0) {
      if (steps > n) {
        status = LSD_SHOT_UNSOLVABLE;
        break;
      }
      const int rc = sparse_step<L, MU, CAP>(G, S, llr, k, true, lane);
      if (rc == 1) {
        status = LSD_SHOT_UNSOLVABLE;
        break;
      }
      if (rc == 3) {
        status = kSpill;
        break;
      }
      ++steps;
      k = collect_invalid(S, lane);
    }
    // ---- LSD-mu ----
    if constexpr (MU) {
      if (status == LSD_SHOT_OK_LSD) {
        for (int e = 0; e < a.order; ++e) {
          k = collect_all(S, lane);
          const int rc = sparse_step<L, MU, CAP>(G, S, llr, k, false, lane);
          if (rc == 3) {
            status = kSpill;
            break;
          }
          if (rc == 2) break;
        }
        if (status == LSD_SHOT_OK_LSD) {
          if (a.osd_cs >= 0)
            sparse_osd_cs(a, S, lane);
          else
            sparse_osd_e(a, S, lane);
        }
      }
    }
    if (status == kSpill) {
      if (lane == 0) {
        if (spill) {
          const unsigned long long q = atomicAdd(spill_count, 1ULL);
          spill[q] = (int)qi;
        } else {
          if (a.status) a.status[shot] = LSD_SHOT_UNSOLVABLE;
        }
      }
      if (!spill) {
        if (cw)
          for (int w = lane; w < packed_words(n); w += 32) cw[w] = 0u;
        else
          for (int j = lane; j < n; j += 32) co[j] = 0;
        unsolv += 1;
      }
      __syncwarp();
      continue;
    }

    // ---- statistics ----
    const int nseed = S.scal()[S_NSEED];
    for (int x = lane; x < nseed; x += 32) S.mark()[x] = 0u;
    __syncwarp();
    // every fault in a cluster was a candidate first: count them from the candidate history
    // is not kept, so count over all faults of the claimed detectors' rows
    {
      const int nsl = S.scal()[S_SLOTS];
      for (int sl = lane; sl < nsl; sl += 32) {
        const int d = S.dslot()[sl];
        for (int e = G.chk_ptr[d]; e < G.chk_ptr[d + 1]; ++e) {
          const int f = G.chk_var[e];
          const int lab = S.fst[f];
          // count each clustered fault once: at its lowest claimed detector
          if (lab >= 0) {
            int lowest = INT_MAX;
            for (int q = G.var_ptr[f]; q < G.var_ptr[f + 1]; ++q) lowest = min(lowest, (int)G.var_chk[q]);
            if (lowest == d) atomicAdd(&S.mark()[S.parent()[lab]], 1u);
          }
        }
      }
    }
    __syncwarp();
    int nu = 0, kappa = 0;
    for (int x = lane; x < nseed; x += 32) {
      if (S.parent()[x] == x) {
        ++nu;
        kappa = max(kappa, (int)S.mark()[x]);
      }
    }
    for (int off = 16; off > 0; off >>= 1) {
      nu += __shfl_xor_sync(kFull, nu, off);
      kappa = max(kappa, __shfl_xor_sync(kFull, kappa, off));
    }
    for (int x = lane; x < nseed; x += 32) S.mark()[x] = 0u;

    // ---- corrections ----
    if (cw)
      for (int w = lane; w < packed_words(n); w += 32) cw[w] = 0u;
    else
      for (int j = lane; j < n; j += 32) co[j] = 0;
    __syncwarp();
    if (status == LSD_SHOT_OK_LSD) {
      auto set = [&](int j) {
        if (cw)
          atomicOr(cw + (j >> 5), 1u << (j & 31));
        else
          co[j] = 1;
      };
      const int nsl = S.scal()[S_SLOTS];
      for (int sl = lane; sl < nsl; sl += 32)
        if (bit_of(S.xsol(), sl)) set(S.pcol()[sl]);
      if constexpr (MU) {
        const int ne = S.scal()[S_EXT];
        for (int t = lane; t < ne; t += 32) set(S.ext()[t]);
      }
    }
    __syncwarp();
    if (lane == 0) {
      if (a.status) a.status[shot] = (uint8_t)status;
      if (a.shot_info) {
        a.shot_info[3 * shot] = nu;
        a.shot_info[3 * shot + 1] = kappa;
        a.shot_info[3 * shot + 2] = steps;
      }
    }
    steps_acc += steps;
    unsolv += status == LSD_SHOT_UNSOLVABLE ? 1 : 0;
    kappa_max = max(kappa_max, kappa);
    nu_max = max(nu_max, nu);
    __syncwarp();
  }
  if (lane == 0) {
    if (steps_acc) atomicAdd(&a.ctr->lsd_steps, steps_acc);
    if (unsolv) atomicAdd(&a.ctr->unsolvable, unsolv);
    atomicMax(&a.ctr->kappa_max, kappa_max);
    atomicMax(&a.ctr->nu_max, nu_max);
  }
}

constexpr int kSmallCap = 256, kSmallSeeds = 256, kBigCap = 4096, kBigSeeds = 4096;
constexpr int kSparseWarps = 4;

template <bool MU>
size_t small_smem() {
  return (size_t)kSparseWarps * (SLay<kSmallCap, kSmallSeeds, MU>::sm_total +
                                 SLay<kSmallCap, kSmallSeeds, MU>::rt_total);
}
constexpr int kBigWarpsPerSm = 4;  // spill-instance warps (one per CTA) per SM

}  // namespace

// Scratch ints per warp: dlab, slot (m each), fst, front (n each); the big instance adds the
// elimination arrays.
size_t sparse_scratch_ints(int m, int n, bool big, bool mu) {
  size_t s = (size_t)2 * m + (size_t)2 * n;
  if (big)
    s += (mu ? SLay<kBigCap, kBigSeeds, true>::rt_total + SLay<kBigCap, kBigSeeds, true>::sm_total
             : SLay<kBigCap, kBigSeeds, false>::rt_total + SLay<kBigCap, kBigSeeds, false>::sm_total) / 4 +
         (size_t)kMaskSeeds * ((n + 31) / 32);  // candidate masks
  return (s + 3) & ~(size_t)3;
}

cudaError_t sparse_config(const DevGraph& g, int order, int* grid_small, int* grid_big) {
  int dev = 0, sms = 0, max_smem = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const bool mu = order > 0;
  const void* fs = mu ? (const void*)lsd_sparse_kernel<kSmallCap, kSmallSeeds, true, false>
                      : (const void*)lsd_sparse_kernel<kSmallCap, kSmallSeeds, false, false>;
  const size_t ss = mu ? small_smem<true>() : small_smem<false>();
  if (ss > (size_t)max_smem) return cudaErrorInvalidValue;
  err = allow_max_dynamic_smem(fs, max_smem);
  if (err != cudaSuccess) return err;
  int per_sm = 0;
  err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fs, kSparseWarps * 32, ss);
  if (err != cudaSuccess) return err;
  if (per_sm < 1) return cudaErrorInvalidValue;
  *grid_small = per_sm * sms;
  *grid_big = sms * kBigWarpsPerSm;  // each spill warp holds megabytes of global scratch
  return cudaSuccess;
}

int sparse_warps_small() { return kSparseWarps; }

cudaError_t launch_sparse(const LSDArgs& a, bool big, int grid, int* scratch, size_t stride,
                          int* spill, unsigned long long* spill_count, const int* items,
                          const unsigned long long* item_count, cudaStream_t st) {
  const bool mu = a.order > 0;
  if (!big) {
    const size_t smem = mu ? small_smem<true>() : small_smem<false>();
    if (mu)
      lsd_sparse_kernel<kSmallCap, kSmallSeeds, true, false><<<grid, kSparseWarps * 32, smem, st>>>(
          a, scratch, stride, spill, spill_count, items, item_count);
    else
      lsd_sparse_kernel<kSmallCap, kSmallSeeds, false, false><<<grid, kSparseWarps * 32, smem, st>>>(
          a, scratch, stride, spill, spill_count, items, item_count);
  } else {
    if (mu)
      lsd_sparse_kernel<kBigCap, kBigSeeds, true, true><<<grid, 32, 0, st>>>(
          a, scratch, stride, nullptr, nullptr, items, item_count);
    else
      lsd_sparse_kernel<kBigCap, kBigSeeds, false, true><<<grid, 32, 0, st>>>(
          a, scratch, stride, nullptr, nullptr, items, item_count);
  }
  return cudaGetLastError();
}

}  // namespace lsdgb
