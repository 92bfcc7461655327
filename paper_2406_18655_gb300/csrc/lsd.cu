// Localized statistics decoding kernel (Alg. 1 of Sec. 4.1, on-the-fly elimination of
// Sec. 4.2, LSD-mu of App. D).
//
// One warp owns one shot; a persistent grid pulls shots from a device work queue (the
// unconverged shots BP appended, or every shot for lsd_postprocess_batch).
//
// Per-shot state in shared memory (m detectors, n faults, W = ceil(m/32), Wn = ceil(n/32)):
//   rank[n], fat[n] the reliability order: the shot's (LLR, index) keys are sorted once
//              (bitonic sort) and every later comparison is a comparison of 16-bit ranks.
//   dlab[m]    cluster label of each detector (-1: in no cluster).  Labels are the seed
//              detectors (one cluster per flipped detector, Alg. 1 init).
//   parent[m]  union-find forest over labels; a merge links the larger root under the
//              smaller one with a CAS (Alg. 2's parallel_union), so a cluster's root is its
//              smallest seed.  Labels are flattened to roots after every step.
//   flab[n]    label of the cluster a fault belongs to (-1: none).
//   cand[m][Wn] candidate set Lambda(C) of every cluster (Def. 4.3) as a bitmask over
//              ranks, so a cluster's pick is its lowest set bit.  A detector joining a
//              cluster adds its free faults; a merge ORs the masks; a fault joining a
//              cluster is cleared.  (When the masks do not fit, a scan over the free faults
//              with a 32-bit atomicMin per neighbouring cluster replaces them.)
//   R[m][W], T[m][W], pcol[m]: the elimination state of every cluster at once.  A pivot
//              column is stored at its pivot row d: R[d] is the reduced column (bit d set,
//              zero at every other pivot row), T[d] the set of pivot rows whose original
//              columns XOR to R[d], pcol[d] the fault it came from.  Rows of different
//              clusters never mix, so the factorization of a merged cluster is the union of
//              its parts: the block-swap of Sec. 4.2 is free.
//   sred[W]    s reduced by the pivots; xsol[W] the pivot rows whose columns XOR to s - sred.
//              A cluster is valid (Def. 4.2) iff sred has no bit on its rows.
//
// A growth step: every growing cluster takes its lowest-rank candidate, all picks are applied
// together, clusters that now share a detector (or a fault) are merged, then the new columns
// are eliminated one by one in rank order: b' = b + sum of R[d] over pivot rows d in supp(b)
// (one W-word XOR per nonzero of the sparse column), a new pivot at the lowest set bit of
// b', and back-elimination of that row from the other pivots.  Validity is re-read from sred.
#include <climits>

#include "lsd_internal.cuh"

namespace lsdgb {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr unsigned kNone = 0xffffffffu;
// candidate masks are used when they take at most this many bytes per warp
constexpr size_t kMaskBudget = 32 << 10;
// the Tanner graph is staged in shared memory when it takes at most this many bytes
constexpr size_t kGraphBudget = 48 << 10;

__host__ __device__ constexpr size_t al16(size_t x) { return (x + 15) & ~(size_t)15; }
__host__ __device__ constexpr int pow2_at_least(int x) {
  int p = 32;
  while (p < x) p <<= 1;
  return p;
}
__host__ __device__ constexpr size_t max_sz(size_t a, size_t b) { return a > b ? a : b; }
__host__ __device__ inline size_t graph_bytes(int m, int n, int E) {
  return al16((size_t)(m + 1 + n + 1) * 4 + (size_t)E * 4);
}

// Per-warp shared-memory layout of a size class (at most MM detectors and NN faults),
// with every offset a compile-time constant.  U holds the sort keys at init, the
// candidate masks during growth and the staged correction bytes at the end.
template <int MM, int NN, bool MU>
struct Lay {
  static constexpr int W = (MM + 31) / 32;
  static constexpr int Wn = (NN + 31) / 32;
  static constexpr int N2 = pow2_at_least(NN);
  static constexpr bool kMasks = (size_t)MM * Wn * 4 <= kMaskBudget;
  // small classes rank the keys with shuffles and need no sort buffer
  static constexpr bool kShuffleRank = NN <= 192;
  static constexpr size_t U = 0;
  static constexpr size_t R = al16(max_sz(kShuffleRank ? 0 : (size_t)N2 * 8,
                                          max_sz(kMasks ? (size_t)MM * Wn * 4 : 0, (size_t)NN)));
  static constexpr size_t T = R + (size_t)MM * W * 4;
  static constexpr size_t flab = T + (size_t)MM * W * 4;
  static constexpr size_t dlab = flab + (size_t)NN * 4;
  static constexpr size_t parent = dlab + (size_t)MM * 4;
  static constexpr size_t best = parent + (size_t)MM * 4;
  static constexpr size_t mark = best + (size_t)MM * 4;
  static constexpr size_t words = mark + (size_t)MM * 4;
  static constexpr size_t scal = words + (size_t)4 * W * 4;
  static constexpr size_t npr = scal + 16 * 4;
  static constexpr size_t npN = npr + (MU ? (size_t)NN * 4 : 0);
  static constexpr size_t ext = npN + (MU ? (size_t)NN * W * 4 : 0);
  static constexpr size_t pcol = ext + (MU ? (size_t)NN * 4 : 0);
  static constexpr size_t inv = pcol + (size_t)MM * 2;
  static constexpr size_t mlist = inv + (size_t)MM * 2;
  static constexpr size_t dnew = mlist + (size_t)MM * 2;
  static constexpr size_t newr = dnew + (size_t)MM * 2;
  static constexpr size_t srt = newr + (size_t)MM * 2;
  static constexpr size_t rank = srt + (size_t)MM * 2;
  static constexpr size_t fat = rank + (size_t)NN * 2;
  static constexpr size_t rflag = fat + (size_t)NN * 2;
  static constexpr size_t total = al16(rflag + (size_t)MM);
};

struct Graph {
  const int32_t* chk_ptr;
  const uint16_t* chk_var;
  const int32_t* var_ptr;
  const uint16_t* var_chk;
  int max_col_deg, max_row_deg;
  // lanes over (pick, detector slot) pairs in the union of a growth step: lane = pl * D + ps
  // for the largest column degree D <= 32 (ppass = 32 / D picks per pass, one slot pass);
  // beyond 32, one pick per pass and dslots = D slots in passes of 32
  int pl, ps, ppass, dslots;
  // the same over (new detector, edge slot) pairs with the largest row degree: lane =
  // dl * D + de, dpass detectors per pass, edges de, de + estep, ... of each
  int dl, de, dpass, estep;
  // log2 of the column degree rounded up to a power of two (column gathers of add_column)
  int gshift;
};

__device__ __forceinline__ void set_lanes(Graph& G, int lane) {
  const int D = max(G.max_col_deg, 1);
  if (D <= 32) {
    G.pl = lane / D;
    G.ps = lane - G.pl * D;
    G.ppass = 32 / D;
    G.dslots = 1;
  } else {
    G.pl = 0;
    G.ps = lane;
    G.ppass = 1;
    G.dslots = D;
  }
  G.gshift = 0;
  while ((1 << G.gshift) < D) ++G.gshift;
  const int Dr = max(G.max_row_deg, 1);
  if (Dr <= 32) {
    G.dl = lane / Dr;
    G.de = lane - G.dl * Dr;
    G.dpass = 32 / Dr;
    G.estep = Dr;
  } else {
    G.dl = 0;
    G.de = lane;
    G.dpass = 1;
    G.estep = 32;
  }
}

// Accessors of one warp's shot state: one base pointer plus compile-time offsets.
template <class L>
struct Shot {
  unsigned char* base;
  template <class T>
  __device__ __forceinline__ T* at(size_t off) const {
    return reinterpret_cast<T*>(base + off);
  }
  __device__ __forceinline__ unsigned long long* keys() const { return at<unsigned long long>(L::U); }
  __device__ __forceinline__ uint32_t* cand() const { return at<uint32_t>(L::U); }
  __device__ __forceinline__ uint8_t* cs() const { return at<uint8_t>(L::U); }
  __device__ __forceinline__ uint32_t* R() const { return at<uint32_t>(L::R); }
  __device__ __forceinline__ uint32_t* T() const { return at<uint32_t>(L::T); }
  __device__ __forceinline__ int* flab() const { return at<int>(L::flab); }
  __device__ __forceinline__ int* dlab() const { return at<int>(L::dlab); }
  __device__ __forceinline__ int* parent() const { return at<int>(L::parent); }
  __device__ __forceinline__ int16_t* pcol() const { return at<int16_t>(L::pcol); }
  __device__ __forceinline__ uint32_t* best() const { return at<uint32_t>(L::best); }
  __device__ __forceinline__ unsigned* mark() const { return at<unsigned>(L::mark); }
  __device__ __forceinline__ uint16_t* inv() const { return at<uint16_t>(L::inv); }
  __device__ __forceinline__ uint16_t* mlist() const { return at<uint16_t>(L::mlist); }
  __device__ __forceinline__ uint16_t* dnew() const { return at<uint16_t>(L::dnew); }
  __device__ __forceinline__ uint16_t* newr() const { return at<uint16_t>(L::newr); }
  __device__ __forceinline__ uint16_t* srt() const { return at<uint16_t>(L::srt); }
  __device__ __forceinline__ uint32_t* syn() const { return at<uint32_t>(L::words); }
  __device__ __forceinline__ uint32_t* sred() const { return at<uint32_t>(L::words + L::W * 4); }
  __device__ __forceinline__ uint32_t* xsol() const { return at<uint32_t>(L::words + 2 * L::W * 4); }
  __device__ __forceinline__ uint32_t* cm() const { return at<uint32_t>(L::words + 3 * L::W * 4); }
  __device__ __forceinline__ int* scal() const { return at<int>(L::scal); }
  __device__ __forceinline__ uint32_t* npr() const { return at<uint32_t>(L::npr); }
  __device__ __forceinline__ uint32_t* npN() const { return at<uint32_t>(L::npN); }
  __device__ __forceinline__ int* ext() const { return at<int>(L::ext); }
  __device__ __forceinline__ uint16_t* rank() const { return at<uint16_t>(L::rank); }
  __device__ __forceinline__ uint16_t* fat() const { return at<uint16_t>(L::fat); }
  __device__ __forceinline__ unsigned char* rflag() const { return at<unsigned char>(L::rflag); }
};

// Order key of fault j: (LLR ascending, index ascending).  -0.0 is folded into +0.0 so that
// the key order is the float order, with ties broken by the index.
__device__ __forceinline__ unsigned llr_bits(float x) {
  x = __fadd_rn(x, 0.0f);
  const unsigned u = __float_as_uint(x);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ unsigned long long llr_key(float x, int j) {
  return ((unsigned long long)llr_bits(x) << 32) | (unsigned)j;
}

__device__ __forceinline__ int uf_find(const volatile int* parent, int x) {
  int p = parent[x];
  while (p != x) {
    x = p;
    p = parent[x];
  }
  return x;
}

// Union of the sets of a and b; a root that gets linked under another is recorded in the
// merged list so that its candidate mask can be folded into the new root.
template <class L>
__device__ __forceinline__ void uf_unite(const Shot<L>& S, int a, int b) {
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
      const int slot = atomicAdd(&S.scal()[3], 1);
      S.mlist()[slot] = (uint16_t)a;
      return;
    }
  }
}

__device__ __forceinline__ bool bit_of(const uint32_t* v, int i) {
  return (v[i >> 5] >> (i & 31)) & 1u;
}

// Bitonic sort of keys[0..N2) ascending (one warp).
template <int N2>
__device__ void warp_sort(unsigned long long* keys, int lane) {
#pragma unroll 1
  for (int k = 2; k <= N2; k <<= 1) {
#pragma unroll 1
    for (int j = k >> 1; j > 0; j >>= 1) {
#pragma unroll
      for (int i0 = 0; i0 < N2; i0 += 32) {
        const int i = i0 + lane;
        const int ixj = i ^ j;
        if (ixj > i) {
          const unsigned long long x = keys[i], y = keys[ixj];
          const bool up = (i & k) == 0;
          if ((x > y) == up) {
            keys[i] = y;
            keys[ixj] = x;
          }
        }
      }
      __syncwarp();
    }
  }
}

// Roots of all clusters, or of the invalid ones, into inv[].  A cluster is invalid iff the
// reduced syndrome has a bit on one of its rows (labels are flattened, so dlab of a row is
// its cluster's root); each such root is listed once, in no particular order (growth is
// synchronous, so the order of the list does not matter).
template <class L>
__device__ int collect_roots(const LSDArgs& a, const Shot<L>& S, int m, bool only_invalid,
                             int lane) {
  if (only_invalid && L::W <= 4) {
    // each invalid row marks its root in a bitmask over labels (cm, free until reprocessing);
    // the roots are then listed in ascending order by ballots, and the mask is cleared
    uint32_t* msk = S.cm();
#pragma unroll
    for (int i = 0; i < L::W; ++i) {
      const int d = lane + 32 * i;
      if ((S.sred()[i] >> lane) & 1u) {
        const int root = S.dlab()[d];
        if (root >= 0) atomicOr(&msk[root >> 5], 1u << (root & 31));
      }
    }
    __syncwarp();
    uint32_t mw[L::W];
#pragma unroll
    for (int i = 0; i < L::W; ++i) mw[i] = msk[i];
    __syncwarp();
    if (lane < L::W) msk[lane] = 0;
    int count = 0;
#pragma unroll
    for (int i = 0; i < L::W; ++i) {
      if ((mw[i] >> lane) & 1u) S.inv()[count + __popc(mw[i] & ((1u << lane) - 1u))] = (uint16_t)(lane + 32 * i);
      count += __popc(mw[i]);
    }
    __syncwarp();
    return count;
  }
  if (only_invalid) {
    if (lane == 0) S.scal()[5] = 0;
    __syncwarp();
    if (lane < L::W) {
      uint32_t bits = S.sred()[lane];
      while (bits) {
        const int d = lane * 32 + __ffs(bits) - 1;
        bits &= bits - 1;
        const int root = S.dlab()[d];
        if (root >= 0 && atomicCAS(&S.mark()[root], 0u, 1u) == 0u) {
          const int slot = atomicAdd(&S.scal()[5], 1);
          S.inv()[slot] = (uint16_t)root;
        }
      }
    }
    __syncwarp();
    const int count = S.scal()[5];
    for (int t = lane; t < count; t += 32) S.mark()[S.inv()[t]] = 0u;
    __syncwarp();
    return count;
  }
  int count = 0;
  for (int base = 0; base < m; base += 32) {
    const int d = base + lane;
    const bool seed = d < m && (a.single_cluster ? d == 0 : bit_of(S.syn(), d));
    const bool pred = seed && S.parent()[d] == d;
    const unsigned bal = __ballot_sync(kFull, pred);
    if (pred) S.inv()[count + __popc(bal & ((1u << lane) - 1u))] = (uint16_t)d;
    count += __popc(bal);
  }
  __syncwarp();
  return count;
}

// Adds the fault of rank `rk` to its cluster's factorization.
template <class L, bool MU>
__device__ void add_column(const Graph& G, const Shot<L>& S, int m, int rk, int gcol, int q0,
                           int q1, int lane) {
  constexpr int W = L::W;
  uint32_t bw = 0, tw = 0;
  if ((W << G.gshift) <= 32) {
    // lane (word wd, detector slot sl) reads one detector's contribution to one word; the
    // 2^gshift slots of a word are XOR-reduced with shuffles and word w lands on lane w
    const int wd = lane >> G.gshift, sl = lane & ((1 << G.gshift) - 1);
    if (wd < W) {
      const int q = q0 + sl;
      if (q < q1) {
        const int d = G.var_chk[q];
        if ((d >> 5) == wd) bw = 1u << (d & 31);
        if (S.pcol()[d] >= 0) {
          bw ^= S.R()[d * W + wd];
          tw = S.T()[d * W + wd];
        }
      }
    }
    for (int off = 1; off < (1 << G.gshift); off <<= 1) {
      bw ^= __shfl_xor_sync(kFull, bw, off);
      tw ^= __shfl_xor_sync(kFull, tw, off);
    }
    bw = __shfl_sync(kFull, bw, (lane << G.gshift) & 31);
    tw = __shfl_sync(kFull, tw, (lane << G.gshift) & 31);
    if (lane >= W) bw = tw = 0;
  } else if (lane < W) {
    for (int q = q0; q < q1; ++q) {
      const int d = G.var_chk[q];
      if ((d >> 5) == lane) bw ^= 1u << (d & 31);
      if (S.pcol()[d] >= 0) {
        bw ^= S.R()[d * W + lane];
        tw ^= S.T()[d * W + lane];
      }
    }
  }
  const unsigned nz = __ballot_sync(kFull, lane < W && bw != 0);
  if (nz == 0) {
    // dependent column: remember its representation for LSD-mu's OSD-E
    if constexpr (MU) {
      const int slot = __shfl_sync(kFull, S.scal()[1], 0);
      if (lane < W) S.npN()[slot * W + lane] = tw;
      __syncwarp();
      if (lane == 0) {
        S.npr()[slot] = (uint32_t)rk;
        S.scal()[1] = slot + 1;
      }
      __syncwarp();
    }
    return;
  }
  const int wl = __ffs(nz) - 1;
  const uint32_t word = __shfl_sync(kFull, bw, wl);
  const int p = wl * 32 + __ffs(word) - 1;
  const int pw = p >> 5;
  const uint32_t pb = 1u << (p & 31);
  if (lane == pw) tw ^= pb;
  const bool sflag = (S.sred()[pw] & pb) != 0;
  if (lane < W) {
    S.R()[p * W + lane] = bw;
    S.T()[p * W + lane] = tw;
  }
  if (lane == 0) S.pcol()[p] = (int16_t)gcol;
  __syncwarp();
  if constexpr (W <= 4) {
    // back-elimination with the new pivot's words taken from the lanes that hold them and
    // every row's test issued before the row updates
    uint32_t rp[W], tp[W];
#pragma unroll
    for (int w = 0; w < W; ++w) {
      rp[w] = __shfl_sync(kFull, bw, w);
      tp[w] = __shfl_sync(kFull, tw, w);
    }
    bool hit[W];
#pragma unroll
    for (int i = 0; i < W; ++i) {
      const int d = lane + 32 * i;
      hit[i] = d < m && d != p && S.pcol()[d] >= 0 && (S.R()[d * W + pw] & pb) != 0;
    }
#pragma unroll
    for (int i = 0; i < W; ++i) {
      if (hit[i]) {
        const int d = lane + 32 * i;
#pragma unroll
        for (int w = 0; w < W; ++w) {
          S.R()[d * W + w] ^= rp[w];
          S.T()[d * W + w] ^= tp[w];
        }
      }
    }
  } else {
    for (int d = lane; d < m; d += 32) {
      if (d == p || S.pcol()[d] < 0) continue;
      if (S.R()[d * W + pw] & pb) {
#pragma unroll
        for (int w = 0; w < W; ++w) {
          S.R()[d * W + w] ^= S.R()[p * W + w];
          S.T()[d * W + w] ^= S.T()[p * W + w];
        }
      }
    }
  }
  if (sflag && lane < W) {
    S.sred()[lane] ^= bw;
    S.xsol()[lane] ^= tw;
  }
  __syncwarp();
}

// add_column for the fault of rank rk (its column and CSC range read from shared memory).
template <class L, bool MU>
__device__ __forceinline__ void add_column(const Graph& G, const Shot<L>& S, int m, int rk,
                                           int lane) {
  const int gcol = S.fat()[rk];
  add_column<L, MU>(G, S, m, rk, gcol, G.var_ptr[gcol], G.var_ptr[gcol + 1], lane);
}

// The growth step of lsd_step when the clusters' candidate masks are kept and at most 32
// clusters grow: lane t carries cluster inv[t]'s pick (rank, fault, CSC range) from the
// search through the union to the column order, instead of passing it through shared memory.
// Same result as the general step: the merges, claims and mask updates commute.
template <class L, bool MU>
__device__ int lsd_step_small(const Graph& G, const Shot<L>& S, int m, int k, bool strict,
                              int lane) {
  constexpr int Wn = L::Wn;
  // ---- find_candidate: the lowest set bit of the cluster's mask ----
  int r = 0;
  unsigned pick = kNone;
  if (lane < k) {
    r = S.inv()[lane];
    const uint32_t* c = S.cand() + (size_t)r * Wn;
    if constexpr (Wn <= 8) {
      uint32_t v[Wn];
#pragma unroll
      for (int w = 0; w < Wn; ++w) v[w] = c[w];
#pragma unroll
      for (int w = Wn - 1; w >= 0; --w)
        if (v[w]) pick = (unsigned)(w * 32 + __ffs(v[w]) - 1);
    } else {
      for (int w = 0; w < Wn; ++w) {
        const uint32_t v = c[w];
        if (v) {
          pick = (unsigned)(w * 32 + __ffs(v) - 1);
          break;
        }
      }
    }
  }
  const bool has = pick != kNone;
  const unsigned hb = __ballot_sync(kFull, has);
  const unsigned all = k == 32 ? kFull : ((1u << k) - 1u);
  const bool none = hb != all;
  if ((strict && none) || hb == 0) return (strict && none) ? 1 : 2;
  if (lane == 0) S.scal()[3] = 0;  // merged labels
  __syncwarp();
  // ---- parallel_union ----
  const unsigned below = (1u << lane) - 1u;
  int gcol = 0, q0 = 0, q1 = 0;
  bool fresh = false;
  if (has) {
    gcol = S.fat()[pick];
    const int old = atomicCAS(&S.flab()[gcol], -1, r);
    fresh = old == -1;
    if (!fresh) uf_unite(S, r, old);
    q0 = G.var_ptr[gcol];
    q1 = G.var_ptr[gcol + 1];
  }
  const unsigned bf = __ballot_sync(kFull, fresh);
  const int n_new = __popc(bf);
  int n_det = 0;
  for (int tb = 0; tb < k; tb += G.ppass) {
    const int src = tb + G.pl;
    const int rs = __shfl_sync(kFull, r, src & 31);
    const int qs0 = __shfl_sync(kFull, q0, src & 31);
    const int qs1 = __shfl_sync(kFull, q1, src & 31);
    for (int so = 0; so < G.dslots; so += 32) {
      const int q = qs0 + G.ps + so;
      int d = 0;
      bool claim = false;
      if (G.pl < G.ppass && src < k && q < qs1) {
        d = G.var_chk[q];
        const int o = atomicCAS(&S.dlab()[d], -1, rs);
        claim = o == -1;
        if (!claim && o != rs) uf_unite(S, rs, o);
      }
      const unsigned bd = __ballot_sync(kFull, claim);
      if (claim) S.dnew()[n_det + __popc(bd & below)] = (uint16_t)d;
      n_det += __popc(bd);
    }
  }
  __syncwarp();
  // ---- flatten labels to roots; only after a merge ----
  const int merged = S.scal()[3];
  if (merged) {
    for (int x = lane; x < m; x += 32) {
      const int root = uf_find(S.parent(), x);
      S.parent()[x] = root;
      const int l = S.dlab()[x];
      if (l >= 0) S.dlab()[x] = uf_find(S.parent(), l);
    }
    __syncwarp();
  }
  // ---- masks: fold merged labels into their roots, add the new detectors' free faults ----
  for (int idx = lane; idx < merged * Wn; idx += 32) {
    const int x = S.mlist()[idx / Wn], w = idx % Wn;
    const uint32_t v = S.cand()[(size_t)x * Wn + w];
    if (v) atomicOr(&S.cand()[(size_t)S.parent()[x] * Wn + w], v);
  }
  for (int tb = 0; tb < n_det; tb += G.dpass) {
    const int t = tb + G.dl;
    if (G.dl < G.dpass && t < n_det) {
      const int d = S.dnew()[t];
      uint32_t* c = S.cand() + (size_t)S.dlab()[d] * Wn;
      const int c1 = G.chk_ptr[d + 1];
      for (int e = G.chk_ptr[d] + G.de; e < c1; e += G.estep) {
        const int f = G.chk_var[e];
        if (S.flab()[f] < 0) {
          const unsigned rk = S.rank()[f];
          atomicOr(&c[rk >> 5], 1u << (rk & 31));
        }
      }
    }
  }
  __syncwarp();
  // the step's new faults are no longer candidates (a fresh pick's fault carries label r)
  if (fresh) {
    const int root = S.parent()[r];
    atomicAnd(&S.cand()[(size_t)root * Wn + (pick >> 5)], ~(1u << (pick & 31)));
  }
  __syncwarp();
  // ---- the new columns in rank order: the warp minimum of the fresh picks, n_new times ----
  unsigned kt = fresh ? pick : kNone;
  for (int t = 0; t < n_new; ++t) {
    const unsigned v = __reduce_min_sync(kFull, kt);
    const int src = __ffs(__ballot_sync(kFull, kt == v)) - 1;
    if (kt == v) kt = kNone;
    add_column<L, MU>(G, S, m, (int)v, __shfl_sync(kFull, gcol, src),
                      __shfl_sync(kFull, q0, src), __shfl_sync(kFull, q1, src), lane);
  }
  return 0;
}

// One synchronous growth step of the k clusters listed in inv[].
// Returns 0 if clusters grew, 1 if strict and a cluster had no candidate, 2 if none grew.
template <class L, bool MU>
__device__ int lsd_step(const Graph& G, const Shot<L>& S, int m, int n, int k, bool strict,
                        int lane) {
  constexpr int Wn = L::Wn;
  if constexpr (L::kMasks)
    if (k <= 32) return lsd_step_small<L, MU>(G, S, m, k, strict, lane);
  // ---- find_candidate: the lowest-rank candidate of every growing cluster ----
  if constexpr (L::kMasks) {
    for (int t = lane; t < k; t += 32) {
      const int r = S.inv()[t];
      const uint32_t* c = S.cand() + (size_t)r * Wn;
      unsigned pick = kNone;
      for (int w = 0; w < Wn; ++w) {
        const uint32_t v = c[w];
        if (v) {
          pick = (unsigned)(w * 32 + __ffs(v) - 1);
          break;
        }
      }
      S.best()[r] = pick;
    }
    __syncwarp();
  } else {
    for (int t = lane; t < k; t += 32) {
      const int r = S.inv()[t];
      S.best()[r] = kNone;
      S.rflag()[r] = 1;
    }
    __syncwarp();
    for (int j = lane; j < n; j += 32) {
      if (S.flab()[j] >= 0) continue;
      const unsigned rk = S.rank()[j];
      const int v1 = G.var_ptr[j + 1];
      for (int q = G.var_ptr[j]; q < v1; ++q) {
        const int lab = S.dlab()[G.var_chk[q]];
        if (lab >= 0 && S.rflag()[lab]) atomicMin(&S.best()[lab], rk);
      }
    }
    __syncwarp();
    for (int t = lane; t < k; t += 32) S.rflag()[S.inv()[t]] = 0;
  }
  bool none = false, some = false;
  for (int t = lane; t < k; t += 32) {
    if (S.best()[S.inv()[t]] == kNone) none = true;
    else some = true;
  }
  none = __any_sync(kFull, none);
  some = __any_sync(kFull, some);
  if ((strict && none) || !some) {
    __syncwarp();
    return (strict && none) ? 1 : 2;
  }
  if (lane == 0) S.scal()[3] = 0;  // merged labels
  __syncwarp();
  // ---- parallel_union: apply every pick, merge clusters sharing a detector or a fault ----
  // (the lists of new faults and newly claimed detectors are filled by ballots)
  const unsigned below = (1u << lane) - 1u;
  int n_new = 0, n_det = 0;
  for (int base = 0; base < k; base += 32) {
    const int t = base + lane;
    const int r = t < k ? S.inv()[t] : 0;
    const unsigned rk = t < k ? S.best()[r] : kNone;
    const bool pick = rk != kNone;
    int gcol = 0, q0 = 0, q1 = 0;
    bool fresh = false;
    if (pick) {
      gcol = S.fat()[rk];
      const int old = atomicCAS(&S.flab()[gcol], -1, r);
      fresh = old == -1;
      if (!fresh) uf_unite(S, r, old);
      q0 = G.var_ptr[gcol];
      q1 = G.var_ptr[gcol + 1];
    }
    const unsigned bf = __ballot_sync(kFull, fresh);
    if (fresh) S.newr()[n_new + __popc(bf & below)] = (uint16_t)rk;
    n_new += __popc(bf);
    // the picks' detectors: lane (pick pl, slot ps) claims detector ps of pick tb + pl, so a
    // pass covers ppass picks (the pick's owner lane passes its cluster and column range)
    const int cnt = min(32, k - base);
    for (int tb = 0; tb < cnt; tb += G.ppass) {
      const int src = tb + G.pl;
      const int rs = __shfl_sync(kFull, r, src & 31);
      const int qs0 = __shfl_sync(kFull, q0, src & 31);
      const int qs1 = __shfl_sync(kFull, q1, src & 31);
      for (int so = 0; so < G.dslots; so += 32) {
        const int q = qs0 + G.ps + so;
        int d = 0;
        bool claim = false;
        if (G.pl < G.ppass && src < cnt && q < qs1) {
          d = G.var_chk[q];
          const int o = atomicCAS(&S.dlab()[d], -1, rs);
          claim = o == -1;
          if (!claim && o != rs) uf_unite(S, rs, o);
        }
        const unsigned bd = __ballot_sync(kFull, claim);
        if (claim) S.dnew()[n_det + __popc(bd & below)] = (uint16_t)d;
        n_det += __popc(bd);
      }
    }
  }
  __syncwarp();
  // ---- flatten labels to roots (later finds take one step); only after a merge ----
  const int merged = S.scal()[3];
  if (merged) {
    for (int x = lane; x < m; x += 32) {
      const int root = uf_find(S.parent(), x);
      S.parent()[x] = root;
      const int l = S.dlab()[x];
      if (l >= 0) S.dlab()[x] = uf_find(S.parent(), l);
    }
    __syncwarp();
  }
  if constexpr (L::kMasks) {
    // fold the masks of merged labels into their roots; add the free faults next to the
    // newly claimed detectors
    const int nm = merged, nd = n_det;
    for (int idx = lane; idx < nm * Wn; idx += 32) {
      const int x = S.mlist()[idx / Wn], w = idx % Wn;
      const uint32_t v = S.cand()[(size_t)x * Wn + w];
      if (v) atomicOr(&S.cand()[(size_t)S.parent()[x] * Wn + w], v);
    }
    // lanes over (new detector, edge slot) pairs
    for (int tb = 0; tb < nd; tb += G.dpass) {
      const int t = tb + G.dl;
      if (G.dl < G.dpass && t < nd) {
        const int d = S.dnew()[t];
        uint32_t* c = S.cand() + (size_t)S.dlab()[d] * Wn;
        const int c1 = G.chk_ptr[d + 1];
        for (int e = G.chk_ptr[d] + G.de; e < c1; e += G.estep) {
          const int f = G.chk_var[e];
          if (S.flab()[f] < 0) {
            const unsigned rk = S.rank()[f];
            atomicOr(&c[rk >> 5], 1u << (rk & 31));
          }
        }
      }
    }
    __syncwarp();
    // the step's new faults are no longer candidates
    const int nn = n_new;
    for (int t = lane; t < nn; t += 32) {
      const unsigned rk = S.newr()[t];
      const int root = S.parent()[S.flab()[S.fat()[rk]]];
      atomicAnd(&S.cand()[(size_t)root * Wn + (rk >> 5)], ~(1u << (rk & 31)));
    }
    __syncwarp();
  }
  // ---- the step's new columns in reliability (rank) order ----
  if (n_new <= 32) {  // lane t holds new column t; the warp minimum is taken n_new times
    unsigned kt = lane < n_new ? (unsigned)S.newr()[lane] : kNone;
    for (int t = 0; t < n_new; ++t) {
      const unsigned v = __reduce_min_sync(kFull, kt);
      if (kt == v) kt = kNone;
      add_column<L, MU>(G, S, m, (int)v, lane);
    }
    return 0;
  }
  for (int t = lane; t < n_new; t += 32) {
    const unsigned kt = S.newr()[t];
    int pos = 0;
    for (int u = 0; u < n_new; ++u) pos += (S.newr()[u] < kt) ? 1 : 0;
    S.srt()[pos] = (uint16_t)kt;
  }
  __syncwarp();
  for (int t = 0; t < n_new; ++t) add_column<L, MU>(G, S, m, (int)S.srt()[t], lane);
  return 0;
}

// LSD-mu reprocessing (App. D): exhaustive OSD over the first min(mu, #dependent) dependent
// columns of each cluster, in reliability order; cost = sum of 2^-32 fixed-point channel
// weights; ties go to the smaller pattern.  Updates xsol and appends the chosen dependent
// columns to ext[].
template <class L>
__device__ void osd_e(const LSDArgs& a, const Shot<L>& S, int m, int lane) {
  constexpr int W = L::W;
  const long long* wfix = a.g.wfix;
  const int order = a.order;
  const int nroots = collect_roots(a, S, m, false, lane);
  const int n_np = S.scal()[1];
  for (int ci = 0; ci < nroots; ++ci) {
    const int r = S.inv()[ci];
#pragma unroll
    for (int c = 0; c < W; ++c) {
      const int d = c * 32 + lane;
      const bool in = d < m && S.dlab()[d] == r;
      const unsigned bal = __ballot_sync(kFull, in);
      if (lane == 0) S.cm()[c] = bal;
    }
    __syncwarp();
    int sel[kMaxOrder];
    int nt = 0;
    unsigned last = 0;
    for (int it = 0; it < order; ++it) {
      unsigned bk = kNone;
      int bi = -1;
      for (int u = lane; u < n_np; u += 32) {
        const unsigned ku = S.npr()[u];
        if (it > 0 && ku <= last) continue;
        if (S.parent()[S.flab()[S.fat()[ku]]] != r) continue;
        if (ku < bk) {
          bk = ku;
          bi = u;
        }
      }
      for (int off = 16; off > 0; off >>= 1) {
        const unsigned ok = __shfl_xor_sync(kFull, bk, off);
        const int oi = __shfl_xor_sync(kFull, bi, off);
        if (ok < bk) {
          bk = ok;
          bi = oi;
        }
      }
      if (bk == kNone) break;
      sel[nt++] = bi;
      last = bk;
    }
    if (nt == 0) continue;
    long long bcost = LLONG_MAX;
    int bt = 0;
    for (int t = lane; t < (1 << nt); t += 32) {
      long long cost = 0;
#pragma unroll
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
        if ((t >> k2) & 1) cost += wfix[S.fat()[S.npr()[sel[k2]]]];
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
    if (lane < W) {
      uint32_t delta = 0;
      for (int k2 = 0; k2 < nt; ++k2)
        if ((bt >> k2) & 1) delta ^= S.npN()[sel[k2] * W + lane];
      S.xsol()[lane] ^= delta;
    }
    if (lane == 0) {
      int ne = S.scal()[2];
      for (int k2 = 0; k2 < nt; ++k2)
        if ((bt >> k2) & 1) S.ext()[ne++] = S.fat()[S.npr()[sel[k2]]];
      S.scal()[2] = ne;
    }
    __syncwarp();
  }
}

// Cost of cluster r's local solution (xsol masked by cm) with the dependent columns of slots
// u1 and u2 flipped (-1 = none).
template <class L>
__device__ __forceinline__ long long pattern_cost(const LSDArgs& a, const Shot<L>& S, int u1,
                                                  int u2) {
  constexpr int W = L::W;
  const long long* wfix = a.g.wfix;
  long long cost = 0;
#pragma unroll
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
  if (u1 >= 0) cost += wfix[S.fat()[S.npr()[u1]]];
  if (u2 >= 0) cost += wfix[S.fat()[S.npr()[u2]]];
  return cost;
}

// LSD-mu reprocessing with the combination sweep OSD-CS-w (App. D's BB experiment): per
// cluster the patterns are no flip, every single dependent column, and every pair among the
// first w dependent columns in reliability order; the least cost wins, ties going to the
// earlier pattern in that order.  A pattern is ranked by (cost, class, key): class 0 = no
// flip, 1 = single (key = the column's rank), 2 = pair (key = i * 16 + j).
template <class L>
__device__ void osd_cs(const LSDArgs& a, const Shot<L>& S, int m, int lane) {
  constexpr int W = L::W;
  const int nroots = collect_roots(a, S, m, false, lane);
  const int n_np = S.scal()[1];
  const int w_cs = a.osd_cs;
  for (int ci = 0; ci < nroots; ++ci) {
    const int r = S.inv()[ci];
#pragma unroll
    for (int c = 0; c < W; ++c) {
      const int d = c * 32 + lane;
      const bool in = d < m && S.dlab()[d] == r;
      const unsigned bal = __ballot_sync(kFull, in);
      if (lane == 0) S.cm()[c] = bal;
    }
    __syncwarp();
    // the first w dependent columns of the cluster, by repeated minimum over the ranks
    int sel[kMaxCsOrder];
    int nt = 0;
    unsigned last = 0;
    for (int it = 0; it < w_cs; ++it) {
      unsigned bk = kNone;
      int bi = -1;
      for (int u = lane; u < n_np; u += 32) {
        const unsigned ku = S.npr()[u];
        if (it > 0 && ku <= last) continue;
        if (S.parent()[S.flab()[S.fat()[ku]]] != r) continue;
        if (ku < bk) {
          bk = ku;
          bi = u;
        }
      }
      for (int off = 16; off > 0; off >>= 1) {
        const unsigned ok = __shfl_xor_sync(kFull, bk, off);
        const int oi = __shfl_xor_sync(kFull, bi, off);
        if (ok < bk) {
          bk = ok;
          bi = oi;
        }
      }
      if (bk == kNone) break;
      sel[nt++] = bi;
      last = bk;
    }
    long long bc = LLONG_MAX;
    int bcls = 3, bkey = 0, b1 = -1, b2 = -1;
    auto consider = [&](long long c, int cls, int key, int u1, int u2) {
      if (c < bc || (c == bc && (cls < bcls || (cls == bcls && key < bkey)))) {
        bc = c;
        bcls = cls;
        bkey = key;
        b1 = u1;
        b2 = u2;
      }
    };
    if (lane == 0) consider(pattern_cost(a, S, -1, -1), 0, 0, -1, -1);
    for (int u = lane; u < n_np; u += 32) {
      const unsigned ku = S.npr()[u];
      if (S.parent()[S.flab()[S.fat()[ku]]] != r) continue;
      consider(pattern_cost(a, S, u, -1), 1, (int)ku, u, -1);
    }
    const int npairs = nt * (nt - 1) / 2;
    for (int t = lane; t < npairs; t += 32) {
      int i = 0, rem = t;
      while (rem >= nt - 1 - i) {
        rem -= nt - 1 - i;
        ++i;
      }
      const int j = i + 1 + rem;
      consider(pattern_cost(a, S, sel[i], sel[j]), 2, i * 16 + j, sel[i], sel[j]);
    }
    for (int off = 16; off > 0; off >>= 1) {
      const long long oc = __shfl_xor_sync(kFull, bc, off);
      const int ocls = __shfl_xor_sync(kFull, bcls, off);
      const int okey = __shfl_xor_sync(kFull, bkey, off);
      const int o1 = __shfl_xor_sync(kFull, b1, off);
      const int o2 = __shfl_xor_sync(kFull, b2, off);
      consider(oc, ocls, okey, o1, o2);
    }
    if (b1 < 0) continue;  // no flip: OSD-0's local solution stands
    if (lane < W) {
      uint32_t delta = S.npN()[b1 * W + lane];
      if (b2 >= 0) delta ^= S.npN()[b2 * W + lane];
      S.xsol()[lane] ^= delta;
    }
    if (lane == 0) {
      int ne = S.scal()[2];
      S.ext()[ne++] = S.fat()[S.npr()[b1]];
      if (b2 >= 0) S.ext()[ne++] = S.fat()[S.npr()[b2]];
      S.scal()[2] = ne;
    }
    __syncwarp();
  }
}

// Per-warp running statistics of the shots a warp decodes.
struct LsdAcc {
  unsigned long long steps = 0, unsolvable = 0;
  int kappa_max = 0, nu_max = 0;
};

__device__ __forceinline__ void lsd_flush(const LSDArgs& a, const LsdAcc& acc, int lane) {
  if (lane == 0) {
    if (acc.steps) atomicAdd(&a.ctr->lsd_steps, acc.steps);
    if (acc.unsolvable) atomicAdd(&a.ctr->unsolvable, acc.unsolvable);
    atomicMax(&a.ctr->kappa_max, acc.kappa_max);
    atomicMax(&a.ctr->nu_max, acc.nu_max);
  }
}

// LSD (Alg. 1, LSD-mu of App. D) of one shot by one warp: lsrc = the shot's soft
// information (global or shared memory), ssrc = its syndrome; writes its correction and
// status.
template <int MM, int NN, bool MU, bool PK>
__device__ __forceinline__ void lsd_shot(const LSDArgs& a, const Graph& G,
                                         const Shot<Lay<MM, NN, MU>>& S, const float* lsrc,
                                         const uint8_t* ssrc, long long shot, int lane,
                                         LsdAcc& acc) {
  using L = Lay<MM, NN, MU>;
  constexpr int W = L::W, Wn = L::Wn, N2 = L::N2;
  const int m = a.g.m, n = a.g.n;
  // ---- the shot's reliability order ----
  if constexpr (L::kShuffleRank) {
    // rank of fault j = number of keys (bits', j') before (bits, j), counted with shuffles
    // of the 32-bit LLR bits; the index tie-break is known from the positions: fault
    // j' = src + 32 t2 precedes j = lane + 32 t on equal bits iff t2 < t, or t2 == t and
    // src < lane.  Padding entries (j >= n) carry the largest bits and the largest index.
    constexpr int KPL = (NN + 31) / 32;
    unsigned myk[KPL];
    int rk[KPL];
#pragma unroll
    for (int t = 0; t < KPL; ++t) {
      const int j = lane + 32 * t;
      myk[t] = j < n ? llr_bits(lsrc[j]) : 0xffffffffu;
      rk[t] = 0;
    }
#pragma unroll 1
    for (int src = 0; src < 32; ++src) {
      const bool before = src < lane;
#pragma unroll
      for (int t2 = 0; t2 < KPL; ++t2) {
        const unsigned other = __shfl_sync(kFull, myk[t2], src);
#pragma unroll
        for (int t = 0; t < KPL; ++t) {
          if (t2 < t) rk[t] += (other <= myk[t]) ? 1 : 0;
          else if (t2 > t) rk[t] += (other < myk[t]) ? 1 : 0;
          else rk[t] += (other < myk[t] || (before && other == myk[t])) ? 1 : 0;
        }
      }
    }
#pragma unroll
    for (int t = 0; t < KPL; ++t) {
      const int j = lane + 32 * t;
      if (j < n) {
        S.rank()[j] = (uint16_t)rk[t];
        S.fat()[rk[t]] = (uint16_t)j;
      }
    }
  } else {
#pragma unroll
    for (int j0 = 0; j0 < N2; j0 += 32) {
      const int j = j0 + lane;
      S.keys()[j] = j < n ? llr_key(lsrc[j], j) : ~0ull;
    }
    __syncwarp();
    warp_sort<N2>(S.keys(), lane);
    for (int r = lane; r < n; r += 32) {
      const int j = (int)(S.keys()[r] & 0xffffffffu);
      S.fat()[r] = (uint16_t)j;
      S.rank()[j] = (uint16_t)r;
    }
  }
  __syncwarp();

  // ---- init: one cluster per flipped detector ----
  // (candidate masks are read only for cluster roots, which are seeds: each seed's lane
  // clears its mask below; the single cluster's mask is cleared here)
  if constexpr (L::kMasks)
    if (a.single_cluster && lane < Wn) S.cand()[lane] = 0;
  for (int j = lane; j < n; j += 32) S.flab()[j] = -1;
  for (int d = lane; d < m; d += 32) {
    S.dlab()[d] = -1;
    S.parent()[d] = d;
    S.pcol()[d] = -1;
    S.rflag()[d] = 0;
    S.mark()[d] = 0u;
  }
#pragma unroll
  for (int c = 0; c < W; ++c) {
    const int d = c * 32 + lane;
    unsigned bv;
    if constexpr (PK) {  // ssrc points at the shot's words; bits past m are ignored
      const int base = c * 32;
      bv = base < m ? reinterpret_cast<const uint32_t*>(ssrc)[c] : 0u;
      if (base + 32 > m && base < m) bv &= (1u << (m - base)) - 1u;
    } else {
      bv = __ballot_sync(kFull, d < m && ssrc[d] != 0);
    }
    if (lane == 0) {
      S.syn()[c] = bv;
      S.sred()[c] = bv;
      S.xsol()[c] = 0;
      S.cm()[c] = 0;
    }
  }
  if (lane < 8) S.scal()[lane] = 0;
  __syncwarp();
  int k = 0;
  if (a.single_cluster) {
    for (int d = lane; d < m; d += 32) S.dlab()[d] = 0;
    if constexpr (L::kMasks) {
      for (int r = lane; r < n; r += 32) {
        const int j = S.fat()[r];
        if (G.var_ptr[j + 1] > G.var_ptr[j]) atomicOr(&S.cand()[r >> 5], 1u << (r & 31));
      }
    }
    bool anys = false;
#pragma unroll
    for (int c = 0; c < W; ++c) anys = anys || S.syn()[c] != 0;
    k = anys ? 1 : 0;
    if (lane == 0) S.inv()[0] = 0;
  } else {
    for (int b0 = 0; b0 < m; b0 += 32) {
      const int d = b0 + lane;
      const bool f = d < m && bit_of(S.syn(), d);
      const unsigned bal = __ballot_sync(kFull, f);
      if (f) {
        S.dlab()[d] = d;
        S.inv()[k + __popc(bal & ((1u << lane) - 1u))] = (uint16_t)d;
        if constexpr (L::kMasks) {
          uint32_t* c = S.cand() + (size_t)d * Wn;
#pragma unroll
          for (int w = 0; w < Wn; ++w) c[w] = 0;
          const int c1 = G.chk_ptr[d + 1];
          for (int e = G.chk_ptr[d]; e < c1; ++e) {
            const unsigned rk = S.rank()[G.chk_var[e]];
            c[rk >> 5] |= 1u << (rk & 31);
          }
        }
      }
      k += __popc(bal);
    }
  }
  __syncwarp();

  // ---- LSD-0: grow every invalid cluster until all are valid ----
  int status = LSD_SHOT_OK_LSD, steps = 0;
  while (k > 0) {
    if (steps > n) {  // each step adds a column: cannot be reached
      status = LSD_SHOT_UNSOLVABLE;
      break;
    }
    if (lsd_step<L, MU>(G, S, m, n, k, true, lane) == 1) {
      status = LSD_SHOT_UNSOLVABLE;
      break;
    }
    ++steps;
    k = collect_roots(a, S, m, true, lane);
  }
  // ---- LSD-mu: mu more steps for every cluster, then local OSD-E ----
  if constexpr (MU) {
    if (status == LSD_SHOT_OK_LSD) {
      for (int e = 0; e < a.order; ++e) {
        k = collect_roots(a, S, m, false, lane);
        if (lsd_step<L, MU>(G, S, m, n, k, false, lane) == 2) break;
      }
      if (a.osd_cs >= 0)
        osd_cs(a, S, m, lane);
      else
        osd_e(a, S, m, lane);
    }
  }

  // ---- statistics: nu clusters, kappa = largest cluster in columns ----
  for (int d = lane; d < m; d += 32) S.best()[d] = 0;
  __syncwarp();
  for (int j = lane; j < n; j += 32) {
    const int lab = S.flab()[j];
    if (lab >= 0) atomicAdd(&S.best()[S.parent()[lab]], 1u);
  }
  __syncwarp();
  int nu = 0, kappa = 0;
  for (int d = lane; d < m; d += 32) {
    const bool seed = a.single_cluster ? d == 0 : bit_of(S.syn(), d);
    if (seed && S.parent()[d] == d) {
      ++nu;
      kappa = max(kappa, (int)S.best()[d]);
    }
  }
  for (int off = 16; off > 0; off >>= 1) {
    nu += __shfl_xor_sync(kFull, nu, off);
    kappa = max(kappa, __shfl_xor_sync(kFull, kappa, off));
  }

  // ---- global decoding: union of the local solutions (Eq. 2) ----
  uint8_t* cs = S.cs();  // the masks are no longer needed
  for (int j = lane; j < n; j += 32) cs[j] = 0;
  __syncwarp();
  if (status == LSD_SHOT_OK_LSD) {
    for (int d = lane; d < m; d += 32)
      if (bit_of(S.xsol(), d)) cs[S.pcol()[d]] = 1;
    if constexpr (MU) {
      const int ne = S.scal()[2];
      for (int t = lane; t < ne; t += 32) cs[S.ext()[t]] = 1;
    }
  }
  __syncwarp();
  if constexpr (PK) {
    uint32_t* co = reinterpret_cast<uint32_t*>(a.corrections) + shot * packed_words(n);
    for (int base = 0; base < n; base += 32) {  // one ballot per word
      const int j = base + lane;
      const unsigned b = __ballot_sync(kFull, j < n && cs[j] != 0);
      if (lane == 0) co[base >> 5] = b;
    }
  } else {
    uint8_t* co = a.corrections + shot * n;
    for (int j = lane; j < n; j += 32) co[j] = cs[j];
  }
  if (lane == 0) {
    if (a.status) a.status[shot] = (uint8_t)status;
    if (a.shot_info) {
      a.shot_info[3 * shot] = nu;
      a.shot_info[3 * shot + 1] = kappa;
      a.shot_info[3 * shot + 2] = steps;
    }
  }
  acc.steps += steps;
  acc.unsolvable += status == LSD_SHOT_UNSOLVABLE ? 1 : 0;
  acc.kappa_max = max(acc.kappa_max, kappa);
  acc.nu_max = max(acc.nu_max, nu);
  __syncwarp();
}

template <int MM, int NN, bool MU, bool PK>
__global__ void __launch_bounds__(256, MU ? 3 : 4) lsd_kernel(LSDArgs a, int graph_smem) {
  using L = Lay<MM, NN, MU>;
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int m = a.g.m, n = a.g.n, E = a.g.E;
  const int nwarps = blockDim.x >> 5;
  Graph G;
  if (graph_smem) {
    int32_t* cp = reinterpret_cast<int32_t*>(smem + (size_t)nwarps * L::total);
    int32_t* vp = cp + (m + 1);
    uint16_t* cv = reinterpret_cast<uint16_t*>(vp + (n + 1));
    uint16_t* vc = cv + E;
    for (int i = threadIdx.x; i <= m; i += blockDim.x) cp[i] = a.g.chk_ptr[i];
    for (int j = threadIdx.x; j <= n; j += blockDim.x) vp[j] = a.g.var_ptr[j];
    for (int e = threadIdx.x; e < E; e += blockDim.x) {
      cv[e] = a.g.chk_var[e];
      vc[e] = a.g.var_chk[e];
    }
    __syncthreads();
    G.chk_ptr = cp;
    G.var_ptr = vp;
    G.chk_var = cv;
    G.var_chk = vc;
    G.max_col_deg = a.g.max_col_deg;
  } else {
    G.chk_ptr = a.g.chk_ptr;
    G.var_ptr = a.g.var_ptr;
    G.chk_var = a.g.chk_var;
    G.var_chk = a.g.var_chk;
    G.max_col_deg = a.g.max_col_deg;
  }
  G.max_row_deg = a.g.max_row_deg;
  set_lanes(G, lane);
  Shot<L> S{smem + (size_t)warp * L::total};

  const long long count = a.count_from_ctr ? (long long)a.ctr->lsd_count : a.count;
  LsdAcc acc;
  // the next work item is requested while the current one is decoded (lane 0 reads the
  // atomic's result only after the shot), hiding the atomic's round trip
  unsigned long long pending = 0;
  if (lane == 0) pending = atomicAdd(&a.ctr->lsd_next, 1ULL);
  for (;;) {
    const unsigned long long item = __shfl_sync(kFull, pending, 0);
    if (item >= (unsigned long long)count) break;
    if (lane == 0) pending = atomicAdd(&a.ctr->lsd_next, 1ULL);
    const long long shot = a.queue ? (long long)a.queue[item] : (long long)item;
    const float* lsrc = a.llr + (a.llr_by_item ? (long long)item : shot) * n;
    const uint8_t* ssrc =
        PK ? reinterpret_cast<const uint8_t*>(reinterpret_cast<const uint32_t*>(a.syndromes) +
                                              shot * packed_words(m))
           : a.syndromes + shot * m;
    lsd_shot<MM, NN, MU, PK>(a, G, S, lsrc, ssrc, shot, lane, acc);
  }
  lsd_flush(a, acc, lane);
}

inline bool graph_in_smem(const DevGraph& g) { return graph_bytes(g.m, g.n, g.E) <= kGraphBudget; }

// Size classes (max detectors, max faults) the kernel is instantiated for.
struct SizeClass {
  int mm, nn;
};
constexpr SizeClass kClasses[] = {{40, 80}, {72, 144}, {96, 192}, {144, 288}, {256, 768}, {512, 2048}};
constexpr int kNumClasses = sizeof(kClasses) / sizeof(kClasses[0]);

int size_class(int m, int n) {
  for (int c = 0; c < kNumClasses; ++c)
    if (m <= kClasses[c].mm && n <= kClasses[c].nn) return c;
  return -1;
}

#define LSD_CLASS_CASES(X)                                                       \
  X(0, 40, 80) X(1, 72, 144) X(2, 96, 192) X(3, 144, 288) X(4, 256, 768) X(5, 512, 2048)

size_t class_bytes(int c, bool mu) {
  switch (c) {
#define X(i, M, N) \
  case i: return mu ? Lay<M, N, true>::total : Lay<M, N, false>::total;
    LSD_CLASS_CASES(X)
#undef X
    default: return 0;
  }
}

// The kernel of a size class; `pk`: the instance with bit-packed syndromes and corrections.
const void* class_kernel(int c, bool mu, bool pk = false) {
  switch (c) {
#define X(i, M, N)                                                                      \
  case i:                                                                               \
    return pk ? (mu ? (const void*)lsd_kernel<M, N, true, true>                          \
                    : (const void*)lsd_kernel<M, N, false, true>)                        \
              : (mu ? (const void*)lsd_kernel<M, N, true, false>                         \
                    : (const void*)lsd_kernel<M, N, false, false>);
    LSD_CLASS_CASES(X)
#undef X
    default: return nullptr;
  }
}
#undef LSD_CLASS_CASES

}  // namespace

cudaError_t lsd_config(const DevGraph& g, int order, int warps, int* warps_out, int* grid,
                       size_t* smem, int* words) {
  int dev = 0, sms = 0, max_smem = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const int c = size_class(g.m, g.n);
  if (c < 0) return cudaErrorInvalidValue;
  const bool mu = order > 0;
  const size_t per = class_bytes(c, mu);
  const size_t gb = graph_in_smem(g) ? graph_bytes(g.m, g.n, g.E) : 0;
  int w = warps > 0 ? warps : 4;
  while (w > 1 && gb + per * w > (size_t)max_smem) --w;
  if (gb + per * w > (size_t)max_smem) return cudaErrorInvalidValue;
  *smem = gb + per * w;
  *words = (g.m + 31) / 32;
  *warps_out = w;
  const void* fn = class_kernel(c, mu);
  cudaFuncAttributes fa{};
  err = cudaFuncGetAttributes(&fa, fn);
  if (err != cudaSuccess) return err;
  if (w * 32 > fa.maxThreadsPerBlock) return cudaErrorInvalidValue;
  err = allow_max_dynamic_smem(fn, max_smem);
  if (err == cudaSuccess) err = allow_max_dynamic_smem(class_kernel(c, mu, true), max_smem);
  if (err != cudaSuccess) return err;
  int per_sm = 0;
  err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, w * 32, *smem);
  if (err != cudaSuccess) return err;
  if (per_sm < 1) return cudaErrorInvalidValue;
  *grid = per_sm * sms;
  return cudaSuccess;
}

cudaError_t launch_lsd(const LSDArgs& a, int warps, int grid, size_t smem, cudaStream_t st) {
  const int c = size_class(a.g.m, a.g.n);
  if (c < 0) return cudaErrorInvalidValue;
  const bool mu = a.order > 0;
  const int gs = graph_in_smem(a.g) ? 1 : 0;
  void* args[] = {const_cast<LSDArgs*>(&a), const_cast<int*>(&gs)};
  return cudaLaunchKernel(class_kernel(c, mu, a.packed != 0), dim3(grid), dim3(warps * 32), args,
                          smem, st);
}

}  // namespace lsdgb
