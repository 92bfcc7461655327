// One giant shot decoded by the whole GPU: BP (Sec. 4.3) with one thread per check and per
// variable, every iteration in one cooperative launch (grid barriers between the check and
// variable halves), then P-LSD (App. B, Alg. 2): every invalid cluster grows in parallel, clusters
// merge through a lock-free union-find, and each cluster keeps its own on-the-fly
// elimination (Sec. 4.2) in a block of a device arena.
//
// Results are those of the batch decoder (and of the oracle) on the same shot: growth is
// synchronous, ties are broken by the (LLR, index) key, and a cluster's pivot columns do not
// depend on how its elimination rows are numbered.
//
// Cluster state.  Clusters are named by seed ordinal (flipped detectors in the order the
// seeding kernel meets them; the labels do not affect any result).  A cluster root r owns a
// block of cap[r] slots (a multiple of 32; W = cap/32 words per row):
//   R[cap][W]   reduced pivot rows over the cluster's slots (row p exists iff pcol[p] >= 0)
//   T[cap][W]   the combination of pivot columns giving each row
//   pcol[cap]   pivot column of a slot (-1 none), det[cap] detector of a slot
//   sred[W]     the cluster's syndrome reduced by the pivots (zero iff valid, Def. 4.2)
//   xsol[W]     the pivot columns whose sum gives the cleared part of the syndrome
// A detector's slot in its cluster is lslot[d].  When clusters merge, the absorbed blocks
// are copied into the root's (new) block at an offset, rows shifted by that many bits: the
// row supports are disjoint, so the merged rows stay reduced.
//
// Per growth step (one host round trip):
//   find      every candidate fault offers its key to the growing clusters next to it
//   union     each invalid cluster takes its best candidate; collisions unite clusters
//   flatten   union-find paths compressed to one hop
//   plan      slot offsets of absorbed clusters and of newly claimed detectors, per root
//   relocate  a root that merged or outgrew its block moves to a new, larger block
//   absorb    absorbed blocks copied (shifted) into their root's block
//   claim     new detectors get slots; faults next to them become candidates
//   add       each changed root adds its new columns in key order (on-the-fly elimination)
//   collect   the invalid roots of the next step
#include <algorithm>
#include <climits>
#include <cstddef>
#include <cstdint>
#include <cstring>
#include <new>
#include <utility>
#include <vector>

#include "lsd_internal.cuh"

using namespace lsdgb;

namespace {

constexpr unsigned kFullMask = 0xffffffffu;
constexpr unsigned long long kNoKey = ~0ull;
constexpr int kWcMax = 8;                     // reduction words per lane
constexpr int kMaxSlots = 32 * 32 * kWcMax;   // 8192 detectors per cluster
constexpr int kUfLimit = 1 << 20;             // bound on union-find retries and path length
// a minimum over an empty set (a check of degree 1): 2^100, as in the batch kernels
constexpr float kEmptyMinF = 1267650600228229401496703205376.0f;

struct GCtr {
  // whole call
  int ns, nfront, unsolvable, overflow, uf_fail, too_big, ndep, dep_top;
  int bp_stop, bp_unsat[2], bp_iters, bp_conv, bp_fail;
  unsigned bar_arrive;  // grid barrier of the persistent BP launch
  int nu, kappa;
  int ninv[2];
  // reset every step
  int nmerged, nchg, nnew, nclaim, bucket_top, pad;
  unsigned long long arena_top;  // words
};

struct GD {
  int m, n;
  const int *chk_ptr, *chk_var, *var_ptr, *var_chk;
  const float* prior;
  // BP: position-major (ELL) tables padded with -1: ell_col[k * m + i] = column of the k-th
  // edge of check i; ell_pos[k * n + j] = position (k' * m + i) of the k-th edge of column j
  // in ascending row order.  Messages r[dc * m] live at those positions.
  int dc, dv;
  const int *ell_col, *ell_pos;
  float *r, *lam;
  // per detector / per fault
  int *dlab, *lslot, *fst, *front;
  // per seed ordinal (at most m)
  int *parent, *inv0, *inv1, *mlist, *chg, *cap, *nsl, *ncol, *valid, *grow, *mark, *extra,
      *newslots, *aoff, *newcnt, *boff;
  unsigned long long *best, *blk;
  // per step lists (at most m entries each)
  int *nc_g, *nc_r, *nc_rank, *bucket, *cl_d, *cl_r, *cl_rel;
  unsigned long long* nc_key;
  unsigned* arena;
  unsigned long long arena_words;
  GCtr* ctr;
  // LSD-mu (App. D): growth steps, reprocessing (-1 OSD-E, w >= 0 OSD-CS-w), cost weights;
  // dependent columns met by the elimination [n] and their per-root buckets
  int order, osd_cs;
  const long long* wfix;
  int *dep_f, *dep_rank, *dep_bucket, *depcnt, *depoff;
};

__host__ __device__ inline size_t blk_words(int C) {
  const int W = C >> 5;
  return 2 * (size_t)C * W + 2 * (size_t)C + 2 * (size_t)W;
}

struct Blk {
  unsigned* b;
  int C, W;
  __device__ unsigned* R(int p) const { return b + (size_t)p * W; }
  __device__ unsigned* T(int p) const { return b + (size_t)C * W + (size_t)p * W; }
  __device__ int* pcol() const { return reinterpret_cast<int*>(b + 2 * (size_t)C * W); }
  __device__ int* det() const { return pcol() + C; }
  __device__ unsigned* sred() const { return reinterpret_cast<unsigned*>(det() + C); }
  __device__ unsigned* xsol() const { return sred() + W; }
};

__device__ __forceinline__ Blk blk_at(const GD& g, unsigned long long off, int C) {
  Blk B;
  B.b = g.arena + off;
  B.C = C;
  B.W = C >> 5;
  return B;
}

__device__ __forceinline__ Blk blk_of(const GD& g, int r) {
  return blk_at(g, g.blk[r], g.cap[r]);
}

__device__ long long arena_alloc(const GD& g, size_t words) {
  const unsigned long long off = atomicAdd(&g.ctr->arena_top, (unsigned long long)words);
  if (off + words > g.arena_words) {
    atomicOr(&g.ctr->overflow, 1);
    return -1;
  }
  return (long long)off;
}

__device__ __forceinline__ unsigned long long llr_key(float x, int j) {
  x = __fadd_rn(x, 0.0f);  // -0 -> +0
  unsigned u = __float_as_uint(x);
  u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
  return ((unsigned long long)u << 32) | (unsigned)j;
}

__device__ __forceinline__ long long gtid() {
  return (long long)blockIdx.x * blockDim.x + threadIdx.x;
}
__device__ __forceinline__ long long gstride() { return (long long)gridDim.x * blockDim.x; }
__device__ __forceinline__ long long gwarp() { return gtid() >> 5; }
__device__ __forceinline__ long long gwarps() { return gstride() >> 5; }

// ---------------------------------------------------------------------------------------
// BP over one shot (flooding min-sum, every operation rounded to float in the order of the
// batch kernels and of the oracle's FP32 mirror)
// ---------------------------------------------------------------------------------------

__global__ void __launch_bounds__(256) gbp_init(GD g) {
  const long long slots = (long long)g.dc * g.m;
  for (long long k = gtid(); k < slots; k += gstride()) g.r[k] = 0.0f;
  for (long long j = gtid(); j < g.n; j += gstride()) g.lam[j] = g.prior[j];
}

// Iteration t (t >= 1): q = Lam - r on every edge of a check, then the scaled min-sum
// message.  For t >= 2 it also tests the hard decision [Lam < 0] of iteration t-1 against s
// (Sec. 4.3's early exit; sign bits stand for "< 0": no Lam is -0), accumulating into
// bp_unsat[t & 1]; gbp_var(t) stops the shot, keeping Lam of iteration t-1, when it passed.
// A warp reads 32 consecutive checks' k-th edges: the column indices and messages are
// contiguous, Lam is gathered.
template <int DCMAX>
__device__ __forceinline__ void check_phase(const GD& g, const uint8_t* __restrict__ s,
                                            float alpha, int t) {
  bool bad = false;
  for (long long i = gtid(); i < g.m; i += gstride()) {
    unsigned hp = s[i] ? 0x80000000u : 0u;  // bit 31: syndrome ^ signs of Lam
    unsigned sx = 0u;                        // bit 31: signs of q
    float m1 = kEmptyMinF, m2 = kEmptyMinF;
    int am = -1, deg = 0;
    unsigned qb[DCMAX];
#pragma unroll
    for (int k = 0; k < DCMAX; ++k) {
      qb[k] = 0u;
      const int j = k < g.dc ? g.ell_col[(long long)k * g.m + i] : -1;
      if (j < 0) continue;
      const float L = __ldcg(&g.lam[j]);  // L2: written by other blocks
      hp ^= __float_as_uint(L);
      const float q = __fsub_rn(L, __ldcg(&g.r[(long long)k * g.m + i]));
      qb[k] = __float_as_uint(q);
      sx ^= qb[k];
      const float a = fabsf(q);
      if (a < m1) {
        m2 = m1;
        m1 = a;
        am = k;
      } else if (a < m2) {
        m2 = a;
      }
      deg = k + 1;
    }
    bad |= (hp >> 31) != 0u;
    const unsigned par = (s[i] ? 0x80000000u : 0u) ^ sx;
    const float mag1 = __fmul_rn(alpha, m1), mag2 = __fmul_rn(alpha, m2);
#pragma unroll
    for (int k = 0; k < DCMAX; ++k) {
      if (k >= deg) continue;
      const float mag = k == am ? mag2 : mag1;
      g.r[(long long)k * g.m + i] =
          __uint_as_float(__float_as_uint(mag) | ((par ^ qb[k]) & 0x80000000u));
    }
  }
  if (t >= 2 && __any_sync(kFullMask, bad) && (threadIdx.x & 31) == 0)
    atomicOr(&g.ctr->bp_unsat[t & 1], 1);
}

template <int DCMAX>
__global__ void __launch_bounds__(256) gbp_check(GD g, const uint8_t* __restrict__ s,
                                                  float alpha, int t) {
  if (*(volatile int*)&g.ctr->bp_stop) return;
  check_phase<DCMAX>(g, s, alpha, t);
}

// Lam of iteration t: prior plus the incoming messages in ascending check order.
__device__ __forceinline__ void var_phase(const GD& g) {
  for (long long j = gtid(); j < g.n; j += gstride()) {
    float L = g.prior[j];
    for (int k = 0; k < g.dv; ++k) {
      const int p = g.ell_pos[(long long)k * g.n + j];
      if (p < 0) break;
      L = __fadd_rn(L, __ldcg(&g.r[p]));
    }
    g.lam[j] = L;
  }
}

// Iteration t's decision before its variable half: stop (true) when iteration t-1
// satisfied the syndrome, keeping its posteriors; else clear the next test's slot.
__device__ __forceinline__ bool bp_converged_before(const GD& g, int t) {
  if (t >= 2 && *(volatile int*)&g.ctr->bp_unsat[t & 1] == 0) {
    if (gtid() == 0) {
      g.ctr->bp_conv = 1;
      g.ctr->bp_iters = t - 1;
      g.ctr->bp_stop = 1;
    }
    return true;
  }
  if (gtid() == 0) {
    g.ctr->bp_unsat[(t + 1) & 1] = 0;
    g.ctr->bp_iters = t;
  }
  return false;
}

__global__ void __launch_bounds__(256) gbp_var(GD g, int t) {
  if (*(volatile int*)&g.ctr->bp_stop) return;
  if (bp_converged_before(g, t)) return;
  var_phase(g);
}

// The test after the last iteration T (slot (T+1) & 1, cleared by iteration T).
__device__ __forceinline__ void syn_phase(const GD& g, const uint8_t* __restrict__ s, int slot) {
  bool bad = false;
  for (long long i = gtid(); i < g.m; i += gstride()) {
    unsigned hp = s[i] ? 0x80000000u : 0u;
    for (int k = 0; k < g.dc; ++k) {
      const int j = g.ell_col[(long long)k * g.m + i];
      if (j < 0) break;
      hp ^= __float_as_uint(__ldcg(&g.lam[j]));
    }
    bad |= (hp >> 31) != 0u;
  }
  if (__any_sync(kFullMask, bad) && (threadIdx.x & 31) == 0) atomicOr(&g.ctr->bp_unsat[slot], 1);
}

__global__ void __launch_bounds__(256) gbp_syn(GD g, const uint8_t* __restrict__ s, int slot) {
  if (*(volatile int*)&g.ctr->bp_stop) return;
  syn_phase(g, s, slot);
}

// Grid-wide barrier of the persistent launch (all blocks co-resident: cooperative launch).
// The arrival counter only grows; barrier b waits for b * gridDim.x arrivals.  The wait is
// bounded by limit_ns of the global timer: past it the block flags bp_fail and every block
// leaves at its next barrier, the host reporting LSD_ERR_TIMEOUT.  `arrive` false (the
// timeout test only) withholds this block's arrival.
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool grid_barrier(const GD& g, unsigned target, long long limit_ns,
                                             bool arrive = true) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (arrive) atomicAdd(&g.ctr->bar_arrive, 1u);
    const unsigned long long t0 = global_ns();
    while (*(volatile unsigned*)&g.ctr->bar_arrive < target &&
           !*(volatile int*)&g.ctr->bp_fail) {
      if ((long long)(global_ns() - t0) > limit_ns) {
        atomicOr(&g.ctr->bp_fail, 1);
        break;
      }
      __nanosleep(64);
    }
    __threadfence();
  }
  __syncthreads();
  return *(volatile int*)&g.ctr->bp_fail == 0;
}

// All T iterations in one launch: check half, barrier, decision, variable half, barrier.
// hold != 0 (the timeout test only): block 0 withholds its first arrival.
template <int DCMAX>
__global__ void __launch_bounds__(256) gbp_persistent(GD g, const uint8_t* __restrict__ s,
                                                       float alpha, int T, long long limit_ns,
                                                       int hold) {
  unsigned target = 0;
  const unsigned nb = gridDim.x;
  for (int t = 1; t <= T; ++t) {
    check_phase<DCMAX>(g, s, alpha, t);
    target += nb;
    if (!grid_barrier(g, target, limit_ns, !(hold && t == 1 && blockIdx.x == 0))) return;
    if (bp_converged_before(g, t)) return;
    var_phase(g);
    target += nb;
    if (!grid_barrier(g, target, limit_ns)) return;
  }
  const int slot = (T + 1) & 1;
  syn_phase(g, s, slot);
  target += nb;
  if (!grid_barrier(g, target, limit_ns)) return;
  if (gtid() == 0) {
    g.ctr->bp_conv = g.ctr->bp_unsat[slot] == 0;
    g.ctr->bp_stop = 1;
  }
}

__global__ void gbp_final(GD g, int slot) {
  if (g.ctr->bp_stop) return;
  g.ctr->bp_conv = g.ctr->bp_unsat[slot] == 0;
  g.ctr->bp_stop = 1;
}

__global__ void __launch_bounds__(256) gcopy_hard(GD g, uint8_t* __restrict__ corr) {
  for (long long j = gtid(); j < g.n; j += gstride()) corr[j] = g.lam[j] < 0.0f ? 1 : 0;
}

// ---------------------------------------------------------------------------------------
// P-LSD
// ---------------------------------------------------------------------------------------

__device__ int gfind(const GD& g, int x) {
  const volatile int* par = g.parent;
  for (int it = 0; it < kUfLimit; ++it) {
    const int p = par[x];
    if (p == x) return x;
    x = p;
  }
  atomicOr(&g.ctr->uf_fail, 1);
  return x;
}

// Links the larger root under the smaller; the absorbed root is listed once in mlist.
__device__ void gunite(const GD& g, int a, int b) {
  for (int it = 0; it < kUfLimit; ++it) {
    a = gfind(g, a);
    b = gfind(g, b);
    if (a == b) return;
    if (a < b) {
      const int t = a;
      a = b;
      b = t;
    }
    if (atomicCAS(g.parent + a, a, b) == a) {
      const int k = atomicAdd(&g.ctr->nmerged, 1);
      g.mlist[k] = a;
      return;
    }
  }
  atomicOr(&g.ctr->uf_fail, 1);
}

__device__ __forceinline__ void add_candidates(const GD& g, int d) {
  for (int e = g.chk_ptr[d]; e < g.chk_ptr[d + 1]; ++e) {
    const int f = g.chk_var[e];
    if (atomicCAS(&g.fst[f], -2, -1) == -2) g.front[atomicAdd(&g.ctr->nfront, 1)] = f;
  }
}

__global__ void __launch_bounds__(256) glsd_reset(GD g) {
  for (long long d = gtid(); d < g.m; d += gstride()) g.dlab[d] = -1;
  for (long long j = gtid(); j < g.n; j += gstride()) g.fst[j] = -2;
}

// One cluster per flipped detector (Alg. 2's initialization), each in a 32-slot block.
__global__ void __launch_bounds__(256) glsd_seed(GD g, const uint8_t* __restrict__ s) {
  constexpr int C = 32;
  const size_t words = blk_words(C);
  for (long long d = gtid(); d < g.m; d += gstride()) {
    if (!s[d]) continue;
    const int ord = atomicAdd(&g.ctr->ns, 1);
    g.dlab[d] = ord;
    g.lslot[d] = 0;
    g.parent[ord] = ord;
    g.inv0[ord] = ord;
    const long long off = arena_alloc(g, words);
    if (off < 0) continue;
    g.blk[ord] = (unsigned long long)off;
    g.cap[ord] = C;
    g.nsl[ord] = 1;
    g.ncol[ord] = 0;
    g.valid[ord] = 0;
    g.grow[ord] = 1;
    g.best[ord] = kNoKey;
    g.mark[ord] = 0;
    g.extra[ord] = 0;
    g.newslots[ord] = 0;
    g.newcnt[ord] = 0;
    g.depcnt[ord] = 0;
    const Blk B = blk_at(g, (unsigned long long)off, C);
    for (size_t w = 0; w < words; ++w) B.b[w] = 0u;
    for (int p = 0; p < C; ++p) B.pcol()[p] = -1;
    B.det()[0] = (int)d;
    B.sred()[0] = 1u;
    add_candidates(g, (int)d);
  }
}

__global__ void glsd_seed_count(GD g) { g.ctr->ninv[0] = g.ctr->ns; }

// find_candidate: every live candidate offers its key to the growing roots next to it.
__global__ void __launch_bounds__(256) glsd_find(GD g, const float* __restrict__ llr) {
  const int nf = g.ctr->nfront;
  for (long long i = gtid(); i < nf; i += gstride()) {
    const int f = g.front[i];
    if (g.fst[f] != -1) continue;
    const unsigned long long key = llr_key(llr[f], f);
    for (int q = g.var_ptr[f]; q < g.var_ptr[f + 1]; ++q) {
      const int c = g.dlab[g.var_chk[q]];
      if (c < 0) continue;
      const int R = g.parent[c];
      if (g.grow[R]) atomicMin(&g.best[R], key);
    }
  }
}

// parallel_union: each invalid cluster takes its pick; collisions unite.
__global__ void __launch_bounds__(256) glsd_union(GD g, int par, int strict) {
  const int cnt = g.ctr->ninv[par];
  const int* inv = par ? g.inv1 : g.inv0;
  for (long long t = gtid(); t < cnt; t += gstride()) {
    const int r = inv[t];
    const unsigned long long key = g.best[r];
    if (key == kNoKey) {
      if (strict) atomicOr(&g.ctr->unsolvable, 1);  // LSD-mu: a full cluster just stops
      continue;
    }
    const int f = (int)(key & 0xffffffffu);
    const int old = atomicCAS(&g.fst[f], -1, r);
    if (old == -1) {
      const int k = atomicAdd(&g.ctr->nnew, 1);
      g.nc_g[k] = f;
      g.nc_r[k] = r;
      g.nc_key[k] = key;
    } else {
      gunite(g, r, old);
    }
    for (int q = g.var_ptr[f]; q < g.var_ptr[f + 1]; ++q) {
      const int d = g.var_chk[q];
      const int o = atomicCAS(&g.dlab[d], -1, r);
      if (o == -1) {
        const int k = atomicAdd(&g.ctr->nclaim, 1);
        g.cl_d[k] = d;
        g.cl_r[k] = r;
      } else if (o != r) {
        gunite(g, r, o);
      }
    }
  }
}

__global__ void __launch_bounds__(256) glsd_flatten(GD g) {
  const int ns = g.ctr->ns;
  for (long long x = gtid(); x < ns; x += gstride()) g.parent[x] = gfind(g, (int)x);
}

__device__ __forceinline__ void mark_changed(const GD& g, int R) {
  if (atomicCAS(&g.mark[R], 0, 1) == 0) g.chg[atomicAdd(&g.ctr->nchg, 1)] = R;
}

// Offsets inside each root's grown block: absorbed clusters, then new detectors; ranks of
// the new columns.
__global__ void __launch_bounds__(256) glsd_plan(GD g) {
  const int nm = g.ctr->nmerged, nc = g.ctr->nclaim, nn = g.ctr->nnew;
  for (long long t = gtid(); t < (long long)nm + nc + nn; t += gstride()) {
    if (t < nm) {
      const int A = g.mlist[t];
      const int R = g.parent[A];
      g.aoff[A] = atomicAdd(&g.extra[R], g.nsl[A]);
      mark_changed(g, R);
    } else if (t < nm + nc) {
      const int k = (int)(t - nm);
      const int R = g.parent[g.cl_r[k]];
      g.cl_rel[k] = atomicAdd(&g.newslots[R], 1);
      mark_changed(g, R);
    } else {
      const int k = (int)(t - nm - nc);
      const int R = g.parent[g.nc_r[k]];
      g.nc_rank[k] = atomicAdd(&g.newcnt[R], 1);
      mark_changed(g, R);
    }
  }
}

// A root that merged or outgrew its block moves to a new zeroed block (its own slots copied
// at the same positions); every changed root reserves room for its new columns' list.
__global__ void __launch_bounds__(256) glsd_relocate(GD g) {
  const int lane = threadIdx.x & 31;
  const int nchg = g.ctr->nchg;
  for (long long t = gwarp(); t < nchg; t += gwarps()) {
    const int R = g.chg[t];
    const int base = g.nsl[R];
    const int need = base + g.extra[R] + g.newslots[R];
    if (lane == 0) g.boff[R] = atomicAdd(&g.ctr->bucket_top, g.newcnt[R]);
    if (need > kMaxSlots) {
      if (lane == 0) atomicOr(&g.ctr->too_big, 1);
      continue;
    }
    const Blk O = blk_of(g, R);
    if (g.extra[R] == 0 && need <= O.C) {
      for (int p = base + lane; p < need; p += 32) O.pcol()[p] = -1;
      continue;
    }
    const int want = need + need / 2;
    const int C = max(O.C, min(kMaxSlots, max(32, (want + 31) & ~31)));  // never shrinks
    const size_t words = blk_words(C);
    long long off = 0;
    if (lane == 0) off = arena_alloc(g, words);
    off = __shfl_sync(kFullMask, off, 0);
    if (off < 0) continue;
    const Blk N = blk_at(g, (unsigned long long)off, C);
    for (size_t w = lane; w < words; w += 32) N.b[w] = 0u;
    __syncwarp();
    for (int p = lane; p < C; p += 32) N.pcol()[p] = p < base ? O.pcol()[p] : -1;
    for (int p = lane; p < base; p += 32) N.det()[p] = O.det()[p];
    for (int w = lane; w < O.W; w += 32) {
      N.sred()[w] = O.sred()[w];
      N.xsol()[w] = O.xsol()[w];
    }
    for (int p = 0; p < base; ++p) {
      if (O.pcol()[p] < 0) continue;
      for (int w = lane; w < O.W; w += 32) {
        N.R(p)[w] = O.R(p)[w];
        N.T(p)[w] = O.T(p)[w];
      }
    }
    __syncwarp();
    if (lane == 0) {
      g.blk[R] = (unsigned long long)off;
      g.cap[R] = C;
    }
  }
}

// Word w of a bit vector `src` (sw words) shifted up by `sh` bits.
__device__ __forceinline__ unsigned shifted_word(const unsigned* src, int sw, int sh, int w) {
  const int q = sh >> 5, b = sh & 31;
  const int i = w - q;
  unsigned v = (i >= 0 && i < sw) ? src[i] << b : 0u;
  if (b && i - 1 >= 0 && i - 1 < sw) v |= src[i - 1] >> (32 - b);
  return v;
}

// Absorbed clusters copied into their root's block at their offset (rows shifted).
__global__ void __launch_bounds__(256) glsd_absorb(GD g) {
  const int lane = threadIdx.x & 31;
  const int nm = g.ctr->nmerged;
  for (long long t = gwarp(); t < nm; t += gwarps()) {
    const int A = g.mlist[t];
    const int R = g.parent[A];
    if (g.ctr->too_big || g.ctr->overflow) continue;
    const Blk S = blk_of(g, A), D = blk_of(g, R);
    const int o = g.nsl[R] + g.aoff[A];
    const int nA = g.nsl[A];
    for (int p = lane; p < nA; p += 32) {
      D.pcol()[o + p] = S.pcol()[p];
      const int d = S.det()[p];
      D.det()[o + p] = d;
      g.lslot[d] = o + p;
    }
    const int w0 = o >> 5, w1 = min(D.W, ((o + nA + 31) >> 5) + 1);
    for (int w = w0 + lane; w < w1; w += 32) {
      const unsigned a = shifted_word(S.sred(), S.W, o, w);
      const unsigned b = shifted_word(S.xsol(), S.W, o, w);
      if (a) atomicOr(&D.sred()[w], a);
      if (b) atomicOr(&D.xsol()[w], b);
    }
    for (int p = 0; p < nA; ++p) {
      if (S.pcol()[p] < 0) continue;
      for (int w = w0 + lane; w < w1; w += 32) {
        D.R(o + p)[w] = shifted_word(S.R(p), S.W, o, w);
        D.T(o + p)[w] = shifted_word(S.T(p), S.W, o, w);
      }
    }
    if (lane == 0) atomicAdd(&g.ncol[R], g.ncol[A]);
  }
}

// New detectors take their slots; faults next to them become candidates (Def. 4.3); the new
// columns are placed in their root's list.
__global__ void __launch_bounds__(256) glsd_claim(GD g) {
  const int nc = g.ctr->nclaim, nn = g.ctr->nnew;
  if (g.ctr->too_big || g.ctr->overflow) return;
  for (long long t = gtid(); t < (long long)nc + nn; t += gstride()) {
    if (t < nc) {
      const int k = (int)t;
      const int d = g.cl_d[k];
      const int R = g.parent[g.cl_r[k]];
      const int slot = g.nsl[R] + g.extra[R] + g.cl_rel[k];
      const Blk D = blk_of(g, R);
      D.det()[slot] = d;
      g.lslot[d] = slot;
      add_candidates(g, d);
    } else {
      const int k = (int)(t - nc);
      const int R = g.parent[g.nc_r[k]];
      g.bucket[g.boff[R] + g.nc_rank[k]] = k;
    }
  }
}

// Adds fault f to the elimination of block D (nslots slots in use), as the batch kernels do.
__device__ void gadd_column(const GD& g, const Blk& D, int nslots, int f, int lane) {
  const int wc = (nslots + 31) >> 5;
  unsigned bw[kWcMax], tw[kWcMax];
#pragma unroll
  for (int c = 0; c < kWcMax; ++c) bw[c] = tw[c] = 0u;
  for (int q = g.var_ptr[f]; q < g.var_ptr[f + 1]; ++q) {
    const int sl = g.lslot[g.var_chk[q]];
    const bool piv = D.pcol()[sl] >= 0;
#pragma unroll
    for (int c = 0; c < kWcMax; ++c) {
      const int w = c * 32 + lane;
      if (w < wc) {
        if ((sl >> 5) == w) bw[c] ^= 1u << (sl & 31);
        if (piv) {
          bw[c] ^= D.R(sl)[w];
          tw[c] ^= D.T(sl)[w];
        }
      }
    }
  }
  int p = -1;
#pragma unroll
  for (int c = 0; c < kWcMax; ++c) {
    const unsigned nz = __ballot_sync(kFullMask, bw[c] != 0u);
    if (p < 0 && nz) {
      const int wl = __ffs(nz) - 1;
      const unsigned word = __shfl_sync(kFullMask, bw[c], wl);
      p = (c * 32 + wl) * 32 + __ffs(word) - 1;
    }
  }
  if (p < 0) {  // dependent column: the span does not change; LSD-mu lists it
    if (g.order > 0 && lane == 0) g.dep_f[atomicAdd(&g.ctr->ndep, 1)] = f;
    return;
  }
  const int pw = p >> 5;
  const unsigned pb = 1u << (p & 31);
#pragma unroll
  for (int c = 0; c < kWcMax; ++c)
    if (c * 32 + lane == pw) tw[c] ^= pb;
  const bool sflag = (D.sred()[pw] & pb) != 0u;
  __syncwarp();
#pragma unroll
  for (int c = 0; c < kWcMax; ++c) {
    const int w = c * 32 + lane;
    if (w < wc) {
      D.R(p)[w] = bw[c];
      D.T(p)[w] = tw[c];
    }
  }
  if (lane == 0) D.pcol()[p] = f;
  __syncwarp();
  for (int d0 = 0; d0 < nslots; d0 += 32) {
    const int d = d0 + lane;
    const bool hit = d < nslots && d != p && D.pcol()[d] >= 0 && (D.R(d)[pw] & pb) != 0u;
    unsigned bal = __ballot_sync(kFullMask, hit);
    while (bal) {
      const int dd = d0 + __ffs(bal) - 1;
      bal &= bal - 1;
#pragma unroll
      for (int c = 0; c < kWcMax; ++c) {
        const int w = c * 32 + lane;
        if (w < wc) {
          D.R(dd)[w] ^= bw[c];
          D.T(dd)[w] ^= tw[c];
        }
      }
    }
    __syncwarp();
  }
  if (sflag) {
#pragma unroll
    for (int c = 0; c < kWcMax; ++c) {
      const int w = c * 32 + lane;
      if (w < wc) {
        D.sred()[w] ^= bw[c];
        D.xsol()[w] ^= tw[c];
      }
    }
  }
  __syncwarp();
}

// on_the_fly_elimination of every changed root: its new columns in key order, then its
// validity.
__global__ void __launch_bounds__(256) glsd_add(GD g) {
  const int lane = threadIdx.x & 31;
  const int nchg = g.ctr->nchg;
  if (g.ctr->too_big || g.ctr->overflow) return;
  for (long long t = gwarp(); t < nchg; t += gwarps()) {
    const int R = g.chg[t];
    const int nslots = g.nsl[R] + g.extra[R] + g.newslots[R];
    const Blk D = blk_of(g, R);
    const int cnt = g.newcnt[R];
    const int* bk = g.bucket + g.boff[R];
    unsigned long long last = 0;
    for (int it = 0; it < cnt; ++it) {
      unsigned long long best = kNoKey;
      int bi = -1;
      for (int u = lane; u < cnt; u += 32) {
        const int k = bk[u];
        const unsigned long long key = g.nc_key[k];
        if ((it == 0 || key > last) && key < best) {
          best = key;
          bi = k;
        }
      }
      for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long ob = __shfl_xor_sync(kFullMask, best, off);
        const int oi = __shfl_xor_sync(kFullMask, bi, off);
        if (ob < best) {
          best = ob;
          bi = oi;
        }
      }
      last = best;
      gadd_column(g, D, nslots, g.nc_g[bi], lane);
    }
    bool any = false;
    for (int w = lane; w < ((nslots + 31) >> 5); w += 32) any |= D.sred()[w] != 0u;
    any = __any_sync(kFullMask, any);
    if (lane == 0) {
      g.valid[R] = any ? 0 : 1;
      g.ncol[R] += cnt;
      g.nsl[R] = nslots;
      g.extra[R] = 0;
      g.newslots[R] = 0;
      g.newcnt[R] = 0;
      g.mark[R] = 0;
    }
  }
}

__global__ void __launch_bounds__(256) glsd_collect(GD g, int par_next) {
  const int ns = g.ctr->ns;
  int* inv = par_next ? g.inv1 : g.inv0;
  for (long long x = gtid(); x < ns; x += gstride()) {
    const bool invalid = g.parent[x] == x && !g.valid[x];
    g.grow[x] = invalid ? 1 : 0;
    if (invalid) {
      g.best[x] = kNoKey;
      inv[atomicAdd(&g.ctr->ninv[par_next], 1)] = (int)x;
    }
  }
}

// LSD-mu: every root grows (App. D's extra steps).
__global__ void __launch_bounds__(256) glsd_collect_all(GD g, int par) {
  const int ns = g.ctr->ns;
  int* inv = par ? g.inv1 : g.inv0;
  for (long long x = gtid(); x < ns; x += gstride()) {
    const bool root = g.parent[x] == x;
    g.grow[x] = root ? 1 : 0;
    if (root) {
      g.best[x] = kNoKey;
      inv[atomicAdd(&g.ctr->ninv[par], 1)] = (int)x;
    }
  }
}

// Dependent columns grouped by final root: rank in the root's bucket, bucket offsets, placement.
__global__ void __launch_bounds__(256) glsd_dep_rank(GD g) {
  const int nd = g.ctr->ndep;
  for (long long k = gtid(); k < nd; k += gstride())
    g.dep_rank[k] = atomicAdd(&g.depcnt[g.parent[g.fst[g.dep_f[k]]]], 1);
}

__global__ void __launch_bounds__(256) glsd_dep_offsets(GD g) {
  const int ns = g.ctr->ns;
  for (long long x = gtid(); x < ns; x += gstride())
    if (g.parent[x] == x && g.depcnt[x] > 0) g.depoff[x] = atomicAdd(&g.ctr->dep_top, g.depcnt[x]);
}

__global__ void __launch_bounds__(256) glsd_dep_place(GD g) {
  const int nd = g.ctr->ndep;
  for (long long k = gtid(); k < nd; k += gstride()) {
    const int R = g.parent[g.fst[g.dep_f[k]]];
    g.dep_bucket[g.depoff[R] + g.dep_rank[k]] = g.dep_f[k];
  }
}

// Cost of root block D's local solution (xsol) with the dependent columns i1, i2 of the
// sorted list flipped (-1 none): tw vectors at tw + i * wc.
__device__ long long gpattern_cost(const GD& g, const Blk& D, int wc, const unsigned* tw,
                                   const int* cols, int i1, int i2) {
  long long cost = 0;
  for (int w = 0; w < wc; ++w) {
    unsigned v = D.xsol()[w];
    if (i1 >= 0) v ^= tw[(size_t)i1 * wc + w];
    if (i2 >= 0) v ^= tw[(size_t)i2 * wc + w];
    while (v) {
      const int b = __ffs(v) - 1;
      v &= v - 1;
      cost += g.wfix[D.pcol()[w * 32 + b]];
    }
  }
  if (i1 >= 0) cost += g.wfix[cols[i1]];
  if (i2 >= 0) cost += g.wfix[cols[i2]];
  return cost;
}

// LSD-mu reprocessing of every root with dependent columns (App. D), as the batch kernels:
// OSD-E over the first min(mu, #dependent) in key order (ties to the smaller pattern), or
// the combination sweep OSD-CS-w (no flip, every single, every pair among the first w; ties
// to the earlier pattern).  A dependent column's representation tw over the pivots is
// recomputed from the root's final rows (the pivots only grow, so it is the same unique
// combination).  Chosen dependent columns go straight to the correction; xsol takes their tw.
__global__ void __launch_bounds__(256) glsd_reprocess(GD g, const float* __restrict__ llr,
                                                       uint8_t* __restrict__ corr) {
  const int lane = threadIdx.x & 31;
  const int ns = g.ctr->ns;
  for (long long x = gwarp(); x < ns; x += gwarps()) {
    if (g.parent[x] != x) continue;
    const int cnt = g.depcnt[x];
    if (cnt == 0) continue;
    const Blk D = blk_of(g, (int)x);
    const int wc = (g.nsl[x] + 31) >> 5;
    const int* bk = g.dep_bucket + g.depoff[x];
    long long off = 0;
    if (lane == 0) off = arena_alloc(g, 1 + 2 * (size_t)cnt + (size_t)cnt * (1 + wc));
    off = __shfl_sync(kFullMask, off, 0);
    if (off < 0) continue;
    off += off & 1;  // 8-byte alignment of the keys
    unsigned long long* keys = reinterpret_cast<unsigned long long*>(g.arena + off);  // [cnt]
    int* cols = reinterpret_cast<int*>(g.arena + off + 2 * (size_t)cnt);            // [cnt]
    unsigned* tw = g.arena + off + 3 * (size_t)cnt;                                  // [cnt][wc]
    // sort the bucket by (LLR, index) key: rank of each entry among the bucket
    for (int u = lane; u < cnt; u += 32) {
      const int f = bk[u];
      const unsigned long long ku = llr_key(llr[f], f);
      int pos = 0;
      for (int v = 0; v < cnt; ++v) {
        const int fv = bk[v];
        pos += llr_key(llr[fv], fv) < ku ? 1 : 0;
      }
      cols[pos] = f;
      keys[pos] = ku;
    }
    __syncwarp();
    // representations over the pivots
    for (int i = 0; i < cnt; ++i) {
      const int f = cols[i];
      for (int w = lane; w < wc; w += 32) {
        unsigned t = 0u;
        for (int q = g.var_ptr[f]; q < g.var_ptr[f + 1]; ++q) {
          const int sl = g.lslot[g.var_chk[q]];
          if (D.pcol()[sl] >= 0) t ^= D.T(sl)[w];
        }
        tw[(size_t)i * wc + w] = t;
      }
    }
    __syncwarp();
    long long bc = LLONG_MAX;
    int b1 = -1, b2 = -1;
    if (g.osd_cs < 0) {
      const int nt = min(g.order, cnt);
      int bt = 0;
      for (int t = lane; t < (1 << nt); t += 32) {
        long long cost = 0;
        for (int w = 0; w < wc; ++w) {
          unsigned v = D.xsol()[w];
          for (int k = 0; k < nt; ++k)
            if ((t >> k) & 1) v ^= tw[(size_t)k * wc + w];
          while (v) {
            const int b = __ffs(v) - 1;
            v &= v - 1;
            cost += g.wfix[D.pcol()[w * 32 + b]];
          }
        }
        for (int k = 0; k < nt; ++k)
          if ((t >> k) & 1) cost += g.wfix[cols[k]];
        if (cost < bc) {
          bc = cost;
          bt = t;
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const long long oc = __shfl_xor_sync(kFullMask, bc, o);
        const int ot = __shfl_xor_sync(kFullMask, bt, o);
        if (oc < bc || (oc == bc && ot < bt)) {
          bc = oc;
          bt = ot;
        }
      }
      if (bt == 0) continue;
      for (int w = lane; w < wc; w += 32) {
        unsigned delta = 0u;
        for (int k = 0; k < nt; ++k)
          if ((bt >> k) & 1) delta ^= tw[(size_t)k * wc + w];
        D.xsol()[w] ^= delta;
      }
      for (int k = lane; k < nt; k += 32)
        if ((bt >> k) & 1) corr[cols[k]] = 1;
      __syncwarp();
      continue;
    }
    // combination sweep
    const int wp = min(g.osd_cs, cnt);
    int bcls = 3;
    unsigned long long bkey = 0;
    auto consider = [&](long long c, int cls, unsigned long long key, int i1, int i2) {
      if (c < bc || (c == bc && (cls < bcls || (cls == bcls && key < bkey)))) {
        bc = c;
        bcls = cls;
        bkey = key;
        b1 = i1;
        b2 = i2;
      }
    };
    if (lane == 0) consider(gpattern_cost(g, D, wc, tw, cols, -1, -1), 0, 0, -1, -1);
    for (int i = lane; i < cnt; i += 32)
      consider(gpattern_cost(g, D, wc, tw, cols, i, -1), 1, keys[i], i, -1);
    const int npairs = wp * (wp - 1) / 2;
    for (int t = lane; t < npairs; t += 32) {
      int i = 0, rem = t;
      while (rem >= wp - 1 - i) {
        rem -= wp - 1 - i;
        ++i;
      }
      const int j = i + 1 + rem;
      consider(gpattern_cost(g, D, wc, tw, cols, i, j), 2, (unsigned long long)(i * 16 + j), i, j);
    }
    for (int o = 16; o > 0; o >>= 1) {
      const long long oc = __shfl_xor_sync(kFullMask, bc, o);
      const int ocls = __shfl_xor_sync(kFullMask, bcls, o);
      const unsigned long long okey = __shfl_xor_sync(kFullMask, bkey, o);
      const int o1 = __shfl_xor_sync(kFullMask, b1, o);
      const int o2 = __shfl_xor_sync(kFullMask, b2, o);
      consider(oc, ocls, okey, o1, o2);
    }
    if (b1 < 0) continue;
    for (int w = lane; w < wc; w += 32) {
      unsigned delta = tw[(size_t)b1 * wc + w];
      if (b2 >= 0) delta ^= tw[(size_t)b2 * wc + w];
      D.xsol()[w] ^= delta;
    }
    if (lane == 0) {
      corr[cols[b1]] = 1;
      if (b2 >= 0) corr[cols[b2]] = 1;
    }
    __syncwarp();
  }
}

// Local solutions (Eq. 2): the pivot columns in each root's xsol; nu and kappa.
__global__ void __launch_bounds__(256) glsd_solve(GD g, uint8_t* __restrict__ corr, int write) {
  const int lane = threadIdx.x & 31;
  const int ns = g.ctr->ns;
  for (long long x = gwarp(); x < ns; x += gwarps()) {
    if (g.parent[x] != x) continue;
    if (lane == 0) {
      atomicAdd(&g.ctr->nu, 1);
      atomicMax(&g.ctr->kappa, g.ncol[x]);
    }
    if (!write) continue;
    const Blk D = blk_of(g, (int)x);
    const int nx = g.nsl[x];
    for (int p = lane; p < nx; p += 32) {
      const int c = D.pcol()[p];
      if (c >= 0 && ((D.xsol()[p >> 5] >> (p & 31)) & 1u)) corr[c] = 1;
    }
  }
}

__global__ void __launch_bounds__(256) gzero(uint8_t* __restrict__ p, long long nbytes) {
  for (long long i = gtid(); i < nbytes; i += gstride()) p[i] = 0;
}

}  // namespace

struct lsd_giant {
  int m = 0, n = 0;
  long long E = 0;
  int bp_iters = 0;
  float alpha = 0.625f;
  cudaStream_t st = nullptr;
  int sms = 0;
  GD g{};
  GCtr* h_ctr = nullptr;  // pinned
  std::vector<void*> allocs;
  size_t bytes = 0;
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  int64_t launches = 0;
  int coop_grid = 0;  // blocks of the persistent BP launch (0: launch per half-iteration)
  long long bar_limit_ns = 1000000000LL;  // bound of a grid-barrier wait
  int hold_barrier = 0;                   // timeout test: block 0 withholds an arrival
};

namespace {

int gfail(cudaError_t e) {
  record_cuda_error(e);
  return e == cudaErrorMemoryAllocation ? LSD_ERR_OOM : LSD_ERR_CUDA;
}

template <class T>
int galloc(lsd_giant* G, T** p, size_t count) {
  const size_t bytes = std::max<size_t>(count * sizeof(T), 16);
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    return gfail(e);
  }
  G->allocs.push_back(*p);
  G->bytes += bytes;
  return LSD_OK;
}

int grid_threads(const lsd_giant* G) { return G->sms * 8; }

int read_ctr(lsd_giant* G) {
  cudaError_t e = cudaMemcpyAsync(G->h_ctr, G->g.ctr, sizeof(GCtr), cudaMemcpyDeviceToHost,
                                  G->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(G->st);
  return e == cudaSuccess ? LSD_OK : gfail(e);
}

int check_launch(lsd_giant* G) {
  G->launches++;
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? LSD_OK : gfail(e);
}

// P-LSD of the shot; writes corr (zero unless solved) and the info fields.
int run_plsd(lsd_giant* G, const float* llr, const uint8_t* s, uint8_t* corr,
             lsd_giant_info* info) {
  const GD& g = G->g;
  const int grid = grid_threads(G);
  int rc;
  // counters of the whole call (BP fields are kept)
  {
    cudaError_t e = cudaMemsetAsync(g.ctr, 0, offsetof(GCtr, bp_stop), G->st);
    if (e == cudaSuccess)
      e = cudaMemsetAsync(&g.ctr->nu, 0, sizeof(GCtr) - offsetof(GCtr, nu), G->st);
    if (e != cudaSuccess) return gfail(e);
  }
  glsd_reset<<<grid, 256, 0, G->st>>>(g);
  if ((rc = check_launch(G))) return rc;
  glsd_seed<<<grid, 256, 0, G->st>>>(g, s);
  if ((rc = check_launch(G))) return rc;
  glsd_seed_count<<<1, 1, 0, G->st>>>(g);
  if ((rc = check_launch(G))) return rc;
  gzero<<<grid, 256, 0, G->st>>>(corr, G->n);
  if ((rc = check_launch(G))) return rc;
  int status = LSD_SHOT_OK_LSD, steps = 0, par = 0;
  if ((rc = read_ctr(G))) return rc;
  for (;;) {
    const GCtr& h = *G->h_ctr;
    if (h.overflow) return LSD_ERR_ADMISSION;
    if (h.uf_fail) return LSD_ERR_TIMEOUT;
    if (h.too_big) return LSD_ERR_UNSUPPORTED;
    if (h.unsolvable) {
      status = LSD_SHOT_UNSOLVABLE;
      break;
    }
    if (h.ninv[par] == 0) break;
    if (steps > G->n) {
      status = LSD_SHOT_UNSOLVABLE;
      break;
    }
    const int nxt = par ^ 1;
    cudaError_t e = cudaMemsetAsync(&g.ctr->nmerged, 0, 6 * sizeof(int), G->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(&g.ctr->ninv[nxt], 0, sizeof(int), G->st);
    if (e != cudaSuccess) return gfail(e);
    glsd_find<<<grid, 256, 0, G->st>>>(g, llr);
    if ((rc = check_launch(G))) return rc;
    glsd_union<<<grid, 256, 0, G->st>>>(g, par, 1);
    if ((rc = check_launch(G))) return rc;
    glsd_flatten<<<grid, 256, 0, G->st>>>(g);
    if ((rc = check_launch(G))) return rc;
    glsd_plan<<<grid, 256, 0, G->st>>>(g);
    if ((rc = check_launch(G))) return rc;
    glsd_relocate<<<grid, 256, 0, G->st>>>(g);
    if ((rc = check_launch(G))) return rc;
    glsd_absorb<<<grid, 256, 0, G->st>>>(g);
    if ((rc = check_launch(G))) return rc;
    glsd_claim<<<grid, 256, 0, G->st>>>(g);
    if ((rc = check_launch(G))) return rc;
    glsd_add<<<grid, 256, 0, G->st>>>(g);
    if ((rc = check_launch(G))) return rc;
    glsd_collect<<<grid, 256, 0, G->st>>>(g, nxt);
    if ((rc = check_launch(G))) return rc;
    // a step in which some invalid cluster found no candidate does not count (Alg. 1)
    if ((rc = read_ctr(G))) return rc;
    if (G->h_ctr->unsolvable) {
      status = LSD_SHOT_UNSOLVABLE;
      break;
    }
    ++steps;
    par = nxt;
  }
  // ---- LSD-mu: mu more steps in which every cluster grows, then local reprocessing ----
  if (status == LSD_SHOT_OK_LSD && g.order > 0) {
    for (int e = 0; e < g.order; ++e) {
      cudaError_t err = cudaMemsetAsync(&g.ctr->nmerged, 0, 6 * sizeof(int), G->st);
      if (err == cudaSuccess) err = cudaMemsetAsync(&g.ctr->ninv[par], 0, sizeof(int), G->st);
      if (err != cudaSuccess) return gfail(err);
      glsd_collect_all<<<grid, 256, 0, G->st>>>(g, par);
      if ((rc = check_launch(G))) return rc;
      glsd_find<<<grid, 256, 0, G->st>>>(g, llr);
      if ((rc = check_launch(G))) return rc;
      glsd_union<<<grid, 256, 0, G->st>>>(g, par, 0);
      if ((rc = check_launch(G))) return rc;
      glsd_flatten<<<grid, 256, 0, G->st>>>(g);
      if ((rc = check_launch(G))) return rc;
      glsd_plan<<<grid, 256, 0, G->st>>>(g);
      if ((rc = check_launch(G))) return rc;
      glsd_relocate<<<grid, 256, 0, G->st>>>(g);
      if ((rc = check_launch(G))) return rc;
      glsd_absorb<<<grid, 256, 0, G->st>>>(g);
      if ((rc = check_launch(G))) return rc;
      glsd_claim<<<grid, 256, 0, G->st>>>(g);
      if ((rc = check_launch(G))) return rc;
      glsd_add<<<grid, 256, 0, G->st>>>(g);
      if ((rc = check_launch(G))) return rc;
      if ((rc = read_ctr(G))) return rc;
      const GCtr& h = *G->h_ctr;
      if (h.overflow) return LSD_ERR_ADMISSION;
      if (h.uf_fail) return LSD_ERR_TIMEOUT;
      if (h.too_big) return LSD_ERR_UNSUPPORTED;
      if (h.nnew == 0 && h.nclaim == 0 && h.nmerged == 0) break;  // nothing could grow
    }
    glsd_dep_rank<<<grid, 256, 0, G->st>>>(g);
    if ((rc = check_launch(G))) return rc;
    glsd_dep_offsets<<<grid, 256, 0, G->st>>>(g);
    if ((rc = check_launch(G))) return rc;
    glsd_dep_place<<<grid, 256, 0, G->st>>>(g);
    if ((rc = check_launch(G))) return rc;
    glsd_reprocess<<<grid, 256, 0, G->st>>>(g, llr, corr);
    if ((rc = check_launch(G))) return rc;
  }
  glsd_solve<<<grid, 256, 0, G->st>>>(g, corr, status == LSD_SHOT_OK_LSD ? 1 : 0);
  if ((rc = check_launch(G))) return rc;
  if ((rc = read_ctr(G))) return rc;
  if (G->h_ctr->overflow) return LSD_ERR_ADMISSION;
  if (info) {
    info->status = status;
    info->nu = G->h_ctr->nu;
    info->kappa = G->h_ctr->kappa;
    info->steps = steps;
    info->arena_bytes_used = (int64_t)G->h_ctr->arena_top * 4;
  }
  return LSD_OK;
}

}  // namespace

extern "C" {

int lsd_giant_create(lsd_giant** out, int32_t m, int32_t n, int64_t nnz, const int32_t* rows,
                     const int32_t* cols, const float* channel_probs, int32_t bp_iters,
                     int32_t lsd_order, size_t arena_bytes, const lsd_options* opt) {
  if (!out) return LSD_ERR_INVALID_ARG;
  *out = nullptr;
  if (m < 1 || n < 1 || nnz < 1 || nnz >= INT32_MAX || !rows || !cols || !channel_probs ||
      bp_iters < 0)
    return LSD_ERR_INVALID_ARG;
  lsd_options o{};
  if (opt) o = *opt;
  if (o.ms_scaling < 0.f || lsd_order < 0 || o.osd_method < 0 || o.osd_method > 1 ||
      o.osd_cs_order < 0 || o.osd_cs_order > kMaxCsOrder ||
      (o.osd_method == 0 && o.osd_cs_order != 0) ||
      lsd_order > (o.osd_method == 1 ? kMaxCsGrowth : kMaxOrder))
    return LSD_ERR_INVALID_ARG;
  for (int j = 0; j < n; ++j)
    if (!(channel_probs[j] > 0.f && channel_probs[j] < 1.f)) return LSD_ERR_INVALID_ARG;
  std::vector<std::pair<int, int>> e((size_t)nnz);
  for (int64_t k = 0; k < nnz; ++k) {
    if (rows[k] < 0 || rows[k] >= m || cols[k] < 0 || cols[k] >= n) return LSD_ERR_INVALID_ARG;
    e[(size_t)k] = {rows[k], cols[k]};
  }
  std::sort(e.begin(), e.end());
  for (size_t k = 1; k < e.size(); ++k)
    if (e[k] == e[k - 1]) return LSD_ERR_INVALID_ARG;
  const int E = (int)e.size();
  std::vector<int> chk_ptr(m + 1, 0), var_ptr(n + 1, 0), chk_var(E), var_edge(E), var_chk(E);
  for (auto& p : e) {
    chk_ptr[p.first + 1]++;
    var_ptr[p.second + 1]++;
  }
  for (int i = 0; i < m; ++i) chk_ptr[i + 1] += chk_ptr[i];
  for (int j = 0; j < n; ++j) var_ptr[j + 1] += var_ptr[j];
  std::vector<int> fill(var_ptr.begin(), var_ptr.end() - 1);
  for (int k = 0; k < E; ++k) {  // ascending (row, column): each column's list ascends in row
    chk_var[k] = e[k].second;
    const int slot = fill[e[k].second]++;
    var_edge[slot] = k;
    var_chk[slot] = e[k].first;
  }
  int dc = 0, dv = 0;
  for (int i = 0; i < m; ++i) dc = std::max(dc, chk_ptr[i + 1] - chk_ptr[i]);
  for (int j = 0; j < n; ++j) dv = std::max(dv, var_ptr[j + 1] - var_ptr[j]);
  if (dc > 32) return LSD_ERR_UNSUPPORTED;  // check degree of the BP kernel
  std::vector<int> ell_col((size_t)dc * m, -1), ell_pos((size_t)dv * n, -1);
  for (int i = 0; i < m; ++i)
    for (int k = chk_ptr[i]; k < chk_ptr[i + 1]; ++k)
      ell_col[(size_t)(k - chk_ptr[i]) * m + i] = chk_var[k];
  for (int j = 0; j < n; ++j)
    for (int a = var_ptr[j]; a < var_ptr[j + 1]; ++a) {
      const int k = var_edge[a], i = var_chk[a];
      ell_pos[(size_t)(a - var_ptr[j]) * n + j] = (k - chk_ptr[i]) * m + i;
    }
  if ((size_t)dc * m >= (size_t)INT32_MAX) return LSD_ERR_UNSUPPORTED;

  lsd_giant* G = new (std::nothrow) lsd_giant();
  if (!G) return LSD_ERR_OOM;
  G->m = m;
  G->n = n;
  G->E = E;
  G->bp_iters = bp_iters;
  G->alpha = o.ms_scaling > 0.f ? o.ms_scaling : 0.625f;
  G->st = static_cast<cudaStream_t>(o.stream);
  GD& g = G->g;
  g.m = m;
  g.n = n;
  const size_t words = arena_bytes ? arena_bytes / 4 : ((size_t)64 << 20);  // 256 MiB
  int rc = LSD_OK;
  int *d_chk_ptr = nullptr, *d_chk_var = nullptr, *d_var_ptr = nullptr, *d_var_chk = nullptr;
  float *d_prior = nullptr, *d_probs = nullptr;
  long long* d_wfix = nullptr;
  auto A = [&](auto** p, size_t count) {
    if (rc == LSD_OK) rc = galloc(G, p, count);
  };
  A(&d_chk_ptr, m + 1);
  A(&d_chk_var, E);
  A(&d_var_ptr, n + 1);
  A(&d_var_chk, E);
  A(&d_prior, n);
  A(&d_probs, n);
  A(&d_wfix, n);
  int *d_ell_col = nullptr, *d_ell_pos = nullptr;
  A(&d_ell_col, (size_t)dc * m);
  A(&d_ell_pos, (size_t)dv * n);
  A(&g.r, (size_t)dc * m);
  A(&g.lam, n);
  A(&g.dlab, m);
  A(&g.lslot, m);
  A(&g.fst, n);
  A(&g.front, n);
  for (int** p : {&g.parent, &g.inv0, &g.inv1, &g.mlist, &g.chg, &g.cap, &g.nsl, &g.ncol,
                  &g.valid, &g.grow, &g.mark, &g.extra, &g.newslots, &g.aoff, &g.newcnt,
                  &g.boff, &g.nc_g, &g.nc_r, &g.nc_rank, &g.bucket, &g.cl_d, &g.cl_r,
                  &g.cl_rel})
    A(p, m);
  A(&g.best, m);
  A(&g.blk, m);
  A(&g.nc_key, m);
  A(&g.dep_f, n);
  A(&g.dep_rank, n);
  A(&g.dep_bucket, n);
  A(&g.depcnt, m);
  A(&g.depoff, m);
  A(&g.arena, words);
  A(&g.ctr, 1);
  g.arena_words = words;
  if (rc == LSD_OK) {
    cudaError_t err = cudaMallocHost(reinterpret_cast<void**>(&G->h_ctr), sizeof(GCtr));
    if (err != cudaSuccess) rc = gfail(err);
  }
  if (rc == LSD_OK) {
    cudaError_t err = cudaMemcpyAsync(d_chk_ptr, chk_ptr.data(), (m + 1) * sizeof(int),
                                      cudaMemcpyHostToDevice, G->st);
    if (err == cudaSuccess)
      err = cudaMemcpyAsync(d_chk_var, chk_var.data(), (size_t)E * sizeof(int),
                            cudaMemcpyHostToDevice, G->st);
    if (err == cudaSuccess)
      err = cudaMemcpyAsync(d_var_ptr, var_ptr.data(), (n + 1) * sizeof(int),
                            cudaMemcpyHostToDevice, G->st);
    if (err == cudaSuccess)
      err = cudaMemcpyAsync(d_var_chk, var_chk.data(), (size_t)E * sizeof(int),
                            cudaMemcpyHostToDevice, G->st);
    if (err == cudaSuccess)
      err = cudaMemcpyAsync(d_ell_col, ell_col.data(), ell_col.size() * sizeof(int),
                            cudaMemcpyHostToDevice, G->st);
    if (err == cudaSuccess)
      err = cudaMemcpyAsync(d_ell_pos, ell_pos.data(), ell_pos.size() * sizeof(int),
                            cudaMemcpyHostToDevice, G->st);
    if (err == cudaSuccess)
      err = cudaMemcpyAsync(d_probs, channel_probs, (size_t)n * sizeof(float),
                            cudaMemcpyHostToDevice, G->st);
    if (err == cudaSuccess) err = launch_priors(d_probs, d_prior, d_wfix, n, G->st);
    if (err == cudaSuccess) err = cudaStreamSynchronize(G->st);
    if (err != cudaSuccess) rc = gfail(err);
  }
  if (rc == LSD_OK) {
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err == cudaSuccess)
      err = cudaDeviceGetAttribute(&G->sms, cudaDevAttrMultiProcessorCount, dev);
    for (int k = 0; k < 3 && err == cudaSuccess; ++k) err = cudaEventCreate(&G->ev[k]);
    // the persistent BP launch: every block must be resident at once (cooperative launch)
    int coop = 0, per_sm = 0;
    if (err == cudaSuccess) err = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    const void* fn = dc <= 8    ? (const void*)gbp_persistent<8>
                     : dc <= 16 ? (const void*)gbp_persistent<16>
                                : (const void*)gbp_persistent<32>;
    if (err == cudaSuccess && coop)
      err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 256, 0);
    if (err == cudaSuccess && coop && per_sm > 0) {
      const long long need = (std::max<long long>(m, n) + 255) / 256;
      G->coop_grid = (int)std::min<long long>(need, (long long)per_sm * G->sms);
    }
    if (err != cudaSuccess) rc = gfail(err);
  }
  g.dc = dc;
  g.dv = dv;
  g.order = lsd_order;
  g.osd_cs = o.osd_method == 1 ? o.osd_cs_order : -1;
  g.wfix = d_wfix;
  g.ell_col = d_ell_col;
  g.ell_pos = d_ell_pos;
  g.chk_ptr = d_chk_ptr;
  g.chk_var = d_chk_var;
  g.var_ptr = d_var_ptr;
  g.var_chk = d_var_chk;
  g.prior = d_prior;
  if (rc != LSD_OK) {
    lsd_giant_destroy(G);
    return rc;
  }
  *out = G;
  return LSD_OK;
}

int lsd_giant_postprocess(lsd_giant* G, const float* llr, const uint8_t* syndrome,
                          uint8_t* correction, lsd_giant_info* info) {
  if (!G || !llr || !syndrome || !correction) return LSD_ERR_INVALID_ARG;
  if (info) std::memset(info, 0, sizeof(*info));
  cudaEventRecord(G->ev[1], G->st);
  const int rc = run_plsd(G, llr, syndrome, correction, info);
  if (rc) return rc;
  cudaEventRecord(G->ev[2], G->st);
  cudaError_t e = cudaEventSynchronize(G->ev[2]);
  if (e != cudaSuccess) return gfail(e);
  if (info) cudaEventElapsedTime(&info->ms_lsd, G->ev[1], G->ev[2]);
  return LSD_OK;
}

int lsd_giant_decode(lsd_giant* G, const uint8_t* syndrome, uint8_t* correction,
                     float* posteriors, lsd_giant_info* info) {
  if (!G || !syndrome || !correction) return LSD_ERR_INVALID_ARG;
  if (info) std::memset(info, 0, sizeof(*info));
  const GD& g = G->g;
  const int grid = grid_threads(G);
  int rc;
  cudaEventRecord(G->ev[0], G->st);
  cudaError_t e = cudaMemsetAsync(g.ctr, 0, sizeof(GCtr), G->st);
  if (e != cudaSuccess) return gfail(e);
  gbp_init<<<grid, 256, 0, G->st>>>(g);
  if ((rc = check_launch(G))) return rc;
  // iterations in chunks of 2, 4, 8, ... with a look at the stop flag after each, so that a
  // shot that converges early is not followed by the remaining iterations' launches
  bool stopped = false;
  if (G->bp_iters > 0 && G->coop_grid > 0) {
    // one persistent launch for every iteration (grid barriers between the halves)
    const uint8_t* sp = syndrome;
    float alpha = G->alpha;
    int T = G->bp_iters;
    long long limit = G->bar_limit_ns;
    int hold = G->hold_barrier;
    void* args[] = {(void*)&g, (void*)&sp, (void*)&alpha, (void*)&T, (void*)&limit, (void*)&hold};
    const void* fn = g.dc <= 8    ? (const void*)gbp_persistent<8>
                     : g.dc <= 16 ? (const void*)gbp_persistent<16>
                                  : (const void*)gbp_persistent<32>;
    e = cudaLaunchCooperativeKernel(fn, G->coop_grid, 256, args, 0, G->st);
    G->launches++;
    if (e != cudaSuccess) return gfail(e);
    stopped = true;
  }
  for (int t = 1, chunk = 2; t <= G->bp_iters && !stopped; chunk *= 2) {
    const int t1 = std::min(G->bp_iters, t + chunk - 1);
    for (; t <= t1; ++t) {
      if (g.dc <= 8)
        gbp_check<8><<<grid, 256, 0, G->st>>>(g, syndrome, G->alpha, t);
      else if (g.dc <= 16)
        gbp_check<16><<<grid, 256, 0, G->st>>>(g, syndrome, G->alpha, t);
      else
        gbp_check<32><<<grid, 256, 0, G->st>>>(g, syndrome, G->alpha, t);
      if ((rc = check_launch(G))) return rc;
      gbp_var<<<grid, 256, 0, G->st>>>(g, t);
      if ((rc = check_launch(G))) return rc;
    }
    if ((rc = read_ctr(G))) return rc;
    stopped = G->h_ctr->bp_stop != 0;
  }
  if (G->bp_iters > 0 && !stopped) {
    const int slot = (G->bp_iters + 1) & 1;
    gbp_syn<<<grid, 256, 0, G->st>>>(g, syndrome, slot);
    if ((rc = check_launch(G))) return rc;
    gbp_final<<<1, 1, 0, G->st>>>(g, slot);
    if ((rc = check_launch(G))) return rc;
  }
  if (posteriors) {
    e = cudaMemcpyAsync(posteriors, g.lam, (size_t)G->n * sizeof(float),
                        cudaMemcpyDeviceToDevice, G->st);
    if (e != cudaSuccess) return gfail(e);
  }
  cudaEventRecord(G->ev[1], G->st);
  if ((rc = read_ctr(G))) return rc;
  if (G->h_ctr->bp_fail) return LSD_ERR_TIMEOUT;
  const int conv = G->h_ctr->bp_conv, iters = G->h_ctr->bp_iters;
  if (conv) {
    gcopy_hard<<<grid, 256, 0, G->st>>>(g, correction);
    if ((rc = check_launch(G))) return rc;
    if (info) info->status = LSD_SHOT_OK_BP;
  } else {
    rc = run_plsd(G, g.lam, syndrome, correction, info);
    if (rc) return rc;
  }
  cudaEventRecord(G->ev[2], G->st);
  e = cudaEventSynchronize(G->ev[2]);
  if (e != cudaSuccess) return gfail(e);
  if (info) {
    info->bp_iterations = iters;
    cudaEventElapsedTime(&info->ms_bp, G->ev[0], G->ev[1]);
    cudaEventElapsedTime(&info->ms_lsd, G->ev[1], G->ev[2]);
  }
  return LSD_OK;
}

int lsd_giant_test_hold_barrier(lsd_giant* G, int32_t hold, int64_t limit_ns) {
  if (!G || limit_ns < 0) return LSD_ERR_INVALID_ARG;
  if (!G->coop_grid) return LSD_ERR_UNSUPPORTED;
  G->hold_barrier = hold ? 1 : 0;
  G->bar_limit_ns = hold ? (long long)limit_ns : 1000000000LL;
  return LSD_OK;
}

int lsd_giant_kernel_launches(const lsd_giant* G, int64_t* count) {
  if (!G || !count) return LSD_ERR_INVALID_ARG;
  *count = G->launches;
  return LSD_OK;
}

int lsd_giant_destroy(lsd_giant* G) {
  if (!G) return LSD_OK;
  cudaStreamSynchronize(G->st);
  for (void* p : G->allocs) cudaFree(p);
  if (G->h_ctr) cudaFreeHost(G->h_ctr);
  for (auto& ev : G->ev)
    if (ev) cudaEventDestroy(ev);
  delete G;
  return LSD_OK;
}

}  // extern "C"
