// Localized statistics decoding kernel (Alg. 1 of Sec. 4.1, on-the-fly elimination of
// Sec. 4.2, LSD-mu of App. D).
//
// One warp owns one shot; a persistent grid pulls shots from a device work queue (the
// unconverged shots BP appended, or every shot for lsd_postprocess_batch).
//
// Per-shot state in shared memory (m detectors, n faults, W = ceil(m/32) words):
//   dlab[m]    cluster label of each detector (-1: in no cluster).  Labels are the
//              seed detectors (one cluster per flipped detector, Alg. 1 init).
//   parent[m]  union-find forest over labels; a merge links the larger root under the
//              smaller one with a CAS (Alg. 2's parallel_union), so a cluster's root is
//              its smallest seed.
//   flab[n]    fault state: -2 untouched, -1 candidate (adjacent to a cluster detector,
//              Def. 4.3's Lambda(C) over all clusters), >= 0 label of its cluster.
//   R[m][W], T[m][W], pcol[m]: the elimination state of every cluster at once.  A
//              pivot column is stored at its pivot row d: R[d] is the reduced column
//              (bit d set, zero at every other pivot row), T[d] the set of pivot rows
//              whose original columns XOR to R[d], pcol[d] the fault it came from.
//              Rows of different clusters never mix, so the factorization of a merged
//              cluster is the union of its parts: the block-swap of Sec. 4.2 is free.
//   sred[W]    s reduced by the pivots; xsol[W] the pivot rows whose columns XOR to
//              s - sred.  A cluster is valid (Def. 4.2) iff sred has no bit on its rows.
//
// A growth step: every growing cluster takes its lowest-(LLR, index) candidate
// (atomicMin on a 64-bit order key), all picks are applied together, clusters that now
// share a detector (or a fault) are merged, then the new columns are eliminated one by
// one in key order: b' = b + sum of R[d] over pivot rows d in supp(b) (one XOR per
// nonzero of the sparse column), a new pivot at the lowest set bit of b', and
// back-elimination of that row from the other pivots.  Validity is re-read from sred.
#include <climits>

#include "lsd_internal.cuh"

namespace lsdgb {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr unsigned long long kNoKey = ~0ull;

__host__ __device__ inline size_t al8(size_t x) { return (x + 7) & ~(size_t)7; }
__host__ __device__ inline size_t al16(size_t x) { return (x + 15) & ~(size_t)15; }

struct Lay {
  size_t R, T, best, newk, srt, dlab, parent, pcol, inv, flab, llr, words, scal, rflag, npk, npN,
      ext, total;
};

__host__ __device__ inline Lay lsd_layout(int m, int n, int W, int order) {
  Lay L;
  size_t o = 0;
  L.R = o; o += (size_t)m * W * 4;
  L.T = o; o += (size_t)m * W * 4;
  o = al8(o);
  L.best = o; o += (size_t)m * 8;
  L.newk = o; o += (size_t)m * 8;
  L.srt = o; o += (size_t)m * 8;
  L.npk = o; o += order > 0 ? (size_t)n * 8 : 0;
  L.dlab = o; o += (size_t)m * 4;
  L.parent = o; o += (size_t)m * 4;
  L.pcol = o; o += (size_t)m * 4;
  L.inv = o; o += (size_t)m * 4;
  L.flab = o; o += (size_t)n * 4;
  L.llr = o; o += (size_t)n * 4;
  L.words = o; o += (size_t)4 * W * 4;
  L.scal = o; o += 16 * 4;
  L.npN = o; o += order > 0 ? (size_t)n * W * 4 : 0;
  L.ext = o; o += order > 0 ? (size_t)n * 4 : 0;
  L.rflag = o; o += (size_t)m;
  L.total = al16(o);
  return L;
}

struct Shot {
  uint32_t *R, *T, *syn, *sred, *xsol, *cm, *npN;
  unsigned long long *best, *newk, *srt, *npk;
  int *dlab, *parent, *pcol, *inv, *flab, *scal, *ext;
  float* llr;
  unsigned char* rflag;
};

// Order key of fault j: (LLR ascending, index ascending).  -0.0 is folded into +0.0 so
// that the key order is the float order, with ties broken by the index.
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

__device__ __forceinline__ void uf_unite(int* parent, int a, int b) {
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
    if (atomicCAS(parent + a, a, b) == a) return;
  }
}

__device__ __forceinline__ bool bit_of(const uint32_t* v, int i) {
  return (v[i >> 5] >> (i & 31)) & 1u;
}

// Roots of all clusters (pred = every alive seed) or of the invalid ones (sred bits).
__device__ int collect_roots(const LSDArgs& a, Shot& S, int m, bool only_invalid, int lane) {
  if (only_invalid) {
    for (int d = lane; d < m; d += 32) S.rflag[d] = 0;
    __syncwarp();
    for (int d = lane; d < m; d += 32) {
      if (bit_of(S.sred, d)) {
        const int lab = S.dlab[d];
        if (lab >= 0) S.rflag[uf_find(S.parent, lab)] = 1;
      }
    }
    __syncwarp();
  }
  int count = 0;
  for (int base = 0; base < m; base += 32) {
    const int d = base + lane;
    const bool seed = d < m && (a.single_cluster ? d == 0 : bit_of(S.syn, d));
    const bool pred = seed && S.parent[d] == d && (!only_invalid || S.rflag[d]);
    const unsigned bal = __ballot_sync(kFull, pred);
    if (pred) S.inv[count + __popc(bal & ((1u << lane) - 1u))] = d;
    count += __popc(bal);
  }
  __syncwarp();
  if (only_invalid) {
    for (int d = lane; d < m; d += 32) S.rflag[d] = 0;
    __syncwarp();
  }
  return count;
}

// Adds fault column gcol (key = its order key) to its cluster's factorization.
__device__ void add_column(const LSDArgs& a, Shot& S, int m, int W, int gcol,
                           unsigned long long key, int lane) {
  const DevGraph& g = a.g;
  uint32_t bw = 0, tw = 0;
  if (lane < W) {
    const int v1 = g.var_ptr[gcol + 1];
    for (int q = g.var_ptr[gcol]; q < v1; ++q) {
      const int d = g.var_chk[q];
      if ((d >> 5) == lane) bw ^= 1u << (d & 31);
      if (S.pcol[d] >= 0) {
        bw ^= S.R[d * W + lane];
        tw ^= S.T[d * W + lane];
      }
    }
  }
  const unsigned nz = __ballot_sync(kFull, lane < W && bw != 0);
  if (nz == 0) {
    // dependent column: remember its representation for LSD-mu's OSD-E
    if (a.order > 0) {
      const int slot = __shfl_sync(kFull, S.scal[1], 0);
      if (lane < W) S.npN[slot * W + lane] = tw;
      if (lane == 0) {
        S.npk[slot] = key;
        S.scal[1] = slot + 1;
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
  const bool sflag = (S.sred[pw] & pb) != 0;
  if (lane < W) {
    S.R[p * W + lane] = bw;
    S.T[p * W + lane] = tw;
  }
  if (lane == 0) S.pcol[p] = gcol;
  __syncwarp();
  for (int d = lane; d < m; d += 32) {
    if (d == p || S.pcol[d] < 0) continue;
    if (S.R[d * W + pw] & pb) {
      for (int w = 0; w < W; ++w) {
        S.R[d * W + w] ^= S.R[p * W + w];
        S.T[d * W + w] ^= S.T[p * W + w];
      }
    }
  }
  if (sflag && lane < W) {
    S.sred[lane] ^= bw;
    S.xsol[lane] ^= tw;
  }
  __syncwarp();
}

// One synchronous growth step of the k clusters listed in S.inv.
// Returns 0 if clusters grew, 1 if strict and a cluster had no candidate, 2 if none grew.
__device__ int lsd_step(const LSDArgs& a, Shot& S, int m, int n, int W, int k, bool strict,
                        int lane) {
  const DevGraph& g = a.g;
  for (int t = lane; t < k; t += 32) {
    const int r = S.inv[t];
    S.best[r] = kNoKey;
    S.rflag[r] = 1;
  }
  __syncwarp();
  // find_candidate: every candidate fault offers itself to the growing clusters it touches
  for (int j = lane; j < n; j += 32) {
    if (S.flab[j] != -1) continue;
    const unsigned long long key = llr_key(S.llr[j], j);
    const int v1 = g.var_ptr[j + 1];
    for (int q = g.var_ptr[j]; q < v1; ++q) {
      const int lab = S.dlab[g.var_chk[q]];
      if (lab < 0) continue;
      const int root = uf_find(S.parent, lab);
      if (S.rflag[root]) atomicMin(&S.best[root], key);
    }
  }
  __syncwarp();
  bool none = false, some = false;
  for (int t = lane; t < k; t += 32) {
    if (S.best[S.inv[t]] == kNoKey) none = true;
    else some = true;
  }
  none = __any_sync(kFull, none);
  some = __any_sync(kFull, some);
  if ((strict && none) || !some) {
    for (int t = lane; t < k; t += 32) S.rflag[S.inv[t]] = 0;
    __syncwarp();
    return (strict && none) ? 1 : 2;
  }
  if (lane == 0) S.scal[0] = 0;
  __syncwarp();
  // parallel_union: apply every pick, merge clusters that now share a detector or a fault
  for (int t = lane; t < k; t += 32) {
    const int r = S.inv[t];
    S.rflag[r] = 0;
    const unsigned long long key = S.best[r];
    if (key == kNoKey) continue;
    const int gcol = (int)(key & 0xffffffffu);
    const int old = atomicCAS(&S.flab[gcol], -1, r);
    if (old == -1) {
      const int slot = atomicAdd(&S.scal[0], 1);
      S.newk[slot] = key;
    } else {
      uf_unite(S.parent, r, old);
    }
    const int v1 = g.var_ptr[gcol + 1];
    for (int q = g.var_ptr[gcol]; q < v1; ++q) {
      const int d = g.var_chk[q];
      const int o = atomicCAS(&S.dlab[d], -1, r);
      if (o == -1) {
        const int c1 = g.chk_ptr[d + 1];
        for (int e = g.chk_ptr[d]; e < c1; ++e) atomicCAS(&S.flab[g.chk_var[e]], -2, -1);
      } else if (o != r) {
        uf_unite(S.parent, r, o);
      }
    }
  }
  __syncwarp();
  // the step's new columns in reliability order (rank by counting; keys are distinct)
  const int n_new = S.scal[0];
  for (int t = lane; t < n_new; t += 32) {
    const unsigned long long kt = S.newk[t];
    int rank = 0;
    for (int u = 0; u < n_new; ++u) rank += (S.newk[u] < kt) ? 1 : 0;
    S.srt[rank] = kt;
  }
  __syncwarp();
  for (int t = 0; t < n_new; ++t) {
    const unsigned long long key = S.srt[t];
    add_column(a, S, m, W, (int)(key & 0xffffffffu), key, lane);
  }
  return 0;
}

// LSD-mu reprocessing (App. D): exhaustive OSD over the first min(mu, #dependent) dependent
// columns of each cluster, in reliability order; cost = sum of 2^-32 fixed-point channel
// weights; ties go to the smaller pattern.  Updates xsol and appends the chosen dependent
// columns to S.ext.
__device__ void osd_e(const LSDArgs& a, Shot& S, int m, int W, int lane) {
  const DevGraph& g = a.g;
  const int order = a.order;
  const int nroots = collect_roots(a, S, m, false, lane);
  const int n_np = S.scal[1];
  for (int ci = 0; ci < nroots; ++ci) {
    const int r = S.inv[ci];
    for (int c = 0; c < W; ++c) {
      const int d = c * 32 + lane;
      const bool in = d < m && S.dlab[d] >= 0 && uf_find(S.parent, S.dlab[d]) == r;
      const unsigned bal = __ballot_sync(kFull, in);
      if (lane == 0) S.cm[c] = bal;
    }
    __syncwarp();
    int sel[kMaxOrder];
    int nt = 0;
    unsigned long long last = 0;
    for (int it = 0; it < order; ++it) {
      unsigned long long bk = kNoKey;
      int bi = -1;
      for (int u = lane; u < n_np; u += 32) {
        const unsigned long long ku = S.npk[u];
        if (it > 0 && ku <= last) continue;
        const int gu = (int)(ku & 0xffffffffu);
        if (uf_find(S.parent, S.flab[gu]) != r) continue;
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
        uint32_t mw = S.xsol[w] & S.cm[w];
        for (int k2 = 0; k2 < nt; ++k2)
          if ((t >> k2) & 1) mw ^= S.npN[sel[k2] * W + w];
        while (mw) {
          const int b = __ffs(mw) - 1;
          mw &= mw - 1;
          cost += g.wfix[S.pcol[w * 32 + b]];
        }
      }
      for (int k2 = 0; k2 < nt; ++k2)
        if ((t >> k2) & 1) cost += g.wfix[(int)(S.npk[sel[k2]] & 0xffffffffu)];
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
        if ((bt >> k2) & 1) delta ^= S.npN[sel[k2] * W + lane];
      S.xsol[lane] ^= delta;
    }
    if (lane == 0) {
      int ne = S.scal[2];
      for (int k2 = 0; k2 < nt; ++k2)
        if ((bt >> k2) & 1) S.ext[ne++] = (int)(S.npk[sel[k2]] & 0xffffffffu);
      S.scal[2] = ne;
    }
    __syncwarp();
  }
}

__global__ void __launch_bounds__(256) lsd_kernel(LSDArgs a, int W) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int m = a.g.m, n = a.g.n;
  const Lay L = lsd_layout(m, n, W, a.order);
  unsigned char* base = smem + (size_t)warp * L.total;
  Shot S;
  S.R = reinterpret_cast<uint32_t*>(base + L.R);
  S.T = reinterpret_cast<uint32_t*>(base + L.T);
  S.best = reinterpret_cast<unsigned long long*>(base + L.best);
  S.newk = reinterpret_cast<unsigned long long*>(base + L.newk);
  S.srt = reinterpret_cast<unsigned long long*>(base + L.srt);
  S.npk = reinterpret_cast<unsigned long long*>(base + L.npk);
  S.dlab = reinterpret_cast<int*>(base + L.dlab);
  S.parent = reinterpret_cast<int*>(base + L.parent);
  S.pcol = reinterpret_cast<int*>(base + L.pcol);
  S.inv = reinterpret_cast<int*>(base + L.inv);
  S.flab = reinterpret_cast<int*>(base + L.flab);
  S.llr = reinterpret_cast<float*>(base + L.llr);
  S.syn = reinterpret_cast<uint32_t*>(base + L.words);
  S.sred = S.syn + W;
  S.xsol = S.sred + W;
  S.cm = S.xsol + W;
  S.scal = reinterpret_cast<int*>(base + L.scal);
  S.npN = reinterpret_cast<uint32_t*>(base + L.npN);
  S.ext = reinterpret_cast<int*>(base + L.ext);
  S.rflag = base + L.rflag;

  const long long count = a.count_from_ctr ? (long long)a.ctr->lsd_count : a.count;
  unsigned long long steps_acc = 0, unsolv = 0;
  int kappa_max = 0, nu_max = 0;
  for (;;) {
    unsigned long long item = 0;
    if (lane == 0) item = atomicAdd(&a.ctr->lsd_next, 1ULL);
    item = __shfl_sync(kFull, item, 0);
    if (item >= (unsigned long long)count) break;
    const long long shot = a.queue ? (long long)a.queue[item] : (long long)item;
    const float* lsrc = a.llr + (a.llr_by_item ? (long long)item : shot) * n;
    const uint8_t* ssrc = a.syndromes + shot * m;

    // ---- init: one cluster per flipped detector ----
    for (int j = lane; j < n; j += 32) {
      S.llr[j] = lsrc[j];
      S.flab[j] = -2;
    }
    for (int d = lane; d < m; d += 32) {
      S.dlab[d] = -1;
      S.parent[d] = d;
      S.pcol[d] = -1;
      S.rflag[d] = 0;
    }
    for (int c = 0; c < W; ++c) {
      const int d = c * 32 + lane;
      const unsigned bv = __ballot_sync(kFull, d < m && ssrc[d] != 0);
      if (lane == 0) {
        S.syn[c] = bv;
        S.sred[c] = bv;
        S.xsol[c] = 0;
      }
    }
    if (lane < 4) S.scal[lane] = 0;
    __syncwarp();
    int k = 0;
    if (a.single_cluster) {
      for (int d = lane; d < m; d += 32) S.dlab[d] = 0;
      for (int j = lane; j < n; j += 32)
        if (a.g.var_ptr[j + 1] > a.g.var_ptr[j]) S.flab[j] = -1;
      bool anys = false;
      for (int c = 0; c < W; ++c) anys = anys || S.syn[c] != 0;
      k = anys ? 1 : 0;
      if (lane == 0) S.inv[0] = 0;
    } else {
      for (int b0 = 0; b0 < m; b0 += 32) {
        const int d = b0 + lane;
        const bool f = d < m && bit_of(S.syn, d);
        const unsigned bal = __ballot_sync(kFull, f);
        if (f) {
          S.dlab[d] = d;
          S.inv[k + __popc(bal & ((1u << lane) - 1u))] = d;
          const int c1 = a.g.chk_ptr[d + 1];
          for (int e = a.g.chk_ptr[d]; e < c1; ++e) S.flab[a.g.chk_var[e]] = -1;
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
      if (lsd_step(a, S, m, n, W, k, true, lane) == 1) {
        status = LSD_SHOT_UNSOLVABLE;
        break;
      }
      ++steps;
      k = collect_roots(a, S, m, true, lane);
    }
    // ---- LSD-mu: mu more steps for every cluster, then local OSD-E ----
    if (status == LSD_SHOT_OK_LSD && a.order > 0) {
      for (int e = 0; e < a.order; ++e) {
        k = collect_roots(a, S, m, false, lane);
        if (lsd_step(a, S, m, n, W, k, false, lane) == 2) break;
      }
      osd_e(a, S, m, W, lane);
    }

    // ---- statistics: nu clusters, kappa = largest cluster in columns ----
    for (int d = lane; d < m; d += 32) S.best[d] = 0;
    __syncwarp();
    for (int j = lane; j < n; j += 32) {
      const int lab = S.flab[j];
      if (lab >= 0) atomicAdd(&S.best[uf_find(S.parent, lab)], 1ULL);
    }
    __syncwarp();
    int nu = 0, kappa = 0;
    for (int d = lane; d < m; d += 32) {
      const bool seed = a.single_cluster ? d == 0 : bit_of(S.syn, d);
      if (seed && S.parent[d] == d) {
        ++nu;
        kappa = max(kappa, (int)S.best[d]);
      }
    }
    for (int off = 16; off > 0; off >>= 1) {
      nu += __shfl_xor_sync(kFull, nu, off);
      kappa = max(kappa, __shfl_xor_sync(kFull, kappa, off));
    }

    // ---- global decoding: union of the local solutions (Eq. 2) ----
    uint8_t* cs = reinterpret_cast<uint8_t*>(S.llr);  // LLRs are no longer needed
    for (int j = lane; j < n; j += 32) cs[j] = 0;
    __syncwarp();
    if (status == LSD_SHOT_OK_LSD) {
      for (int d = lane; d < m; d += 32)
        if (bit_of(S.xsol, d)) cs[S.pcol[d]] = 1;
      const int ne = S.scal[2];
      for (int t = lane; t < ne; t += 32) cs[S.ext[t]] = 1;
    }
    __syncwarp();
    uint8_t* co = a.corrections + shot * n;
    for (int j = lane; j < n; j += 32) co[j] = cs[j];
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

}  // namespace

cudaError_t lsd_config(const DevGraph& g, int order, int warps, int* warps_out, int* grid,
                       size_t* smem, int* words) {
  int dev = 0, sms = 0, max_smem = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const int W = (g.m + 31) / 32;
  if (W > kMaxLsdWords) return cudaErrorInvalidValue;
  const size_t per = lsd_layout(g.m, g.n, W, order).total;
  int w = warps > 0 ? warps : 8;
  while (w > 1 && per * w > (size_t)max_smem) --w;
  if (per * w > (size_t)max_smem) return cudaErrorInvalidValue;
  *smem = per * w;
  *words = W;
  *warps_out = w;
  // the limit is a property of the function, shared by every decoder: allow the maximum
  err = cudaFuncSetAttribute(lsd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
  if (err != cudaSuccess) return err;
  int per_sm = 0;
  err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lsd_kernel, w * 32, *smem);
  if (err != cudaSuccess) return err;
  if (per_sm < 1) return cudaErrorInvalidValue;
  *grid = per_sm * sms;
  return cudaSuccess;
}

cudaError_t launch_lsd(const LSDArgs& a, int warps, int grid, size_t smem, cudaStream_t st) {
  const int W = (a.g.m + 31) / 32;
  lsd_kernel<<<grid, warps * 32, smem, st>>>(a, W);
  return cudaGetLastError();
}

}  // namespace lsdgb
