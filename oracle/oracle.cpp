// CPU oracle for BP + localized statistics decoding (LSD).
//
// TEST INFRASTRUCTURE ONLY.  This file is a plain, slow restatement of the
// method (arXiv 2406.18655) used to check the GPU library.  It shares no code,
// header, table or constant generator with the CUDA path, and nothing in the
// product imports it: only tests/, __graft_entry__.smoke() and bench.py's CPU
// baseline call it.
//
// Parts and the passages they follow:
//   * BP: min-sum (scaling alpha, flooding schedule, early exit on H.e = s),
//     Sec. 4.3 "Numerical decoding simulations" (min-sum, alpha = 0.625,
//     parallel schedule) and App. C.4 (BP runs first; LSD only if BP fails).
//     The paper does not print the update rules; the standard min-sum and
//     sum-product rules are used (reading O1).  Arithmetic in double, or in an
//     FP32 mirror mode that rounds every operation to float in a fixed order.
//   * GF(2): column echelon form, reduction in pivot-creation order (plain
//     Gaussian elimination; Sec. 4.2 names PLU, any exact elimination gives
//     the same greedy pivot set and the same solution on it).
//   * OSD-0: Sec. 2.2 "Inversion decoding": columns in reliability order, the
//     greedy independent set I, e_[I] = H_[I]^-1 s.
//   * LSD: Alg. 1 (Sec. 4.1) with Defs. 4.1-4.4: one cluster per flipped
//     detector, growth by the most reliable candidate (lowest LLR, ties to the
//     lower column index), merge on shared detectors, validity
//     s_[C] in image(H_[C]), local solve, union of local solutions (Eq. 2).
//     Growth is synchronous: every invalid cluster picks from the same
//     snapshot, then all picks are applied and colliding clusters merge
//     (the find_candidate / parallel_union split of Alg. 2).
//     Every validity check re-eliminates the cluster from scratch (no
//     on-the-fly elimination here).
//   * LSD-mu: App. D: after LSD-0, up to mu extra synchronous growth steps on
//     every cluster (merges allowed, clusters stay valid), then exhaustive
//     OSD-E over the first min(mu, #non-pivots) non-pivot columns of each
//     cluster.  Costs are sums of channel-prior weights in 2^-32 fixed point.
//     Alternatively (the BB experiment of App. D, which fixes the local
//     reprocessing to OSD-CS-4) the combination sweep of order w over the
//     cluster's non-pivot columns in reliability order: no flip, every single
//     non-pivot column, every pair among the first w; the first pattern of
//     least cost in that order wins.
//   * Logical failure: residual r = e + e_hat is a logical error iff
//     r is not in the row space of H_Z (rank test).
//
// Parity status: every function above is pinned by tests/test_oracle_*.py
// (brute force, tree exactness, closed forms, invariants, worked example); the
// FP32 mirror of sum-product is pinned to exact tree inference within a
// rounding bound derived from float tanh/atanh.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <thread>
#include <vector>

namespace {

typedef std::vector<uint64_t> Bits;

inline int nwords(int nbits) { return (nbits + 63) / 64; }
inline bool bit(const Bits& b, int i) { return (b[i >> 6] >> (i & 63)) & 1u; }
inline void setbit(Bits& b, int i) { b[i >> 6] |= (uint64_t)1 << (i & 63); }
inline void xorin(Bits& a, const Bits& b) { for (size_t k = 0; k < a.size(); ++k) a[k] ^= b[k]; }
inline bool anybit(const Bits& a) { for (uint64_t w : a) if (w) return true; return false; }
inline int lowbit(const Bits& a) {
  for (size_t k = 0; k < a.size(); ++k)
    if (a[k]) return (int)(k * 64 + __builtin_ctzll(a[k]));
  return -1;
}
inline bool intersects(const Bits& a, const Bits& b) {
  for (size_t k = 0; k < a.size(); ++k) if (a[k] & b[k]) return true;
  return false;
}

// Tanner graph of H: rows (checks / detectors) and columns (variables / faults).
struct Graph {
  int m = 0, n = 0;
  std::vector<int> rptr, rcol;   // row i -> columns, ascending
  std::vector<int> cptr, crow;   // column j -> rows, ascending
  std::vector<Bits> colbits;     // column j as an m-bit vector
};

int build_graph(int m, int n, int64_t nnz, const int32_t* rows, const int32_t* cols, Graph& g) {
  if (m < 0 || n < 0 || nnz < 0) return -1;
  std::vector<std::pair<int, int>> e((size_t)nnz);
  for (int64_t k = 0; k < nnz; ++k) {
    if (rows[k] < 0 || rows[k] >= m || cols[k] < 0 || cols[k] >= n) return -1;
    e[(size_t)k] = {rows[k], cols[k]};
  }
  std::sort(e.begin(), e.end());
  for (size_t k = 1; k < e.size(); ++k) if (e[k] == e[k - 1]) return -1;
  g.m = m; g.n = n;
  g.rptr.assign(m + 1, 0); g.cptr.assign(n + 1, 0);
  for (auto& p : e) { g.rptr[p.first + 1]++; g.cptr[p.second + 1]++; }
  for (int i = 0; i < m; ++i) g.rptr[i + 1] += g.rptr[i];
  for (int j = 0; j < n; ++j) g.cptr[j + 1] += g.cptr[j];
  g.rcol.resize(e.size()); g.crow.resize(e.size());
  std::vector<int> rf(g.rptr.begin(), g.rptr.end() - 1), cf(g.cptr.begin(), g.cptr.end() - 1);
  for (auto& p : e) { g.rcol[rf[p.first]++] = p.second; }
  // column lists ascending in row: e is sorted by (row, col), so filling in this order works
  for (auto& p : e) { g.crow[cf[p.second]++] = p.first; }
  g.colbits.assign(n, Bits(nwords(m), 0));
  for (auto& p : e) setbit(g.colbits[p.second], p.first);
  return 0;
}

// --------------------------------------------------------------------------
// BP
// --------------------------------------------------------------------------

// Magnitude used for a minimum over an empty set (a check of degree 1):
// a large finite value instead of infinity, 2^100 exactly in both precisions.
const double kEmptyMin = 1267650600228229401496703205376.0;  // 2^100

// One shot of BP.  Edge k of the row-major list (check i, its t-th column) has
// message slots q[k] (variable -> check) and r[k] (check -> variable).
template <typename R>
void bp_shot(const Graph& g, const std::vector<int>& col_edges_ptr, const std::vector<int>& col_edges,
             const R* lam, const uint8_t* s, int iters, R alpha, int method, int early_exit,
             R* Lam, uint8_t* hard, int* iters_used, uint8_t* converged) {
  const int m = g.m, n = g.n;
  const size_t E = g.rcol.size();
  std::vector<R> q(E), r(E);
  for (int i = 0; i < m; ++i)
    for (int k = g.rptr[i]; k < g.rptr[i + 1]; ++k) q[k] = lam[g.rcol[k]];
  for (int j = 0; j < n; ++j) { Lam[j] = lam[j]; hard[j] = 0; }
  int used = 0;
  bool ok = false;
  for (int t = 1; t <= iters; ++t) {
    // check update: r_{i->j} from the other edges of check i
    for (int i = 0; i < m; ++i) {
      for (int k = g.rptr[i]; k < g.rptr[i + 1]; ++k) {
        if (method == 0) {
          bool neg = s[i] != 0;
          R mn = (R)kEmptyMin;
          for (int k2 = g.rptr[i]; k2 < g.rptr[i + 1]; ++k2) {
            if (k2 == k) continue;
            if (q[k2] < (R)0) neg = !neg;
            R a = std::fabs(q[k2]);
            if (a < mn) mn = a;
          }
          R mag = alpha * mn;
          r[k] = neg ? -mag : mag;
        } else {
          R prod = (R)1;
          for (int k2 = g.rptr[i]; k2 < g.rptr[i + 1]; ++k2) {
            if (k2 == k) continue;
            prod = prod * std::tanh(q[k2] / (R)2);
          }
          const R lim = (R)1 - (R)1e-15;
          if (sizeof(R) == 4) {
            // 1 - 1e-15 rounds to 1 in float; clamp to the largest float below 1
            const R flim = (R)0.99999994f;
            if (prod > flim) prod = flim;
            if (prod < -flim) prod = -flim;
          } else {
            if (prod > lim) prod = lim;
            if (prod < -lim) prod = -lim;
          }
          R v = (R)2 * std::atanh(prod);
          r[k] = s[i] ? -v : v;
        }
      }
    }
    // variable update: Lambda_j = lambda_j + sum of incoming r, ascending check order
    for (int j = 0; j < n; ++j) {
      R L = lam[j];
      for (int a = col_edges_ptr[j]; a < col_edges_ptr[j + 1]; ++a) L = L + r[col_edges[a]];
      Lam[j] = L;
      for (int a = col_edges_ptr[j]; a < col_edges_ptr[j + 1]; ++a) q[col_edges[a]] = L - r[col_edges[a]];
      hard[j] = (L < (R)0) ? 1 : 0;
    }
    used = t;
    // H.e_hat = s ?
    ok = true;
    for (int i = 0; i < m && ok; ++i) {
      int par = s[i] ? 1 : 0;
      for (int k = g.rptr[i]; k < g.rptr[i + 1]; ++k) par ^= hard[g.rcol[k]];
      if (par) ok = false;
    }
    if (ok && early_exit) break;
  }
  *iters_used = used;
  *converged = ok ? 1 : 0;
}

// edges of column j (indices into the row-major edge list), ascending row
void column_edges(const Graph& g, std::vector<int>& ptr, std::vector<int>& idx) {
  ptr.assign(g.n + 1, 0);
  for (int i = 0; i < g.m; ++i)
    for (int k = g.rptr[i]; k < g.rptr[i + 1]; ++k) ptr[g.rcol[k] + 1]++;
  for (int j = 0; j < g.n; ++j) ptr[j + 1] += ptr[j];
  idx.assign(g.rcol.size(), 0);
  std::vector<int> fill(ptr.begin(), ptr.end() - 1);
  for (int i = 0; i < g.m; ++i)  // ascending i, so each column list is ascending in row
    for (int k = g.rptr[i]; k < g.rptr[i + 1]; ++k) idx[fill[g.rcol[k]]++] = k;
}

double prior_llr(double p) { return std::log((1.0 - p) / p); }

template <typename F>
void parallel_for(int64_t count, int nthreads, F fn) {
  if (nthreads <= 0) nthreads = (int)std::thread::hardware_concurrency();
  if (nthreads <= 1 || count <= 1) { for (int64_t k = 0; k < count; ++k) fn(k); return; }
  std::atomic<int64_t> next(0);
  std::vector<std::thread> th;
  for (int t = 0; t < nthreads; ++t)
    th.emplace_back([&]() {
      for (;;) {
        int64_t k = next.fetch_add(1);
        if (k >= count) break;
        fn(k);
      }
    });
  for (auto& t : th) t.join();
}

// --------------------------------------------------------------------------
// GF(2) elimination (column echelon form, reduction in pivot-creation order)
// --------------------------------------------------------------------------

struct Echelon {
  int cw;                       // words of a combination set (over column positions)
  std::vector<Bits> vec, comb;  // reduced basis vectors and their column combinations
  std::vector<int> prow;        // pivot row of each basis vector
  std::vector<int> pos;         // column position of each basis vector
  explicit Echelon(int ncols) : cw(nwords(std::max(ncols, 1))) {}

  // Adds column ``v`` at position ``p``; true if it is independent of the basis.
  bool add(Bits v, int p) {
    Bits c(cw, 0);
    setbit(c, p);
    for (size_t k = 0; k < vec.size(); ++k)
      if (bit(v, prow[k])) { xorin(v, vec[k]); xorin(c, comb[k]); }
    int r = lowbit(v);
    if (r < 0) return false;
    vec.push_back(v); comb.push_back(c); prow.push_back(r); pos.push_back(p);
    return true;
  }
  // Reduces ``v``; returns true if v is in the span, with the combination in ``c``.
  bool reduce(Bits v, Bits& c) const {
    c.assign(cw, 0);
    for (size_t k = 0; k < vec.size(); ++k)
      if (bit(v, prow[k])) { xorin(v, vec[k]); xorin(c, comb[k]); }
    return !anybit(v);
  }
};

// --------------------------------------------------------------------------
// LSD (Alg. 1, synchronous growth) and LSD-mu (App. D)
// --------------------------------------------------------------------------

struct Cluster {
  Bits dets;              // V_D^C
  Bits colset;            // V_F^C as a set
  std::vector<int> cols;  // V_F^C in column order
  bool valid = false;
  bool alive = true;
};

enum { ST_OK_BP = 1, ST_OK_LSD = 2, ST_UNSOLVABLE = 3 };

struct LsdOut { int status, nu, kappa, steps; };

LsdOut lsd_shot(const Graph& g, const uint8_t* s, const double* llr, const int64_t* wfix,
                int order, int osd_cs, int single, uint8_t* out, int32_t* det_lab,
                int32_t* fault_lab) {
  const int m = g.m, n = g.n, W = nwords(std::max(m, 1)), NW = nwords(std::max(n, 1));
  auto before = [&](int a, int b) { return llr[a] < llr[b] || (llr[a] == llr[b] && a < b); };
  Bits S(W, 0);
  for (int d = 0; d < m; ++d) if (s[d]) setbit(S, d);

  std::vector<Cluster> cl;
  if (single) {
    Cluster c;
    c.dets.assign(W, 0);
    for (int d = 0; d < m; ++d) setbit(c.dets, d);
    c.colset.assign(NW, 0);
    c.valid = !anybit(S);
    cl.push_back(c);
  } else {
    for (int d = 0; d < m; ++d) {
      if (!s[d]) continue;
      Cluster c;
      c.dets.assign(W, 0); setbit(c.dets, d);
      c.colset.assign(NW, 0);
      c.valid = false;  // s_[C] = (1) is not in the span of no columns
      cl.push_back(c);
    }
  }

  auto is_valid = [&](const Cluster& c) {
    Echelon e((int)c.cols.size());
    for (size_t p = 0; p < c.cols.size(); ++p) e.add(g.colbits[c.cols[p]], (int)p);
    Bits t(W);
    for (int k = 0; k < W; ++k) t[k] = S[k] & c.dets[k];
    Bits comb;
    return e.reduce(t, comb);
  };

  // One synchronous growth step.  growers: only invalid clusters (LSD-0) or all (LSD-mu).
  // Returns 0 if something grew, 1 if an invalid cluster had no candidate, 2 if nothing grew.
  auto step = [&](bool only_invalid) -> int {
    const int K = (int)cl.size();
    std::vector<int> pick(K, -1);
    bool any = false;
    for (int k = 0; k < K; ++k) {
      if (!cl[k].alive || (only_invalid && cl[k].valid)) continue;
      int best = -1;
      for (int d = 0; d < m; ++d) {
        if (!bit(cl[k].dets, d)) continue;
        for (int a = g.rptr[d]; a < g.rptr[d + 1]; ++a) {
          int j = g.rcol[a];
          if (bit(cl[k].colset, j)) continue;
          if (best < 0 || before(j, best)) best = j;
        }
      }
      if (best < 0) {
        if (only_invalid) return 1;
        continue;
      }
      pick[k] = best;
      any = true;
    }
    if (!any) return 2;
    for (int k = 0; k < K; ++k)
      if (pick[k] >= 0)
        for (int w = 0; w < W; ++w) cl[k].dets[w] |= g.colbits[pick[k]][w];
    // merge clusters whose detector sets intersect (transitively); root = lowest index
    std::vector<int> par(K);
    for (int k = 0; k < K; ++k) par[k] = k;
    auto find = [&](int x) { while (par[x] != x) x = par[x]; return x; };
    for (int a = 0; a < K; ++a) {
      if (!cl[a].alive) continue;
      for (int b = a + 1; b < K; ++b) {
        if (!cl[b].alive) continue;
        if (intersects(cl[a].dets, cl[b].dets)) {
          int ra = find(a), rb = find(b);
          if (ra != rb) { if (ra < rb) par[rb] = ra; else par[ra] = rb; }
        }
      }
    }
    std::vector<char> changed(K, 0);
    for (int r = 0; r < K; ++r) {
      if (!cl[r].alive || find(r) != r) continue;
      std::vector<int> members;
      for (int k = r; k < K; ++k) if (cl[k].alive && find(k) == r) members.push_back(k);
      if (members.size() == 1) {
        if (pick[r] >= 0) {
          cl[r].cols.push_back(pick[r]);
          setbit(cl[r].colset, pick[r]);
          changed[r] = 1;
        }
        continue;
      }
      std::vector<int> newcols;
      for (int k : members) if (pick[k] >= 0) newcols.push_back(pick[k]);
      std::sort(newcols.begin(), newcols.end(), [&](int a, int b) { return before(a, b); });
      newcols.erase(std::unique(newcols.begin(), newcols.end()), newcols.end());
      for (size_t t = 1; t < members.size(); ++t) {
        Cluster& o = cl[members[t]];
        cl[r].cols.insert(cl[r].cols.end(), o.cols.begin(), o.cols.end());
        for (int w = 0; w < W; ++w) cl[r].dets[w] |= o.dets[w];
        for (int w = 0; w < NW; ++w) cl[r].colset[w] |= o.colset[w];
        o.alive = false;
      }
      for (int j : newcols) { cl[r].cols.push_back(j); setbit(cl[r].colset, j); }
      changed[r] = 1;
    }
    for (int k = 0; k < K; ++k)
      if (changed[k] && cl[k].alive) cl[k].valid = is_valid(cl[k]);
    return 0;
  };

  LsdOut res{ST_OK_LSD, 0, 0, 0};
  std::memset(out, 0, (size_t)n);
  for (;;) {
    bool any_invalid = false;
    for (auto& c : cl) if (c.alive && !c.valid) any_invalid = true;
    if (!any_invalid) break;
    int r = step(true);
    if (r == 1) { res.status = ST_UNSOLVABLE; break; }
    res.steps++;
  }
  if (res.status == ST_OK_LSD && order > 0) {
    for (int t = 0; t < order; ++t) {
      if (step(false) == 2) break;
      for (auto& c : cl)
        if (c.alive && !c.valid) { res.status = ST_UNSOLVABLE; break; }  // cannot happen (App. D)
    }
  }

  // local solves and the global decoding
  int label = 0;
  if (det_lab) for (int d = 0; d < m; ++d) det_lab[d] = -1;
  if (fault_lab) for (int j = 0; j < n; ++j) fault_lab[j] = -1;
  for (auto& c : cl) {
    if (!c.alive) continue;
    res.nu++;
    res.kappa = std::max(res.kappa, (int)c.cols.size());
    if (det_lab) for (int d = 0; d < m; ++d) if (bit(c.dets, d)) det_lab[d] = label;
    if (fault_lab) for (int j : c.cols) fault_lab[j] = label;
    label++;
    if (res.status != ST_OK_LSD) continue;
    Echelon e((int)c.cols.size());
    std::vector<int> nonpiv;
    for (size_t p = 0; p < c.cols.size(); ++p)
      if (!e.add(g.colbits[c.cols[p]], (int)p)) nonpiv.push_back((int)p);
    std::sort(nonpiv.begin(), nonpiv.end(),
              [&](int a, int b) { return before(c.cols[a], c.cols[b]); });
    // the flip patterns (sets of non-pivot positions), in the order that breaks cost ties
    std::vector<std::vector<int>> patterns;
    if (order > 0 && osd_cs >= 0) {  // combination sweep of order osd_cs
      patterns.push_back({});
      for (int k = 0; k < (int)nonpiv.size(); ++k) patterns.push_back({k});
      const int wp = std::min<int>(osd_cs, (int)nonpiv.size());
      for (int i = 0; i < wp; ++i)
        for (int j = i + 1; j < wp; ++j) patterns.push_back({i, j});
    } else {  // exhaustive over the first min(mu, #non-pivots)
      const int nt = std::min<int>(order, (int)nonpiv.size());
      for (int64_t t = 0; t < ((int64_t)1 << nt); ++t) {
        std::vector<int> pat;
        for (int k = 0; k < nt; ++k) if ((t >> k) & 1) pat.push_back(k);
        patterns.push_back(pat);
      }
    }
    Bits target(W);
    for (int w = 0; w < W; ++w) target[w] = S[w] & c.dets[w];
    int64_t best_cost = std::numeric_limits<int64_t>::max();
    std::vector<int> best_sol;
    for (const auto& pat : patterns) {
      Bits rhs = target;
      for (int k : pat) xorin(rhs, g.colbits[c.cols[nonpiv[k]]]);
      Bits comb;
      if (!e.reduce(rhs, comb)) { res.status = ST_UNSOLVABLE; break; }
      std::vector<int> sol;
      for (size_t p = 0; p < c.cols.size(); ++p) if (bit(comb, (int)p)) sol.push_back(c.cols[p]);
      for (int k : pat) sol.push_back(c.cols[nonpiv[k]]);
      if (patterns.size() == 1) { best_sol = sol; break; }
      int64_t cost = 0;
      for (int j : sol) cost += wfix[j];
      if (cost < best_cost) { best_cost = cost; best_sol = sol; }
    }
    for (int j : best_sol) out[j] = 1;
  }
  if (res.status == ST_UNSOLVABLE) std::memset(out, 0, (size_t)n);
  return res;
}

// 2^-32 fixed-point weight of the FP32 channel-prior LLR of each column.
void fixed_weights(int n, const double* probs, std::vector<int64_t>& w) {
  w.assign(n, 0);
  for (int j = 0; j < n; ++j) {
    float lf = (float)prior_llr(probs[j]);
    w[j] = (int64_t)std::llrint((double)lf * 4294967296.0);
  }
}

}  // namespace

extern "C" {

// lambda_j = ln((1-p_j)/p_j) in double; precision 1 rounds it to float.
int orc_priors(int32_t n, const double* probs, int32_t precision, double* out) {
  for (int j = 0; j < n; ++j) {
    double v = prior_llr(probs[j]);
    out[j] = precision == 1 ? (double)(float)v : v;
  }
  return 0;
}

// BP over a batch.  precision 0 = double, 1 = FP32 mirror.  llr_out, hard_out [shots][n].
int orc_bp(int32_t m, int32_t n, int64_t nnz, const int32_t* rows, const int32_t* cols,
           const double* probs, int64_t shots, const uint8_t* syndromes, int32_t iters,
           double alpha, int32_t method, int32_t early_exit, int32_t precision, int32_t nthreads,
           double* llr_out, uint8_t* hard_out, int32_t* iters_used, uint8_t* converged) {
  Graph g;
  if (build_graph(m, n, nnz, rows, cols, g)) return -1;
  std::vector<int> cep, ce;
  column_edges(g, cep, ce);
  std::vector<double> lamd(n);
  std::vector<float> lamf(n);
  for (int j = 0; j < n; ++j) { lamd[j] = prior_llr(probs[j]); lamf[j] = (float)lamd[j]; }
  parallel_for(shots, nthreads, [&](int64_t k) {
    const uint8_t* s = syndromes + (size_t)k * m;
    int used; uint8_t conv;
    if (precision == 1) {
      std::vector<float> L(n);
      bp_shot<float>(g, cep, ce, lamf.data(), s, iters, (float)alpha, method, early_exit, L.data(),
                     hard_out + (size_t)k * n, &used, &conv);
      for (int j = 0; j < n; ++j) llr_out[(size_t)k * n + j] = L[j];
    } else {
      bp_shot<double>(g, cep, ce, lamd.data(), s, iters, alpha, method, early_exit,
                      llr_out + (size_t)k * n, hard_out + (size_t)k * n, &used, &conv);
    }
    iters_used[k] = used;
    converged[k] = conv;
  });
  return 0;
}

// Rank over GF(2) of a dense row-major 0/1 matrix.
int32_t orc_gf2_rank(int32_t nrows, int32_t ncols, const uint8_t* a) {
  Echelon e(ncols);
  int rank = 0;
  for (int c = 0; c < ncols; ++c) {
    Bits v(nwords(std::max(nrows, 1)), 0);
    for (int r = 0; r < nrows; ++r) if (a[(size_t)r * ncols + c]) setbit(v, r);
    if (e.add(v, c)) rank++;
  }
  return rank;
}

// Solve A x = b (dense row-major m x n) on the greedy independent set of columns
// taken in index order.  pivots_out[j] = 1 for the basis columns.  Returns 1 if
// b is in the column span (x_out holds the unique solution supported on the
// basis), else 0.
int32_t orc_gf2_solve(int32_t m, int32_t n, const uint8_t* a, const uint8_t* b,
                      uint8_t* x_out, uint8_t* pivots_out) {
  Echelon e(n);
  const int W = nwords(std::max(m, 1));
  for (int c = 0; c < n; ++c) {
    Bits v(W, 0);
    for (int r = 0; r < m; ++r) if (a[(size_t)r * n + c]) setbit(v, r);
    pivots_out[c] = e.add(v, c) ? 1 : 0;
  }
  Bits t(W, 0);
  for (int r = 0; r < m; ++r) if (b[r]) setbit(t, r);
  Bits comb;
  bool ok = e.reduce(t, comb);
  for (int c = 0; c < n; ++c) x_out[c] = ok && bit(comb, c) ? 1 : 0;
  return ok ? 1 : 0;
}

// OSD-0: columns sorted by (llr, index); greedy basis; the solution on it.
int32_t orc_osd0(int32_t m, int32_t n, int64_t nnz, const int32_t* rows, const int32_t* cols,
                 const uint8_t* syndrome, const double* llr, uint8_t* out) {
  Graph g;
  if (build_graph(m, n, nnz, rows, cols, g)) return -1;
  std::vector<int> order(n);
  for (int j = 0; j < n; ++j) order[j] = j;
  std::sort(order.begin(), order.end(), [&](int a, int b) {
    return llr[a] < llr[b] || (llr[a] == llr[b] && a < b);
  });
  Echelon e(n);
  for (int p = 0; p < n; ++p) e.add(g.colbits[order[p]], p);
  Bits t(nwords(std::max(m, 1)), 0);
  for (int d = 0; d < m; ++d) if (syndrome[d]) setbit(t, d);
  Bits comb;
  std::memset(out, 0, (size_t)n);
  if (!e.reduce(t, comb)) return 0;
  for (int p = 0; p < n; ++p) if (bit(comb, p)) out[order[p]] = 1;
  return 1;
}

// LSD on given soft information.  llrs [shots][n]; probs (for LSD-mu costs) may be
// null when order == 0.  info [shots][3] = (nu, kappa, steps).  det_lab [shots][m]
// and fault_lab [shots][n] (nullable) receive the final cluster label of each node.
int orc_lsd(int32_t m, int32_t n, int64_t nnz, const int32_t* rows, const int32_t* cols,
            int64_t shots, const uint8_t* syndromes, const double* llrs, const double* probs,
            int32_t order, int32_t osd_cs, int32_t single_cluster, int32_t nthreads,
            uint8_t* corrections, uint8_t* status, int32_t* info, int32_t* det_lab,
            int32_t* fault_lab) {
  Graph g;
  if (build_graph(m, n, nnz, rows, cols, g)) return -1;
  std::vector<int64_t> w;
  if (order > 0) {
    if (!probs) return -1;
    fixed_weights(n, probs, w);
  }
  parallel_for(shots, nthreads, [&](int64_t k) {
    LsdOut r = lsd_shot(g, syndromes + (size_t)k * m, llrs + (size_t)k * n, w.data(), order,
                        osd_cs, single_cluster, corrections + (size_t)k * n,
                        det_lab ? det_lab + (size_t)k * m : nullptr,
                        fault_lab ? fault_lab + (size_t)k * n : nullptr);
    status[k] = (uint8_t)r.status;
    if (info) { info[3 * k] = r.nu; info[3 * k + 1] = r.kappa; info[3 * k + 2] = r.steps; }
  });
  return 0;
}

// BP then LSD (App. C.4): if BP's hard decision satisfies the syndrome it is the
// correction (status 1), otherwise LSD runs on BP's last posteriors (status 2/3).
// precision as in orc_bp.  llr_out [shots][n] nullable; info [shots][3] nullable.
int orc_decode(int32_t m, int32_t n, int64_t nnz, const int32_t* rows, const int32_t* cols,
               const double* probs, int64_t shots, const uint8_t* syndromes, int32_t bp_iters,
               double alpha, int32_t lsd_order, int32_t osd_cs, int32_t precision,
               int32_t nthreads, uint8_t* corrections, uint8_t* status, int32_t* bp_iters_used,
               int32_t* info, double* llr_out) {
  Graph g;
  if (build_graph(m, n, nnz, rows, cols, g)) return -1;
  std::vector<int> cep, ce;
  column_edges(g, cep, ce);
  std::vector<double> lamd(n);
  std::vector<float> lamf(n);
  for (int j = 0; j < n; ++j) { lamd[j] = prior_llr(probs[j]); lamf[j] = (float)lamd[j]; }
  std::vector<int64_t> w;
  fixed_weights(n, probs, w);
  parallel_for(shots, nthreads, [&](int64_t k) {
    const uint8_t* s = syndromes + (size_t)k * m;
    uint8_t* out = corrections + (size_t)k * n;
    std::vector<double> L(n);
    int used; uint8_t conv;
    if (precision == 1) {
      std::vector<float> Lf(n);
      bp_shot<float>(g, cep, ce, lamf.data(), s, bp_iters, (float)alpha, 0, 1, Lf.data(), out,
                     &used, &conv);
      for (int j = 0; j < n; ++j) L[j] = Lf[j];
    } else {
      bp_shot<double>(g, cep, ce, lamd.data(), s, bp_iters, alpha, 0, 1, L.data(), out, &used,
                      &conv);
    }
    if (bp_iters_used) bp_iters_used[k] = used;
    if (llr_out) for (int j = 0; j < n; ++j) llr_out[(size_t)k * n + j] = L[j];
    if (conv) {
      status[k] = ST_OK_BP;
      if (info) { info[3 * k] = 0; info[3 * k + 1] = 0; info[3 * k + 2] = 0; }
      return;
    }
    LsdOut r = lsd_shot(g, s, L.data(), w.data(), lsd_order, osd_cs, 0, out, nullptr, nullptr);
    status[k] = (uint8_t)r.status;
    if (info) { info[3 * k] = r.nu; info[3 * k + 1] = r.kappa; info[3 * k + 2] = r.steps; }
  });
  return 0;
}

// Logical failure by the rank test: fail[k] = 1 iff residual k is not in the row
// space of H_Z (dense row-major mz x n).
int orc_logical_failures(int32_t mz, int32_t n, const uint8_t* hz, int64_t shots,
                         const uint8_t* residuals, int32_t nthreads, uint8_t* fail) {
  // echelon basis of the rows of H_Z (vectors over n coordinates)
  Echelon e(mz);
  const int W = nwords(std::max(n, 1));
  for (int r = 0; r < mz; ++r) {
    Bits v(W, 0);
    for (int c = 0; c < n; ++c) if (hz[(size_t)r * n + c]) setbit(v, c);
    e.add(v, r);
  }
  parallel_for(shots, nthreads, [&](int64_t k) {
    Bits v(W, 0);
    for (int c = 0; c < n; ++c) if (residuals[(size_t)k * n + c]) setbit(v, c);
    Bits comb;
    fail[k] = e.reduce(v, comb) ? 0 : 1;
  });
  return 0;
}

}  // extern "C"
