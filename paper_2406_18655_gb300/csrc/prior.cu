// Learned prior: edge-MLP message passing on the Tanner graph, BF16 tensor-core matrix
// products with FP32 accumulation (forward, backward, Adam), and a device-side sampler of
// training pairs.  The paper has no learned component; the model is defined in
// include/lsd.h (lsd_prior_create) and restated by the CPU oracle.
//
// Model (hidden width 32, R rounds, weights shared by the rounds, one MLP per direction):
//   sigma_c = 1 - 2 s_c;  h_v = relu(lambda_v a0 + a1);  h_c = sigma_c u0 + u1
//   round: h_v += sum_c MLP_cv([h_c, h_v, sigma_c]);  h_c += sum_v MLP_vc([h_v, h_c, sigma_c])
//   LLR_v = lambda_v + w_o . h_v + b_o
//   MLP(x) = W2 relu(W1 x + b1) + b2   (W1: 32 x 65, W2: 32 x 32)
//
// Inference (prior_fwd_kernel) and training (prior_train_kernel) both evaluate the model
// on per-node products (see the comment above prior_fwd_kernel); Adam updates the FP32
// master parameters (adam_kernel) and sample_kernel draws training pairs.

#include <cuda_bf16.h>

#include "lsd_internal.cuh"
#include "prior_params.cuh"

namespace lsdgb {

namespace {

using prior_params::DIN;
using prior_params::HD;
using prior_params::POff;

__host__ __device__ inline size_t a16(size_t x) { return (x + 15) & ~(size_t)15; }

// ---- mma.sync helpers (PTX ISA fragment layouts for m16n8k16 .bf16) ----
__device__ __forceinline__ void mma16816(float c[4], const uint32_t a[4], const uint32_t b[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}
__device__ __forceinline__ uint32_t ld32(const __nv_bfloat16* p) {
  return *reinterpret_cast<const uint32_t*>(p);
}
__device__ __forceinline__ uint32_t pack_bf(const __nv_bfloat16 lo, const __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g,
                            float* __restrict__ mom, float* __restrict__ vel, int count, float lr,
                            float b1, float b2, float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const float gi = g[i];
  const float mi = b1 * mom[i] + (1.f - b1) * gi;
  const float vi = b2 * vel[i] + (1.f - b2) * gi * gi;
  mom[i] = mi;
  vel[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// Training pairs: fault j of shot k is 1 with probability p_j, drawn from the xoshiro256**
// stream of shot k (seeded by splitmix64 from seed ^ (k+1) * 0xD1B54A32D192ED03) in
// ascending column order, u = (x >> 11) * 2^-53 < p_j in double; then s = H e.
__device__ __forceinline__ unsigned long long rotl64(unsigned long long x, int k) {
  return (x << k) | (x >> (64 - k));
}

__global__ void sample_kernel(unsigned long long seed, long long first, long long shots, int m,
                              int n, const float* __restrict__ probs,
                              const int32_t* __restrict__ chk_ptr,
                              const uint16_t* __restrict__ chk_var, uint8_t* __restrict__ errors,
                              uint8_t* __restrict__ syndromes) {
  const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k >= shots) return;
  unsigned long long x = seed ^ ((unsigned long long)(first + k + 1) * 0xD1B54A32D192ED03ull);
  unsigned long long s[4];
  for (int i = 0; i < 4; ++i) {
    x += 0x9E3779B97F4A7C15ull;
    unsigned long long z = x;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    s[i] = z ^ (z >> 31);
  }
  uint8_t* e = errors + k * n;
  for (int j = 0; j < n; ++j) {
    const unsigned long long r = rotl64(s[1] * 5ull, 7) * 9ull;
    const unsigned long long t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl64(s[3], 45);
    const double u = (double)(r >> 11) * 0x1.0p-53;
    e[j] = u < (double)probs[j] ? 1 : 0;
  }
  uint8_t* sy = syndromes + k * m;
  for (int i = 0; i < m; ++i) {
    int par = 0;
    for (int q = chk_ptr[i]; q < chk_ptr[i + 1]; ++q) par ^= e[chk_var[q]];
    sy[i] = (uint8_t)par;
  }
}



// ======================================================================================
// Forward-only kernel on per-node projections (inference).
//
// Split the layer-1 matrix of a direction by input block, W1 = [W_first | W_second | w_s]:
//   W1 x_e + b1 = W_first h_first + W_second h_second + sigma_c w_s + b1,
// so layer 1 needs one product per node, not per edge; and since layer 2 is affine, the
// messages into a node sum to
//   sum_e (W2 relu(z_e) + b2) = W2 (sum_e relu(z_e)) + deg * b2,
// one product per destination node on the summed activations.  The model is unchanged
// (same function, different rounding order).  With
//   A_c = W1cv[:, 0:32] h_c + sigma_c W1cv[:, 64] + b1cv,   B_v = W1cv[:, 32:64] h_v,
//   C_v = W1vc[:, 0:32] h_v,   D_c = W1vc[:, 32:64] h_c + sigma_c W1vc[:, 64] + b1vc,
// one round is
//   X2: S_v = sum_{c in N(v)} relu(A_c + B_v)          (gather, FP32)
//   G1: h_v += W2cv S_v + deg_v b2cv;  C_v, B_v from the new h_v
//   X1: T_c = sum_{v in N(c)} relu(C_v + D_c)
//   G2: h_c += W2vc T_c + deg_c b2vc;  A_c, D_c from the new h_c
// and the last round stops after G1 with LLR_v = lambda_v + w_o . h_v + b_o.  The G steps
// run on the tensor cores (mma.sync m16n8k16, BF16 operands, FP32 accumulation): a warp
// owns 16 node rows, starts the accumulators from the FP32 state, and re-packs the updated
// state from the accumulator fragments as the A operand of the projection product.
// One CTA owns one shot at a time; all node arrays live in shared memory.
// ======================================================================================

constexpr int kFwdWarps = 8;    // training kernel (warps 0-5 own the weight gradients)
constexpr int kInfWarps = 9;    // inference kernel: 9 warps give BB144's 9 variable tiles one each

struct FwdArgs {
  int m, n, rounds;
  const int32_t* chk_ptr;
  const uint16_t* chk_var;
  const int32_t* var_ptr;
  const uint16_t* var_chk;
  const float* prior;
  const float* params;
  long long shots;
  const uint8_t* syndromes;
  float* llr_out;          // [shots][n] output LLRs, or null in decode mode:
  // decode mode: the hard decision [LLR < 0] of a shot that satisfies its syndrome is its
  // correction (status LSD_SHOT_OK_BP); any other shot is queued for LSD with its LLR row
  uint8_t* corrections;
  uint8_t* status;
  int32_t* queue;
  float* queue_llr;
  DevCounters* ctr;
};

struct FLay {
  int npad, mpad;
  size_t hv, hc, cv, bv, ac, dc, w, vec, sig, lam, degv, degc, llr, total;
};

// FP32 states h_v, h_c; BF16 projections C_v, B_v, A_c, D_c.  The summed activations S_v
// (T_c) overwrite B_v (D_c) in place: each is read once, by the thread that then writes
// the same columns of the same row.
__host__ __device__ inline FLay fwd_layout(int m, int n) {
  FLay L;
  L.npad = (n + 15) & ~15;
  L.mpad = (m + 15) & ~15;
  const size_t fv = (size_t)L.npad * HD * 4, fc = (size_t)L.mpad * HD * 4;
  size_t o = 0;
  L.hv = o; o += fv;
  L.hc = o; o += fc;
  L.cv = o; o += fv / 2;
  L.bv = o; o += fv / 2;
  L.ac = o; o += fc / 2;
  L.dc = o; o += fc / 2;
  L.w = o; o += (size_t)6 * HD * HD * 2;   // W2cv | Wv (C rows, B rows) | W2vc | Wc (A, D rows)
  L.vec = o; o += (size_t)12 * HD * 4;
  L.sig = o; o += a16((size_t)L.mpad * 4);
  L.lam = o; o += a16((size_t)L.npad * 4);
  L.degv = o; o += a16((size_t)L.npad * 4);
  L.degc = o; o += a16((size_t)L.mpad * 4);
  L.llr = o; o += a16((size_t)L.npad * 4);
  L.total = o;
  return L;
}

// vec slots of the forward kernel (x32 floats each)
enum { F_a0 = 0, F_a1, F_u0, F_u1, F_b2cv, F_b2vc, F_wscv, F_b1cv, F_wsvc, F_b1vc, F_wo, F_bo };

// FP32 [rows][32] arrays: the 4-float block b of row r is stored at block b ^ 2(r & 3), so
// the accumulator-fragment accesses (float2, rows r0+g, columns 8j+2t) and the gather
// accesses (float4 per lane, 8 lanes per row) are free of bank conflicts.
__device__ __forceinline__ int fsw(int r, int col) {
  return (r << 5) + ((((col >> 2) ^ ((r & 3) << 1)) << 2) | (col & 3));
}
// BF16 [rows][32] arrays: the 8-value block b of row r is stored at block b ^ ((r >> 1) & 3)
// (conflict-free 32-bit fragment loads).
__device__ __forceinline__ int bsw(int r, int col) {
  return (r << 5) + ((((col >> 3) ^ ((r >> 1) & 3)) << 3) | (col & 7));
}

__device__ __forceinline__ void fa_sw(uint32_t a[4], const __nv_bfloat16* base, int r0, int k0,
                                      int lane) {
  const int g = lane >> 2, t = lane & 3;
  a[0] = ld32(base + bsw(r0 + g, k0 + 2 * t));
  a[1] = ld32(base + bsw(r0 + g + 8, k0 + 2 * t));
  a[2] = ld32(base + bsw(r0 + g, k0 + 2 * t + 8));
  a[3] = ld32(base + bsw(r0 + g + 8, k0 + 2 * t + 8));
}
__device__ __forceinline__ void fb_sw(uint32_t b[2], const __nv_bfloat16* base, int n0, int k0,
                                      int lane) {
  const int g = lane >> 2, t = lane & 3;
  b[0] = ld32(base + bsw(n0 + g, k0 + 2 * t));
  b[1] = ld32(base + bsw(n0 + g, k0 + 2 * t + 8));
}

struct FwdSmem {
  float *hv, *hc, *vec, *sig, *lam, *degv, *degc, *llr;
  __nv_bfloat16 *cv, *bv, *ac, *dc, *W2cv, *Wv, *W2vc, *Wc;
};

// G step on node rows r0..r0+15 (CHECK: check nodes, else variable nodes).
//   has_agg: h += W2 agg + deg b2 (written back; agg = T_c in dc, S_v in bv);  proj: the
//   two projections of the new h into (ac, dc) or (cv, bv);  otherwise (variables, last
//   round) the output LLRs.
//   init (syn != null): the initial states h_v = relu(lambda_v a0 + a1), h_c = sigma_c u0 + u1
//   are formed in registers (and sigma_c recorded) instead of read.
template <bool CHECK>
__device__ __forceinline__ void g_step(const FwdSmem& S, int rows, int r0, bool has_agg, bool proj,
                                       float* llr, int lane, const uint8_t* syn = nullptr,
                                       __nv_bfloat16* save = nullptr) {
  const int g = lane >> 2, t = lane & 3;
  const int ra = r0 + g, rb = r0 + g + 8;
  float* h = CHECK ? S.hc : S.hv;
  float c[4][4];
  if (syn) {
    float xa = 0.f, xb = 0.f;  // lambda_v or sigma_c of the two rows (0 on padding rows)
    if (CHECK) {
      xa = ra < rows ? (syn[ra] ? -1.f : 1.f) : 0.f;
      xb = rb < rows ? (syn[rb] ? -1.f : 1.f) : 0.f;
      if (t == 0) {
        S.sig[ra] = xa;
        S.sig[rb] = xb;
      }
    } else {
      xa = S.lam[ra];
      xb = S.lam[rb];
    }
    const float* w0 = S.vec + (CHECK ? F_u0 : F_a0) * HD;
    const float* w1 = S.vec + (CHECK ? F_u1 : F_a1) * HD;
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int col = nt * 8 + 2 * t + q;
        float za = fmaf(xa, w0[col], w1[col]), zb = fmaf(xb, w0[col], w1[col]);
        if (!CHECK) {
          za = fmaxf(za, 0.f);
          zb = fmaxf(zb, 0.f);
        }
        c[nt][q] = ra < rows ? za : 0.f;
        c[nt][2 + q] = rb < rows ? zb : 0.f;
      }
      const int col = nt * 8 + 2 * t;
      if (ra < rows) *reinterpret_cast<float2*>(h + fsw(ra, col)) = make_float2(c[nt][0], c[nt][1]);
      if (rb < rows) *reinterpret_cast<float2*>(h + fsw(rb, col)) = make_float2(c[nt][2], c[nt][3]);
    }
  } else {
    const float* b2 = S.vec + (CHECK ? F_b2vc : F_b2cv) * HD;
    const float* deg = CHECK ? S.degc : S.degv;
    const float da = has_agg ? deg[ra] : 0.f, db = has_agg ? deg[rb] : 0.f;
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      const int col = nt * 8 + 2 * t;
      const float2 x = *reinterpret_cast<const float2*>(h + fsw(ra, col));
      const float2 y = *reinterpret_cast<const float2*>(h + fsw(rb, col));
      c[nt][0] = fmaf(da, b2[col], x.x);
      c[nt][1] = fmaf(da, b2[col + 1], x.y);
      c[nt][2] = fmaf(db, b2[col], y.x);
      c[nt][3] = fmaf(db, b2[col + 1], y.y);
    }
  }
  if (has_agg) {
    const __nv_bfloat16* W2 = CHECK ? S.W2vc : S.W2cv;
    const __nv_bfloat16* agg = CHECK ? S.dc : S.bv;
    uint32_t af[2][4];
    fa_sw(af[0], agg, r0, 0, lane);
    fa_sw(af[1], agg, r0, 16, lane);
    __syncwarp();  // the aggregate rows are overwritten by this warp's projections below
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        uint32_t bf[2];
        fb_sw(bf, W2, nt * 8, j * 16, lane);
        mma16816(c[nt], af[j], bf);
      }
      const int col = nt * 8 + 2 * t;
      if (ra < rows) *reinterpret_cast<float2*>(h + fsw(ra, col)) = make_float2(c[nt][0], c[nt][1]);
      if (rb < rows) *reinterpret_cast<float2*>(h + fsw(rb, col)) = make_float2(c[nt][2], c[nt][3]);
    }
  }
  if (save) {  // training: the new state rounded to BF16, row-major, for the backward pass
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      const int col = nt * 8 + 2 * t;
      if (ra < rows) *reinterpret_cast<uint32_t*>(save + ra * HD + col) = pack2(c[nt][0], c[nt][1]);
      if (rb < rows) *reinterpret_cast<uint32_t*>(save + rb * HD + col) = pack2(c[nt][2], c[nt][3]);
    }
  }
  if (!proj) {  // variables, last round: LLR_v = lambda_v + w_o . h_v + b_o
    const float* wo = S.vec + F_wo * HD;
    float pa = 0.f, pb = 0.f;
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      const int col = nt * 8 + 2 * t;
      pa = fmaf(c[nt][0], wo[col], fmaf(c[nt][1], wo[col + 1], pa));
      pb = fmaf(c[nt][2], wo[col], fmaf(c[nt][3], wo[col + 1], pb));
    }
    pa += __shfl_xor_sync(0xffffffffu, pa, 1);
    pa += __shfl_xor_sync(0xffffffffu, pa, 2);
    pb += __shfl_xor_sync(0xffffffffu, pb, 1);
    pb += __shfl_xor_sync(0xffffffffu, pb, 2);
    const float bo = S.vec[F_bo * HD];
    if (t == 0 && ra < rows) llr[ra] = S.lam[ra] + pa + bo;
    if (t == 0 && rb < rows) llr[rb] = S.lam[rb] + pb + bo;
    return;
  }
  uint32_t ah[2][4];
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    ah[j][0] = pack2(c[2 * j][0], c[2 * j][1]);
    ah[j][1] = pack2(c[2 * j][2], c[2 * j][3]);
    ah[j][2] = pack2(c[2 * j + 1][0], c[2 * j + 1][1]);
    ah[j][3] = pack2(c[2 * j + 1][2], c[2 * j + 1][3]);
  }
  const __nv_bfloat16* Wp = CHECK ? S.Wc : S.Wv;
  const float sa = CHECK ? S.sig[ra] : 0.f, sb = CHECK ? S.sig[rb] : 0.f;
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    const int col = (nt & 3) * 8 + 2 * t;
    float u[4] = {0.f, 0.f, 0.f, 0.f};
    if (CHECK) {
      const float* ws = S.vec + (nt < 4 ? F_wscv : F_wsvc) * HD;
      const float* b1 = S.vec + (nt < 4 ? F_b1cv : F_b1vc) * HD;
      u[0] = fmaf(sa, ws[col], b1[col]);
      u[1] = fmaf(sa, ws[col + 1], b1[col + 1]);
      u[2] = fmaf(sb, ws[col], b1[col]);
      u[3] = fmaf(sb, ws[col + 1], b1[col + 1]);
    }
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      uint32_t bf[2];
      fb_sw(bf, Wp, nt * 8, j * 16, lane);
      mma16816(u, ah[j], bf);
    }
    __nv_bfloat16* P = nt < 4 ? (CHECK ? S.ac : S.cv) : (CHECK ? S.dc : S.bv);
    if (ra < rows) *reinterpret_cast<uint32_t*>(P + bsw(ra, col)) = pack2(u[0], u[1]);
    if (rb < rows) *reinterpret_cast<uint32_t*>(P + bsw(rb, col)) = pack2(u[2], u[3]);
  }
}

__device__ __forceinline__ void unpack8(const uint4 v, float f[8]) {
  const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    f[2 * i] = __uint_as_float(w[i] << 16);
    f[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
  }
}

// The gather step for the 16 destination rows r0..r0+15 of one warp (4 lanes per row).
__device__ __forceinline__ void x_tile(int count, int r0, const int32_t* __restrict__ ptr,
                                       const uint16_t* __restrict__ adj,
                                       const __nv_bfloat16* src, __nv_bfloat16* dst, int lane) {
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int task = lane + 32 * i, d = r0 + (task >> 2), b = task & 3;
    if (d >= count) continue;
    uint4* dp = reinterpret_cast<uint4*>(dst + bsw(d, 8 * b));
    float q[8], acc[8];
    unpack8(*dp, q);
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] = 0.f;
    const int e1 = __ldg(ptr + d + 1);
    for (int e = __ldg(ptr + d); e < e1; ++e) {
      float p[8];
      unpack8(*reinterpret_cast<const uint4*>(src + bsw(__ldg(adj + e), 8 * b)), p);
#pragma unroll
      for (int k = 0; k < 8; ++k) acc[k] += fmaxf(p[k] + q[k], 0.f);
    }
    *dp = make_uint4(pack2(acc[0], acc[1]), pack2(acc[2], acc[3]), pack2(acc[4], acc[5]),
                     pack2(acc[6], acc[7]));
  }
  __syncwarp();
}

__global__ void __launch_bounds__(kInfWarps * 32, 3) prior_fwd_kernel(FwdArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int m = a.m, n = a.n;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const FLay L = fwd_layout(m, n);
  FwdSmem S;
  S.hv = reinterpret_cast<float*>(smem + L.hv);
  S.hc = reinterpret_cast<float*>(smem + L.hc);
  S.cv = reinterpret_cast<__nv_bfloat16*>(smem + L.cv);
  S.bv = reinterpret_cast<__nv_bfloat16*>(smem + L.bv);
  S.ac = reinterpret_cast<__nv_bfloat16*>(smem + L.ac);
  S.dc = reinterpret_cast<__nv_bfloat16*>(smem + L.dc);
  S.W2cv = reinterpret_cast<__nv_bfloat16*>(smem + L.w);
  S.Wv = S.W2cv + HD * HD;
  S.W2vc = S.Wv + 2 * HD * HD;
  S.Wc = S.W2vc + HD * HD;
  S.vec = reinterpret_cast<float*>(smem + L.vec);
  S.sig = reinterpret_cast<float*>(smem + L.sig);
  S.lam = reinterpret_cast<float*>(smem + L.lam);
  S.degv = reinterpret_cast<float*>(smem + L.degv);
  S.degc = reinterpret_cast<float*>(smem + L.degc);
  S.llr = reinterpret_cast<float*>(smem + L.llr);

  // ---- parameters (BF16 weight tiles, FP32 vectors), graph degrees, zeroed padding ----
  const float* P = a.params;
  for (int i = threadIdx.x; i < HD * HD; i += blockDim.x) {
    const int r = i >> 5, k = i & 31;
    S.W2cv[bsw(r, k)] = __float2bfloat16_rn(P[POff::W2cv + r * HD + k]);
    S.W2vc[bsw(r, k)] = __float2bfloat16_rn(P[POff::W2vc + r * HD + k]);
    S.Wv[bsw(r, k)] = __float2bfloat16_rn(P[POff::W1vc + r * DIN + k]);            // C
    S.Wv[bsw(r + HD, k)] = __float2bfloat16_rn(P[POff::W1cv + r * DIN + HD + k]);  // B
    S.Wc[bsw(r, k)] = __float2bfloat16_rn(P[POff::W1cv + r * DIN + k]);            // A
    S.Wc[bsw(r + HD, k)] = __float2bfloat16_rn(P[POff::W1vc + r * DIN + HD + k]);  // D
  }
  for (int i = threadIdx.x; i < HD; i += blockDim.x) {
    S.vec[F_a0 * HD + i] = P[POff::a0 + i];
    S.vec[F_a1 * HD + i] = P[POff::a1 + i];
    S.vec[F_u0 * HD + i] = P[POff::u0 + i];
    S.vec[F_u1 * HD + i] = P[POff::u1 + i];
    S.vec[F_b2cv * HD + i] = P[POff::b2cv + i];
    S.vec[F_b2vc * HD + i] = P[POff::b2vc + i];
    S.vec[F_wscv * HD + i] = P[POff::W1cv + i * DIN + 2 * HD];
    S.vec[F_b1cv * HD + i] = P[POff::b1cv + i];
    S.vec[F_wsvc * HD + i] = P[POff::W1vc + i * DIN + 2 * HD];
    S.vec[F_b1vc * HD + i] = P[POff::b1vc + i];
    S.vec[F_wo * HD + i] = P[POff::wo + i];
    S.vec[F_bo * HD + i] = i == 0 ? P[POff::bo] : 0.f;
  }
  for (int j = threadIdx.x; j < L.npad; j += blockDim.x) {
    S.lam[j] = j < n ? a.prior[j] : 0.f;
    S.degv[j] = j < n ? (float)(a.var_ptr[j + 1] - a.var_ptr[j]) : 0.f;
  }
  for (int i = threadIdx.x; i < L.mpad; i += blockDim.x) {
    S.degc[i] = i < m ? (float)(a.chk_ptr[i + 1] - a.chk_ptr[i]) : 0.f;
    S.sig[i] = 0.f;
  }
  // padding rows (read by the last 16-row tile, never written) stay zero
  for (int i = n * HD + threadIdx.x; i < L.npad * HD; i += blockDim.x) S.hv[i] = 0.f;
  for (int i = m * HD + threadIdx.x; i < L.mpad * HD; i += blockDim.x) S.hc[i] = 0.f;
  for (int i = n * HD / 2 + threadIdx.x; i < L.npad * HD / 2; i += blockDim.x)
    reinterpret_cast<uint32_t*>(S.bv)[i] = 0u;
  for (int i = m * HD / 2 + threadIdx.x; i < L.mpad * HD / 2; i += blockDim.x)
    reinterpret_cast<uint32_t*>(S.dc)[i] = 0u;
  __syncthreads();
  const int vt = L.npad >> 4, ct = L.mpad >> 4, R = a.rounds;

  for (long long shot = blockIdx.x; shot < a.shots; shot += gridDim.x) {
    const uint8_t* sp = a.syndromes + shot * m;
    // initial states and their projections, one 16-row tile per warp
    for (int tile = warp; tile < vt + ct; tile += kInfWarps) {
      if (tile < vt) g_step<false>(S, n, tile * 16, false, true, nullptr, lane, sp);
      else g_step<true>(S, m, (tile - vt) * 16, false, true, nullptr, lane, sp);
    }
    __syncthreads();
    float* llr = a.llr_out ? a.llr_out + shot * n : S.llr;
    // a round: each warp gathers the aggregates of its own rows and updates them at once
    // (the gathers read the other node type's projections, complete after the barrier)
    for (int r = 0; r < R; ++r) {
      const bool last = r == R - 1;
      for (int tile = warp; tile < vt; tile += kInfWarps) {
        x_tile(n, tile * 16, a.var_ptr, a.var_chk, S.ac, S.bv, lane);
        g_step<false>(S, n, tile * 16, true, !last, llr, lane);
      }
      __syncthreads();
      if (last) break;
      for (int tile = warp; tile < ct; tile += kInfWarps) {
        x_tile(m, tile * 16, a.chk_ptr, a.chk_var, S.cv, S.dc, lane);
        g_step<true>(S, m, tile * 16, true, true, nullptr, lane);
      }
      __syncthreads();
    }
    if (a.llr_out) continue;
    // ---- decode mode: hard decision of the LLRs ----
    bool bad = false;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
      unsigned par = sp[i] ? 1u : 0u;
      const int e1 = __ldg(a.chk_ptr + i + 1);
      for (int e = __ldg(a.chk_ptr + i); e < e1; ++e) par ^= S.llr[__ldg(a.chk_var + e)] < 0.f;
      bad = bad || par;
    }
    if (__syncthreads_or(bad)) {
      __shared__ unsigned long long s_slot;
      if (threadIdx.x == 0) {
        s_slot = atomicAdd(&a.ctr->lsd_count, 1ULL);
        a.queue[s_slot] = (int32_t)shot;
      }
      __syncthreads();
      float* lo = a.queue_llr + (long long)s_slot * n;
      for (int j = threadIdx.x; j < n; j += blockDim.x) lo[j] = S.llr[j];
    } else {
      uint8_t* co = a.corrections + shot * n;
      for (int j = threadIdx.x; j < n; j += blockDim.x) co[j] = S.llr[j] < 0.f ? 1 : 0;
      if (threadIdx.x == 0) {
        if (a.status) a.status[shot] = LSD_SHOT_OK_BP;
        atomicAdd(&a.ctr->bp_converged, 1ULL);
      }
    }
    __syncthreads();
  }
}


// ======================================================================================
// Training on per-node products: the forward pass of prior_fwd_kernel (the states of every
// round saved in BF16 to a per-CTA scratch), the loss, and the backward pass of the same
// decomposition, round by round in reverse.  With W1cv = [Ucv | Vcv | w_s] (h_c, h_v, sigma
// blocks) and W1vc = [Uvc | Vvc | w_s'] (h_v', h_c, sigma blocks), for round t with output
// gradients g_hv' = dL/dh_v^{t+1} and g_hc' = dL/dh_c^{t+1}:
//   vc half:  gT_c = W2vc^T g_hc'       y_e = C_v + D_c
//             gC_v = sum_c gT_c [y_e > 0]    gD_c = gT_c * #{v in N(c) : y_e > 0}
//             g_hv' += Uvc^T gC_v             g_hc = g_hc' + Vvc^T gD_c
//   cv half:  gS_v = W2cv^T g_hv'       z_e = A_c + B_v
//             gA_c = sum_v gS_v [z_e > 0]    gB_v = gS_v * #{c in N(v) : z_e > 0}
//             g_hc += Ucv^T gA_c              g_hv = g_hv' + Vcv^T gB_v
//   weights:  dW2vc += sum_c g_hc' T_c^T, dVvc += sum_c gD_c h_c^T, dUvc += sum_v gC_v h_v'^T,
//             dW2cv += sum_v g_hv' S_v^T, dUcv += sum_c gA_c h_c^T, dVcv += sum_v gB_v h_v^T;
//             db2 = sum deg g_h', db1 = sum gD (gA), dw_s = sum sigma gD (gA).
// All products run on mma.sync with BF16 operands and FP32 accumulation.  Warps 0-5 each own
// one weight gradient and keep it in registers across every shot of the launch; warps 6-7
// accumulate the vector gradients.  One CTA (8 warps) per SM and shot.
// ======================================================================================

struct TrainArgs {
  int m, n, rounds;
  const int32_t* chk_ptr;
  const uint16_t* chk_var;
  const int32_t* var_ptr;
  const uint16_t* var_chk;
  const float* prior;
  const float* params;
  long long shots;
  const uint8_t* syndromes;
  const uint8_t* errors;
  __nv_bfloat16* scratch;  // per CTA: (R + 1) n + R m rows of 32 BF16 states
  float* grads;
  double* loss;
  float inv_norm;
};

struct TLay {
  int npad, mpad;
  size_t hv, hc, cv, bv, ac, dc, hvA, hvB, hcA, Sv, Tc, gT, gD, gA, gC, gS, gB, ghv, ghc;
  size_t w, wt, vec, vg, sig, lam, degv, degc, llr, total;
};

__host__ __device__ inline TLay train_layout(int m, int n) {
  TLay L;
  L.npad = (n + 15) & ~15;
  L.mpad = (m + 15) & ~15;
  const size_t fv = (size_t)L.npad * HD * 4, fc = (size_t)L.mpad * HD * 4;
  const size_t bv = fv / 2, bc = fc / 2;
  size_t o = 0;
  L.hv = o; o += fv;
  L.hc = o; o += fc;
  L.cv = o; o += bv;
  L.bv = o; o += bv;
  L.hvA = o; o += bv;
  L.hvB = o; o += bv;
  L.Sv = o; o += bv;
  L.gC = o; o += bv;
  L.gS = o; o += bv;
  L.gB = o; o += bv;
  L.ghv = o; o += bv;
  L.ac = o; o += bc;
  L.dc = o; o += bc;
  L.hcA = o; o += bc;
  L.Tc = o; o += bc;
  L.gT = o; o += bc;
  L.gD = o; o += bc;
  L.gA = o; o += bc;
  L.ghc = o; o += bc;
  L.w = o; o += (size_t)6 * HD * HD * 2;
  L.wt = o; o += (size_t)6 * HD * HD * 2;
  L.vec = o; o += (size_t)12 * HD * 4;
  L.vg = o; o += (size_t)12 * HD * 4;
  L.sig = o; o += a16((size_t)L.mpad * 4);
  L.lam = o; o += a16((size_t)L.npad * 4);
  L.degv = o; o += a16((size_t)L.npad * 4);
  L.degc = o; o += a16((size_t)L.mpad * 4);
  L.llr = o; o += a16((size_t)L.npad * 4);
  L.total = o;
  return L;
}

// vector-gradient slots
enum { VG_b2cv = 0, VG_b2vc, VG_wscv, VG_b1cv, VG_wsvc, VG_b1vc, VG_a0, VG_a1, VG_u0, VG_u1,
       VG_wo, VG_bo };

// acc[NT] += A[r0 .. r0+15][0..32) (BF16, swizzled) x W[w0 .. w0 + 8 NT)^T
template <int NT>
__device__ __forceinline__ void tile_mm(float acc[NT][4], const __nv_bfloat16* A, int r0,
                                        const __nv_bfloat16* Wt, int w0, int lane) {
  uint32_t af[2][4];
  fa_sw(af[0], A, r0, 0, lane);
  fa_sw(af[1], A, r0, 16, lane);
#pragma unroll
  for (int nt = 0; nt < NT; ++nt)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      uint32_t bf[2];
      fb_sw(bf, Wt, w0 + nt * 8, j * 16, lane);
      mma16816(acc[nt], af[j], bf);
    }
}

template <int NT>
__device__ __forceinline__ void tile_store_bf16(__nv_bfloat16* dst, int r0, int rows,
                                                const float acc[NT][4], int lane) {
  const int g = lane >> 2, t = lane & 3, ra = r0 + g, rb = r0 + g + 8;
#pragma unroll
  for (int nt = 0; nt < NT; ++nt) {
    const int col = nt * 8 + 2 * t;
    if (ra < rows) *reinterpret_cast<uint32_t*>(dst + bsw(ra, col)) = pack2(acc[nt][0], acc[nt][1]);
    if (rb < rows) *reinterpret_cast<uint32_t*>(dst + bsw(rb, col)) = pack2(acc[nt][2], acc[nt][3]);
  }
}

// FP32 state rows r0..r0+15 += A x W^T (in place), optionally copied out in BF16.
__device__ __forceinline__ void tile_update_f32(float* h, const __nv_bfloat16* A, int r0, int rows,
                                                const __nv_bfloat16* Wt, __nv_bfloat16* copy,
                                                int lane) {
  const int g = lane >> 2, t = lane & 3, ra = r0 + g, rb = r0 + g + 8;
  float acc[4][4];
#pragma unroll
  for (int nt = 0; nt < 4; ++nt) {
    const int col = nt * 8 + 2 * t;
    const float2 x = *reinterpret_cast<const float2*>(h + fsw(ra, col));
    const float2 y = *reinterpret_cast<const float2*>(h + fsw(rb, col));
    acc[nt][0] = x.x;
    acc[nt][1] = x.y;
    acc[nt][2] = y.x;
    acc[nt][3] = y.y;
  }
  tile_mm<4>(acc, A, r0, Wt, 0, lane);
#pragma unroll
  for (int nt = 0; nt < 4; ++nt) {
    const int col = nt * 8 + 2 * t;
    if (ra < rows) *reinterpret_cast<float2*>(h + fsw(ra, col)) = make_float2(acc[nt][0], acc[nt][1]);
    if (rb < rows) *reinterpret_cast<float2*>(h + fsw(rb, col)) = make_float2(acc[nt][2], acc[nt][3]);
  }
  if (copy) tile_store_bf16<4>(copy, r0, rows, acc, lane);
}

__device__ __forceinline__ float bf_at(const __nv_bfloat16* base, int r, int c) {
  return __bfloat162float(base[bsw(r, c)]);
}
__device__ __forceinline__ uint32_t bf_pair(const __nv_bfloat16* base, int r0, int r1, int c) {
  return pack_bf(base[bsw(r0, c)], base[bsw(r1, c)]);
}

// acc (32 x 32, j x k) += sum over rows of G[row][j] H[row][k]  (rows 0..K, K % 16 == 0; the
// padding rows of G and H are zero)
__device__ __forceinline__ void wgrad_mm(float acc[2][4][4], const __nv_bfloat16* G,
                                         const __nv_bfloat16* H, int K, int lane) {
  const int g = lane >> 2, t = lane & 3;
  for (int k0 = 0; k0 < K; k0 += 16) {
    const int ka = k0 + 2 * t, kb = ka + 8;
    uint32_t af[2][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
      const int j = mt * 16 + g;
      af[mt][0] = bf_pair(G, ka, ka + 1, j);
      af[mt][1] = bf_pair(G, ka, ka + 1, j + 8);
      af[mt][2] = bf_pair(G, kb, kb + 1, j);
      af[mt][3] = bf_pair(G, kb, kb + 1, j + 8);
    }
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      uint32_t bf[2];
      const int kk = nt * 8 + g;
      bf[0] = bf_pair(H, ka, ka + 1, kk);
      bf[1] = bf_pair(H, kb, kb + 1, kk);
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) mma16816(acc[mt][nt], af[mt], bf);
    }
  }
}

// Copy `rows` rows of 32 BF16 values (row-major, global) into a swizzled shared array.
__device__ __forceinline__ void load_rows(__nv_bfloat16* dst, const __nv_bfloat16* src, int rows) {
  for (int i = threadIdx.x; i < rows * 4; i += blockDim.x) {
    const int r = i >> 2, b = i & 3;
    *reinterpret_cast<uint4*>(dst + bsw(r, 8 * b)) =
        *reinterpret_cast<const uint4*>(src + r * HD + 8 * b);
  }
}

__global__ void __launch_bounds__(kFwdWarps * 32, 1) prior_train_kernel(TrainArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int m = a.m, n = a.n, R = a.rounds;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const TLay L = train_layout(m, n);
  auto BF = [&](size_t off) { return reinterpret_cast<__nv_bfloat16*>(smem + off); };
  FwdSmem S;
  S.hv = reinterpret_cast<float*>(smem + L.hv);
  S.hc = reinterpret_cast<float*>(smem + L.hc);
  S.cv = BF(L.cv);
  S.bv = BF(L.bv);
  S.ac = BF(L.ac);
  S.dc = BF(L.dc);
  S.W2cv = BF(L.w);
  S.Wv = S.W2cv + HD * HD;
  S.W2vc = S.Wv + 2 * HD * HD;
  S.Wc = S.W2vc + HD * HD;
  S.vec = reinterpret_cast<float*>(smem + L.vec);
  S.sig = reinterpret_cast<float*>(smem + L.sig);
  S.lam = reinterpret_cast<float*>(smem + L.lam);
  S.degv = reinterpret_cast<float*>(smem + L.degv);
  S.degc = reinterpret_cast<float*>(smem + L.degc);
  S.llr = reinterpret_cast<float*>(smem + L.llr);
  __nv_bfloat16 *hvA = BF(L.hvA), *hvB = BF(L.hvB), *hcA = BF(L.hcA), *Sv = BF(L.Sv),
                *Tc = BF(L.Tc), *gT = BF(L.gT), *gD = BF(L.gD), *gA = BF(L.gA), *gC = BF(L.gC),
                *gS = BF(L.gS), *gB = BF(L.gB), *ghv = BF(L.ghv), *ghc = BF(L.ghc);
  __nv_bfloat16* WT = BF(L.wt);  // transposed weights: W2vc, Vvc, Uvc, W2cv, Ucv, Vcv
  float* vg = reinterpret_cast<float*>(smem + L.vg);
  float* gv = S.hv;  // after the forward pass: dL/dh_v, dL/dh_c
  float* gc = S.hc;

  // ---- parameters, graph degrees, zero padding ----
  const float* P = a.params;
  for (int i = threadIdx.x; i < HD * HD; i += blockDim.x) {
    const int r = i >> 5, k = i & 31;
    const float w2cv = P[POff::W2cv + r * HD + k], w2vc = P[POff::W2vc + r * HD + k];
    const float ucv = P[POff::W1cv + r * DIN + k], vcv = P[POff::W1cv + r * DIN + HD + k];
    const float uvc = P[POff::W1vc + r * DIN + k], vvc = P[POff::W1vc + r * DIN + HD + k];
    S.W2cv[bsw(r, k)] = __float2bfloat16_rn(w2cv);
    S.W2vc[bsw(r, k)] = __float2bfloat16_rn(w2vc);
    S.Wv[bsw(r, k)] = __float2bfloat16_rn(uvc);        // C
    S.Wv[bsw(r + HD, k)] = __float2bfloat16_rn(vcv);   // B
    S.Wc[bsw(r, k)] = __float2bfloat16_rn(ucv);        // A
    S.Wc[bsw(r + HD, k)] = __float2bfloat16_rn(vvc);   // D
    // transposes (row k, column r)
    WT[0 * HD * HD + bsw(k, r)] = __float2bfloat16_rn(w2vc);
    WT[1 * HD * HD + bsw(k, r)] = __float2bfloat16_rn(vvc);
    WT[2 * HD * HD + bsw(k, r)] = __float2bfloat16_rn(uvc);
    WT[3 * HD * HD + bsw(k, r)] = __float2bfloat16_rn(w2cv);
    WT[4 * HD * HD + bsw(k, r)] = __float2bfloat16_rn(ucv);
    WT[5 * HD * HD + bsw(k, r)] = __float2bfloat16_rn(vcv);
  }
  for (int i = threadIdx.x; i < HD; i += blockDim.x) {
    S.vec[F_a0 * HD + i] = P[POff::a0 + i];
    S.vec[F_a1 * HD + i] = P[POff::a1 + i];
    S.vec[F_u0 * HD + i] = P[POff::u0 + i];
    S.vec[F_u1 * HD + i] = P[POff::u1 + i];
    S.vec[F_b2cv * HD + i] = P[POff::b2cv + i];
    S.vec[F_b2vc * HD + i] = P[POff::b2vc + i];
    S.vec[F_wscv * HD + i] = P[POff::W1cv + i * DIN + 2 * HD];
    S.vec[F_b1cv * HD + i] = P[POff::b1cv + i];
    S.vec[F_wsvc * HD + i] = P[POff::W1vc + i * DIN + 2 * HD];
    S.vec[F_b1vc * HD + i] = P[POff::b1vc + i];
    S.vec[F_wo * HD + i] = P[POff::wo + i];
    S.vec[F_bo * HD + i] = i == 0 ? P[POff::bo] : 0.f;
  }
  for (int i = threadIdx.x; i < 12 * HD; i += blockDim.x) vg[i] = 0.f;
  for (int j = threadIdx.x; j < L.npad; j += blockDim.x) {
    S.lam[j] = j < n ? a.prior[j] : 0.f;
    S.degv[j] = j < n ? (float)(a.var_ptr[j + 1] - a.var_ptr[j]) : 0.f;
  }
  for (int i = threadIdx.x; i < L.mpad; i += blockDim.x) {
    S.degc[i] = i < m ? (float)(a.chk_ptr[i + 1] - a.chk_ptr[i]) : 0.f;
    S.sig[i] = 0.f;
  }
  // every node array starts zero, so its padding rows stay zero
  {
    uint32_t* z = reinterpret_cast<uint32_t*>(smem + L.hv);
    const size_t words = (L.w - L.hv) / 4;
    for (size_t i = threadIdx.x; i < words; i += blockDim.x) z[i] = 0u;
  }
  __syncthreads();
  const int vt = L.npad >> 4, ct = L.mpad >> 4;
  __nv_bfloat16* save = a.scratch + (size_t)blockIdx.x * ((size_t)(R + 1) * n + (size_t)R * m) * HD;
  auto save_hv = [&](int t) { return save + (size_t)t * n * HD; };
  auto save_hc = [&](int t) { return save + (size_t)(R + 1) * n * HD + (size_t)t * m * HD; };

  float wacc[2][4][4];  // warps 0-5: one weight gradient (32 x 32)
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) wacc[i][j][q] = 0.f;
  double loss_acc = 0.0;

  for (long long shot = blockIdx.x; shot < a.shots; shot += gridDim.x) {
    const uint8_t* sp = a.syndromes + shot * m;
    const uint8_t* ep = a.errors + shot * n;
    // ================= forward (prior_fwd_kernel, saving every state) =================
    for (int tile = warp; tile < vt + ct; tile += kFwdWarps) {
      if (tile < vt) g_step<false>(S, n, tile * 16, false, true, nullptr, lane, sp, save_hv(0));
      else g_step<true>(S, m, (tile - vt) * 16, false, true, nullptr, lane, sp, save_hc(0));
    }
    __syncthreads();
    for (int r = 0; r < R; ++r) {
      const bool last = r == R - 1;
      for (int tile = warp; tile < vt; tile += kFwdWarps) {
        x_tile(n, tile * 16, a.var_ptr, a.var_chk, S.ac, S.bv, lane);
        g_step<false>(S, n, tile * 16, true, !last, S.llr, lane, nullptr, save_hv(r + 1));
      }
      __syncthreads();
      if (last) break;
      for (int tile = warp; tile < ct; tile += kFwdWarps) {
        x_tile(m, tile * 16, a.chk_ptr, a.chk_var, S.cv, S.dc, lane);
        g_step<true>(S, m, tile * 16, true, true, nullptr, lane, nullptr, save_hc(r + 1));
      }
      __syncthreads();
    }
    // ================= loss, dL/dLLR, output layer =================
    for (int v = threadIdx.x; v < n; v += blockDim.x) {
      const float l = S.llr[v];
      const float y = ep[v] ? 1.f : 0.f;
      const float sp_l = l > 0.f ? l + log1pf(__expf(-l)) : log1pf(__expf(l));
      loss_acc += (double)(sp_l - (1.f - y) * l);
      S.llr[v] = (1.f / (1.f + __expf(-l)) - (1.f - y)) * a.inv_norm;
    }
    __syncthreads();
    {
      float dwo = 0.f, dbo = 0.f;
      for (int v = warp; v < n; v += kFwdWarps) {
        dwo = fmaf(S.llr[v], S.hv[fsw(v, lane)], dwo);
        dbo += S.llr[v];
      }
      atomicAdd(&vg[VG_wo * HD + lane], dwo);
      if (lane == 0) atomicAdd(&vg[VG_bo * HD], dbo);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n * HD; i += blockDim.x) {
      const int v = i >> 5, k = i & 31;
      gv[fsw(v, k)] = S.llr[v] * S.vec[F_wo * HD + k];
    }
    for (int i = threadIdx.x; i < m * HD; i += blockDim.x) gc[fsw(i >> 5, i & 31)] = 0.f;
    __syncthreads();
    // ================= backward, rounds in reverse =================
    for (int r = R - 1; r >= 0; --r) {
      // states of the round and the BF16 copy of dL/dh_c^{r+1}
      load_rows(hvB, save_hv(r + 1), n);
      load_rows(hvA, save_hv(r), n);
      load_rows(hcA, save_hc(r), m);
      for (int i = threadIdx.x; i < m * HD / 2; i += blockDim.x) {
        const int c = i >> 4, k = 2 * (i & 15);
        const float2 x = *reinterpret_cast<const float2*>(gc + fsw(c, k));
        *reinterpret_cast<uint32_t*>(ghc + bsw(c, k)) = pack2(x.x, x.y);
      }
      __syncthreads();
      // projections A, D (checks), B, C (variables); gT = W2vc^T g_hc'
      for (int tile = warp; tile < vt + ct; tile += kFwdWarps) {
        const int g = lane >> 2, t = lane & 3;
        if (tile < vt) {
          const int r0 = tile * 16;
          float accB[4][4] = {}, accC[4][4] = {};
          tile_mm<4>(accB, hvA, r0, S.Wv, HD, lane);
          tile_mm<4>(accC, hvB, r0, S.Wv, 0, lane);
          tile_store_bf16<4>(S.bv, r0, n, accB, lane);
          tile_store_bf16<4>(S.cv, r0, n, accC, lane);
        } else {
          const int r0 = (tile - vt) * 16, ra = r0 + g, rb = r0 + g + 8;
          const float sa = S.sig[ra], sb = S.sig[rb];
          float accA[4][4], accD[4][4], accT[4][4] = {};
#pragma unroll
          for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int q = 0; q < 2; ++q) {
              const int col = nt * 8 + 2 * t + q;
              accA[nt][q] = fmaf(sa, S.vec[F_wscv * HD + col], S.vec[F_b1cv * HD + col]);
              accA[nt][2 + q] = fmaf(sb, S.vec[F_wscv * HD + col], S.vec[F_b1cv * HD + col]);
              accD[nt][q] = fmaf(sa, S.vec[F_wsvc * HD + col], S.vec[F_b1vc * HD + col]);
              accD[nt][2 + q] = fmaf(sb, S.vec[F_wsvc * HD + col], S.vec[F_b1vc * HD + col]);
            }
          tile_mm<4>(accA, hcA, r0, S.Wc, 0, lane);
          tile_mm<4>(accD, hcA, r0, S.Wc, HD, lane);
          tile_mm<4>(accT, ghc, r0, WT, 0, lane);
          tile_store_bf16<4>(S.ac, r0, m, accA, lane);
          tile_store_bf16<4>(S.dc, r0, m, accD, lane);
          tile_store_bf16<4>(gT, r0, m, accT, lane);
        }
      }
      __syncthreads();
      // gathers of the vc half (and S for dW2cv): 4 lanes of 8 columns per node
      for (int i = threadIdx.x; i < (n + m) * 4; i += blockDim.x) {
        const int b = i & 3;
        float x0[8], acc1[8], acc2[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) acc1[k] = acc2[k] = 0.f;
        if (i < n * 4) {  // variable v: S_v, gC_v
          const int v = i >> 2;
          float bvv[8];
          unpack8(*reinterpret_cast<const uint4*>(S.cv + bsw(v, 8 * b)), x0);
          unpack8(*reinterpret_cast<const uint4*>(S.bv + bsw(v, 8 * b)), bvv);
          for (int e = a.var_ptr[v]; e < a.var_ptr[v + 1]; ++e) {
            const int c = a.var_chk[e];
            float av[8], dv[8], tv[8];
            unpack8(*reinterpret_cast<const uint4*>(S.ac + bsw(c, 8 * b)), av);
            unpack8(*reinterpret_cast<const uint4*>(S.dc + bsw(c, 8 * b)), dv);
            unpack8(*reinterpret_cast<const uint4*>(gT + bsw(c, 8 * b)), tv);
#pragma unroll
            for (int k = 0; k < 8; ++k) {
              acc1[k] += fmaxf(av[k] + bvv[k], 0.f);
              acc2[k] += (x0[k] + dv[k] > 0.f) ? tv[k] : 0.f;
            }
          }
          *reinterpret_cast<uint4*>(Sv + bsw(v, 8 * b)) =
              make_uint4(pack2(acc1[0], acc1[1]), pack2(acc1[2], acc1[3]), pack2(acc1[4], acc1[5]),
                         pack2(acc1[6], acc1[7]));
          *reinterpret_cast<uint4*>(gC + bsw(v, 8 * b)) =
              make_uint4(pack2(acc2[0], acc2[1]), pack2(acc2[2], acc2[3]), pack2(acc2[4], acc2[5]),
                         pack2(acc2[6], acc2[7]));
        } else {  // check c: T_c, gD_c
          const int c = (i >> 2) - n;
          float tv[8];
          unpack8(*reinterpret_cast<const uint4*>(S.dc + bsw(c, 8 * b)), x0);
          unpack8(*reinterpret_cast<const uint4*>(gT + bsw(c, 8 * b)), tv);
          for (int e = a.chk_ptr[c]; e < a.chk_ptr[c + 1]; ++e) {
            const int v = a.chk_var[e];
            float cvv[8];
            unpack8(*reinterpret_cast<const uint4*>(S.cv + bsw(v, 8 * b)), cvv);
#pragma unroll
            for (int k = 0; k < 8; ++k) {
              const float y = cvv[k] + x0[k];
              acc1[k] += fmaxf(y, 0.f);
              acc2[k] += y > 0.f ? 1.f : 0.f;
            }
          }
#pragma unroll
          for (int k = 0; k < 8; ++k) acc2[k] *= tv[k];
          *reinterpret_cast<uint4*>(Tc + bsw(c, 8 * b)) =
              make_uint4(pack2(acc1[0], acc1[1]), pack2(acc1[2], acc1[3]), pack2(acc1[4], acc1[5]),
                         pack2(acc1[6], acc1[7]));
          *reinterpret_cast<uint4*>(gD + bsw(c, 8 * b)) =
              make_uint4(pack2(acc2[0], acc2[1]), pack2(acc2[2], acc2[3]), pack2(acc2[4], acc2[5]),
                         pack2(acc2[6], acc2[7]));
        }
      }
      __syncthreads();
      // g_hv' += Uvc^T gC (and its BF16 copy);  g_hc = g_hc' + Vvc^T gD
      for (int tile = warp; tile < vt + ct; tile += kFwdWarps) {
        if (tile < vt) tile_update_f32(gv, gC, tile * 16, n, WT + 2 * HD * HD, ghv, lane);
        else tile_update_f32(gc, gD, (tile - vt) * 16, m, WT + 1 * HD * HD, nullptr, lane);
      }
      __syncthreads();
      // gS = W2cv^T g_hv'
      for (int tile = warp; tile < vt; tile += kFwdWarps) {
        float acc[4][4] = {};
        tile_mm<4>(acc, ghv, tile * 16, WT + 3 * HD * HD, 0, lane);
        tile_store_bf16<4>(gS, tile * 16, n, acc, lane);
      }
      __syncthreads();
      // gathers of the cv half: gA_c, gB_v
      for (int i = threadIdx.x; i < (n + m) * 4; i += blockDim.x) {
        const int b = i & 3;
        float x0[8], acc[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) acc[k] = 0.f;
        if (i < n * 4) {  // variable v: gB_v = gS_v * #{c : A_c + B_v > 0}
          const int v = i >> 2;
          float sv[8];
          unpack8(*reinterpret_cast<const uint4*>(S.bv + bsw(v, 8 * b)), x0);
          unpack8(*reinterpret_cast<const uint4*>(gS + bsw(v, 8 * b)), sv);
          for (int e = a.var_ptr[v]; e < a.var_ptr[v + 1]; ++e) {
            float av[8];
            unpack8(*reinterpret_cast<const uint4*>(S.ac + bsw(a.var_chk[e], 8 * b)), av);
#pragma unroll
            for (int k = 0; k < 8; ++k) acc[k] += (av[k] + x0[k] > 0.f) ? 1.f : 0.f;
          }
#pragma unroll
          for (int k = 0; k < 8; ++k) acc[k] *= sv[k];
          *reinterpret_cast<uint4*>(gB + bsw(v, 8 * b)) =
              make_uint4(pack2(acc[0], acc[1]), pack2(acc[2], acc[3]), pack2(acc[4], acc[5]),
                         pack2(acc[6], acc[7]));
        } else {  // check c: gA_c = sum_v gS_v [A_c + B_v > 0]
          const int c = (i >> 2) - n;
          unpack8(*reinterpret_cast<const uint4*>(S.ac + bsw(c, 8 * b)), x0);
          for (int e = a.chk_ptr[c]; e < a.chk_ptr[c + 1]; ++e) {
            const int v = a.chk_var[e];
            float bvv[8], sv[8];
            unpack8(*reinterpret_cast<const uint4*>(S.bv + bsw(v, 8 * b)), bvv);
            unpack8(*reinterpret_cast<const uint4*>(gS + bsw(v, 8 * b)), sv);
#pragma unroll
            for (int k = 0; k < 8; ++k) acc[k] += (x0[k] + bvv[k] > 0.f) ? sv[k] : 0.f;
          }
          *reinterpret_cast<uint4*>(gA + bsw(c, 8 * b)) =
              make_uint4(pack2(acc[0], acc[1]), pack2(acc[2], acc[3]), pack2(acc[4], acc[5]),
                         pack2(acc[6], acc[7]));
        }
      }
      __syncthreads();
      // g_hc += Ucv^T gA;  g_hv = g_hv' + Vcv^T gB;  then the parameter gradients of the round
      for (int tile = warp; tile < vt + ct; tile += kFwdWarps) {
        if (tile < vt) tile_update_f32(gv, gB, tile * 16, n, WT + 5 * HD * HD, nullptr, lane);
        else tile_update_f32(gc, gA, (tile - vt) * 16, m, WT + 4 * HD * HD, nullptr, lane);
      }
      switch (warp) {
        case 0: wgrad_mm(wacc, ghc, Tc, L.mpad, lane); break;   // dW2vc
        case 1: wgrad_mm(wacc, gD, hcA, L.mpad, lane); break;   // dVvc
        case 2: wgrad_mm(wacc, gC, hvB, L.npad, lane); break;   // dUvc
        case 3: wgrad_mm(wacc, ghv, Sv, L.npad, lane); break;   // dW2cv
        case 4: wgrad_mm(wacc, gA, hcA, L.mpad, lane); break;   // dUcv
        case 5: wgrad_mm(wacc, gB, hvA, L.npad, lane); break;   // dVcv
        case 6: {
          float b2 = 0.f, ws = 0.f, b1 = 0.f;
          for (int c = 0; c < m; ++c) {
            const float gd = bf_at(gD, c, lane);
            b2 = fmaf(S.degc[c], bf_at(ghc, c, lane), b2);
            ws = fmaf(S.sig[c], gd, ws);
            b1 += gd;
          }
          vg[VG_b2vc * HD + lane] += b2;
          vg[VG_wsvc * HD + lane] += ws;
          vg[VG_b1vc * HD + lane] += b1;
          break;
        }
        default: {
          float b2 = 0.f, ws = 0.f, b1 = 0.f;
          for (int v = 0; v < n; ++v) b2 = fmaf(S.degv[v], bf_at(ghv, v, lane), b2);
          for (int c = 0; c < m; ++c) {
            const float ga = bf_at(gA, c, lane);
            ws = fmaf(S.sig[c], ga, ws);
            b1 += ga;
          }
          vg[VG_b2cv * HD + lane] += b2;
          vg[VG_wscv * HD + lane] += ws;
          vg[VG_b1cv * HD + lane] += b1;
          break;
        }
      }
      __syncthreads();
    }
    // ================= the initial states =================
    if (warp == 0) {
      float d0 = 0.f, d1 = 0.f;
      for (int v = 0; v < n; ++v) {
        const float z = fmaf(S.lam[v], S.vec[F_a0 * HD + lane], S.vec[F_a1 * HD + lane]);
        const float gz = z > 0.f ? gv[fsw(v, lane)] : 0.f;
        d0 = fmaf(gz, S.lam[v], d0);
        d1 += gz;
      }
      vg[VG_a0 * HD + lane] += d0;
      vg[VG_a1 * HD + lane] += d1;
    } else if (warp == 1) {
      float d0 = 0.f, d1 = 0.f;
      for (int c = 0; c < m; ++c) {
        const float gcv = gc[fsw(c, lane)];
        d0 = fmaf(S.sig[c], gcv, d0);
        d1 += gcv;
      }
      vg[VG_u0 * HD + lane] += d0;
      vg[VG_u1 * HD + lane] += d1;
    }
    __syncthreads();
  }
  // ---- flush the CTA's gradients ----
  float* G = a.grads;
  if (warp < 6) {
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int nt = 0; nt < 4; ++nt)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int j = mt * 16 + g + (q >> 1) * 8, k = nt * 8 + 2 * t + (q & 1);
          int idx;
          switch (warp) {
            case 0: idx = POff::W2vc + j * HD + k; break;
            case 1: idx = POff::W1vc + j * DIN + HD + k; break;
            case 2: idx = POff::W1vc + j * DIN + k; break;
            case 3: idx = POff::W2cv + j * HD + k; break;
            case 4: idx = POff::W1cv + j * DIN + k; break;
            default: idx = POff::W1cv + j * DIN + HD + k; break;
          }
          atomicAdd(&G[idx], wacc[mt][nt][q]);
        }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < HD; k += blockDim.x) {
    atomicAdd(&G[POff::b2cv + k], vg[VG_b2cv * HD + k]);
    atomicAdd(&G[POff::b2vc + k], vg[VG_b2vc * HD + k]);
    atomicAdd(&G[POff::W1cv + k * DIN + 2 * HD], vg[VG_wscv * HD + k]);
    atomicAdd(&G[POff::b1cv + k], vg[VG_b1cv * HD + k]);
    atomicAdd(&G[POff::W1vc + k * DIN + 2 * HD], vg[VG_wsvc * HD + k]);
    atomicAdd(&G[POff::b1vc + k], vg[VG_b1vc * HD + k]);
    atomicAdd(&G[POff::a0 + k], vg[VG_a0 * HD + k]);
    atomicAdd(&G[POff::a1 + k], vg[VG_a1 * HD + k]);
    atomicAdd(&G[POff::u0 + k], vg[VG_u0 * HD + k]);
    atomicAdd(&G[POff::u1 + k], vg[VG_u1 * HD + k]);
    atomicAdd(&G[POff::wo + k], vg[VG_wo * HD + k]);
  }
  if (threadIdx.x == 0) atomicAdd(&G[POff::bo], vg[VG_bo * HD]);
  for (int off = 16; off > 0; off >>= 1) loss_acc += __shfl_xor_sync(0xffffffffu, loss_acc, off);
  if (lane == 0 && loss_acc != 0.0) atomicAdd(a.loss, loss_acc);
}

}  // namespace


int prior_num_params() { return POff::total; }

size_t prior_smem(int m, int n, int E, bool train) {
  (void)E;
  return train ? train_layout(m, n).total : fwd_layout(m, n).total;
}

size_t prior_scratch_floats(int m, int n, int rounds, int grid) {
  // BF16 states: (R + 1) variable and R check rows of 32 values per CTA
  return ((size_t)grid * ((size_t)(rounds + 1) * n + (size_t)rounds * m) * HD + 1) / 2;
}

cudaError_t prior_config(int m, int n, int E, bool train, int* grid) {
  int dev = 0, sms = 0, max_smem = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const size_t smem = prior_smem(m, n, E, train);
  if (smem > (size_t)max_smem) return cudaErrorInvalidValue;
  const void* fn = train ? (const void*)prior_train_kernel : (const void*)prior_fwd_kernel;
  const int threads = (train ? kFwdWarps : kInfWarps) * 32;
  err = allow_max_dynamic_smem(fn, max_smem);
  if (err != cudaSuccess) return err;
  int per_sm = 0;
  err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem);
  if (err != cudaSuccess) return err;
  if (per_sm < 1) return cudaErrorInvalidValue;
  *grid = per_sm * sms;
  return cudaSuccess;
}

cudaError_t launch_prior_decode(int grid, const DevGraph& g, int rounds, const float* params,
                                long long shots, const uint8_t* syndromes, float* llr_out,
                                uint8_t* corrections, uint8_t* status, int32_t* queue,
                                float* queue_llr, DevCounters* ctr, cudaStream_t st) {
  if (!llr_out && (!corrections || !queue || !queue_llr || !ctr)) return cudaErrorInvalidValue;
  FwdArgs f{};
  f.m = g.m;
  f.n = g.n;
  f.rounds = rounds;
  f.chk_ptr = g.chk_ptr;
  f.chk_var = g.chk_var;
  f.var_ptr = g.var_ptr;
  f.var_chk = g.var_chk;
  f.prior = g.prior;
  f.params = params;
  f.shots = shots;
  f.syndromes = syndromes;
  f.llr_out = llr_out;
  f.corrections = corrections;
  f.status = status;
  f.queue = queue;
  f.queue_llr = queue_llr;
  f.ctr = ctr;
  const long long blocks = shots < grid ? shots : grid;
  if (blocks <= 0) return cudaSuccess;
  prior_fwd_kernel<<<(int)blocks, kInfWarps * 32, fwd_layout(g.m, g.n).total, st>>>(f);
  return cudaGetLastError();
}

cudaError_t launch_prior(bool train, int grid, const DevGraph& g, int rounds, const float* params,
                         long long shots, const uint8_t* syndromes, const uint8_t* errors,
                         float* llr_out, float* scratch, float* grads, double* loss,
                         cudaStream_t st) {
  if (!train) {
    if (!llr_out) return cudaErrorInvalidValue;
    return launch_prior_decode(grid, g, rounds, params, shots, syndromes, llr_out, nullptr,
                               nullptr, nullptr, nullptr, nullptr, st);
  }
  TrainArgs a{};
  a.m = g.m;
  a.n = g.n;
  a.rounds = rounds;
  a.chk_ptr = g.chk_ptr;
  a.chk_var = g.chk_var;
  a.var_ptr = g.var_ptr;
  a.var_chk = g.var_chk;
  a.prior = g.prior;
  a.params = params;
  a.shots = shots;
  a.syndromes = syndromes;
  a.errors = errors;
  a.scratch = reinterpret_cast<__nv_bfloat16*>(scratch);
  a.grads = grads;
  a.loss = loss;
  a.inv_norm = shots > 0 ? (float)(1.0 / ((double)shots * g.n)) : 0.f;
  (void)llr_out;
  const long long blocks = shots < grid ? shots : grid;
  if (blocks <= 0) return cudaSuccess;
  prior_train_kernel<<<(int)blocks, kFwdWarps * 32, train_layout(g.m, g.n).total, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_adam(float* p, const float* g, float* m, float* v, int count, float lr,
                        int step, cudaStream_t st) {
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  adam_kernel<<<(count + 255) / 256, 256, 0, st>>>(p, g, m, v, count, lr, b1, b2, 1e-8f, c1, c2);
  return cudaGetLastError();
}

cudaError_t launch_sample(const DevGraph& g, const float* probs, unsigned long long seed,
                          long long first, long long shots, uint8_t* errors, uint8_t* syndromes,
                          cudaStream_t st) {
  if (shots <= 0) return cudaSuccess;
  const int threads = 128;
  sample_kernel<<<(int)((shots + threads - 1) / threads), threads, 0, st>>>(
      seed, first, shots, g.m, g.n, probs, g.chk_ptr, g.chk_var, errors, syndromes);
  return cudaGetLastError();
}

}  // namespace lsdgb
