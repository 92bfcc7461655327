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
// One CTA owns one shot at a time; node states (FP32) live in shared memory.  A warp
// handles 16 edges at a time: it gathers X = [h_first | h_second | sigma | 1 | 0...]
// (16 x 80, BF16) into its staging tile, runs the two layers with mma.sync m16n8k16
// (the layer-1 accumulator fragments are re-packed in registers as the A operand of layer
// 2), and scatter-adds the 16 x 32 messages into the destination accumulators.  The
// backward pass recomputes layer 1 from the saved node states, forms da1 = dm W2 and
// dx = dz1 W1 on the tensor cores, and the weight gradients dW2 = dm^T a1 and
// dW1 = dz1^T X (its column 65 is the bias gradient) with transposed operand loads from
// the staging tiles.
#include <cuda_bf16.h>

#include "lsd_internal.cuh"

namespace lsdgb {

namespace {

constexpr int HD = 32;        // hidden width
constexpr int XK = 80;        // padded layer-1 input: 32 + 32 + sigma + one + 14 zeros
constexpr int DIN = 2 * HD + 1;
constexpr int NWARP = 8;
constexpr int kPriorThreads = NWARP * 32;

__host__ __device__ inline size_t a16(size_t x) { return (x + 15) & ~(size_t)15; }

// offsets of the flat parameter vector
struct POff {
  static constexpr int a0 = 0, a1 = 32, u0 = 64, u1 = 96;
  static constexpr int W1cv = 128, b1cv = W1cv + HD * DIN, W2cv = b1cv + HD, b2cv = W2cv + HD * HD;
  static constexpr int W1vc = b2cv + HD, b1vc = W1vc + HD * DIN, W2vc = b1vc + HD,
                       b2vc = W2vc + HD * HD;
  static constexpr int wo = b2vc + HD, bo = wo + HD, total = bo + 1;
};

// Shared-memory layout of the prior kernel (runtime n, m, E).
struct PLay {
  size_t hv, hc, accv, accc, gv, gc, W1, W2, W1T, W2T, vec, dW1, dW2, db2, stage, ec, ev, sig,
      lam, llr, err, total;
};

__host__ __device__ inline PLay prior_layout(int m, int n, int E, bool train) {
  PLay L;
  size_t o = 0;
  L.hv = o; o += a16((size_t)n * HD * 4);
  L.hc = o; o += a16((size_t)m * HD * 4);
  L.accv = o; o += a16((size_t)n * HD * 4);
  L.accc = o; o += a16((size_t)m * HD * 4);
  L.gv = o; o += train ? a16((size_t)n * HD * 4) : 0;
  L.gc = o; o += train ? a16((size_t)m * HD * 4) : 0;
  L.W1 = o; o += 2 * (size_t)HD * XK * 2;     // [dir][32][80] bf16
  L.W2 = o; o += 2 * (size_t)HD * HD * 2;     // [dir][32][32]
  L.W1T = o; o += 2 * (size_t)XK * HD * 2;    // [dir][80][32]
  L.W2T = o; o += 2 * (size_t)HD * HD * 2;    // [dir][32][32]
  L.vec = o; o += 16 * HD * 4;                 // a0 a1 u0 u1 b1cv b2cv b1vc b2vc wo (+bo)
  L.dW1 = o; o += train ? 2 * (size_t)HD * XK * 4 : 0;
  L.dW2 = o; o += train ? 2 * (size_t)HD * HD * 4 : 0;
  L.db2 = o; o += train ? 16 * HD * 4 : 0;     // db2cv db2vc da0 da1 du0 du1 dwo dbo
  L.stage = o; o += (size_t)NWARP * (16 * XK * 2 + 3 * 16 * HD * 2);
  L.ec = o; o += a16((size_t)E * 2);
  L.ev = o; o += a16((size_t)E * 2);
  L.sig = o; o += a16((size_t)m * 4);
  L.lam = o; o += a16((size_t)n * 4);
  L.llr = o; o += a16((size_t)n * 4);
  L.err = o; o += a16((size_t)n);
  L.total = a16(o);
  return L;
}

struct PriorArgs {
  int m, n, E, rounds;
  const int32_t* chk_ptr;
  const uint16_t* chk_var;
  const float* prior;      // lambda_j
  const float* params;     // flat FP32 parameters
  long long shots;
  const uint8_t* syndromes;
  const uint8_t* errors;   // training targets (train only)
  float* llr_out;          // [shots][n] (forward only, nullable)
  float* scratch;          // per-CTA saved node states (train only)
  float* grads;            // flat FP32 gradient accumulator (train only)
  double* loss;            // loss sum accumulator (train only)
  float inv_norm;          // 1 / (shots * n)
};

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

// A[r][k] = base[r*ld + k] (row-major tile), rows r0.., cols k0..k0+15
__device__ __forceinline__ void frag_a_row(uint32_t a[4], const __nv_bfloat16* base, int ld,
                                           int r0, int k0, int lane) {
  const int g = lane >> 2, t = lane & 3;
  a[0] = ld32(base + (r0 + g) * ld + k0 + 2 * t);
  a[1] = ld32(base + (r0 + g + 8) * ld + k0 + 2 * t);
  a[2] = ld32(base + (r0 + g) * ld + k0 + 2 * t + 8);
  a[3] = ld32(base + (r0 + g + 8) * ld + k0 + 2 * t + 8);
}
// A[r][k] = base[k*ld + r] (transposed source)
__device__ __forceinline__ void frag_a_col(uint32_t a[4], const __nv_bfloat16* base, int ld,
                                           int r0, int k0, int lane) {
  const int g = lane >> 2, t = lane & 3;
  const int r = r0 + g, k = k0 + 2 * t;
  a[0] = pack_bf(base[k * ld + r], base[(k + 1) * ld + r]);
  a[1] = pack_bf(base[k * ld + r + 8], base[(k + 1) * ld + r + 8]);
  a[2] = pack_bf(base[(k + 8) * ld + r], base[(k + 9) * ld + r]);
  a[3] = pack_bf(base[(k + 8) * ld + r + 8], base[(k + 9) * ld + r + 8]);
}
// B[k][n] = base[n*ld + k] ([N][K] storage)
__device__ __forceinline__ void frag_b_nk(uint32_t b[2], const __nv_bfloat16* base, int ld,
                                          int n0, int k0, int lane) {
  const int g = lane >> 2, t = lane & 3;
  b[0] = ld32(base + (n0 + g) * ld + k0 + 2 * t);
  b[1] = ld32(base + (n0 + g) * ld + k0 + 2 * t + 8);
}
// B[k][n] = base[k*ld + n] ([K][N] storage)
__device__ __forceinline__ void frag_b_kn(uint32_t b[2], const __nv_bfloat16* base, int ld,
                                          int k0, int n0, int lane) {
  const int g = lane >> 2, t = lane & 3;
  const int k = k0 + 2 * t, n = n0 + g;
  b[0] = pack_bf(base[k * ld + n], base[(k + 1) * ld + n]);
  b[1] = pack_bf(base[(k + 8) * ld + n], base[(k + 9) * ld + n]);
}

struct Smem {
  float *hv, *hc, *accv, *accc, *gv, *gc, *vec, *dW1, *dW2, *db2, *sig, *lam, *llr;
  __nv_bfloat16 *W1, *W2, *W1T, *W2T;
  unsigned char* stage;
  uint16_t *ec, *ev;
  uint8_t* err;
};

// vec slots (x32 floats each)
enum { V_a0 = 0, V_a1, V_u0, V_u1, V_b1cv, V_b2cv, V_b1vc, V_b2vc, V_wo, V_bo };
// db2 slots
enum { G_b2cv = 0, G_b2vc, G_a0, G_a1, G_u0, G_u1, G_wo, G_bo };

// Gathers X for edges tile*16.. into the warp's staging tile (BF16 [16][80]).
// dir 0 (check -> variable): X = [h_c, h_v, sigma_c, 1]; dir 1: X = [h_v, h_c, sigma_c, 1].
__device__ __forceinline__ void stage_x(const Smem& S, const PriorArgs& a, int dir, int tile,
                                        __nv_bfloat16* Xs, int lane) {
  for (int idx = lane; idx < 16 * (XK / 2); idx += 32) {
    const int row = idx / (XK / 2), col = 2 * (idx % (XK / 2));
    const int e = tile * 16 + row;
    float x0 = 0.f, x1 = 0.f;
    if (e < a.E) {
      const int c = S.ec[e], v = S.ev[e];
      const float* first = dir == 0 ? S.hc + c * HD : S.hv + v * HD;
      const float* second = dir == 0 ? S.hv + v * HD : S.hc + c * HD;
      if (col < HD) {
        x0 = first[col];
        x1 = first[col + 1];
      } else if (col < 2 * HD) {
        x0 = second[col - HD];
        x1 = second[col - HD + 1];
      } else if (col == 2 * HD) {
        x0 = S.sig[c];
        x1 = 1.f;
      }
    }
    *reinterpret_cast<uint32_t*>(Xs + row * XK + col) = pack2(x0, x1);
  }
  __syncwarp();
}

// Layer 1 of direction dir on the staged X: z1 (16 x 32) as four accumulator fragments.
__device__ __forceinline__ void layer1(const Smem& S, int dir, const __nv_bfloat16* Xs,
                                       float z[4][4], int lane) {
  const int t = lane & 3;
  const float* b1 = S.vec + (dir == 0 ? V_b1cv : V_b1vc) * HD;
  const __nv_bfloat16* W1 = S.W1 + dir * HD * XK;
#pragma unroll
  for (int nt = 0; nt < 4; ++nt) {
    z[nt][0] = z[nt][2] = b1[nt * 8 + 2 * t];
    z[nt][1] = z[nt][3] = b1[nt * 8 + 2 * t + 1];
  }
#pragma unroll
  for (int ks = 0; ks < XK / 16; ++ks) {
    uint32_t af[4];
    frag_a_row(af, Xs, XK, 0, ks * 16, lane);
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      uint32_t bf[2];
      frag_b_nk(bf, W1, XK, nt * 8, ks * 16, lane);
      mma16816(z[nt], af, bf);
    }
  }
}

// One message half-round (forward): messages of direction dir into the destination
// accumulators.
__device__ void pass_forward(const Smem& S, const PriorArgs& a, int dir, int warp, int lane) {
  const int g = lane >> 2, t = lane & 3;
  __nv_bfloat16* Xs = reinterpret_cast<__nv_bfloat16*>(S.stage + warp * (16 * XK * 2 + 3 * 16 * HD * 2));
  const float* b2 = S.vec + (dir == 0 ? V_b2cv : V_b2vc) * HD;
  const __nv_bfloat16* W2 = S.W2 + dir * HD * HD;
  float* acc = dir == 0 ? S.accv : S.accc;
  const int ntiles = (a.E + 15) / 16;
  for (int tile = warp; tile < ntiles; tile += NWARP) {
    stage_x(S, a, dir, tile, Xs, lane);
    float z[4][4];
    layer1(S, dir, Xs, z, lane);
    uint32_t a2[2][4];
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      a2[j][0] = pack2(fmaxf(z[2 * j][0], 0.f), fmaxf(z[2 * j][1], 0.f));
      a2[j][1] = pack2(fmaxf(z[2 * j][2], 0.f), fmaxf(z[2 * j][3], 0.f));
      a2[j][2] = pack2(fmaxf(z[2 * j + 1][0], 0.f), fmaxf(z[2 * j + 1][1], 0.f));
      a2[j][3] = pack2(fmaxf(z[2 * j + 1][2], 0.f), fmaxf(z[2 * j + 1][3], 0.f));
    }
    const int e0 = tile * 16 + g, e1 = e0 + 8;
    const int d0 = e0 < a.E ? (dir == 0 ? S.ev[e0] : S.ec[e0]) : -1;
    const int d1 = e1 < a.E ? (dir == 0 ? S.ev[e1] : S.ec[e1]) : -1;
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      float c[4];
      c[0] = c[2] = b2[nt * 8 + 2 * t];
      c[1] = c[3] = b2[nt * 8 + 2 * t + 1];
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        uint32_t bf[2];
        frag_b_nk(bf, W2, HD, nt * 8, j * 16, lane);
        mma16816(c, a2[j], bf);
      }
      if (d0 >= 0) {
        atomicAdd(&acc[d0 * HD + nt * 8 + 2 * t], c[0]);
        atomicAdd(&acc[d0 * HD + nt * 8 + 2 * t + 1], c[1]);
      }
      if (d1 >= 0) {
        atomicAdd(&acc[d1 * HD + nt * 8 + 2 * t], c[2]);
        atomicAdd(&acc[d1 * HD + nt * 8 + 2 * t + 1], c[3]);
      }
    }
    __syncwarp();
  }
}

// One message half-round (backward) of direction dir: gradient dm of every message is the
// gradient state of its destination; adds dx to the source accumulators and the weight
// gradients to the CTA accumulators.
__device__ void pass_backward(const Smem& S, const PriorArgs& a, int dir, int warp, int lane) {
  const int g = lane >> 2, t = lane & 3;
  unsigned char* wb = S.stage + warp * (16 * XK * 2 + 3 * 16 * HD * 2);
  __nv_bfloat16* Xs = reinterpret_cast<__nv_bfloat16*>(wb);
  __nv_bfloat16* A1s = Xs + 16 * XK;
  __nv_bfloat16* DMs = A1s + 16 * HD;
  __nv_bfloat16* DZs = DMs + 16 * HD;
  const __nv_bfloat16* W1T = S.W1T + dir * XK * HD;
  const __nv_bfloat16* W2T = S.W2T + dir * HD * HD;
  const float* gdst = dir == 0 ? S.gv : S.gc;          // gradient of the destination states
  float* acc_first = dir == 0 ? S.accc : S.accv;      // x[0:32]
  float* acc_second = dir == 0 ? S.accv : S.accc;     // x[32:64]
  float* dW1 = S.dW1 + dir * HD * XK;
  float* dW2 = S.dW2 + dir * HD * HD;
  float db2 = 0.f;  // lane's column of db2
  const int ntiles = (a.E + 15) / 16;
  for (int tile = warp; tile < ntiles; tile += NWARP) {
    stage_x(S, a, dir, tile, Xs, lane);
    float z[4][4];
    layer1(S, dir, Xs, z, lane);
    const int e0 = tile * 16 + g, e1 = e0 + 8;
    // a1 tile (for dW2) and dm tile (gathered gradient of the destinations)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      *reinterpret_cast<uint32_t*>(A1s + g * HD + nt * 8 + 2 * t) =
          pack2(fmaxf(z[nt][0], 0.f), fmaxf(z[nt][1], 0.f));
      *reinterpret_cast<uint32_t*>(A1s + (g + 8) * HD + nt * 8 + 2 * t) =
          pack2(fmaxf(z[nt][2], 0.f), fmaxf(z[nt][3], 0.f));
    }
    for (int idx = lane; idx < 16 * (HD / 2); idx += 32) {
      const int row = idx / (HD / 2), col = 2 * (idx % (HD / 2));
      const int e = tile * 16 + row;
      float v0 = 0.f, v1 = 0.f;
      if (e < a.E) {
        const int d = dir == 0 ? S.ev[e] : S.ec[e];
        v0 = gdst[d * HD + col];
        v1 = gdst[d * HD + col + 1];
      }
      *reinterpret_cast<uint32_t*>(DMs + row * HD + col) = pack2(v0, v1);
    }
    __syncwarp();
    // db2: column sums of dm (lane = column)
    for (int row = 0; row < 16; ++row) db2 += __bfloat162float(DMs[row * HD + lane]);
    // da1 = dm W2 ; dz1 = da1 * [z1 > 0]
    float dz[4][4];
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) dz[nt][0] = dz[nt][1] = dz[nt][2] = dz[nt][3] = 0.f;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      uint32_t af[4];
      frag_a_row(af, DMs, HD, 0, j * 16, lane);
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        uint32_t bf[2];
        frag_b_nk(bf, W2T, HD, nt * 8, j * 16, lane);
        mma16816(dz[nt], af, bf);
      }
    }
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
#pragma unroll
      for (int q = 0; q < 4; ++q) dz[nt][q] = z[nt][q] > 0.f ? dz[nt][q] : 0.f;
      *reinterpret_cast<uint32_t*>(DZs + g * HD + nt * 8 + 2 * t) = pack2(dz[nt][0], dz[nt][1]);
      *reinterpret_cast<uint32_t*>(DZs + (g + 8) * HD + nt * 8 + 2 * t) =
          pack2(dz[nt][2], dz[nt][3]);
    }
    __syncwarp();
    // dx = dz1 W1 (columns 0..63), scattered to the two endpoint accumulators
    {
      uint32_t af[2][4];
      frag_a_row(af[0], DZs, HD, 0, 0, lane);
      frag_a_row(af[1], DZs, HD, 0, 16, lane);
      const int c0 = e0 < a.E ? S.ec[e0] : -1, v0 = e0 < a.E ? S.ev[e0] : -1;
      const int c1 = e1 < a.E ? S.ec[e1] : -1, v1 = e1 < a.E ? S.ev[e1] : -1;
      const int f0 = dir == 0 ? c0 : v0, s0 = dir == 0 ? v0 : c0;
      const int f1 = dir == 0 ? c1 : v1, s1 = dir == 0 ? v1 : c1;
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          uint32_t bf[2];
          frag_b_nk(bf, W1T, HD, nt * 8, j * 16, lane);
          mma16816(c, af[j], bf);
        }
        const int col = (nt & 3) * 8 + 2 * t;
        float* dst0 = nt < 4 ? (f0 >= 0 ? acc_first + f0 * HD : nullptr)
                             : (s0 >= 0 ? acc_second + s0 * HD : nullptr);
        float* dst1 = nt < 4 ? (f1 >= 0 ? acc_first + f1 * HD : nullptr)
                             : (s1 >= 0 ? acc_second + s1 * HD : nullptr);
        if (dst0) {
          atomicAdd(dst0 + col, c[0]);
          atomicAdd(dst0 + col + 1, c[1]);
        }
        if (dst1) {
          atomicAdd(dst1 + col, c[2]);
          atomicAdd(dst1 + col + 1, c[3]);
        }
      }
    }
    // dW2 += dm^T a1  (32 x 32, k = the 16 edges)
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
      uint32_t af[4];
      frag_a_col(af, DMs, HD, mt * 16, 0, lane);
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        uint32_t bf[2];
        frag_b_kn(bf, A1s, HD, 0, nt * 8, lane);
        float c[4] = {0.f, 0.f, 0.f, 0.f};
        mma16816(c, af, bf);
        float* w = dW2 + (mt * 16 + g) * HD + nt * 8 + 2 * t;
        atomicAdd(w, c[0]);
        atomicAdd(w + 1, c[1]);
        atomicAdd(w + 8 * HD, c[2]);
        atomicAdd(w + 8 * HD + 1, c[3]);
      }
    }
    // dW1 += dz1^T X  (32 x 72 used: inputs 0..64 and the bias column 65)
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
      uint32_t af[4];
      frag_a_col(af, DZs, HD, mt * 16, 0, lane);
#pragma unroll
      for (int nt = 0; nt < 9; ++nt) {
        uint32_t bf[2];
        frag_b_kn(bf, Xs, XK, 0, nt * 8, lane);
        float c[4] = {0.f, 0.f, 0.f, 0.f};
        mma16816(c, af, bf);
        float* w = dW1 + (mt * 16 + g) * XK + nt * 8 + 2 * t;
        atomicAdd(w, c[0]);
        atomicAdd(w + 1, c[1]);
        atomicAdd(w + 8 * XK, c[2]);
        atomicAdd(w + 8 * XK + 1, c[3]);
      }
    }
    __syncwarp();
  }
  atomicAdd(&S.db2[(dir == 0 ? G_b2cv : G_b2vc) * HD + lane], db2);
}

__device__ __forceinline__ void cta_zero(float* p, int count) {
  for (int i = threadIdx.x; i < count; i += blockDim.x) p[i] = 0.f;
}

// h_dst += acc (and optionally copies h_dst to `save`)
__device__ __forceinline__ void cta_add(float* h, const float* acc, int count, float* save) {
  for (int i = threadIdx.x; i < count; i += blockDim.x) {
    const float v = h[i] + acc[i];
    h[i] = v;
    if (save) save[i] = v;
  }
}

template <bool TRAIN>
__global__ void __launch_bounds__(kPriorThreads) prior_kernel(PriorArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int m = a.m, n = a.n, E = a.E;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const PLay L = prior_layout(m, n, E, TRAIN);
  Smem S;
  S.hv = reinterpret_cast<float*>(smem + L.hv);
  S.hc = reinterpret_cast<float*>(smem + L.hc);
  S.accv = reinterpret_cast<float*>(smem + L.accv);
  S.accc = reinterpret_cast<float*>(smem + L.accc);
  S.gv = reinterpret_cast<float*>(smem + L.gv);
  S.gc = reinterpret_cast<float*>(smem + L.gc);
  S.W1 = reinterpret_cast<__nv_bfloat16*>(smem + L.W1);
  S.W2 = reinterpret_cast<__nv_bfloat16*>(smem + L.W2);
  S.W1T = reinterpret_cast<__nv_bfloat16*>(smem + L.W1T);
  S.W2T = reinterpret_cast<__nv_bfloat16*>(smem + L.W2T);
  S.vec = reinterpret_cast<float*>(smem + L.vec);
  S.dW1 = reinterpret_cast<float*>(smem + L.dW1);
  S.dW2 = reinterpret_cast<float*>(smem + L.dW2);
  S.db2 = reinterpret_cast<float*>(smem + L.db2);
  S.stage = smem + L.stage;
  S.ec = reinterpret_cast<uint16_t*>(smem + L.ec);
  S.ev = reinterpret_cast<uint16_t*>(smem + L.ev);
  S.sig = reinterpret_cast<float*>(smem + L.sig);
  S.lam = reinterpret_cast<float*>(smem + L.lam);
  S.llr = reinterpret_cast<float*>(smem + L.llr);
  S.err = reinterpret_cast<uint8_t*>(smem + L.err);

  // ---- parameters: BF16 weight tiles (and their transposes), FP32 vectors ----
  const float* P = a.params;
  for (int i = threadIdx.x; i < 2 * HD * XK; i += blockDim.x) {
    const int dir = i / (HD * XK), r = (i / XK) % HD, k = i % XK;
    const float v = k < DIN ? P[(dir ? POff::W1vc : POff::W1cv) + r * DIN + k] : 0.f;
    const __nv_bfloat16 b = __float2bfloat16_rn(v);
    S.W1[i] = b;
    S.W1T[dir * XK * HD + k * HD + r] = b;
  }
  for (int i = threadIdx.x; i < 2 * HD * HD; i += blockDim.x) {
    const int dir = i / (HD * HD), r = (i / HD) % HD, k = i % HD;
    const __nv_bfloat16 b = __float2bfloat16_rn(P[(dir ? POff::W2vc : POff::W2cv) + r * HD + k]);
    S.W2[i] = b;
    S.W2T[dir * HD * HD + k * HD + r] = b;
  }
  for (int i = threadIdx.x; i < HD; i += blockDim.x) {
    S.vec[V_a0 * HD + i] = P[POff::a0 + i];
    S.vec[V_a1 * HD + i] = P[POff::a1 + i];
    S.vec[V_u0 * HD + i] = P[POff::u0 + i];
    S.vec[V_u1 * HD + i] = P[POff::u1 + i];
    S.vec[V_b1cv * HD + i] = P[POff::b1cv + i];
    S.vec[V_b2cv * HD + i] = P[POff::b2cv + i];
    S.vec[V_b1vc * HD + i] = P[POff::b1vc + i];
    S.vec[V_b2vc * HD + i] = P[POff::b2vc + i];
    S.vec[V_wo * HD + i] = P[POff::wo + i];
  }
  if (threadIdx.x == 0) S.vec[V_bo * HD] = P[POff::bo];
  for (int i = threadIdx.x; i < m; i += blockDim.x)
    for (int e = a.chk_ptr[i]; e < a.chk_ptr[i + 1]; ++e) {
      S.ec[e] = (uint16_t)i;
      S.ev[e] = a.chk_var[e];
    }
  for (int j = threadIdx.x; j < n; j += blockDim.x) S.lam[j] = a.prior[j];
  if (TRAIN) {
    cta_zero(S.dW1, 2 * HD * XK);
    cta_zero(S.dW2, 2 * HD * HD);
    cta_zero(S.db2, 16 * HD);
  }
  __syncthreads();
  const int R = a.rounds;
  float* save = TRAIN ? a.scratch + (size_t)blockIdx.x * (R + 1) * (n + m) * HD : nullptr;
  double loss_acc = 0.0;

  for (long long shot = blockIdx.x; shot < a.shots; shot += gridDim.x) {
    // ---- init ----
    const uint8_t* sp = a.syndromes + shot * m;
    for (int i = threadIdx.x; i < m; i += blockDim.x) S.sig[i] = sp[i] ? -1.f : 1.f;
    if (TRAIN)
      for (int j = threadIdx.x; j < n; j += blockDim.x) S.err[j] = a.errors[shot * n + j];
    __syncthreads();
    for (int i = threadIdx.x; i < n * HD; i += blockDim.x) {
      const int v = i / HD, k = i % HD;
      const float z = fmaf(S.lam[v], S.vec[V_a0 * HD + k], S.vec[V_a1 * HD + k]);
      S.hv[i] = fmaxf(z, 0.f);
      if (TRAIN) save[i] = S.hv[i];
    }
    for (int i = threadIdx.x; i < m * HD; i += blockDim.x) {
      const int c = i / HD, k = i % HD;
      S.hc[i] = fmaf(S.sig[c], S.vec[V_u0 * HD + k], S.vec[V_u1 * HD + k]);
      if (TRAIN) save[n * HD + i] = S.hc[i];
    }
    __syncthreads();
    // ---- rounds ----
    for (int r = 0; r < R; ++r) {
      float* sv = TRAIN ? save + (size_t)(r + 1) * (n + m) * HD : nullptr;
      cta_zero(S.accv, n * HD);
      __syncthreads();
      pass_forward(S, a, 0, warp, lane);
      __syncthreads();
      cta_add(S.hv, S.accv, n * HD, sv);
      cta_zero(S.accc, m * HD);
      __syncthreads();
      pass_forward(S, a, 1, warp, lane);
      __syncthreads();
      cta_add(S.hc, S.accc, m * HD, sv ? sv + n * HD : nullptr);
      __syncthreads();
    }
    // ---- output LLRs ----
    for (int v = warp; v < n; v += NWARP) {
      float d = S.hv[v * HD + lane] * S.vec[V_wo * HD + lane];
      for (int off = 16; off > 0; off >>= 1) d += __shfl_xor_sync(0xffffffffu, d, off);
      if (lane == 0) {
        const float l = S.lam[v] + d + S.vec[V_bo * HD];
        S.llr[v] = l;
        if (!TRAIN && a.llr_out) a.llr_out[shot * n + v] = l;
      }
    }
    __syncthreads();
    if (!TRAIN) continue;

    // ---- loss and dL/dLLR ----
    for (int v = threadIdx.x; v < n; v += blockDim.x) {
      const float l = S.llr[v];
      const float y = S.err[v] ? 1.f : 0.f;
      const float sp_l = l > 0.f ? l + log1pf(__expf(-l)) : log1pf(__expf(l));
      loss_acc += (double)(sp_l - (1.f - y) * l);
      const float sg = 1.f / (1.f + __expf(-l));
      S.llr[v] = (sg - (1.f - y)) * a.inv_norm;  // now dLLR
    }
    __syncthreads();
    // dw_o, db_o (lane = hidden unit), g_v = dLLR w_o, g_c = 0
    {
      float dwo = 0.f, dbo = 0.f;
      for (int v = warp; v < n; v += NWARP) {
        dwo += S.llr[v] * S.hv[v * HD + lane];
        dbo += lane == 0 ? S.llr[v] : 0.f;
      }
      atomicAdd(&S.db2[G_wo * HD + lane], dwo);
      if (lane == 0) atomicAdd(&S.db2[G_bo * HD], dbo);
    }
    for (int i = threadIdx.x; i < n * HD; i += blockDim.x)
      S.gv[i] = S.llr[i / HD] * S.vec[V_wo * HD + (i % HD)];
    cta_zero(S.gc, m * HD);
    __syncthreads();
    for (int r = R - 1; r >= 0; --r) {
      const float* st0 = save + (size_t)r * (n + m) * HD;        // h_v^r, h_c^r
      const float* st1 = save + (size_t)(r + 1) * (n + m) * HD;  // h_v^{r+1}, h_c^{r+1}
      // direction v -> c of round r: inputs h_v^{r+1}, h_c^r
      for (int i = threadIdx.x; i < n * HD; i += blockDim.x) S.hv[i] = st1[i];
      for (int i = threadIdx.x; i < m * HD; i += blockDim.x) S.hc[i] = st0[n * HD + i];
      cta_zero(S.accv, n * HD);
      cta_zero(S.accc, m * HD);
      __syncthreads();
      pass_backward(S, a, 1, warp, lane);
      __syncthreads();
      cta_add(S.gv, S.accv, n * HD, nullptr);
      cta_add(S.gc, S.accc, m * HD, nullptr);
      // direction c -> v of round r: inputs h_c^r, h_v^r
      for (int i = threadIdx.x; i < n * HD; i += blockDim.x) S.hv[i] = st0[i];
      cta_zero(S.accv, n * HD);
      cta_zero(S.accc, m * HD);
      __syncthreads();
      pass_backward(S, a, 0, warp, lane);
      __syncthreads();
      cta_add(S.gv, S.accv, n * HD, nullptr);
      cta_add(S.gc, S.accc, m * HD, nullptr);
      __syncthreads();
    }
    // init-layer gradients (hv holds h_v^0 = relu(z_v^0): z > 0 iff h > 0)
    {
      float da0 = 0.f, da1 = 0.f, du0 = 0.f, du1 = 0.f;
      for (int v = warp; v < n; v += NWARP) {
        const float z = fmaf(S.lam[v], S.vec[V_a0 * HD + lane], S.vec[V_a1 * HD + lane]);
        const float gz = z > 0.f ? S.gv[v * HD + lane] : 0.f;
        da0 += gz * S.lam[v];
        da1 += gz;
      }
      for (int c = warp; c < m; c += NWARP) {
        du0 += S.gc[c * HD + lane] * S.sig[c];
        du1 += S.gc[c * HD + lane];
      }
      atomicAdd(&S.db2[G_a0 * HD + lane], da0);
      atomicAdd(&S.db2[G_a1 * HD + lane], da1);
      atomicAdd(&S.db2[G_u0 * HD + lane], du0);
      atomicAdd(&S.db2[G_u1 * HD + lane], du1);
    }
    __syncthreads();
  }
  if (!TRAIN) return;
  // ---- flush the CTA's gradients ----
  __syncthreads();
  float* G = a.grads;
  for (int i = threadIdx.x; i < 2 * HD * XK; i += blockDim.x) {
    const int dir = i / (HD * XK), r = (i / XK) % HD, k = i % XK;
    const float v = S.dW1[i];
    if (k < DIN) atomicAdd(&G[(dir ? POff::W1vc : POff::W1cv) + r * DIN + k], v);
    else if (k == DIN) atomicAdd(&G[(dir ? POff::b1vc : POff::b1cv) + r], v);
  }
  for (int i = threadIdx.x; i < 2 * HD * HD; i += blockDim.x) {
    const int dir = i / (HD * HD), rk = i % (HD * HD);
    atomicAdd(&G[(dir ? POff::W2vc : POff::W2cv) + rk], S.dW2[i]);
  }
  for (int i = threadIdx.x; i < HD; i += blockDim.x) {
    atomicAdd(&G[POff::b2cv + i], S.db2[G_b2cv * HD + i]);
    atomicAdd(&G[POff::b2vc + i], S.db2[G_b2vc * HD + i]);
    atomicAdd(&G[POff::a0 + i], S.db2[G_a0 * HD + i]);
    atomicAdd(&G[POff::a1 + i], S.db2[G_a1 * HD + i]);
    atomicAdd(&G[POff::u0 + i], S.db2[G_u0 * HD + i]);
    atomicAdd(&G[POff::u1 + i], S.db2[G_u1 * HD + i]);
    atomicAdd(&G[POff::wo + i], S.db2[G_wo * HD + i]);
  }
  if (threadIdx.x == 0) atomicAdd(&G[POff::bo], S.db2[G_bo * HD]);
  for (int off = 16; off > 0; off >>= 1) loss_acc += __shfl_xor_sync(0xffffffffu, loss_acc, off);
  if (lane == 0 && loss_acc != 0.0) atomicAdd(a.loss, loss_acc);
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

constexpr int kFwdWarps = 8;

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
                                       float* llr, int lane, const uint8_t* syn = nullptr) {
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

__global__ void __launch_bounds__(kFwdWarps * 32, 3) prior_fwd_kernel(FwdArgs a) {
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
    for (int tile = warp; tile < vt + ct; tile += kFwdWarps) {
      if (tile < vt) g_step<false>(S, n, tile * 16, false, true, nullptr, lane, sp);
      else g_step<true>(S, m, (tile - vt) * 16, false, true, nullptr, lane, sp);
    }
    __syncthreads();
    float* llr = a.llr_out ? a.llr_out + shot * n : S.llr;
    // a round: each warp gathers the aggregates of its own rows and updates them at once
    // (the gathers read the other node type's projections, complete after the barrier)
    for (int r = 0; r < R; ++r) {
      const bool last = r == R - 1;
      for (int tile = warp; tile < vt; tile += kFwdWarps) {
        x_tile(n, tile * 16, a.var_ptr, a.var_chk, S.ac, S.bv, lane);
        g_step<false>(S, n, tile * 16, true, !last, llr, lane);
      }
      __syncthreads();
      if (last) break;
      for (int tile = warp; tile < ct; tile += kFwdWarps) {
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

}  // namespace


int prior_num_params() { return POff::total; }

size_t prior_smem(int m, int n, int E, bool train) {
  return train ? prior_layout(m, n, E, true).total : fwd_layout(m, n).total;
}

size_t prior_scratch_floats(int m, int n, int rounds, int grid) {
  return (size_t)grid * (rounds + 1) * (n + m) * HD;
}

cudaError_t prior_config(int m, int n, int E, bool train, int* grid) {
  int dev = 0, sms = 0, max_smem = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const size_t smem = prior_smem(m, n, E, train);
  if (smem > (size_t)max_smem) return cudaErrorInvalidValue;
  const void* fn = train ? (const void*)prior_kernel<true> : (const void*)prior_fwd_kernel;
  const int threads = train ? kPriorThreads : kFwdWarps * 32;
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
  prior_fwd_kernel<<<(int)blocks, kFwdWarps * 32, fwd_layout(g.m, g.n).total, st>>>(f);
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
  PriorArgs a{};
  a.m = g.m;
  a.n = g.n;
  a.E = g.E;
  a.rounds = rounds;
  a.chk_ptr = g.chk_ptr;
  a.chk_var = g.chk_var;
  a.prior = g.prior;
  a.params = params;
  a.shots = shots;
  a.syndromes = syndromes;
  a.errors = errors;
  a.llr_out = llr_out;
  a.scratch = scratch;
  a.grads = grads;
  a.loss = loss;
  a.inv_norm = shots > 0 ? (float)(1.0 / ((double)shots * g.n)) : 0.f;
  const size_t smem = prior_smem(g.m, g.n, g.E, train);
  const long long blocks = shots < grid ? shots : grid;
  if (blocks <= 0) return cudaSuccess;
  prior_kernel<true><<<(int)blocks, kPriorThreads, smem, st>>>(a);
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
