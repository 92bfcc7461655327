// Learned prior, inference on the 5th-generation tensor cores: the per-node projections of
// every round live in tensor memory (TMEM) as FP32 accumulators, and each round's dense
// products are tcgen05.mma instructions (BF16 operands from shared memory, FP32 accumulate)
// issued by one thread and tracked by an mbarrier.  The paper has no learned component; the
// model is the one defined in include/lsd.h (see prior.cu for its restatement).
//
// Reformulation.  The projections the gathers read are linear in the node states:
//   P_v = [C_v | B_v] = Wv h_v,   Wv = [W1vc[:, 0:32] ; W1cv[:, 32:64]]            (64 x 32)
//   P_c = [A_c | D_c] = Wc h_c + sigma_c ws + b1,   Wc = [W1cv[:, 0:32] ; W1vc[:, 32:64]]
// and a round adds W2 S + deg b2 to a state, so the projections themselves advance by
//   P_v <- P_v + Mv S_v + deg_v kv,   Mv = Wv W2cv,  kv = Wv b2cv
//   P_c <- P_c + Mc T_c + deg_c kc,   Mc = Wc W2vc,  kc = Wc b2vc
// (S_v = sum_c relu(A_c + B_v), T_c = sum_v relu(C_v + D_c): the gathers).  The states are
// never formed: TMEM holds P^0 + sum_t M S^t per node row, the deg k terms are added in FP32
// when a row is read, and the output LLR_v = lambda_v + w_o . h_v^R + b_o is tracked as
//   y_v = lambda_v + w_o . h_v^0 + b_o + sum_t (W2cv^T w_o) . S_v^t + deg_v (w_o . b2cv).
// The initial projections do not depend on the shot for variables (h_v^0 is a function of
// lambda_v) and take one of two values for checks (sigma_c = +-1): both are tabulated once
// per CTA.  Weights are rounded to BF16, Mv and Mc formed from the rounded factors in FP32
// and rounded to BF16 once; accumulators, biases and LLRs stay FP32.
//
// Layout.  One CTA works on a group of S shots at a time, their node rows stacked: variable
// row s * n8 + v (n8 = n rounded up to 8, so every shot's rows start a core-matrix row group)
// in vt 128-row tiles and check row s * m8 + c in ct tiles, 64 TMEM columns per tile
// (vt + ct <= 8; S is the largest group that fits, at most 8).  The weights are shared by all
// rows, so one MMA per tile serves the whole group and each barrier and completion wait of a
// round is paid once per group, not once per shot.  A round:
//   X2 (all threads, 4 per row, 8 features each): S_v from the A_c rows in shared memory and
//       the row's own B_v; BF16 S_v into the MMA operand buffer; the LLR update
//   MMA (one thread): P_v tiles += S tile x Mv^T (M = 128, N = 64, K = 32: two K = 16 steps)
//   epilogue (the warps whose TMEM lane quarter holds the row): tcgen05.ld of P_v, + deg kv,
//       BF16 C_v and B_v rows into shared memory
//   X1, MMA on the check tiles, epilogue: the same for T_c, P_c, A_c and D_c
// The last round stops after X2 (only the LLR needs it).  Shared-memory operands use the
// canonical K-major layout without swizzle: 8-row x 16-byte core matrices, adjacent along K
// 128 bytes apart, adjacent along M/N 512 bytes apart (a K = 32 BF16 row block).
#include <cuda_bf16.h>

#include <algorithm>

#include "lsd_internal.cuh"
#include "prior_params.cuh"

namespace lsdgb {

namespace {

using prior_params::DIN;
using prior_params::HD;
using prior_params::POff;

constexpr int kTcMinWarps = 8, kTcMaxWarps = 20;
constexpr int kTcMaxTiles = 8;  // variable + check tiles: 64 TMEM columns each, 512 in all
constexpr int kTcMaxGroup = 8;  // shots per CTA group

struct TcArgs {
  int m, n, E, rounds, vt, ct, tmem_cols;
  int S, n8, m8;            // shots per group; rows per shot, rounded up to 8
  uint32_t inv_n8, inv_m8;  // ceil(2^32 / n8), ceil(2^32 / m8): row -> shot by one mul.hi
  const int32_t* chk_ptr;
  const uint16_t* chk_var;
  const int32_t* var_ptr;
  const uint16_t* var_chk;
  const float* prior;
  const float* params;
  long long shots;
  const uint8_t* syndromes;
  float* llr_out;       // [shots][n], or null: decode mode (as prior_fwd_kernel)
  uint8_t* corrections;
  uint8_t* status;
  int32_t* queue;
  float* queue_llr;
  DevCounters* ctr;
  int* timeout_flag;    // set when an MMA completion wait runs out (nullable)
};

struct TcLay {
  size_t mv, mc, op, as, ds, cs, bs, p0, pc0, kv, kc, u, y0, llr, degv, degc, sig, vptr, cptr,
      vadj, cadj, misc, total;
};

__host__ __device__ inline size_t al(size_t x, size_t a) { return (x + a - 1) / a * a; }

__host__ __device__ inline int up8(int x) { return (x + 7) & ~7; }

// Shared memory of a group of S shots: per-row arrays over S n8 / S m8 rows, the tables once.
__host__ __device__ inline TcLay tc_layout(int m, int n, int E, int vt, int ct, int S) {
  TcLay L;
  size_t o = 0;
  const size_t N = (size_t)S * up8(n), M = (size_t)S * up8(m);
  L.mv = o; o += 4096;                                   // Mv: 64 x 32 BF16, K-major
  L.mc = o; o += 4096;                                   // Mc
  // S or T tiles (128 x 32 BF16 each); at set-up, Wv and Wc in FP32 (16 KB)
  L.op = o; o += (size_t)(vt > ct ? (vt > 2 ? vt : 2) : (ct > 2 ? ct : 2)) * 8192;
  L.as = o; o += al(M * 64, 128);                        // BF16 rows [S m8][32] (swizzled)
  L.ds = o; o += al(M * 64, 128);
  L.cs = o; o += al(N * 64, 128);
  L.bs = o; o += al(N * 64, 128);                        // at set-up, with cs: h_v^0 [n][32] FP32
  L.p0 = o; o += (size_t)n * 256;                        // FP32 [n][64], 4-float chunks rotated
  L.pc0 = o; o += 512;                                   // FP32 [2][64]: sigma = +1, -1
  L.kv = o; o += 256;
  L.kc = o; o += 256;
  L.u = o; o += 128;
  L.y0 = o; o += al((size_t)n * 4, 16);
  L.llr = o; o += al(N * 4, 16);
  L.degv = o; o += al((size_t)n * 4, 16);
  L.degc = o; o += al((size_t)m * 4, 16);
  L.sig = o; o += al(M * 4, 16);
  L.vptr = o; o += al((size_t)(n + 1) * 4, 16);          // the graph: CSC / CSR row starts
  L.cptr = o; o += al((size_t)(m + 1) * 4, 16);
  L.vadj = o; o += al((size_t)E * 4, 16);                // per edge: row * 64 | swizzle bits
  L.cadj = o; o += al((size_t)E * 4, 16);
  L.misc = o; o += 64;                                   // kappa, TMEM address, mbarrier, flags
  L.total = o;
  return L;
}

// ---- PTX helpers ----
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
// Shared-memory matrix descriptor of tcgen05.mma: start address, leading (K direction) and
// stride (M/N direction) byte offsets in 16-byte units, the fixed version field 0b001 at
// bits 46-48, no swizzle.
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)(128 >> 4) << 16) |
         ((uint64_t)(512 >> 4) << 32) | ((uint64_t)1 << 46);
}
// Byte offset of element (row r, column k) of a K-major operand with K = 32 per row block.
__device__ __forceinline__ int koff(int r, int k) {
  return (r >> 3) * 512 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}
// Instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both K-major,
// N = 64, M = 128.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((64u >> 3) << 17) |
                            ((128u >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
      :: "r"(tmem_d), "l"(a), "l"(b), "r"(kIdesc), "r"(1));
}
__device__ __forceinline__ void mma_commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
               :: "r"(smem_u32(mbar)) : "memory");
}
__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Waits for the mbarrier phase with the given parity; false after about one second.
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity) {
  const uint32_t a = smem_u32(mbar);
  uint32_t done = 0;
  const unsigned long long t0 = global_ns();
  while (true) {
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done) : "r"(a), "r"(parity) : "memory");
    if (done) return true;
    if (global_ns() - t0 > 1000000000ull) return false;
  }
}

// 16 consecutive FP32 columns of this thread's TMEM lane (warp-collective).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* f) {
  uint32_t v[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) f[i] = __uint_as_float(v[i]);
}
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float* f) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
      "%13,%14,%15,%16};"
      :: "r"(taddr), "r"(__float_as_uint(f[0])), "r"(__float_as_uint(f[1])),
         "r"(__float_as_uint(f[2])), "r"(__float_as_uint(f[3])), "r"(__float_as_uint(f[4])),
         "r"(__float_as_uint(f[5])), "r"(__float_as_uint(f[6])), "r"(__float_as_uint(f[7])),
         "r"(__float_as_uint(f[8])), "r"(__float_as_uint(f[9])), "r"(__float_as_uint(f[10])),
         "r"(__float_as_uint(f[11])), "r"(__float_as_uint(f[12])), "r"(__float_as_uint(f[13])),
         "r"(__float_as_uint(f[14])), "r"(__float_as_uint(f[15]))
      : "memory");
}

// 32 consecutive FP32 columns of this thread's TMEM lane (warp-collective).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* f) {
  uint32_t v[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]),
        "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]),
        "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) f[i] = __uint_as_float(v[i]);
}

__device__ __forceinline__ float bfr(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }
__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}
// acc (8 FP32 values as four f32x2 pairs) += relu(p + q) for 8 BF16 pairs: the sum and the
// relu in one packed BF16 FMA (one rounding), the accumulation in FP32.
__device__ __forceinline__ void relu_acc8(const uint4 p, const uint4 q, unsigned long long acc[4]) {
  const uint32_t pw[4] = {p.x, p.y, p.z, p.w}, qw[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    uint32_t d;
    asm("fma.rn.relu.bf16x2 %0, %1, %2, %3;" : "=r"(d) : "r"(pw[i]), "r"(0x3F803F80u), "r"(qw[i]));
    unsigned long long x;
    asm("mov.b64 %0, {%1, %2};" : "=l"(x) : "r"(d << 16), "r"(d & 0xffff0000u));
    asm("add.rn.f32x2 %0, %0, %1;" : "+l"(acc[i]) : "l"(x));
  }
}
__device__ __forceinline__ void unpack_acc8(const unsigned long long acc[4], float s[8]) {
#pragma unroll
  for (int i = 0; i < 4; ++i) asm("mov.b64 {%0, %1}, %2;" : "=f"(s[2 * i]), "=f"(s[2 * i + 1]) : "l"(acc[i]));
}

// BF16 node rows [rows][32]: the 16-byte chunk b of row r sits at chunk b ^ ((r >> 1) & 3),
// so 32 lanes writing one row each (the epilogue) spread over all banks.
__device__ __forceinline__ uint4* row_chunk(unsigned char* base, int r, int b) {
  return reinterpret_cast<uint4*>(base + (size_t)r * 64 + ((b ^ ((r >> 1) & 3)) << 4));
}

// Chunk b of the row an edge entry x = row * 64 | ((row >> 1) & 3) points at (row_chunk).
__device__ __forceinline__ uint4 edge_chunk(const unsigned char* base, uint32_t x, int b) {
  return *reinterpret_cast<const uint4*>(base + (x & ~63u) + ((((uint32_t)b ^ x) & 3u) << 4));
}

// P0 row v (64 FP32) as 16 chunks of 4: chunk c at position (c + v) mod 16, so that 32 lanes
// reading chunk c of consecutive rows spread over all banks.
__host__ __device__ __forceinline__ int p0_index(int v, int o) {
  return v * 64 + ((((o >> 2) + v) & 15) << 2) + (o & 3);
}

// Epilogue / init of one half (32 columns: hf = 0 the first projection, 1 the second) of a
// 32-row chunk of a tile: rows r0 .. r0+31 (this lane: group row r = r0 + lane, node l of
// its shot, l < 0 for a padding row), TMEM address taddr of the chunk's column 0.  mode 0:
// init from the tables (variables: P0, rows of p0_index; checks: Pc0[sigma]) with tcgen05.st; mode 1:
// read the accumulators and add `nb` deg k.  Writes the BF16 row half to dst (lo for hf = 0,
// hi for hf = 1).
__device__ __forceinline__ void tc_half(uint32_t taddr, int hf, int r, int l, int n, bool check,
                                        int mode, float nb, const float* p0, const float* pc0,
                                        const float* k, const float* deg, const float* sig,
                                        unsigned char* dst) {
  const bool ok = l >= 0;
  float f[32];
  if (mode == 0) {
    // initial values: checks one of the two rows of Pc0, variables row l of P0
    if (check) {
      const float* src = pc0 + (ok && sig[r] < 0.f ? 64 : 0) + hf * 32;
#pragma unroll
      for (int i = 0; i < 32; ++i) f[i] = src[i];
    } else {
      const int v = ok ? l : 0;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const float4 x = *reinterpret_cast<const float4*>(p0 + p0_index(v, 32 * hf + 4 * q));
        f[4 * q] = x.x;
        f[4 * q + 1] = x.y;
        f[4 * q + 2] = x.z;
        f[4 * q + 3] = x.w;
      }
    }
    tmem_st16(taddr + hf * 32, f);
    tmem_st16(taddr + hf * 32 + 16, f + 16);
  } else {
    tmem_ld32(taddr + hf * 32, f);
    const float dk = ok ? nb * deg[l] : 0.f;
#pragma unroll
    for (int i = 0; i < 32; ++i) f[i] = fmaf(dk, k[hf * 32 + i], f[i]);
  }
  if (ok) {
#pragma unroll
    for (int b = 0; b < 4; ++b)
      *row_chunk(dst, r, b) = make_uint4(pack2(f[8 * b], f[8 * b + 1]), pack2(f[8 * b + 2], f[8 * b + 3]),
                                         pack2(f[8 * b + 4], f[8 * b + 5]), pack2(f[8 * b + 6], f[8 * b + 7]));
  }
}

__global__ void __launch_bounds__(kTcMaxWarps * 32, 1) prior_tc_kernel(TcArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int m = a.m, n = a.n, R = a.rounds, vt = a.vt, ct = a.ct;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, T = blockDim.x;
  const int W = T >> 5;
  const TcLay L = tc_layout(m, n, a.E, vt, ct, a.S);
  const int S = a.S, n8 = a.n8, m8 = a.m8, NR = S * n8, MR = S * m8;  // group rows
  unsigned char* mv = smem + L.mv;
  unsigned char* mc = smem + L.mc;
  unsigned char* op = smem + L.op;
  unsigned char* as = smem + L.as;
  unsigned char* ds = smem + L.ds;
  unsigned char* cs = smem + L.cs;
  unsigned char* bs = smem + L.bs;
  float* p0 = reinterpret_cast<float*>(smem + L.p0);
  float* pc0 = reinterpret_cast<float*>(smem + L.pc0);
  float* kv = reinterpret_cast<float*>(smem + L.kv);
  float* kc = reinterpret_cast<float*>(smem + L.kc);
  float* u = reinterpret_cast<float*>(smem + L.u);
  float* y0 = reinterpret_cast<float*>(smem + L.y0);
  float* llr = reinterpret_cast<float*>(smem + L.llr);
  float* degv = reinterpret_cast<float*>(smem + L.degv);
  float* degc = reinterpret_cast<float*>(smem + L.degc);
  float* sig = reinterpret_cast<float*>(smem + L.sig);
  int* vptr = reinterpret_cast<int*>(smem + L.vptr);
  int* cptr = reinterpret_cast<int*>(smem + L.cptr);
  uint32_t* vadj = reinterpret_cast<uint32_t*>(smem + L.vadj);
  uint32_t* cadj = reinterpret_cast<uint32_t*>(smem + L.cadj);
  float* kappa = reinterpret_cast<float*>(smem + L.misc);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + L.misc + 8);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + L.misc + 16);
  const float* P = a.params;

  // ---- tables: Mv, Mc (BF16 operands), kv, kc, P0, Pc0, y0, u, kappa, degrees ----
  // staging: BF16-rounded Wv and Wc (FP32) in the operand buffer, h_v^0 over cs / bs
  float* swv = reinterpret_cast<float*>(op);
  float* swc = swv + 64 * HD;
  float* h0 = reinterpret_cast<float*>(cs);
  for (int i = tid; i < 64 * HD; i += T) {
    const int o = i >> 5, j = i & 31;
    swv[i] = bfr(o < HD ? __ldg(P + POff::W1vc + o * DIN + j) : __ldg(P + POff::W1cv + (o - HD) * DIN + HD + j));
    swc[i] = bfr(o < HD ? __ldg(P + POff::W1cv + o * DIN + j) : __ldg(P + POff::W1vc + (o - HD) * DIN + HD + j));
  }
  for (int i = tid; i < n * HD; i += T) {
    const int v = i >> 5, j = i & 31;
    h0[i] = fmaxf(fmaf(__ldg(a.prior + v), __ldg(P + POff::a0 + j), __ldg(P + POff::a1 + j)), 0.f);
  }
  __syncthreads();
  for (int i = tid; i < 2 * 64 * HD; i += T) {
    const bool chk = i >= 64 * HD;
    const int o = (i >> 5) & 63, kk = i & 31;
    const float* w = (chk ? swc : swv) + o * HD;
    const float* w2 = P + (chk ? POff::W2vc : POff::W2cv) + kk;
    float acc = 0.f;
#pragma unroll 1
    for (int j = 0; j < HD; ++j) acc = fmaf(w[j], bfr(__ldg(w2 + j * HD)), acc);
    *reinterpret_cast<__nv_bfloat16*>((chk ? mc : mv) + koff(o, kk)) = __float2bfloat16_rn(acc);
  }
  for (int o = tid; o < 64; o += T) {
    float a1 = 0.f, a2 = 0.f, sp = 0.f, sm = 0.f;
#pragma unroll 1
    for (int j = 0; j < HD; ++j) {
      const float v = swv[o * HD + j], c = swc[o * HD + j];
      a1 = fmaf(v, __ldg(P + POff::b2cv + j), a1);
      a2 = fmaf(c, __ldg(P + POff::b2vc + j), a2);
      const float u0 = __ldg(P + POff::u0 + j), u1 = __ldg(P + POff::u1 + j);
      sp = fmaf(c, u1 + u0, sp);  // h_c^0 = sigma u0 + u1, sigma = +1
      sm = fmaf(c, u1 - u0, sm);  //                        sigma = -1
    }
    kv[o] = a1;
    kc[o] = a2;
    const float ws = bfr(o < HD ? __ldg(P + POff::W1cv + o * DIN + 2 * HD)
                                : __ldg(P + POff::W1vc + (o - HD) * DIN + 2 * HD));
    const float b1 = o < HD ? __ldg(P + POff::b1cv + o) : __ldg(P + POff::b1vc + o - HD);
    pc0[o] = sp + ws + b1;
    pc0[64 + o] = sm - ws + b1;
  }
  for (int kk = tid; kk < HD; kk += T) {
    float acc = 0.f;
#pragma unroll 1
    for (int o = 0; o < HD; ++o)
      acc = fmaf(bfr(__ldg(P + POff::W2cv + o * HD + kk)), __ldg(P + POff::wo + o), acc);
    u[kk] = acc;
  }
  if (tid == 0) {
    float acc = 0.f;
#pragma unroll 1
    for (int o = 0; o < HD; ++o) acc = fmaf(__ldg(P + POff::wo + o), __ldg(P + POff::b2cv + o), acc);
    *kappa = acc;
  }
  for (int v = tid; v < n; v += T) {  // column-major [64][n]: a thread per variable
    float h[HD];
#pragma unroll
    for (int j = 0; j < HD; ++j) h[j] = h0[v * HD + ((j + v) & (HD - 1))];  // rotated: no conflicts
#pragma unroll 1
    for (int o = 0; o < 64; ++o) {
      float acc = 0.f;
#pragma unroll
      for (int j = 0; j < HD; ++j) acc = fmaf(swv[o * HD + ((j + v) & (HD - 1))], h[j], acc);
      p0[p0_index(v, o)] = acc;
    }
  }
  for (int v = tid; v < n; v += T) {
    float acc = __ldg(a.prior + v) + __ldg(P + POff::bo);
#pragma unroll 1
    for (int j = 0; j < HD; ++j) acc = fmaf(__ldg(P + POff::wo + j), h0[v * HD + j], acc);
    y0[v] = acc;
    degv[v] = (float)(__ldg(a.var_ptr + v + 1) - __ldg(a.var_ptr + v));
  }
  for (int c = tid; c < m; c += T) degc[c] = (float)(__ldg(a.chk_ptr + c + 1) - __ldg(a.chk_ptr + c));
  for (int v = tid; v <= n; v += T) vptr[v] = __ldg(a.var_ptr + v);
  for (int c = tid; c <= m; c += T) cptr[c] = __ldg(a.chk_ptr + c);
  for (int e = tid; e < a.E; e += T) {
    const uint32_t c = __ldg(a.var_chk + e), v = __ldg(a.chk_var + e);
    vadj[e] = (c << 6) | ((c >> 1) & 3u);
    cadj[e] = (v << 6) | ((v >> 1) & 3u);
  }
  __syncthreads();
  {  // the staging is done: operand rows past the last node stay zero (finite)
    const int words = (int)((L.as - L.op) / 16);
    for (int i = tid; i < words; i += T) reinterpret_cast<uint4*>(op)[i] = make_uint4(0, 0, 0, 0);
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_u32(tmem_slot)), "r"(a.tmem_cols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(mbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tbase = *tmem_slot;
  const float kap = *kappa;
  uint32_t phase = 0;
  bool failed = false;

  // warp w serves TMEM lane quarter w % 4; half hf of chunk (tile i, quarter q) goes to warp
  // q + 4 ((2 i + hf + rot) % nq), nq = the number of warps on quarter q
  const int q = warp & 3;
  const int nq = (W - q + 3) >> 2;
  const int wslot = warp >> 2;
  auto chunks = [&](int tiles, int col0, int rot, bool check, int mode, float nb,
                    unsigned char* lo, unsigned char* hi) {
    const int rows = check ? MR : NR, r8 = check ? m8 : n8, nn = check ? m : n;
    const uint32_t inv = check ? a.inv_m8 : a.inv_n8;
    for (int i = 0; i < tiles; ++i) {
      if (i * 128 + q * 32 >= rows) continue;
      const uint32_t taddr = tbase + ((uint32_t)(q * 32) << 16) + (uint32_t)(col0 + 64 * i);
      const int r = i * 128 + q * 32 + lane;
      int l = -1;
      if (r < rows) {
        l = r - (int)__umulhi((uint32_t)r, inv) * r8;
        if (l >= nn) l = -1;
      }
      for (int hf = 0; hf < 2; ++hf) {
        if ((2 * i + hf + rot) % nq != wslot) continue;
        tc_half(taddr, hf, r, l, n, check, mode, nb, p0, pc0, check ? kc : kv,
                check ? degc : degv, sig, hf ? hi : lo);
      }
    }
  };
  // the MMA of `tiles` tiles: accumulators at column col0 + 64 i, operand tile i, weights w.
  // The issuing thread alone waits for completion; the others wait at the barrier.
  auto mma_tiles = [&](int tiles, int col0, const unsigned char* w) -> bool {
    int ok = 1;
    if (tid == 0) {
      fence_after();
      for (int i = 0; i < tiles; ++i)
        for (int j = 0; j < 2; ++j)
          mma_bf16(tbase + (uint32_t)(col0 + 64 * i), umma_desc(smem_u32(op + 8192 * i + 256 * j)),
                   umma_desc(smem_u32(w + 256 * j)));
      mma_commit(mbar);
      ok = mbar_wait(mbar, phase) ? 1 : 0;
    }
    phase ^= 1u;
    ok = __syncthreads_and(ok);
    fence_after();
    return ok != 0;
  };

  __shared__ int s_bad[kTcMaxGroup];
  __shared__ unsigned long long s_slot[kTcMaxGroup];
  for (long long shot0 = (long long)blockIdx.x * S; shot0 < a.shots && !failed;
       shot0 += (long long)gridDim.x * S) {
    const int ns = (int)min((long long)S, a.shots - shot0);  // shots of this group
    // rows of a shot past the batch, and padding rows, read an all-zero syndrome
    for (int rr = tid; rr < MR; rr += T) {
      const int s = (int)__umulhi((uint32_t)rr, a.inv_m8), c = rr - s * m8;
      sig[rr] = (s < ns && c < m && a.syndromes[(shot0 + s) * m + c]) ? -1.f : 1.f;
    }
    for (int rr = tid; rr < NR; rr += T) {
      const int v = rr - (int)__umulhi((uint32_t)rr, a.inv_n8) * n8;
      llr[rr] = v < n ? y0[v] : 0.f;
    }
    if (tid < kTcMaxGroup) s_bad[tid] = 0;
    __syncthreads();
    // initial accumulators and the round-0 gather sources
    chunks(vt, 0, 0, false, 0, 0.f, cs, bs);
    chunks(ct, 64 * vt, 1, true, 0, 0.f, as, ds);
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    fence_before();
    __syncthreads();
    for (int t = 0; t < R; ++t) {
      const bool last = t == R - 1;
      // ---- X2: S_v = sum_c relu(A_c + B_v), 2 threads per row (16 features each), and the
      // LLR update ----
      for (int base = warp * 32; base < 2 * NR; base += T) {
        const int task = base + lane, r = task >> 1, h = task & 1;
        const int sh = (int)__umulhi((uint32_t)r, a.inv_n8), v = r - sh * n8;
        const bool live = task < 2 * NR && v < n;
        float s[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) s[k] = 0.f;
        if (live) {
          const uint4 q0 = *row_chunk(bs, r, 2 * h), q1 = *row_chunk(bs, r, 2 * h + 1);
          unsigned long long acc0[4] = {0ull, 0ull, 0ull, 0ull}, acc1[4] = {0ull, 0ull, 0ull, 0ull};
          const uint32_t xo = (uint32_t)(sh * m8) << 6;  // the shot's check rows
          const int e1 = vptr[v + 1];
          for (int e = vptr[v]; e < e1; ++e) {
            const uint32_t x = vadj[e] + xo;
            relu_acc8(edge_chunk(as, x, 2 * h), q0, acc0);
            relu_acc8(edge_chunk(as, x, 2 * h + 1), q1, acc1);
          }
          unpack_acc8(acc0, s);
          unpack_acc8(acc1, s + 8);
        }
        if (!last && task < 2 * NR) {  // padding rows of the operand are zero
          *reinterpret_cast<uint4*>(op + koff(r, 16 * h)) =
              make_uint4(pack2(s[0], s[1]), pack2(s[2], s[3]), pack2(s[4], s[5]), pack2(s[6], s[7]));
          *reinterpret_cast<uint4*>(op + koff(r, 16 * h + 8)) =
              make_uint4(pack2(s[8], s[9]), pack2(s[10], s[11]), pack2(s[12], s[13]), pack2(s[14], s[15]));
        }
        float dot = 0.f;
#pragma unroll
        for (int k = 0; k < 16; ++k) dot = fmaf(u[16 * h + k], s[k], dot);
        dot += __shfl_xor_sync(0xffffffffu, dot, 1);
        if (live && h == 0) llr[r] += dot + degv[v] * kap;
      }
      if (last) break;
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      if (!mma_tiles(vt, 0, mv)) {
        failed = true;
        break;
      }
      chunks(vt, 0, 0, false, 1, (float)(t + 1), cs, bs);
      fence_before();
      __syncthreads();
      // ---- X1: T_c = sum_v relu(C_v + D_c) ----
      for (int task = tid; task < 4 * MR; task += T) {
        const int r = task >> 2, b = task & 3;
        const int sh = (int)__umulhi((uint32_t)r, a.inv_m8), c = r - sh * m8;
        float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (c < m) {
          const uint4 qd = *row_chunk(ds, r, b);
          unsigned long long acc[4] = {0ull, 0ull, 0ull, 0ull};
          const uint32_t xo = (uint32_t)(sh * n8) << 6;  // the shot's variable rows
          const int e1 = cptr[c + 1];
          for (int e = cptr[c]; e < e1; ++e) relu_acc8(edge_chunk(cs, cadj[e] + xo, b), qd, acc);
          unpack_acc8(acc, s);
        }
        *reinterpret_cast<uint4*>(op + koff(r, 8 * b)) =
            make_uint4(pack2(s[0], s[1]), pack2(s[2], s[3]), pack2(s[4], s[5]), pack2(s[6], s[7]));
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      if (!mma_tiles(ct, 64 * vt, mc)) {
        failed = true;
        break;
      }
      chunks(ct, 64 * vt, 1, true, 1, (float)(t + 1), as, ds);
      fence_before();
      __syncthreads();
    }
    if (failed) break;
    __syncthreads();
    if (a.llr_out) {
      for (int rr = tid; rr < NR; rr += T) {
        const int s = (int)__umulhi((uint32_t)rr, a.inv_n8), v = rr - s * n8;
        if (s < ns && v < n) a.llr_out[(shot0 + s) * n + v] = llr[rr];
      }
      __syncthreads();
      continue;
    }
    // ---- decode mode: per shot, the hard decision of the LLRs, or the shot is queued for
    // LSD ----
    for (int rr = tid; rr < MR; rr += T) {
      const int s = (int)__umulhi((uint32_t)rr, a.inv_m8), c = rr - s * m8;
      if (s >= ns || c >= m) continue;
      unsigned par = sig[rr] < 0.f ? 1u : 0u;
      const float* ls = llr + s * n8;
      const int e1 = cptr[c + 1];
      for (int e = cptr[c]; e < e1; ++e) par ^= ls[cadj[e] >> 6] < 0.f;
      if (par) s_bad[s] = 1;
    }
    __syncthreads();
    if (tid < ns) {
      const long long shot = shot0 + tid;
      if (s_bad[tid]) {
        s_slot[tid] = atomicAdd(&a.ctr->lsd_count, 1ULL);
        a.queue[s_slot[tid]] = (int32_t)shot;
      } else {
        if (a.status) a.status[shot] = LSD_SHOT_OK_BP;
        atomicAdd(&a.ctr->bp_converged, 1ULL);
      }
    }
    __syncthreads();
    for (int rr = tid; rr < NR; rr += T) {
      const int s = (int)__umulhi((uint32_t)rr, a.inv_n8), v = rr - s * n8;
      if (s >= ns || v >= n) continue;
      if (s_bad[s])
        a.queue_llr[(long long)s_slot[s] * n + v] = llr[rr];
      else
        a.corrections[(shot0 + s) * n + v] = llr[rr] < 0.f ? 1 : 0;
    }
    __syncthreads();
  }
  if (failed) {
    // the MMA that did not report is given one more bounded wait before TMEM is released
    mbar_wait(mbar, phase ^ 1u);
    if (tid == 0 && a.timeout_flag) atomicExch(a.timeout_flag, 1);
  }
  fence_before();
  __syncthreads();
  if (warp == 0) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                 :: "r"(tbase), "r"(a.tmem_cols) : "memory");
  }
}

struct TcShape {
  int vt, ct, cols, threads, S;
  size_t smem;
};

// The launch shape for H (m x n with maximal degrees dv, dc), or false when the graph does
// not fit: a group of S shots in at most 8 tiles of 128 rows, the tables in shared memory.
// S is the group that keeps the most shots per SM in flight (TMEM holds 512 / cols CTAs).
bool tc_shape(int m, int n, int E, int dv, int dc, int max_smem, TcShape* s) {
  if (n >= 65535 || m >= 65535) return false;
  int best_inflight = 0;
  for (int S = 1; S <= kTcMaxGroup; ++S) {
    const int vt = (S * up8(n) + 127) / 128, ct = (S * up8(m) + 127) / 128;
    if (vt + ct > kTcMaxTiles) break;
    int cols = 32;
    while (cols < 64 * (vt + ct)) cols <<= 1;
    size_t smem = tc_layout(m, n, E, vt, ct, S).total;
    // at most as many CTAs per SM as TMEM holds: pad shared memory so no more fit
    const int per_sm = 512 / cols;
    const size_t floor_smem = (size_t)(228 * 1024) / (size_t)(per_sm + 1) + 1024;
    if (smem < floor_smem) smem = floor_smem;
    if (smem > (size_t)max_smem) continue;
    if (S * per_sm > best_inflight) {
      best_inflight = S * per_sm;
      s->S = S;
      s->vt = vt;
      s->ct = ct;
      s->cols = cols;
      s->smem = smem;
    }
  }
  if (best_inflight == 0) return false;
  // warps: the count that leaves the fewest idle task slots in the two gathers, the most
  // warps among equals (with one CTA per SM up to 20 warps, else up to 10 so that the CTAs
  // TMEM admits also fit in registers)
  const int NR = s->S * up8(n), MR = s->S * up8(m);
  const int max_w = s->cols == 512 ? kTcMaxWarps : 10;
  double best = -1.0;
  for (int w = kTcMinWarps; w <= max_w; ++w) {
    const int T = 32 * w;
    // X2: 2 tasks per variable row, 16 features each; X1: 4 tasks per check row, 8 each
    const double pv = (double)((2 * NR + T - 1) / T) * T * 2 * dv, pc = (double)((4 * MR + T - 1) / T) * T * dc;
    const double eff = (4.0 * NR * dv + 4.0 * MR * dc) / (pv + pc);
    if (eff > best - 1e-9) {
      best = eff > best ? eff : best;
      s->threads = T;
    }
  }
  return true;
}

}  // namespace

cudaError_t prior_tc_config(const DevGraph& g, int* grid) {
  int dev = 0, sms = 0, max_smem = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  TcShape s;
  if (!tc_shape(g.m, g.n, g.E, g.max_col_deg, g.max_row_deg, max_smem, &s)) return cudaErrorInvalidValue;
  err = allow_max_dynamic_smem((const void*)prior_tc_kernel, max_smem);
  if (err == cudaSuccess)
    err = cudaFuncSetAttribute((const void*)prior_tc_kernel,
                               cudaFuncAttributePreferredSharedMemoryCarveout,
                               cudaSharedmemCarveoutMaxShared);
  if (err != cudaSuccess) return err;
  int per_sm = 0;
  err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, prior_tc_kernel, s.threads, s.smem);
  if (err != cudaSuccess) return err;
  // CTAs per SM from the kernel's own limits: registers (in 256-register warp units), shared
  // memory (with the per-CTA reservation) and threads
  cudaFuncAttributes fa{};
  int regs_sm = 0, smem_sm = 0, reserved = 0, threads_sm = 0;
  err = cudaFuncGetAttributes(&fa, (const void*)prior_tc_kernel);
  if (err == cudaSuccess) err = cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
  if (err == cudaSuccess) err = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  if (err == cudaSuccess) err = cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  if (err == cudaSuccess) err = cudaDeviceGetAttribute(&threads_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
  if (err != cudaSuccess) return err;
  const long warp_regs = ((long)fa.numRegs * 32 + 255) / 256 * 256;
  const long by_regs = regs_sm / (warp_regs * (s.threads / 32));
  const long by_smem = smem_sm / ((long)s.smem + fa.sharedSizeBytes + reserved);
  const long by_threads = threads_sm / s.threads;
  const long own = std::min(std::min(by_regs, by_smem), by_threads);
  if (own > per_sm) per_sm = (int)own;
  if (per_sm < 1) return cudaErrorInvalidValue;
  if (per_sm > 512 / s.cols) per_sm = 512 / s.cols;  // TMEM: 512 columns per SM
  *grid = per_sm * sms;
  return cudaSuccess;
}

cudaError_t launch_prior_tc(int grid, const DevGraph& g, int rounds, const float* params,
                            long long shots, const uint8_t* syndromes, float* llr_out,
                            uint8_t* corrections, uint8_t* status, int32_t* queue,
                            float* queue_llr, DevCounters* ctr, int* timeout_flag,
                            cudaStream_t st) {
  if (!llr_out && (!corrections || !queue || !queue_llr || !ctr)) return cudaErrorInvalidValue;
  int dev = 0, max_smem = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  TcShape s;
  if (!tc_shape(g.m, g.n, g.E, g.max_col_deg, g.max_row_deg, max_smem, &s)) return cudaErrorInvalidValue;
  TcArgs a{};
  a.m = g.m;
  a.n = g.n;
  a.E = g.E;
  a.rounds = rounds;
  a.vt = s.vt;
  a.ct = s.ct;
  a.S = s.S;
  a.n8 = up8(g.n);
  a.m8 = up8(g.m);
  a.inv_n8 = (uint32_t)((0x100000000ull + a.n8 - 1) / a.n8);
  a.inv_m8 = (uint32_t)((0x100000000ull + a.m8 - 1) / a.m8);
  a.tmem_cols = s.cols;
  a.chk_ptr = g.chk_ptr;
  a.chk_var = g.chk_var;
  a.var_ptr = g.var_ptr;
  a.var_chk = g.var_chk;
  a.prior = g.prior;
  a.params = params;
  a.shots = shots;
  a.syndromes = syndromes;
  a.llr_out = llr_out;
  a.corrections = corrections;
  a.status = status;
  a.queue = queue;
  a.queue_llr = queue_llr;
  a.ctr = ctr;
  a.timeout_flag = timeout_flag;
  const long long groups = (shots + s.S - 1) / s.S;
  const long long blocks = groups < grid ? groups : grid;
  if (blocks <= 0) return cudaSuccess;
  prior_tc_kernel<<<(int)blocks, s.threads, s.smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace lsdgb
