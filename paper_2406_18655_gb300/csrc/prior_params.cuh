// Flat parameter layout of the learned prior (the C ABI's order, include/lsd.h), shared by the
// per-node mma.sync kernels (prior.cu) and the TMEM-resident inference kernel (prior_tc.cu).
#pragma once

namespace lsdgb {
namespace prior_params {

constexpr int HD = 32;          // hidden width
constexpr int DIN = 2 * HD + 1; // layer-1 input: two node states and the syndrome sign

// offsets of the flat parameter vector
struct POff {
  static constexpr int a0 = 0, a1 = 32, u0 = 64, u1 = 96;
  static constexpr int W1cv = 128, b1cv = W1cv + HD * DIN, W2cv = b1cv + HD, b2cv = W2cv + HD * HD;
  static constexpr int W1vc = b2cv + HD, b1vc = W1vc + HD * DIN, W2vc = b1vc + HD,
                       b2vc = W2vc + HD * HD;
  static constexpr int wo = b2vc + HD, bo = wo + HD, total = bo + 1;
};

}  // namespace prior_params
}  // namespace lsdgb
