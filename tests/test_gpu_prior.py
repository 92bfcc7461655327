"""Learned prior on the GPU against the CPU oracle (oracle/prior.py), and what training gains.

Tolerances.  The GPU runs the matrix products with BF16 operands (weights and activations,
unit roundoff u = 2^-9 ~ 2e-3) and FP32 accumulation; the test weights are already BF16
values, so only activations are rounded.  The LLR is lambda (exact) plus the 32-term output
product of FP32 states whose per-element rounding errors (each at most u relative, of
random sign) average out over the sums, so the LLR error stays well below u: the test allows
|dLLR| <= 2.5 u * max(1, |LLR|) = 5e-3 (measured: 3e-4).  The gradient is a sum of such
products over thousands of edges: the whole vector must agree within 1e-2 in L2 norm
(measured: 8e-4) and every parameter group within cosine 0.999.
"""
import numpy as np
import pytest
import torch

import oracle.prior as P
from paper_2406_18655_gb300 import inputs as I
from paper_2406_18655_gb300.learned import init_params
from tests.gpu_cases import logicals_hz, sample

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2406_18655_gb300 import build
    build.build()
    from paper_2406_18655_gb300 import lsd
    lsd.lib()
    return lsd


def bf16_weights(theta):
    """Parameters with the two weight matrices of each MLP rounded to BF16 (as on the GPU)."""
    p = P.unflatten(theta)
    for k in ("W1_cv", "W2_cv", "W1_vc", "W2_vc"):
        p[k] = torch.tensor(p[k]).to(torch.bfloat16).to(torch.float64).numpy()
    return P.flatten(p)


def params_case(seed):
    rng = np.random.default_rng(seed)
    pp = P.unflatten(init_params(seed))
    pp["w_o"] = rng.normal(0, 0.3, 32)
    pp["b_o"] = np.array([0.05])
    for d in ("cv", "vc"):
        pp["b1_" + d] = rng.normal(0, 0.1, 32)
        pp["b2_" + d] = rng.normal(0, 0.05, 32)
    return bf16_weights(P.flatten(pp))


def test_sampler_matches_host_generator(L):
    h, probs, _, _ = sample("bb144", 0.05, 1, seed=1)
    d = L.Decoder(h, probs, 10)
    e, s = d.sample(777, 3000, first_shot=12345)
    e_host = I.sample_errors(777, 3000, probs.astype(np.float64), first_shot=12345)
    assert np.array_equal(e.cpu().numpy(), e_host)
    assert np.array_equal(s.cpu().numpy(), I.syndromes(h, e_host))


@pytest.mark.parametrize("kernel", ["mma_sync", "tcgen05"])
@pytest.mark.parametrize("name,rounds", [("bb72", 4), ("bb144", 4), ("bb288", 4),
                                         ("irreg_37x61", 1), ("irreg_37x61", 3)])
def test_forward_matches_oracle(L, name, rounds, kernel):
    """Both inference kernels against the oracle's per-edge MLPs: the per-node mma.sync
    kernel (16-row tiles, ragged last tile) and the tcgen05 kernel (projections in tensor
    memory, 128-row tiles: BB[[288,12,18]] takes 3 variable and 2 check tiles), irregular
    degrees, 1 to 4 rounds."""
    h, probs, e, s = sample(name, 0.06, 64, seed=11)
    theta = params_case(3)
    d = L.Decoder(h, probs, 10)
    pr = L.Prior(d, rounds=rounds, params=theta.astype(np.float32))
    pr.set_kernel(kernel)
    llr = pr.forward(torch.from_numpy(s).cuda()).cpu().numpy().astype(np.float64)
    lam = np.log((1 - probs.astype(np.float64)) / probs.astype(np.float64))
    ref, _ = P.forward(P.Graph(h), theta.astype(np.float32).astype(np.float64), s, lam,
                       rounds=rounds)
    err = np.abs(llr - ref) / np.maximum(1.0, np.abs(ref))
    print(f"forward {kernel} {name} R={rounds}: max rel err {err.max():.3e}, mean {err.mean():.3e}")
    assert err.max() <= 5e-3


def test_tensor_memory_kernel_many_shots_per_cta(L):
    """20000 BB[[144,12,12]] shots (each CTA of the persistent grid takes tens of shots, so
    the tensor-memory state is reinitialised between shots): 64 shots spread over the batch
    against the oracle, and every shot against the mma.sync kernel."""
    h, probs, e, s = sample("bb144", 0.06, 20000, seed=13)
    theta = params_case(5)
    d = L.Decoder(h, probs, 10)
    pr = L.Prior(d, rounds=4, params=theta.astype(np.float32))
    sd = torch.from_numpy(s).cuda()
    pr.set_kernel("tcgen05")
    llr_tc = pr.forward(sd).cpu().numpy().astype(np.float64)
    pr.set_kernel("mma_sync")
    llr_ms = pr.forward(sd).cpu().numpy().astype(np.float64)
    pick = np.linspace(0, 19999, 64).astype(int)
    lam = np.log((1 - probs.astype(np.float64)) / probs.astype(np.float64))
    ref, _ = P.forward(P.Graph(h), theta.astype(np.float32).astype(np.float64), s[pick], lam)
    err = np.abs(llr_tc[pick] - ref) / np.maximum(1.0, np.abs(ref))
    both = np.abs(llr_tc - llr_ms) / np.maximum(1.0, np.abs(llr_ms))
    print(f"tcgen05 vs oracle max rel err {err.max():.3e}; vs mma.sync {both.max():.3e}")
    assert err.max() <= 5e-3
    assert both.max() <= 1e-2


def test_gradient_matches_oracle(L):
    h, probs, e, s = sample("bb144", 0.06, 48, seed=12)
    theta = params_case(4).astype(np.float32).astype(np.float64)
    d = L.Decoder(h, probs, 10)
    pr = L.Prior(d, rounds=4, params=theta.astype(np.float32))
    loss, g = pr.gradient(torch.from_numpy(s).cuda(), torch.from_numpy(e).cuda())
    lam = np.log((1 - probs.astype(np.float64)) / probs.astype(np.float64))
    ref_loss, ref_g, _ = P.loss_and_grad(h, theta, s, e, lam)
    g = g.astype(np.float64)
    rel = np.linalg.norm(g - ref_g) / np.linalg.norm(ref_g)
    cos = g @ ref_g / (np.linalg.norm(g) * np.linalg.norm(ref_g))
    print(f"loss gpu {loss:.6f} oracle {ref_loss:.6f}; grad rel L2 {rel:.3e}, cos {cos:.6f}")
    assert abs(loss - ref_loss) <= 0.01 * abs(ref_loss)
    assert rel <= 1e-2 and cos >= 0.9999
    # every parameter group carries gradient, and the groups agree in direction
    off = 0
    for name, shp in P.param_shapes():
        k = int(np.prod(shp))
        a, b = g[off:off + k], ref_g[off:off + k]
        if np.linalg.norm(b) > 1e-8:
            assert a @ b / (np.linalg.norm(a) * np.linalg.norm(b)) >= 0.999, name
        off += k


def test_training_gains_over_lsd_on_channel_priors(L):
    """Train on device-sampled pairs at p = 0.05, then compare logical error rates on held-out
    shots: LSD on the learned LLRs against LSD on the channel priors alone (BP with 0
    iterations) and against BP+LSD with as many message-passing rounds as the network has
    (BP with 4 iterations, the method without the network at the same budget)."""
    name, p = "bb144", 0.05
    h, probs, _, _ = sample(name, p, 1, seed=1)
    d = L.Decoder(h, probs, 50)
    pr = L.Prior(d, rounds=4, params=init_params(7))
    losses = []
    batch, steps = 2048, 1000  # about 2 M pairs
    for step in range(steps):
        e, s = d.sample(99, batch, first_shot=step * batch)
        lr = 3e-3 if step < 0.8 * steps else 1e-3
        losses.append(pr.train_step(s, e, lr, want_loss=(step % 100 == 0 or step == steps - 1)))
    losses = [x for x in losses if x is not None]
    print("training losses", [round(x, 5) for x in losses])
    assert losses[-1] < 0.9 * losses[0]
    # held-out evaluation shots (a different seed and range)
    _, _, e, s = sample(name, p, 20000, seed=424242)
    sd, ed = torch.from_numpy(s).cuda(), torch.from_numpy(e).cuda()
    corr_l, st_l = d.decode_learned(pr, sd)
    assert torch.equal(torch.remainder(corr_l.float() @ torch.from_numpy(h.T.astype(np.float32)).cuda(), 2).to(torch.uint8), sd)
    d0 = L.Decoder(h, probs, 0)
    corr_0, _ = d0.decode(sd)
    corr_bp, _ = d.decode(sd)
    from paper_2406_18655_gb300.evaluate import LogicalChecker
    chk = LogicalChecker(logicals_hz(name))
    ler_learned = chk.failures(ed, corr_l).float().mean().item()
    ler_prior = chk.failures(ed, corr_0).float().mean().item()
    ler_bp = chk.failures(ed, corr_bp).float().mean().item()
    d4 = L.Decoder(h, probs, 4)  # BP with as many message-passing rounds as the network
    corr_bp4, _ = d4.decode(sd)
    ler_bp4 = chk.failures(ed, corr_bp4).float().mean().item()
    print(f"LER learned+LSD {ler_learned:.4f}  LSD on channel priors {ler_prior:.4f}  "
          f"BP(4)+LSD {ler_bp4:.4f}  BP(50)+LSD {ler_bp:.4f}")
    sigma = np.sqrt(ler_prior * (1 - ler_prior) / 20000)
    assert ler_learned < ler_prior - 3 * sigma
    sigma4 = np.sqrt(ler_bp4 * (1 - ler_bp4) / 20000)
    assert ler_learned < ler_bp4 - 2 * sigma4
    # the same network through the other inference kernel: the two kernels differ only in
    # rounding, so their logical error rates on the same shots agree closely
    kernels = {"mma_sync": None, "tcgen05": None}
    for k in kernels:
        pr.set_kernel(k)
        c_k, _ = d.decode_learned(pr, sd)
        kernels[k] = chk.failures(ed, c_k).float().mean().item()
    print("LER by inference kernel", kernels)
    assert abs(kernels["mma_sync"] - kernels["tcgen05"]) <= 2e-3
