"""Large check matrices on the GPU against the oracle: the CTA-per-shot BP and the sparse LSD
(state sized by what a shot touches), including its large-capacity spill instance."""
import numpy as np
import pytest
import torch

import oracle
from tests.gpu_cases import code, sample

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2406_18655_gb300 import build
    build.build()
    from paper_2406_18655_gb300 import lsd
    lsd.lib()
    return lsd


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def f64(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


@pytest.mark.parametrize("name,p,iters,order,shots", [
    ("st_bb144_d12", 0.01, 50, 0, 300), ("hgp", 0.02, 100, 0, 120), ("hgp", 0.02, 100, 10, 60),
    # percolating regime: a third of the shots reach LSD with clusters of hundreds to
    # thousands of columns (the global-memory spill instance)
    ("hgp", 0.05, 100, 0, 200), ("hgp", 0.05, 100, 10, 100)])
def test_large_decode_matches_oracle(L, name, p, iters, order, shots):
    h, probs, e, s = sample(name, p, shots, seed=31 + order)
    d = L.Decoder(h, probs, iters, order)
    corr, st, stats = d.decode(dev(s), want_stats=True)
    o = oracle.decode(h, f64(probs), s, iters, lsd_order=order, precision=1)
    assert np.array_equal(st.cpu().numpy(), o["status"])
    assert np.array_equal(corr.cpu().numpy(), o["corrections"])
    assert stats["lsd_shots"] == int((o["status"] != 1).sum())
    print(f"{name} p={p}: {stats['lsd_shots']} LSD shots, kappa_max {stats['kappa_max']}, "
          f"spilled {stats['lsd_spilled']}")


@pytest.mark.parametrize("bp_kernel", [0, 1])
def test_large_bp_matches_oracle(L, bp_kernel):
    """HGP (3072 x 6400, rows of weight 7, columns of weight 3 and 4): the register-table CTA
    kernel (auto) and the CTA kernel that reads the graph through the cache (generic)."""
    h, probs, e, s = sample("hgp", 0.03, 40, seed=5)
    d = L.Decoder(h, probs, 40, bp_kernel=bp_kernel)
    post, conv, it = d.bp(dev(s))
    llr, hard, used, convo = oracle.bp(h, f64(probs), s, 40, precision=1)
    assert np.array_equal(it.cpu().numpy(), used)
    assert np.array_equal(post.cpu().numpy().astype(np.float64), llr)


def test_large_autotune_keeps_results(L):
    """Every BP variant the autotuner times on HGP gives the same decode."""
    h, probs, e, s = sample("hgp", 0.04, 300, seed=6)
    d = L.Decoder(h, probs, 100)
    c0, s0 = d.decode(dev(s))
    rep = d.autotune(dev(s))
    assert rep["bp_candidates"] >= 3
    c1, s1 = d.decode(dev(s))
    assert torch.equal(c0, c1) and torch.equal(s0, s1)
    o = oracle.decode(h, f64(probs), s, 100, precision=1)
    assert np.array_equal(c1.cpu().numpy(), o["corrections"])
    print("hgp autotune:", rep)


@pytest.mark.parametrize("order", [0, 6])
def test_sparse_equals_dense(L, order):
    h, probs, e, s = sample("bb144", 0.07, 3000, seed=17 + order)
    llr, *_ = oracle.bp(h, f64(probs), s, 30, precision=1)
    llr = dev(llr.astype(np.float32))
    dd = L.Decoder(h, probs, 30, order, lsd_kernel=1)
    ds = L.Decoder(h, probs, 30, order, lsd_kernel=2)
    c1, s1, i1 = dd.postprocess(llr, dev(s))
    c2, s2, i2 = ds.postprocess(llr, dev(s))
    assert torch.equal(c1, c2) and torch.equal(s1, s2) and torch.equal(i1, i2)


def test_sparse_spill_instance_matches_oracle(L):
    """Shots whose clusters claim more rows than the shared-memory instance holds are decoded
    by the global-memory instance, with the same results."""
    h, probs, e, s = sample("st_bb144_d12", 0.035, 24, seed=8)
    d = L.Decoder(h, probs, 20)
    corr, st, stats = d.decode(dev(s), want_stats=True)
    assert stats["lsd_spilled"] > 0
    o = oracle.decode(h, f64(probs), s, 20, precision=1)
    assert np.array_equal(st.cpu().numpy(), o["status"])
    assert np.array_equal(corr.cpu().numpy(), o["corrections"])
