"""GPU path (through the C ABI) against the CPU oracle, element by element.

Bars (the oracle's FP32 mirror rounds every BP operation in the kernel's order):
  * BP posteriors: |dLLR| <= 1e-4 * max(1, |LLR|), and in practice bit-identical;
    iteration counts and convergence flags identical.
  * LSD given identical soft information: corrections, status, nu, kappa and step
    counts bit-exact.
  * End to end BP + LSD: corrections identical; logical error rates within 2 sigma.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2406_18655_gb300 import inputs as I
from tests.gpu_cases import code, logicals_hz, sample

pytestmark = pytest.mark.gpu

BP_TOL = 1e-4


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


def test_priors_bit_exact(L):
    p = np.array([0.5, 0.25, 0.1, 0.05, 0.01, 1e-3, 1e-5, 0.3, 0.45, 0.999], np.float32)
    h = np.eye(p.size, dtype=np.uint8)
    d = L.Decoder(h, p, 1)
    got = d.priors()
    exp = oracle.priors(f64(p), precision=1).astype(np.float32)
    assert np.array_equal(got, exp)


@pytest.mark.parametrize("kernel", [1, 0])
@pytest.mark.parametrize("lanes", [8, 16, 32])
@pytest.mark.parametrize("name,p,iters,shots", [
    ("bb72", 0.05, 30, 4000), ("bb144", 0.02, 50, 3000), ("bb144", 0.08, 50, 3000),
    ("bb288", 0.04, 50, 1500), ("st_bb72_d6", 0.01, 50, 1500), ("rep_boundary", 0.1, 20, 2000)])
def test_bp_matches_oracle(L, kernel, lanes, name, p, iters, shots):
    """kernel 1: generic (graph in shared memory); 0: automatic choice, which is the
    register-resident kernel for the regular BB codes whenever a shape with these lanes fits."""
    h, probs, e, s = sample(name, p, shots, seed=1000 + int(p * 1000) + lanes)
    d = L.Decoder(h, probs, iters, bp_lanes=lanes, bp_kernel=kernel)
    post, conv, it = d.bp(dev(s))
    torch.cuda.synchronize()
    llr, hard, used, convo = oracle.bp(h, f64(probs), s, iters, precision=1)
    assert np.array_equal(it.cpu().numpy(), used)
    assert np.array_equal(conv.cpu().numpy(), convo)
    g = post.cpu().numpy().astype(np.float64)
    rel = np.abs(g - llr) / np.maximum(1.0, np.abs(llr))
    assert rel.max() <= BP_TOL
    assert np.array_equal(g, llr)


def test_register_kernel_available_for_bb_codes(L):
    for name in ("bb72", "bb144", "bb288"):
        h, probs, e, s = sample(name, 0.05, 300, seed=2)
        d = L.Decoder(h, probs, 30, bp_kernel=2)
        post, conv, it = d.bp(dev(s))
        llr, hard, used, convo = oracle.bp(h, f64(probs), s, 30, precision=1)
        assert np.array_equal(post.cpu().numpy().astype(np.float64), llr)
    with pytest.raises(L.LsdError):  # columns of weight 4: no register shape
        L.Decoder(code("irreg_37x61"), np.full(61, 0.01, np.float32), 30, bp_kernel=2)


def _irregular_rows(name):
    """Check matrices whose rows have different degrees (space-time matrices, hook faults,
    a window with the noiseless last block, a degree-1 boundary check)."""
    from oracle import window as OW
    if name == "hooks_bb144_d6":
        return I.space_time_hooks(code("bb144"), 6, seed=6)[0]
    if name == "hooks_bb72_d3":
        return I.space_time_hooks(code("bb72"), 3, seed=3)[0]
    if name == "window_bb144_final":
        return OW.window_matrix(code("bb144"), 3, 4)
    return code(name)


@pytest.mark.parametrize("kernel", [2, 3])
@pytest.mark.parametrize("name,p,iters,shots", [
    ("st_bb72_d6", 0.01, 50, 3000), ("st_bb72_d6", 0.04, 30, 2000),
    ("st_bb144_d12", 0.004, 50, 1500), ("hooks_bb144_d6", 0.004, 50, 1500),
    ("hooks_bb72_d3", 0.02, 30, 2000), ("window_bb144_final", 0.01, 30, 2000),
    ("rep_boundary", 0.1, 20, 2000), ("st_bb288_d18", 0.004, 30, 300)])
def test_register_cta_kernel_on_irregular_rows(L, kernel, name, p, iters, shots):
    """One CTA per shot with register tables on rows of unequal degree (padded with a dummy
    column that takes part in no minimum and no parity): posteriors, iteration counts and
    convergence bit-exact, and the decode through the LSD queue equals the oracle's.
    kernel 2: the throughput shapes; 3: the latency shapes (the most threads per shot)."""
    h = _irregular_rows(name)
    assert h.sum(1).min() < h.sum(1).max()
    probs = np.full(h.shape[1], p, np.float32)
    e = I.sample_errors(1300 + shots, shots, probs.astype(np.float64))
    s = I.syndromes(h, e)
    d = L.Decoder(h, probs, iters, bp_kernel=kernel)
    post, conv, it = d.bp(dev(s))
    llr, hard, used, convo = oracle.bp(h, f64(probs), s, iters, precision=1)
    assert np.array_equal(it.cpu().numpy(), used)
    assert np.array_equal(conv.cpu().numpy(), convo)
    assert np.array_equal(post.cpu().numpy().astype(np.float64), llr)
    corr, st = d.decode(dev(s))
    o = oracle.decode(h, f64(probs), s, iters, precision=1)
    assert np.array_equal(st.cpu().numpy(), o["status"])
    assert np.array_equal(corr.cpu().numpy(), o["corrections"])


def test_bp_no_early_exit_and_zero_iterations(L):
    h, probs, e, s = sample("bb72", 0.04, 500, seed=5)
    d = L.Decoder(h, probs, 15, no_early_exit=True)
    post, conv, it = d.bp(dev(s))
    llr, hard, used, convo = oracle.bp(h, f64(probs), s, 15, early_exit=0, precision=1)
    assert np.all(it.cpu().numpy() == 15)
    assert np.array_equal(conv.cpu().numpy(), convo)
    assert np.array_equal(post.cpu().numpy().astype(np.float64), llr)
    d0 = L.Decoder(h, probs, 0)
    post0, conv0, it0 = d0.bp(dev(s))
    assert np.all(it0.cpu().numpy() == 0) and not conv0.cpu().numpy().any()
    assert np.array_equal(post0.cpu().numpy(), np.broadcast_to(d0.priors(), post0.shape))


def test_sum_product_exact_on_trees(L):
    """Sum-product (FP32 on the GPU) reproduces exact tree marginals within the BP tolerance."""
    for seed in range(6):
        h = I.random_tree_tanner(seed, 10 + seed)
        n = h.shape[1]
        g = I.Xoshiro256ss(1000 + seed, np.arange(n + h.shape[0], dtype=np.uint64))
        u = g.uniform()
        p = (0.02 + 0.43 * u[:n]).astype(np.float32)
        s = (u[n:] < 0.5).astype(np.uint8)[None]
        xs = ((np.arange(2 ** n)[:, None] >> np.arange(n)[None, :]) & 1)
        ok = np.all((xs @ h.T.astype(np.int64)) % 2 == s[0], axis=1)
        xs = xs[ok]
        pd = f64(p)
        w = np.exp(xs @ np.log(pd) + (1 - xs) @ np.log(1 - pd))
        exact = np.array([np.log(w[xs[:, j] == 0].sum() / w[xs[:, j] == 1].sum()) for j in range(n)])
        d = L.Decoder(h, p, 2 * n, bp_method=1, no_early_exit=True)
        post, conv, it = d.bp(dev(s))
        got = post.cpu().numpy()[0].astype(np.float64)
        assert (np.abs(got - exact) / np.maximum(1.0, np.abs(exact))).max() <= BP_TOL


def _rounded_llrs(shape, seed):
    g = I.Xoshiro256ss(seed, np.arange(int(np.prod(shape)), dtype=np.uint64))
    return np.round(g.uniform() * 5 - 0.5, 1).astype(np.float32).reshape(shape)


@pytest.mark.parametrize("name,p,order,single,soft", [
    ("bb72", 0.05, 0, False, "bp"), ("bb72", 0.1, 0, False, "ties"),
    ("bb144", 0.04, 0, False, "bp"), ("bb144", 0.1, 0, False, "bp"),
    ("bb144", 0.06, 0, False, "ties"), ("bb288", 0.05, 0, False, "bp"),
    ("st_bb72_d6", 0.02, 0, False, "bp"), ("rep_boundary", 0.15, 0, False, "ties"),
    ("bb72", 0.05, 0, True, "bp"), ("bb144", 0.05, 0, True, "ties"),
    ("bb72", 0.08, 6, False, "bp"), ("bb144", 0.06, 6, False, "bp"),
    ("bb144", 0.06, 10, False, "ties"), ("bb72", 0.05, 1, False, "bp"),
    ("ldpc_96x192", 0.06, 0, False, "bp"), ("ldpc_96x192", 0.06, 6, False, "ties"),
    ("ldpc_480x960", 0.04, 0, False, "bp"), ("ldpc_480x960", 0.04, 4, False, "bp")])
def test_lsd_bit_exact_given_identical_soft_information(L, name, p, order, single, soft):
    h, probs, e, s = sample(name, p, 1500, seed=77 + order + int(100 * p))
    if soft == "bp":
        llr, *_ = oracle.bp(h, f64(probs), s, 30, precision=1)
        llr = llr.astype(np.float32)
    else:
        llr = _rounded_llrs((s.shape[0], h.shape[1]), 5 + order)
    d = L.Decoder(h, probs, 30, order, single_cluster=single)
    corr, st, info = d.postprocess(dev(llr), dev(s))
    torch.cuda.synchronize()
    r = oracle.lsd(h, s, llr.astype(np.float64), order=order, probs=f64(probs),
                   single_cluster=single)
    assert np.array_equal(st.cpu().numpy(), r["status"])
    assert np.array_equal(corr.cpu().numpy(), r["corrections"])
    info = info.cpu().numpy()
    assert np.array_equal(info[:, 0], r["nu"])
    assert np.array_equal(info[:, 1], r["kappa"])
    assert np.array_equal(info[:, 2], r["steps"])


@pytest.mark.parametrize("name,p,order,w,soft,kernel", [
    ("bb72", 0.08, 2, 4, "bp", 1), ("bb144", 0.06, 6, 4, "bp", 1),
    ("bb144", 0.06, 3, 7, "ties", 1), ("bb144", 0.08, 29, 4, "bp", 1),
    ("bb144", 0.06, 6, 0, "bp", 1), ("bb144", 0.06, 58, 8, "ties", 1),
    ("bb144", 0.06, 6, 4, "bp", 2), ("bb144", 0.08, 29, 8, "ties", 2),
    ("ldpc_96x192", 0.06, 4, 4, "bp", 0), ("ldpc_480x960", 0.04, 14, 4, "bp", 0),
    ("ldpc_480x960", 0.04, 14, 4, "ties", 2)])
def test_lsd_osd_cs_bit_exact(L, name, p, order, w, soft, kernel):
    """LSD-mu with the combination sweep OSD-CS-w (App. D), dense and sparse LSD kernels,
    growth beyond OSD-E's order limit (29 and 58 steps = 10 % and 20 % of BB144's n)."""
    h, probs, e, s = sample(name, p, 1500, seed=501 + order + w)
    if soft == "bp":
        llr, *_ = oracle.bp(h, f64(probs), s, 30, precision=1)
        llr = llr.astype(np.float32)
    else:
        llr = _rounded_llrs((s.shape[0], h.shape[1]), 7 + order)
    d = L.Decoder(h, probs, 30, order, osd_cs=w, lsd_kernel=kernel)
    corr, st, info = d.postprocess(dev(llr), dev(s))
    torch.cuda.synchronize()
    r = oracle.lsd(h, s, llr.astype(np.float64), order=order, probs=f64(probs), osd_cs=w)
    assert np.array_equal(st.cpu().numpy(), r["status"])
    assert np.array_equal(corr.cpu().numpy(), r["corrections"])
    info = info.cpu().numpy()
    assert np.array_equal(info[:, 0], r["nu"])
    assert np.array_equal(info[:, 1], r["kappa"])


def test_decode_osd_cs_matches_oracle(L):
    h, probs, e, s = sample("bb144", 0.08, 4000, seed=909)
    d = L.Decoder(h, probs, 30, 14, osd_cs=4)
    corr, st, stats = d.decode(dev(s), want_stats=True)
    o = oracle.decode(h, f64(probs), s, 30, lsd_order=14, osd_cs=4, precision=1)
    assert np.array_equal(st.cpu().numpy(), o["status"])
    assert np.array_equal(corr.cpu().numpy(), o["corrections"])


@pytest.mark.parametrize("name,d,p,iters,order,osd_cs", [
    ("bb72", 3, 0.01, 30, 0, None), ("bb72", 3, 0.02, 30, 6, None),
    ("bb144", 3, 0.01, 50, 0, None), ("bb144", 6, 0.005, 50, 0, None),
    ("bb144", 6, 0.008, 30, 12, 4)])
def test_circuit_like_dem_with_non_uniform_priors(L, name, d, p, iters, order, osd_cs):
    """Space-time matrices with mid-round hook faults (weight-2 and weight-3 hyperedges
    across rounds) and seeded non-uniform priors, the shape of a circuit-level detector
    error model; BB144 over 6 rounds (504 x 2160) takes the sparse LSD kernel."""
    h0 = code(name)
    m0, n0 = h0.shape
    h, _ = I.space_time_hooks(h0, d, seed=d)
    probs = I.space_time_hooks_probs(n0, m0, d, p, seed=d + 1).astype(np.float32)
    e = I.sample_errors(83 + d, 3000, probs.astype(np.float64))
    s = I.syndromes(h, e)
    dec = L.Decoder(h, probs, iters, order, osd_cs=osd_cs)
    corr, st = dec.decode(dev(s))
    o = oracle.decode(h, f64(probs), s, iters, lsd_order=order, precision=1,
                      osd_cs=-1 if osd_cs is None else osd_cs)
    assert np.array_equal(st.cpu().numpy(), o["status"])
    assert np.array_equal(corr.cpu().numpy(), o["corrections"])
    assert (o["status"] == 2).sum() > 20


def test_single_cluster_equals_osd0(L):
    h, probs, e, s = sample("bb144", 0.05, 200, seed=9)
    llr, *_ = oracle.bp(h, f64(probs), s, 20, precision=1)
    llr = llr.astype(np.float32)
    d = L.Decoder(h, probs, 20, single_cluster=True)
    corr, st, info = d.postprocess(dev(llr), dev(s))
    corr = corr.cpu().numpy()
    for k in range(s.shape[0]):
        ok, out = oracle.osd0(h, s[k], llr[k].astype(np.float64))
        assert ok and np.array_equal(corr[k], out)


@pytest.mark.parametrize("name,p,iters,order", [
    ("bb72", 0.05, 30, 0), ("bb144", 0.05, 50, 0), ("bb144", 0.08, 50, 6),
    ("bb288", 0.06, 50, 0), ("st_bb72_d6", 0.02, 50, 0), ("ldpc_96x192", 0.05, 50, 0),
    ("ldpc_480x960", 0.07, 50, 0)])
def test_decode_matches_oracle(L, name, p, iters, order):
    h, probs, e, s = sample(name, p, 4000, seed=300 + iters + order)
    d = L.Decoder(h, probs, iters, order)
    corr, st, stats = d.decode(dev(s), want_stats=True)
    o = oracle.decode(h, f64(probs), s, iters, lsd_order=order, precision=1)
    corr = corr.cpu().numpy()
    st = st.cpu().numpy()
    assert np.array_equal(st, o["status"])
    assert np.array_equal(corr, o["corrections"])
    assert np.array_equal((corr.astype(np.int64) @ h.T) % 2, s)
    assert stats["bp_converged"] == int((o["status"] == 1).sum())
    assert stats["lsd_shots"] == int((o["status"] != 1).sum())
    assert stats["bp_iterations"] == int(o["bp_iters"].sum())
    assert stats["kappa_max"] == int(o["kappa"].max())


def test_logical_error_rate_within_two_sigma(L):
    name, p = "bb144", 0.06
    h, probs, e, s = sample(name, p, 20000, seed=4242)
    d = L.Decoder(h, probs, 50)
    corr, st = d.decode(dev(s))
    gpu_fail = oracle.logical_failures(logicals_hz(name), e ^ corr.cpu().numpy())
    o = oracle.decode(h, f64(probs), s, 50, precision=1)
    orc_fail = oracle.logical_failures(logicals_hz(name), e ^ o["corrections"])
    n = s.shape[0]
    pg, po = gpu_fail.mean(), orc_fail.mean()
    sigma = np.sqrt(max(po * (1 - po), 1.0 / n) / n)
    assert abs(pg - po) <= 2 * sigma
    assert np.array_equal(gpu_fail, orc_fail)


def test_edge_cases(L):
    h, probs, e, s = sample("bb72", 0.05, 64, seed=1)
    d = L.Decoder(h, probs, 30)
    # empty batch
    c0, st0 = d.decode(dev(np.zeros((0, h.shape[0]), np.uint8)))
    assert c0.shape == (0, h.shape[1])
    # zero syndromes: BP converges after one iteration with the zero correction
    z = np.zeros((5, h.shape[0]), np.uint8)
    cz, stz = d.decode(dev(z))
    assert not cz.cpu().numpy().any() and np.all(stz.cpu().numpy() == 1)
    post, conv, it = d.bp(dev(z))
    assert np.all(it.cpu().numpy() == 1)
    # a single shot
    c1, st1 = d.decode(dev(s[:1]))
    o = oracle.decode(h, f64(probs), s[:1], 30, precision=1)
    assert np.array_equal(c1.cpu().numpy(), o["corrections"])
    # unsolvable syndrome: duplicated rows, syndrome differs on them
    hu = np.array([[1, 1, 0, 0], [1, 1, 0, 0], [0, 1, 1, 0], [0, 0, 1, 1]], np.uint8)
    su = np.array([[1, 0, 0, 0]], np.uint8)
    du = L.Decoder(hu, np.full(4, 0.1, np.float32), 10)
    cu, stu = du.decode(dev(su))
    assert stu.cpu().numpy()[0] == L.SHOT_UNSOLVABLE and not cu.cpu().numpy().any()
    ro = oracle.lsd(hu, su, np.full((1, 4), 2.0), order=0)
    assert ro["status"][0] == 3
    # ragged: a batch that is not a multiple of anything
    h2, probs2, e2, s2 = sample("bb144", 0.05, 1237, seed=8)
    d2 = L.Decoder(h2, probs2, 50)
    c2, _ = d2.decode(dev(s2))
    o2 = oracle.decode(h2, f64(probs2), s2, 50, precision=1)
    assert np.array_equal(c2.cpu().numpy(), o2["corrections"])


def test_host_buffer_entry_point(L):
    h, probs, e, s = sample("bb144", 0.06, 3000, seed=12)
    d = L.Decoder(h, probs, 50)
    c_dev, st_dev = d.decode(dev(s))
    c_host, st_host = d.decode_host(np.ascontiguousarray(s))
    assert np.array_equal(c_host, c_dev.cpu().numpy())
    assert np.array_equal(st_host, st_dev.cpu().numpy())
    pinned = torch.from_numpy(s).pin_memory()
    out = torch.empty((s.shape[0], h.shape[1]), dtype=torch.uint8).pin_memory()
    stt = torch.empty(s.shape[0], dtype=torch.uint8).pin_memory()
    d.decode_host(pinned, out, stt)
    assert np.array_equal(out.numpy(), c_host)


def test_host_buffer_pipeline_matches_device_decode(L):
    """A batch large enough for the chunked copy/decode pipeline (ragged chunk sizes) gives
    the same corrections and statuses as one device-resident call."""
    h, probs, e, s = sample("bb144", 0.05, 300_001, seed=21)
    d = L.Decoder(h, probs, 50)
    c_dev, st_dev = d.decode(dev(s))
    pinned = torch.from_numpy(s).pin_memory()
    out = torch.empty((s.shape[0], h.shape[1]), dtype=torch.uint8).pin_memory()
    stt = torch.empty(s.shape[0], dtype=torch.uint8).pin_memory()
    for _ in range(2):  # the second call reuses the streams, events and staging buffers
        out.zero_()
        stt.zero_()
        d.decode_host(pinned, out, stt)
        assert torch.equal(out, c_dev.cpu()) and torch.equal(stt, st_dev.cpu())


def test_memory_budget_admission(L):
    h, probs, e, s = sample("bb144", 0.05, 10, seed=3)
    with pytest.raises(L.LsdError) as ei:
        L.Decoder(h, probs, 50, mem_budget=1024)
    assert ei.value.code == L.LSD_ERR_ADMISSION
    d = L.Decoder(h, probs, 50, mem_budget=2 << 20)
    with pytest.raises(L.LsdError) as ei:
        d.decode(dev(np.zeros((100000, h.shape[0]), np.uint8)))
    assert ei.value.code == L.LSD_ERR_ADMISSION


def test_full_size_bb144_million_shots(L):
    """The benchmark workload (BB144, p = 0.05, 10^6 shots, 50 iterations) in the
    benchmark's launch configuration: every correction satisfies H e = s, and a sample of
    shots matches the oracle exactly."""
    shots = 1_000_000
    h, probs, e, s = sample("bb144", 0.05, shots, seed=20240601)
    d = L.Decoder(h, probs, 50)
    sd = dev(s)
    corr, st, stats = d.decode(sd, want_stats=True)
    ht = torch.from_numpy(h.T.astype(np.float32)).cuda()
    syn = torch.remainder(corr.float() @ ht, 2).to(torch.uint8)
    assert torch.equal(syn, sd)
    assert stats["unsolvable"] == 0
    idx = np.sort(np.random.default_rng(0).choice(shots, 3000, replace=False))
    o = oracle.decode(h, f64(probs), s[idx], 50, precision=1)
    assert np.array_equal(corr.cpu().numpy()[idx], o["corrections"])
    assert np.array_equal(st.cpu().numpy()[idx], o["status"])


def test_autotune_keeps_results(L):
    h, probs, e, s = sample("bb144", 0.06, 20000, seed=77)
    d = L.Decoder(h, probs, 50)
    c0, s0 = d.decode(dev(s))
    rep = d.autotune(dev(s[:8000]))
    assert rep["bp_candidates"] >= 3 and rep["lsd_candidates"] >= 2
    assert rep["ms_bp_best"] <= rep["ms_bp_first"] + 1e-6
    c1, s1 = d.decode(dev(s))
    assert torch.equal(c0, c1) and torch.equal(s0, s1)


@pytest.mark.parametrize("name,p", [("window_bb144_final", 0.01), ("hooks_bb72_d3", 0.02)])
def test_autotune_on_irregular_rows_keeps_results(L, name, p):
    """On rows of unequal degree the autotuner times the generic kernels and every padded
    register-table shape that fits; whichever it keeps decodes as the oracle does."""
    h = _irregular_rows(name)
    probs = np.full(h.shape[1], p, np.float32)
    e = I.sample_errors(91, 6000, probs.astype(np.float64))
    s = I.syndromes(h, e)
    d = L.Decoder(h, probs, 30)
    rep = d.autotune(dev(s))
    assert rep["bp_candidates"] >= 4
    assert rep["ms_bp_best"] <= rep["ms_bp_first"] + 1e-6
    corr, st = d.decode(dev(s))
    o = oracle.decode(h, f64(probs), s, 30, precision=1)
    assert np.array_equal(st.cpu().numpy(), o["status"])
    assert np.array_equal(corr.cpu().numpy(), o["corrections"])
