"""Serving runtime: continuous batching over several codes, on the GPU.

The phenomenological space-time matrices of the three BB codes (d = 6, 12, 18 rounds, with
one noiseless final round; p = q = 0.003) are served together.  Every shot's correction is
the same whether it is decoded alone, in a mix with the other codes, or by the decoder
directly (decoding is deterministic per shot, so the tolerance is bit-exact)."""
import numpy as np
import pytest
import torch

from paper_2406_18655_gb300 import inputs as I

pytestmark = pytest.mark.gpu

ROUNDS = {"bb72": 6, "bb144": 12, "bb288": 18}


@pytest.fixture(scope="module")
def L():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2406_18655_gb300 import build
    build.build()
    from paper_2406_18655_gb300 import lsd
    lsd.lib()
    return lsd


def st_code(name, p=0.003):
    hx = getattr(I, name)()[0]
    d = ROUNDS[name]
    h = I.space_time(hx, d)
    probs = I.space_time_probs(hx.shape[1], hx.shape[0], d, p, p).astype(np.float32)
    return h, probs


def pool(L, h, probs, shots, seed):
    dec = L.Decoder(h, probs, 1)
    e, s = dec.sample(seed, shots)
    return s.cpu().pin_memory()


@pytest.fixture(scope="module")
def setup(L):
    codes = [st_code(nm) for nm in ("bb72", "bb144", "bb288")]
    pools = [pool(L, h, p, 600, 40 + k) for k, (h, p) in enumerate(codes)]
    return codes, pools


def test_alone_equals_mixed_equals_direct(L, setup):
    codes, pools = setup
    srv = L.Server([(h, p, 50, 0) for h, p in codes], slots_per_code=3, max_batch=256,
                   max_wait_us=100)
    alone = []
    for c, (h, p) in enumerate(codes):
        out = torch.zeros((pools[c].shape[0], h.shape[1]), dtype=torch.uint8).pin_memory()
        st = torch.zeros(pools[c].shape[0], dtype=torch.uint8).pin_memory()
        for k in range(pools[c].shape[0]):
            srv.submit(c, pools[c][k], out[k], st[k])
        srv.wait_all()
        alone.append((out.clone(), st.clone()))
    # mixed: all codes interleaved, submitted back to back
    outs = [torch.zeros((pools[c].shape[0], h.shape[1]), dtype=torch.uint8).pin_memory()
            for c, (h, p) in enumerate(codes)]
    sts = [torch.zeros(pools[c].shape[0], dtype=torch.uint8).pin_memory() for c in range(3)]
    order = np.random.default_rng(0).permutation(
        [(c, k) for c in range(3) for k in range(pools[c].shape[0])])
    for c, k in order:
        srv.submit(int(c), pools[c][k], outs[c][k], sts[c][k])
    srv.wait_all()
    rep = srv.report()
    assert rep["completed"] == rep["submitted"]
    for c, (h, p) in enumerate(codes):
        assert torch.equal(outs[c], alone[c][0]), f"code {c}: mixed differs from alone"
        assert torch.equal(sts[c], alone[c][1])
        d = L.Decoder(h, p, 50)
        corr, st = d.decode(pools[c].cuda())
        assert torch.equal(corr.cpu(), outs[c]) and torch.equal(st.cpu(), sts[c])
        syn = (outs[c].numpy().astype(np.float32) @ h.T.astype(np.float32)).astype(np.int64) % 2
        assert np.array_equal(syn, pools[c].numpy())
    srv.close()


def test_graphs_equal_plain_launches(L, setup):
    """A slot's captured graph (device-side batch size) decodes exactly like plain launches,
    for every batch size from 1 to max_batch."""
    codes, pools = setup
    h, p = codes[1]
    res = []
    for graphs in (True, False):
        srv = L.Server([(h, p, 50, 0)], slots_per_code=2, max_batch=64, max_wait_us=30,
                       graphs=graphs)
        out = torch.zeros((pools[1].shape[0], h.shape[1]), dtype=torch.uint8).pin_memory()
        st = torch.zeros(pools[1].shape[0], dtype=torch.uint8).pin_memory()
        k = 0
        for b in [1, 2, 3, 7, 31, 64, 65, 100]:
            for j in range(k, min(k + b, pools[1].shape[0])):
                srv.submit(0, pools[1][j], out[j], st[j])
            k += b
            srv.wait_all()
        for j in range(k, pools[1].shape[0]):
            srv.submit(0, pools[1][j], out[j], st[j])
        srv.wait_all()
        assert srv.report()["completed"] == pools[1].shape[0]
        res.append((out, st))
        srv.close()
    assert torch.equal(res[0][0], res[1][0]) and torch.equal(res[0][1], res[1][1])
    assert (res[0][1] > 0).all()


@pytest.mark.parametrize("graphs", [True, False])
def test_rows_solved_by_bp_and_by_lsd_written_back(L, graphs):
    """At a noise level where many shots of a batch need LSD, the rows BP solves (written back
    before the batch's LSD) and the rows LSD solves (written back after it) both equal the
    direct decode, and every request is reported complete once."""
    h, p = st_code("bb144", p=0.008)
    syn = pool(L, h, p, 400, 77)
    srv = L.Server([(h, p, 30, 0)], slots_per_code=2, max_batch=64, max_wait_us=50,
                   graphs=graphs)
    out = torch.zeros((syn.shape[0], h.shape[1]), dtype=torch.uint8).pin_memory()
    st = torch.zeros(syn.shape[0], dtype=torch.uint8).pin_memory()
    for k in range(syn.shape[0]):
        srv.submit(0, syn[k], out[k], st[k])
    srv.wait_all()
    rep = srv.report()
    assert rep["completed"] == rep["submitted"] == syn.shape[0]
    srv.close()
    corr, st_d = L.Decoder(h, p, 30).decode(syn.cuda())
    assert torch.equal(corr.cpu(), out) and torch.equal(st_d.cpu(), st)
    assert (st == 1).sum() > 0 and (st == 2).sum() > 0, "both write-back phases exercised"


def test_admission_by_memory(L, setup):
    codes, pools = setup
    h, p = codes[1]
    per_shot = h.shape[0] + 2 * h.shape[1] + 2 + 4 * (h.shape[1] + 1)
    budget = 40 * per_shot
    srv = L.Server([(h, p, 50, 0)], slots_per_code=4, max_batch=512, max_wait_us=20,
                   mem_budget=budget)
    out = torch.zeros((pools[1].shape[0], h.shape[1]), dtype=torch.uint8).pin_memory()
    for k in range(pools[1].shape[0]):
        srv.submit(0, pools[1][k], out[k])
    srv.wait_all()
    rep = srv.report()
    assert rep["completed"] == pools[1].shape[0]
    assert 0 < rep["peak_inflight_bytes"] <= budget
    assert rep["mean_batch"] <= 40
    d = L.Decoder(h, p, 50)
    corr, _ = d.decode(pools[1].cuda())
    assert torch.equal(corr.cpu(), out)
    srv.close()


@pytest.mark.parametrize("graphs", [True, False])
def test_poisson_load(L, setup, graphs):
    codes, pools = setup
    srv = L.Server([(h, p, 50, 0) for h, p in codes], graphs=graphs)
    rep = srv.run_poisson(2e5, 0.2, [1, 1, 1], pools, seed=3)
    assert rep["completed"] == rep["generated"] > 0
    assert rep["p99_us"] >= rep["p50_us"] > 0
    print(f"poisson 2e5/s graphs={graphs}:", {k: round(v, 2) for k, v in rep.items()})
    srv.close()


def test_rejects_pageable_buffers(L, setup):
    codes, pools = setup
    srv = L.Server([(codes[0][0], codes[0][1], 50, 0)])
    pageable = torch.zeros(codes[0][0].shape[0], dtype=torch.uint8)
    with pytest.raises(L.LsdError):
        srv.submit(0, pageable)
    srv.close()


def _served_windows(L, srv, code, h, seqs, streams, d, mix_with=None):
    """Submits the block sequences `seqs` ([k][(d+1) m], k a multiple of `streams`) round by
    round, stream s playing sequences s, s + S, ...; returns the committed corrections
    [k][d (n+m)] and the largest window status per sequence, assembled from what each
    completing block's request received.  `mix_with` (a callable) is invoked between rounds
    to submit other requests."""
    m, n = h.shape
    F = n + m
    k = seqs.shape[0]
    corr = np.zeros((k, d * F), np.uint8)
    status = np.zeros(k, np.uint8)
    pending = []
    for rep in range(k // streams):
        for b in range(d + 1):
            for s in range(streams):
                j = rep * streams + s
                buf = torch.zeros(d * F, dtype=torch.uint8).pin_memory()
                st = torch.zeros(1, dtype=torch.uint8).pin_memory()
                blk = seqs[j, b * m:(b + 1) * m].contiguous()
                first, rounds = srv.submit_round(code, s, blk, buf, st)
                if rounds:
                    pending.append((j, first, rounds, buf, st))
            if mix_with is not None:
                mix_with()
        srv.wait_all()  # a stream's next sequence reuses its history once these are done
    for j, first, rounds, buf, st in pending:
        corr[j, first * F:(first + rounds) * F] = buf.numpy()[:rounds * F]
        status[j] = max(status[j], int(st[0]))
    return corr, status


@pytest.mark.parametrize("d,w,c", [(6, 3, 1), (7, 4, 2)])
def test_served_windows_match_window_oracle(L, d, w, c):
    """Streams of BB[[72,12,6]] syndrome rounds (p = q = 0.02) served round by round in (w, c)
    windows: the committed corrections and statuses equal the window oracle's and
    lsd_window_decode's, bit for bit, alone and mixed with whole-shot requests of other codes
    submitted between the rounds."""
    import oracle.window as OW
    hx = I.bb72()[0]
    m, n = hx.shape
    p = 0.02
    streams, k = 24, 48
    probs = I.space_time_probs(n, m, d, p, p).astype(np.float32)
    e = I.sample_errors(900 + d, k, probs.astype(np.float64))
    seqs = torch.from_numpy(I.syndromes(I.space_time(hx, d), e))
    wcode = dict(h=hx, p=p, q=p, rounds=d, window=w, commit=c, bp_iters=30, streams=streams)
    h_st, p_st = st_code("bb144")
    shot_pool = pool(L, h_st, p_st, 64, 77)
    srv = L.Server([(h_st, p_st, 50, 0)], slots_per_code=3, max_batch=64, window_codes=[wcode])
    alone = _served_windows(L, srv, 1, hx, seqs, streams, d)
    outs = torch.zeros((64, h_st.shape[1]), dtype=torch.uint8).pin_memory()
    sts = torch.zeros(64, dtype=torch.uint8).pin_memory()
    cursor = [0]

    def shots():  # 5 per round: (d + 1) * (k / streams) * 5 >= 64 shots in all
        for _ in range(5):
            j = cursor[0] % 64
            srv.submit(0, shot_pool[j], outs[j], sts[j])
            cursor[0] += 1

    mixed = _served_windows(L, srv, 1, hx, seqs, streams, d, mix_with=shots)
    srv.wait_all()
    assert cursor[0] >= 64
    np.testing.assert_array_equal(mixed[0], alone[0])
    np.testing.assert_array_equal(mixed[1], alone[1])
    o = OW.window_decode(hx, np.full(n, p, np.float32).astype(np.float64),
                         np.full(m, p, np.float32).astype(np.float64), d, seqs.numpy(),
                         w=w, c=c, bp_iters=30)
    np.testing.assert_array_equal(alone[0], o["corrections"])
    np.testing.assert_array_equal(alone[1], o["status"])
    wd = L.WindowDecoder(hx, np.full(n, p, np.float32), np.full(m, p, np.float32), d, w, c,
                         bp_iters=30)
    c2, s2 = wd.decode(seqs.cuda())
    np.testing.assert_array_equal(alone[0], c2.cpu().numpy())
    # the shot requests of the mix equal the direct decode
    dec = L.Decoder(h_st, p_st, 50)
    c3, s3 = dec.decode(shot_pool.cuda())
    assert torch.equal(outs, c3.cpu()) and torch.equal(sts, s3.cpu())
    rep = srv.code_report(1)
    assert rep["completed"] == rep["submitted"] > 0
    srv.close()


def test_served_windows_under_poisson_load(L):
    """The load generator drives window streams and shots together; every window job and
    shot completes, and per-code latency figures are reported."""
    hx = I.bb72()[0]
    m, n = hx.shape
    d, p = 6, 0.003
    probs = I.space_time_probs(n, m, d, p, p).astype(np.float32)
    e = I.sample_errors(31, 256, probs.astype(np.float64))
    seqs = torch.from_numpy(I.syndromes(I.space_time(hx, d), e))
    h_st, p_st = st_code("bb72")
    shot_pool = pool(L, h_st, p_st, 256, 78)
    srv = L.Server([(h_st, p_st, 30, 0)], window_codes=[dict(h=hx, p=p, q=p, rounds=d,
                                                              streams=64)])
    rep = srv.run_poisson(2e4, 0.3, [1, 1], [shot_pool, seqs], seed=3)
    assert rep["completed"] == rep["submitted"] > 0
    wrep = srv.code_report(1)
    assert wrep["completed"] > 0 and wrep["p99_us"] >= wrep["p50_us"] > 0
    srv.close()
