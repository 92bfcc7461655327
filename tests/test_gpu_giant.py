"""One giant shot on the whole GPU (lsd_giant_*: grid-parallel BP, then P-LSD of Alg. 2)
against the oracle, shot by shot: posteriors and iteration counts of BP bit-exact,
corrections, status, nu, kappa and growth steps of LSD bit-exact."""
import numpy as np
import pytest
import torch

import oracle
from paper_2406_18655_gb300 import inputs as I
from tests.gpu_cases import code

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2406_18655_gb300 import build
    build.build()
    from paper_2406_18655_gb300 import lsd
    lsd.lib()
    return lsd


def f64(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def _shots(h, p, shots, seed):
    probs = np.full(h.shape[1], p, np.float32)
    e = I.sample_errors(seed, shots, probs.astype(np.float64))
    return probs, e, I.syndromes(h, e)


@pytest.mark.parametrize("name,p,iters", [("hgp", 0.03, 50), ("bb144", 0.08, 30),
                                          ("ldpc_480x960", 0.06, 20), ("rep_boundary", 0.2, 8),
                                          ("irreg_37x61", 0.1, 12)])
def test_giant_bp_matches_oracle(L, name, p, iters):
    h = code(name)
    probs, e, s = _shots(h, p, 12, seed=61)
    gd = L.GiantDecoder.from_dense(h, probs, iters)
    llr, hard, used, conv = oracle.bp(h, f64(probs), s, iters, precision=1)
    post = torch.empty(h.shape[1], dtype=torch.float32, device="cuda")
    for k in range(s.shape[0]):
        corr, info = gd.decode(torch.from_numpy(s[k]).cuda(), posteriors=post)
        assert np.array_equal(post.cpu().numpy(), llr[k].astype(np.float32))
        assert info["bp_iterations"] == used[k]
        assert (info["status"] == 1) == bool(conv[k])
        if conv[k]:
            assert np.array_equal(corr.cpu().numpy(), hard[k])


def _rounded(n, seed):
    g = I.Xoshiro256ss(seed, np.arange(n, dtype=np.uint64))
    return np.round(g.uniform() * 5 - 0.5, 1).astype(np.float32)


@pytest.mark.parametrize("name,p,soft,shots", [
    ("hgp", 0.05, "bp", 24), ("hgp", 0.03, "ties", 24), ("bb144", 0.1, "bp", 40),
    ("bb72", 0.08, "ties", 40), ("ldpc_480x960", 0.06, "bp", 30),
    ("rep_boundary", 0.15, "ties", 40), ("st_bb72_d6", 0.03, "bp", 30),
    ("irreg_37x61", 0.08, "ties", 40), ("irreg_37x61", 0.12, "bp", 40)])
def test_plsd_matches_oracle_lsd(L, name, p, soft, shots):
    """P-LSD with many clusters growing, colliding and merging at once gives the serial
    algorithm's clusters and corrections."""
    h = code(name)
    probs, e, s = _shots(h, p, shots, seed=67)
    if soft == "bp":
        llr, *_ = oracle.bp(h, f64(probs), s, 30, precision=1)
        llr = llr.astype(np.float32)
    else:
        llr = np.stack([_rounded(h.shape[1], 100 + k) for k in range(shots)])
    r = oracle.lsd(h, s, llr.astype(np.float64), order=0, probs=f64(probs))
    gd = L.GiantDecoder.from_dense(h, probs, 30)
    for k in range(shots):
        corr, info = gd.postprocess(torch.from_numpy(llr[k]).cuda(), torch.from_numpy(s[k]).cuda())
        assert info["status"] == r["status"][k]
        assert np.array_equal(corr.cpu().numpy(), r["corrections"][k])
        assert (info["nu"], info["kappa"], info["steps"]) == (r["nu"][k], r["kappa"][k],
                                                              r["steps"][k])


@pytest.mark.parametrize("name,p,order,osd_cs,shots", [
    ("bb144", 0.06, 6, None, 30), ("bb144", 0.08, 3, None, 30), ("bb72", 0.08, 10, None, 30),
    ("bb144", 0.06, 14, 4, 30), ("bb144", 0.08, 29, 8, 20), ("hgp", 0.04, 10, None, 12),
    ("hgp", 0.04, 20, 4, 12), ("ldpc_480x960", 0.05, 6, 0, 20)])
def test_plsd_mu_matches_oracle(L, name, p, order, osd_cs, shots):
    """LSD-mu in the giant shot: mu growth steps for every cluster, then OSD-E or OSD-CS-w per
    cluster, as the serial algorithm (App. D)."""
    h = code(name)
    probs, e, s = _shots(h, p, shots, seed=97 + order)
    llr, *_ = oracle.bp(h, f64(probs), s, 30, precision=1)
    llr = llr.astype(np.float32)
    r = oracle.lsd(h, s, llr.astype(np.float64), order=order, probs=f64(probs),
                   osd_cs=-1 if osd_cs is None else osd_cs)
    gd = L.GiantDecoder.from_dense(h, probs, 30, order, osd_cs=osd_cs)
    for k in range(shots):
        corr, info = gd.postprocess(torch.from_numpy(llr[k]).cuda(), torch.from_numpy(s[k]).cuda())
        assert info["status"] == r["status"][k]
        assert np.array_equal(corr.cpu().numpy(), r["corrections"][k])
        assert (info["nu"], info["kappa"], info["steps"]) == (r["nu"][k], r["kappa"][k],
                                                              r["steps"][k])


def test_giant_decode_matches_oracle_and_batch_decoder(L):
    """End to end on the HGP code: the giant path, the batch decoder and the oracle agree."""
    h = code("hgp")
    probs, e, s = _shots(h, 0.04, 30, seed=71)
    o = oracle.decode(h, f64(probs), s, 50, precision=1)
    gd = L.GiantDecoder.from_dense(h, probs, 50)
    bd = L.Decoder(h, probs, 50)
    bc, bs = bd.decode(torch.from_numpy(s).cuda())
    for k in range(s.shape[0]):
        corr, info = gd.decode(torch.from_numpy(s[k]).cuda())
        assert info["status"] == o["status"][k] == int(bs[k])
        assert np.array_equal(corr.cpu().numpy(), o["corrections"][k])
        assert torch.equal(corr, bc[k])


def test_larger_hgp_matches_oracle(L):
    """HGP of a (3,4)-regular 96 x 128 matrix (n = 25600, beyond one warp's comfort): a few
    shots at a noise level where LSD runs on most of them."""
    base = I.random_regular_ldpc(96, 128, 3, 4, seed=11)
    m, n, rows, cols = I.hgp_coo(base)
    h = np.zeros((m, n), np.uint8)
    h[rows, cols] = 1
    probs, e, s = _shots(h, 0.04, 4, seed=73)
    o = oracle.decode(h, f64(probs), s, 30, precision=1)
    gd = L.GiantDecoder(m, n, rows, cols, probs, 30)
    for k in range(s.shape[0]):
        corr, info = gd.decode(torch.from_numpy(s[k]).cuda())
        assert info["status"] == o["status"][k]
        assert np.array_equal(corr.cpu().numpy(), o["corrections"][k])


def test_giant_shot_explains_its_syndrome(L):
    """HGP of a (3,4)-regular 240 x 320 matrix: n = 160000 faults, m = 76800 detectors,
    beyond the batch decoder's 65535 limit.  The correction satisfies H e_hat = s."""
    base = I.random_regular_ldpc(240, 320, 3, 4, seed=13)
    m, n, rows, cols = I.hgp_coo(base)
    gd = L.GiantDecoder(m, n, rows, cols, np.full(n, 0.03, np.float32), 50)
    for seed in (1, 2):
        e = I.sample_errors(seed, 1, np.full(n, 0.03))[0]
        s = I.coo_syndrome(m, rows, cols, e)
        corr, info = gd.decode(torch.from_numpy(s).cuda())
        assert info["status"] in (1, 2)
        assert np.array_equal(I.coo_syndrome(m, rows, cols, corr.cpu().numpy()), s)
        if info["status"] == 2:
            assert info["nu"] > 1 and info["steps"] > 0


def test_largest_giant_shot(L):
    """HGP of a (3,4)-regular 480 x 640 matrix: 640000 faults, 307200 detectors, 2.15 M
    edges, at a noise level where LSD meets thousands of clusters in one shot."""
    base = I.random_regular_ldpc(480, 640, 3, 4, seed=2886)
    m, n, rows, cols = I.hgp_coo(base)
    gd = L.GiantDecoder(m, n, rows, cols, np.full(n, 0.03, np.float32), 30)
    e = I.sample_errors(5, 1, np.full(n, 0.03))[0]
    s = I.coo_syndrome(m, rows, cols, e)
    corr, info = gd.decode(torch.from_numpy(s).cuda())
    assert info["status"] == 2 and info["nu"] > 1000
    assert np.array_equal(I.coo_syndrome(m, rows, cols, corr.cpu().numpy()), s)


def test_unsolvable_and_small_arena(L):
    """A syndrome outside image(H) gives status 3 and a zero correction; an arena too small
    for the clusters raises LSD_ERR_ADMISSION and leaves the decoder usable."""
    h = np.array([[1, 1, 0], [1, 1, 0], [0, 0, 1]], np.uint8)
    gd = L.GiantDecoder.from_dense(h, np.full(3, 0.1, np.float32), 5)
    corr, info = gd.decode(torch.tensor([1, 0, 0], dtype=torch.uint8, device="cuda"))
    assert info["status"] == 3 and not corr.any()
    hh = code("bb144")
    probs, e, s = _shots(hh, 0.1, 2, seed=79)
    small = L.GiantDecoder.from_dense(hh, probs, 0, arena_bytes=2048)
    assert s[0].sum() > 10
    with pytest.raises(L.LsdError) as err:
        small.decode(torch.from_numpy(s[0]).cuda())
    assert err.value.code == L.LSD_ERR_ADMISSION
    corr, info = small.decode(torch.zeros(hh.shape[0], dtype=torch.uint8, device="cuda"))
    assert info["status"] == 2 and not corr.any()
    o = oracle.decode(hh, f64(probs), s, 5, precision=1)
    big = L.GiantDecoder.from_dense(hh, probs, 5)
    corr, info = big.decode(torch.from_numpy(s[1]).cuda())
    assert np.array_equal(corr.cpu().numpy(), o["corrections"][1])


def test_grid_barrier_timeout_leaves_the_device_usable(L):
    """A BP grid barrier whose wait runs out (block 0 withholds its arrival through the test
    facility) makes the decode return LSD_ERR_TIMEOUT after its bound; the next decode, with
    the hold lifted, gives the oracle's answer."""
    h = code("hgp")
    probs, e, s = _shots(h, 0.03, 2, seed=89)
    gd = L.GiantDecoder.from_dense(h, probs, 50)
    gd.test_hold_barrier(True, limit_ns=20_000_000)
    with pytest.raises(L.LsdError) as err:
        gd.decode(torch.from_numpy(s[0]).cuda())
    assert err.value.code == L.LSD_ERR_TIMEOUT
    gd.test_hold_barrier(False)
    o = oracle.decode(h, f64(probs), s, 50, precision=1)
    for k in range(2):
        corr, info = gd.decode(torch.from_numpy(s[k]).cuda())
        assert info["status"] == o["status"][k]
        assert np.array_equal(corr.cpu().numpy(), o["corrections"][k])
