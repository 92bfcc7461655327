"""Overlapping-window decoding on the GPU (lsd_window_*) against the window oracle, bit for bit:
every window is BP + LSD on the window's matrix, so corrections and status must be identical."""
import numpy as np
import pytest
import torch

import oracle
from oracle import window as OW
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


def _case(h, d, p, q, shots, seed):
    m, n = h.shape
    probs = I.space_time_probs(n, m, d, p, q).astype(np.float32).astype(np.float64)
    e = I.sample_errors(seed, shots, probs)
    return I.syndromes(I.space_time(h, d), e)


def _f32(v, k):
    return np.full(k, v, np.float32).astype(np.float64)


@pytest.mark.parametrize("name,d,w,c,p,order,osd_cs", [
    ("bb72", 6, 3, 1, 0.02, 0, None), ("bb72", 6, 3, 1, 0.04, 0, None),
    ("bb144", 12, 3, 1, 0.003, 0, None), ("bb144", 12, 3, 1, 0.01, 0, None),
    ("bb72", 7, 4, 2, 0.02, 0, None), ("bb72", 5, 2, 1, 0.02, 0, None),
    ("bb72", 6, 3, 3, 0.02, 0, None), ("bb72", 6, 3, 1, 0.03, 6, None),
    ("bb72", 6, 3, 1, 0.03, 4, 4), ("irreg_37x61", 5, 3, 1, 0.02, 0, None)])
def test_window_decode_matches_oracle(L, name, d, w, c, p, order, osd_cs):
    h = code(name)
    m, n = h.shape
    s = _case(h, d, p, p, 2000, seed=700 + d + w + int(1000 * p))
    wd = L.WindowDecoder(h, np.full(n, p, np.float32), np.full(m, p, np.float32), d, w, c,
                         bp_iters=30, lsd_order=order, osd_cs=osd_cs)
    corr, st, stats = wd.decode(torch.from_numpy(s).cuda(), want_stats=True)
    o = OW.window_decode(h, _f32(p, n), _f32(p, m), d, s, w=w, c=c, bp_iters=30,
                         lsd_order=order, osd_cs=-1 if osd_cs is None else osd_cs)
    assert np.array_equal(corr.cpu().numpy(), o["corrections"])
    assert np.array_equal(st.cpu().numpy(), o["status"])
    assert stats["shots"] == 2000 * o["windows"]
    hst = I.space_time(h, d).astype(np.int64)
    solvable = o["status"] <= 2
    assert np.array_equal((corr.cpu().numpy()[solvable].astype(np.int64) @ hst.T) % 2,
                          s[solvable])
    # one window kernel per window plus the first gather
    assert wd.kernel_launches() >= o["windows"] + 1


def test_one_window_equals_the_batch_decoder(L):
    """w > d: the only window is the whole space-time matrix."""
    h = code("bb72")
    m, n = h.shape
    d, p = 4, 0.02
    s = _case(h, d, p, p, 3000, seed=41)
    wd = L.WindowDecoder(h, np.full(n, p, np.float32), np.full(m, p, np.float32), d, 6, 1)
    corr, st = wd.decode(torch.from_numpy(s).cuda())
    dec = L.Decoder(I.space_time(h, d), I.space_time_probs(n, m, d, p, p).astype(np.float32), 30)
    c2, s2 = dec.decode(torch.from_numpy(s).cuda())
    assert torch.equal(corr, c2) and torch.equal(st, s2)


def test_byte_path_on_unaligned_buffers(L):
    """Syndrome and correction buffers that start off a 4-byte boundary take the byte-wise
    window kernel; results equal the word-wise path's."""
    h = code("bb72")
    m, n = h.shape
    d, p, shots = 6, 0.03, 1500
    s = _case(h, d, p, p, shots, seed=43)
    wd = L.WindowDecoder(h, np.full(n, p, np.float32), np.full(m, p, np.float32), d)
    ref, rst = wd.decode(torch.from_numpy(s).cuda())
    sl, fl = (d + 1) * m, d * (n + m)
    sbuf = torch.zeros(shots * sl + 1, dtype=torch.uint8, device="cuda")
    sbuf[1:].copy_(torch.from_numpy(s.ravel()).cuda())
    cbuf = torch.zeros(shots * fl + 3, dtype=torch.uint8, device="cuda")
    s_view = sbuf[1:].view(shots, sl)
    c_view = cbuf[3:].view(shots, fl)
    assert s_view.data_ptr() % 4 != 0 and c_view.data_ptr() % 4 != 0
    corr, st = wd.decode(s_view, c_view)
    assert torch.equal(corr, ref) and torch.equal(st, rst)


def test_repeated_calls_and_growing_batches(L):
    """Workspace grows with the batch; a second call on the same decoder gives the same
    answer (nothing carried over between calls)."""
    h = code("bb72")
    m, n = h.shape
    d, p = 6, 0.02
    s = _case(h, d, p, p, 4000, seed=47)
    wd = L.WindowDecoder(h, np.full(n, p, np.float32), np.full(m, p, np.float32), d)
    small, _ = wd.decode(torch.from_numpy(s[:700]).cuda())
    big, _ = wd.decode(torch.from_numpy(s).cuda())
    again, _ = wd.decode(torch.from_numpy(s[:700]).cuda())
    assert torch.equal(small, big[:700]) and torch.equal(small, again)
    o = OW.window_decode(h, _f32(p, n), _f32(p, m), d, s[:700])
    assert np.array_equal(small.cpu().numpy(), o["corrections"])


@pytest.mark.parametrize("d,w,c", [(12, 3, 1), (6, 4, 2), (6, 3, 3), (3, 5, 1)])
def test_streaming_pushes_match_batch_decode(L, d, w, c):
    """Blocks pushed one at a time give the batch decoder's corrections; each push commits the
    rounds of the window it completes, in order, and every round exactly once."""
    h = code("bb72")
    m, n = h.shape
    p, shots = 0.02, 1200
    s = _case(h, d, p, p, shots, seed=53 + d + w + c)
    wd = L.WindowDecoder(h, np.full(n, p, np.float32), np.full(m, p, np.float32), d, w, c)
    s_dev = torch.from_numpy(s).cuda()
    ref, rst = wd.decode(s_dev)
    corr = torch.full((shots, d * (n + m)), 7, dtype=torch.uint8, device="cuda")
    st = torch.empty(shots, dtype=torch.uint8, device="cuda")
    wd.stream_reset(shots)
    blocks = s_dev.view(shots, d + 1, m)
    done = 0
    for b in range(d + 1):
        first, count = wd.stream_push(blocks[:, b].contiguous(), corr, st)
        if count:
            assert first == done
            done += count
    assert done == d
    assert torch.equal(corr, ref) and torch.equal(st, rst)
    with pytest.raises(L.LsdError):
        wd.stream_push(blocks[:, 0].contiguous(), corr, st)


def test_window_decode_with_sparse_lsd_kernel(L):
    """The windows' LSD on the sparse kernel (state sized by what a shot touches) gives the
    same corrections as the oracle."""
    h = code("bb144")
    m, n = h.shape
    d, p = 8, 0.01
    s = _case(h, d, p, p, 1500, seed=59)
    wd = L.WindowDecoder(h, np.full(n, p, np.float32), np.full(m, p, np.float32), d,
                         bp_iters=30, lsd_kernel=2)
    corr, st = wd.decode(torch.from_numpy(s).cuda())
    o = OW.window_decode(h, _f32(p, n), _f32(p, m), d, s, bp_iters=30)
    assert np.array_equal(corr.cpu().numpy(), o["corrections"])
    assert np.array_equal(st.cpu().numpy(), o["status"])
