"""Bit-packed batch I/O (lsd_decode_batch_packed / _host_packed) against the byte-per-bit
path, bit for bit: the kernels read packed syndrome words and write packed corrections
themselves, so every BP kernel family and both LSD kernels are covered, with row lengths
that are not multiples of 32 (the last word's spare bits) and a host batch large enough for
the chunked copy pipeline."""
import numpy as np
import pytest
import torch

from paper_2406_18655_gb300 import inputs as I
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


def _words(L, rows):
    return torch.from_numpy(L.pack_bits(rows).view(np.int32)).cuda()


@pytest.mark.parametrize("name,p,iters,order,opts", [
    ("bb144", 0.06, 50, 0, {}),                   # register warp-group BP, dense LSD
    ("bb144", 0.06, 50, 0, {"bp_lanes": 16}),     # two shots per warp
    ("bb144", 0.06, 50, 0, {"bp_kernel": 1}),     # generic warp-group BP
    ("bb72", 0.06, 30, 4, {}),                    # LSD-mu (OSD-E)
    ("irreg_37x61", 0.05, 30, 0, {}),             # 37 x 61: spare bits in both rows
    ("st_bb72_d6", 0.01, 30, 0, {}),              # padded register-table CTA BP
    ("ldpc_480x960", 0.05, 30, 0, {}),            # largest dense LSD class
    ("hgp", 0.05, 100, 0, {}),                    # sparse LSD, spill instance
])
def test_packed_equals_bytes(L, name, p, iters, order, opts):
    shots = 600 if name == "hgp" else 3000
    h, probs, e, s = sample(name, p, shots, seed=71)
    d = L.Decoder(h, probs, iters, order, **opts)
    ref_c, ref_s = d.decode(torch.from_numpy(s).cuda())
    cw, st = d.decode_packed(_words(L, s))
    got = L.unpack_bits(cw.cpu().numpy().view(np.uint32), h.shape[1])
    assert np.array_equal(got, ref_c.cpu().numpy())
    assert torch.equal(st, ref_s)
    # spare bits of the last word are written as zero
    n = h.shape[1]
    if n % 32:
        last = cw.cpu().numpy().view(np.uint32)[:, -1]
        assert not np.any(last >> np.uint32(n % 32))
    assert (st.cpu().numpy() == L.SHOT_OK_LSD).any()


def test_packed_syndromes_ignore_spare_bits(L):
    """Bits past m in the last syndrome word do not change the decode."""
    h, probs, e, s = sample("irreg_37x61", 0.05, 2000, seed=72)
    d = L.Decoder(h, probs, 30)
    w = L.pack_bits(s)
    c1, s1 = d.decode_packed(torch.from_numpy(w.view(np.int32)).cuda())
    w2 = w.copy()
    w2[:, -1] |= np.uint32(0xFFFFFFFF) << np.uint32(37 % 32)
    c2, s2 = d.decode_packed(torch.from_numpy(w2.view(np.int32)).cuda())
    assert torch.equal(c1, c2) and torch.equal(s1, s2)


def test_host_packed_pipeline(L):
    """2 x 65536 + 1000 BB[[144,12,12]] shots through the host-buffer packed path (chunked
    copy pipeline) equal the device byte path."""
    h, probs, _, _ = sample("bb144", 0.05, 1, seed=73)
    shots = 2 * 65536 + 1000
    e = I.sample_errors(74, shots, probs.astype(np.float64))
    s = I.syndromes(h, e)
    d = L.Decoder(h, probs, 50)
    ref_c, ref_s = d.decode(torch.from_numpy(s).cuda())
    sw = torch.from_numpy(L.pack_bits(s).view(np.int32)).pin_memory()
    cw = torch.empty((shots, (h.shape[1] + 31) // 32), dtype=torch.int32).pin_memory()
    st = torch.empty(shots, dtype=torch.uint8).pin_memory()
    d.decode_host_packed(sw, cw, st)
    got = L.unpack_bits(cw.numpy().view(np.uint32), h.shape[1])
    assert np.array_equal(got, ref_c.cpu().numpy())
    assert np.array_equal(st.numpy(), ref_s.cpu().numpy())
