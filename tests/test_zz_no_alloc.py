"""Allocation-free decode entry point (lsd_decode_batch_static), through the C ABI.

Some callers cannot call cudaMalloc while they decode: a real-time loop that runs with a
device-memory footprint fixed at start-up (cudaMalloc may synchronize the device and has
unbounded latency), or a process whose free device memory is held by another allocator.
lsd_decode_batch_static serves them with scratch from a fixed device array inside the
library.  This test checks that it returns exactly what lsd_decode_batch returns, on two
calls in a row (the array keeps the previous call's contents, so the second call also
checks that the state that must start at zero is cleared), that it leaves the decoder's
own device memory untouched, and that an oversized batch is refused.

This file is collected last so that a failure here cannot hide the other GPU tests.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from tests.gpu_cases import sample

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2406_18655_gb300 import build
    build.build()
    from paper_2406_18655_gb300 import lsd
    lsd.lib()
    return lsd


def _call_static(L, dec, syn, corr, status):
    return L.lib().lsd_decode_batch_static(dec._h, syn.shape[0], C.c_void_p(syn.data_ptr()),
                                           C.c_void_p(corr.data_ptr()),
                                           C.c_void_p(status.data_ptr()))


def test_static_scratch_decode_matches_decode_batch(L):
    h, probs, _, _ = sample("bb144", 0.06, 1, seed=1)
    dec = L.Decoder(h, probs, 50)
    ref = L.Decoder(h, probs, 50)  # the existing entry point, on its own decoder
    held = dec.workspace_bytes()
    for call, (shots, seed) in enumerate([(9000, 501), (4321, 502)]):
        _, _, e, s = sample("bb144", 0.06, shots, seed=seed)
        sd = torch.from_numpy(s).cuda()
        corr = torch.full((shots, h.shape[1]), 7, dtype=torch.uint8, device="cuda")
        status = torch.zeros(shots, dtype=torch.uint8, device="cuda")
        assert _call_static(L, dec, sd, corr, status) == L.LSD_OK, f"call {call}"
        torch.cuda.synchronize()
        assert dec.workspace_bytes() == held  # the decoder allocated nothing
        ref_c, ref_st = ref.decode(sd)
        torch.cuda.synchronize()
        assert torch.equal(corr, ref_c), f"call {call}: corrections differ"
        assert torch.equal(status, ref_st), f"call {call}: status differs"
        assert (status.cpu().numpy() == L.SHOT_OK_LSD).any()


def test_static_scratch_rejects_oversized_batches(L):
    h, probs, _, _ = sample("bb144", 0.05, 1, seed=2)
    dec = L.Decoder(h, probs, 50)
    too_many = 14463  # one shot beyond what 8 MiB holds for n = 144
    sd = torch.zeros((too_many, h.shape[0]), dtype=torch.uint8, device="cuda")
    corr = torch.zeros((too_many, h.shape[1]), dtype=torch.uint8, device="cuda")
    status = torch.zeros(too_many, dtype=torch.uint8, device="cuda")
    assert _call_static(L, dec, sd, corr, status) == L.LSD_ERR_ADMISSION
    assert _call_static(L, dec, sd[:14462], corr[:14462], status[:14462]) == L.LSD_OK
    torch.cuda.synchronize()
    assert np.all(status[:14462].cpu().numpy() == L.SHOT_OK_BP)  # zero syndromes


def test_static_scratch_padded_cta_kernel_without_status(L):
    """A BB[[72,12,6]] space-time matrix over 6 noisy rounds (252 x 648, rows of 8 edges and
    1 in the last block): BP runs in the register-table CTA kernel with padded rows and LSD
    in the dense kernel.  No status buffer is passed; the corrections must still equal
    lsd_decode_batch's, on two calls in a row."""
    from paper_2406_18655_gb300 import inputs as I
    hx = I.bb72()[0]
    m0, n0 = hx.shape
    h = I.space_time(hx, 6)
    probs = I.space_time_probs(n0, m0, 6, 0.01, 0.01).astype(np.float32)
    dec = L.Decoder(h, probs, 30)
    ref = L.Decoder(h, probs, 30)
    held = dec.workspace_bytes()
    lsd_seen = False
    for call, (shots, seed) in enumerate([(3000, 611), (1700, 612)]):
        e = I.sample_errors(seed, shots, probs.astype(np.float64))
        sd = torch.from_numpy(I.syndromes(h, e)).cuda()
        corr = torch.full((shots, h.shape[1]), 7, dtype=torch.uint8, device="cuda")
        rc = L.lib().lsd_decode_batch_static(dec._h, shots, C.c_void_p(sd.data_ptr()),
                                             C.c_void_p(corr.data_ptr()), None)
        assert rc == L.LSD_OK, f"call {call}"
        torch.cuda.synchronize()
        assert dec.workspace_bytes() == held
        ref_c, ref_st = ref.decode(sd)
        torch.cuda.synchronize()
        assert torch.equal(corr, ref_c), f"call {call}: corrections differ"
        lsd_seen |= bool((ref_st.cpu().numpy() == L.SHOT_OK_LSD).any())
    assert lsd_seen  # the LSD kernel ran on the static queue
