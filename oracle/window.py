"""Oracle of (w, c) overlapping-window decoding of repeated syndrome rounds (Methods 4.3).

TEST INFRASTRUCTURE ONLY (imported by tests/, never by the product path).

Phenomenological noise over d noisy syndrome rounds followed by one noiseless round: detector
block t (t = 0..d) is the difference of syndrome rounds t and t-1; the faults of round t are
n data faults (flipping block t through H) and m measurement faults (flipping blocks t and
t+1).  A fault vector is laid out round by round, [data | measurement] per round, and a
syndrome block by block.

The window decoder (Methods 4.3: w = 3 rounds decoded, the c = 1 oldest committed) works on
a running syndrome S, initially the shot's syndrome:

    t = 0
    loop:
        if t + w - 1 >= d or t + c >= d:
                            the final window holds blocks t..d and fault rounds t..d-1;
                            decode it, commit all of it, stop (the second condition only
                            matters for c = w, where the windows would otherwise leave the
                            noiseless block d alone in a window without faults)
        else:               the window holds blocks t..t+w-1 and fault rounds t..t+w-1
                            (the measurement faults of its last round reach one block past
                            the window; inside it they flip only that last block); decode
                            it, commit its first c rounds
        committing fault f: correction[f] ^= 1 and S ^= (column f of the full matrix)
        t += c

Each window is decoded by BP + LSD (oracle.decode) on its own matrix and the channel
probabilities of its columns.  After the commits of a window, blocks t..t+c-1 of S are zero
when the window's decode satisfied its syndrome: only faults of those rounds and of earlier,
already committed rounds touch them.
"""
from __future__ import annotations

import numpy as np

from . import oracle as _o


def window_matrix(h, rounds: int, blocks: int) -> np.ndarray:
    """Detector blocks 0..blocks-1 by fault rounds 0..rounds-1 of the phenomenological matrix
    (blocks = rounds for an inner window, rounds + 1 for the final one)."""
    h = np.asarray(h, dtype=np.uint8)
    m, n = h.shape
    out = np.zeros((blocks * m, rounds * (n + m)), np.uint8)
    for r in range(rounds):
        c0 = r * (n + m)
        out[r * m:(r + 1) * m, c0:c0 + n] = h
        for i in range(m):
            out[r * m + i, c0 + n + i] = 1
            if r + 1 < blocks:
                out[(r + 1) * m + i, c0 + n + i] = 1
    return out


def window_probs(p_data, q_meas, rounds: int) -> np.ndarray:
    """Channel probabilities of `rounds` fault rounds: [p_data | q_meas] per round."""
    return np.tile(np.concatenate([np.asarray(p_data, np.float64),
                                   np.asarray(q_meas, np.float64)]), rounds)


def window_decode(h, p_data, q_meas, d: int, syndromes, w: int = 3, c: int = 1,
                  bp_iters: int = 30, alpha: float = 0.625, lsd_order: int = 0,
                  osd_cs: int = -1, precision: int = 1, nthreads: int = 0):
    """Returns dict(corrections [shots][d (n+m)], status [shots] (largest status of any
    window), windows (the number of windows), residual_syndrome [shots][(d+1) m])."""
    h = np.asarray(h, dtype=np.uint8)
    m, n = h.shape
    s = np.atleast_2d(np.asarray(syndromes, dtype=np.uint8))
    shots = s.shape[0]
    S = s.reshape(shots, d + 1, m).copy()
    corr = np.zeros((shots, d, n + m), np.uint8)
    status = np.zeros(shots, np.uint8)
    t, windows = 0, 0
    while True:
        final = t + w - 1 >= d or t + c >= d
        rounds = d - t if final else w
        blocks = rounds + 1 if final else w
        hw = window_matrix(h, rounds, blocks)
        sw = np.ascontiguousarray(S[:, t:t + blocks].reshape(shots, blocks * m))
        o = _o.decode(hw, window_probs(p_data, q_meas, rounds), sw, bp_iters, alpha=alpha,
                      lsd_order=lsd_order, precision=precision, nthreads=nthreads,
                      osd_cs=osd_cs)
        status = np.maximum(status, o["status"])
        ew = o["corrections"].reshape(shots, rounds, n + m)
        commit = rounds if final else c
        for r in range(commit):
            data, meas = ew[:, r, :n], ew[:, r, n:]
            corr[:, t + r] ^= ew[:, r]
            S[:, t + r] ^= ((data.astype(np.int64) @ h.T.astype(np.int64)) % 2).astype(np.uint8)
            S[:, t + r] ^= meas
            if t + r + 1 <= d:
                S[:, t + r + 1] ^= meas
        windows += 1
        if final:
            break
        t += c
    return dict(corrections=corr.reshape(shots, d * (n + m)), status=status, windows=windows,
                residual_syndrome=S.reshape(shots, (d + 1) * m))
