"""Oracle of (3,1) overlapping-window decoding (Methods 4.3) pinned against the full
space-time matrix, global decoding, the syndrome it must explain and a hand-worked case."""
import numpy as np
import pytest

from paper_2406_18655_gb300 import inputs as I


@pytest.fixture(scope="module")
def W(oracle_lib):
    from oracle import window
    return window


@pytest.mark.parametrize("d", [1, 3, 6])
def test_window_matrices_are_blocks_of_the_space_time_matrix(W, d):
    """The final window over every round is the whole space-time matrix, and an inner window
    of w rounds is its first w detector blocks (generator in inputs.py, written separately)."""
    h = I.bb72()[0]
    m = h.shape[0]
    assert np.array_equal(W.window_matrix(h, d, d + 1), I.space_time(h, d))
    assert np.array_equal(W.window_matrix(h, d, d), I.space_time(h, d)[:d * m])


def _sample(h, d, p, q, shots, seed):
    m, n = h.shape
    probs = I.space_time_probs(n, m, d, p, q)
    e = I.sample_errors(seed, shots, probs)
    return e, I.syndromes(I.space_time(h, d), e)


@pytest.mark.parametrize("d,w", [(3, 4), (3, 9), (6, 7)])
def test_one_window_is_global_decoding(W, oracle_lib, d, w):
    """With w >= d + 1 the first window is already the final one: the whole matrix, decoded
    once."""
    h = I.bb72()[0]
    m, n = h.shape
    e, s = _sample(h, d, 0.02, 0.02, 200, seed=11 + d)
    r = W.window_decode(h, np.full(n, 0.02), np.full(m, 0.02), d, s, w=w, c=1)
    g = oracle_lib.decode(I.space_time(h, d), I.space_time_probs(n, m, d, 0.02, 0.02), s, 30)
    assert r["windows"] == 1
    assert np.array_equal(r["corrections"], g["corrections"])
    assert np.array_equal(r["status"], g["status"])


@pytest.mark.parametrize("d,w,c,p", [(6, 3, 1, 0.01), (6, 3, 1, 0.03), (12, 3, 1, 0.02),
                                     (6, 4, 2, 0.02), (5, 2, 1, 0.02), (6, 3, 3, 0.02),
                                     (7, 3, 3, 0.02), (1, 3, 1, 0.05)])
def test_windowed_correction_explains_the_syndrome(W, d, w, c, p):
    """Committed faults explain every detector: H_st e_hat = s for the full space-time matrix,
    and the running syndrome is left at zero; the windows start at 0, c, 2c, ... up to the
    first that reaches block d or commits the last round."""
    h = I.bb72()[0]
    m, n = h.shape
    e, s = _sample(h, d, p, p, 150, seed=int(1000 * p) + d + w)
    r = W.window_decode(h, np.full(n, p), np.full(m, p), d, s, w=w, c=c)
    assert np.all(r["status"] <= 2)
    hst = I.space_time(h, d).astype(np.int64)
    assert np.array_equal((r["corrections"].astype(np.int64) @ hst.T) % 2, s)
    assert not r["residual_syndrome"].any()
    inner = 0
    t = 0
    while t + w - 1 < d and t + c < d:
        inner += 1
        t += c
    assert r["windows"] == inner + 1


def test_hand_worked_measurement_error(W):
    """Repetition code of 3 bits (checks x0+x1, x1+x2), d = 4 noisy rounds, (3,1) windows,
    one measurement error on check 0 in round 1: detector block 1 and block 2 fire on row 0.
    Window 0 (blocks 0..2) explains both by that measurement fault (weight 1) and commits
    round 0 (nothing); window 1 (blocks 1..3) finds it again in its first round and commits
    it, clearing block 2; the final window (blocks 2..4) then sees no syndrome.  The result is
    exactly the one measurement fault."""
    h = np.array([[1, 1, 0], [0, 1, 1]], np.uint8)
    m, n, d = 2, 3, 4
    e = np.zeros((1, d * (n + m)), np.uint8)
    e[0, 1 * (n + m) + n + 0] = 1
    s = I.syndromes(I.space_time(h, d), e)
    assert s[0].tolist() == [0, 0, 1, 0, 1, 0, 0, 0, 0, 0]
    r = W.window_decode(h, np.full(n, 0.05), np.full(m, 0.05), d, s, w=3, c=1)
    assert r["windows"] == 3
    assert np.array_equal(r["corrections"], e)
