"""Seeded input generators: code constructions and the PRNG (no GPU)."""
import numpy as np
import pytest

from paper_2406_18655_gb300 import inputs as I


def test_splitmix_xoshiro_published_values():
    # splitmix64 from state 0 yields 0xE220A8397B1DCDAF first (Vigna's reference output).
    g = I.Xoshiro256ss.__new__(I.Xoshiro256ss)
    x = np.array([0], dtype=np.uint64) + I._GOLDEN
    z = x
    z = (z ^ (z >> np.uint64(30))) * I._SM_M1
    z = (z ^ (z >> np.uint64(27))) * I._SM_M2
    z = z ^ (z >> np.uint64(31))
    assert int(z[0]) == 0xE220A8397B1DCDAF
    # xoshiro256** state update: with s = (1, 2, 3, 4) the first output is rotl(2*5, 7)*9 = 11520
    g.s0, g.s1, g.s2, g.s3 = (np.array([v], dtype=np.uint64) for v in (1, 2, 3, 4))
    assert int(g.next_u64()[0]) == 11520
    assert int(g.next_u64()[0]) == 0  # s1 becomes 0 after the first update: rotl(0)*9 = 0


def test_streams_are_reproducible_by_shot():
    p = np.full(50, 0.2)
    a = I.sample_errors(11, 40, p)
    b = I.sample_errors(11, 10, p, first_shot=30)
    assert np.array_equal(a[30:], b)
    assert 0.1 < a.mean() < 0.3


@pytest.mark.parametrize("fn,n", [(I.bb72, 72), (I.bb144, 144), (I.bb288, 288)])
def test_bb_codes(fn, n):
    hx, hz = fn()
    assert hx.shape == (n // 2, n) and hz.shape == (n // 2, n)
    assert np.all(hx.sum(0) == 3) and np.all(hx.sum(1) == 6)
    assert not np.any((hx.astype(int) @ hz.T.astype(int)) % 2)


def test_hgp_instance():
    h = I.random_regular_ldpc(48, 64, 3, 4, 2406)
    assert np.all(h.sum(0) == 3) and np.all(h.sum(1) == 4)
    ov = h.astype(int) @ h.T.astype(int)
    np.fill_diagonal(ov, 0)
    assert ov.max() <= 1  # no two rows share two columns: girth >= 6
    hx, hz = I.hgp(h)
    assert hx.shape == (3072, 6400)
    assert np.all(hx.sum(1) == 7)
    assert sorted(set(hx.sum(0).tolist())) == [3, 4]
    # float32 products are exact here (entries are counts below 2^24)
    assert not np.any((hx.astype(np.float32) @ hz.T.astype(np.float32)) % 2)


def test_space_time_structure():
    hx, _ = I.bb72()
    d = 6
    st = I.space_time(hx, d)
    assert st.shape == ((d + 1) * 36, d * (72 + 36))
    assert st.sum() == d * (3 * 72 + 2 * 36)
    # measurement faults flip the same detector in two consecutive blocks
    col = st[:, 72]
    assert col.sum() == 2 and col[0] == 1 and col[36] == 1
    e = np.zeros((1, st.shape[1]), np.uint8)
    e[0, 5] = 1                      # data fault of round 0
    e[0, 108 + 5] = 1                # the same data fault again in round 1
    assert not np.any(I.space_time_data_residual(e, 72, 36, d))


def test_hgp_coo_equals_the_dense_product():
    h = I.random_regular_ldpc(12, 16, 3, 4, seed=9)
    hx = I.hgp(h)[0]
    m, n, rows, cols = I.hgp_coo(h)
    assert (m, n) == hx.shape
    dense = np.zeros((m, n), np.uint8)
    dense[rows, cols] = 1
    assert np.array_equal(dense, hx) and rows.size == int(hx.sum())
    e = I.sample_errors(3, 4, np.full(n, 0.1))
    for k in range(4):
        assert np.array_equal(I.coo_syndrome(m, rows, cols, e[k]), I.syndromes(hx, e[k:k + 1])[0])


def test_space_time_hooks_structure():
    """Hook columns split a qubit's checks between two consecutive blocks; with every hook
    removed the matrix is the phenomenological one; a hook together with the data fault of
    the same qubit and round fires exactly the checks moved to the next block, twice
    (cancelling in block t)."""
    h = I.bb72()[0]
    m, n = h.shape
    d = 3
    hs, split = I.space_time_hooks(h, d, seed=5)
    F = 2 * n + m
    keep = np.concatenate([np.arange(t * F, t * F + n + m) for t in range(d)])
    assert np.array_equal(hs[:, keep], I.space_time(h, d))
    for t in range(d):
        for j in range(n):
            col = hs[:, t * F + n + m + j]
            assert col.sum() == h[:, j].sum() == 3
            assert 1 <= split[t, j] < 3
            assert col[t * m:(t + 1) * m].sum() == split[t, j]
            both = (col.astype(int) + hs[:, t * F + j]) % 2
            assert both[t * m:(t + 1) * m].sum() == 3 - split[t, j]
            assert np.array_equal(both[(t + 1) * m:(t + 2) * m], col[(t + 1) * m:(t + 2) * m])
    p = I.space_time_hooks_probs(n, m, d, 0.01, seed=6)
    assert p.size == d * F and p.min() >= 0.00125 and p.max() < 0.0175 and np.unique(p).size > 100
