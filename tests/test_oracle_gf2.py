"""GF(2) rank / solve and OSD-0 of the oracle against brute force (no GPU)."""
import itertools

import numpy as np
import pytest

from paper_2406_18655_gb300 import inputs as I


def _all_x(n):
    return ((np.arange(2 ** n)[:, None] >> np.arange(n)[None, :]) & 1).astype(np.int64)


def _span_size(a):
    """Number of distinct vectors A x over all 2^n vectors x (brute force)."""
    n = a.shape[1]
    if n == 0:
        return 1
    img = (_all_x(n) @ a.T.astype(np.int64)) % 2
    keys = img @ (1 << np.arange(a.shape[0], dtype=np.int64))
    return len(np.unique(keys))


def _rand(seed, m, n, density=0.4):
    g = I.Xoshiro256ss(seed, np.arange(m * n, dtype=np.uint64))
    return (g.uniform() < density).astype(np.uint8).reshape(m, n)


@pytest.mark.parametrize("seed", range(12))
def test_rank_vs_brute_force(oracle_lib, seed):
    m, n = 3 + seed % 6, 4 + seed % 9
    a = _rand(seed, m, n)
    assert 2 ** oracle_lib.gf2_rank(a) == _span_size(a)


@pytest.mark.parametrize("seed", range(12))
def test_solve_vs_brute_force(oracle_lib, seed):
    m, n = 4 + seed % 5, 5 + seed % 8
    a = _rand(100 + seed, m, n)
    x_true = _rand(200 + seed, 1, n)[0]
    b = (a.astype(int) @ x_true) % 2
    if seed % 3 == 0:  # also unsolvable right-hand sides
        b = _rand(300 + seed, 1, m)[0]
    ok, x, piv = oracle_lib.gf2_solve(a, b)
    # brute-force greedy basis: column c is a pivot iff it raises the rank of columns 0..c
    sizes = [1] + [_span_size(a[:, :c + 1]) for c in range(n)]
    piv_bf = np.array([sizes[c + 1] > sizes[c] for c in range(n)], np.uint8)
    assert np.array_equal(piv, piv_bf)
    sols = []
    for bits in itertools.product((0, 1), repeat=int(piv_bf.sum())):
        xx = np.zeros(n, np.int64)
        xx[np.nonzero(piv_bf)[0]] = bits
        if np.array_equal((a.astype(int) @ xx) % 2, b):
            sols.append(xx)
    solvable_bf = bool(np.any(np.all((_all_x(n) @ a.T.astype(np.int64)) % 2 == b, axis=1)))
    assert ok == solvable_bf
    if ok:
        assert len(sols) == 1 and np.array_equal(x, sols[0])


@pytest.mark.parametrize("seed", range(10))
def test_osd0_vs_brute_force(oracle_lib, seed):
    """OSD-0 (Sec. 2.2): the unique solution on the greedy basis of reliability-sorted columns."""
    m, n = 5 + seed % 3, 9 + seed % 4
    a = _rand(400 + seed, m, n, 0.35)
    e = _rand(500 + seed, 1, n, 0.25)[0]
    s = (a.astype(int) @ e) % 2
    g = I.Xoshiro256ss(600 + seed, np.arange(n, dtype=np.uint64))
    llr = np.round(g.uniform() * 4 - 1, 1)  # coarse values: ties happen
    ok, out = oracle_lib.osd0(a, s, llr)
    order = sorted(range(n), key=lambda j: (llr[j], j))
    ap = a[:, order]
    sizes = [1] + [_span_size(ap[:, :c + 1]) for c in range(n)]
    basis = [order[c] for c in range(n) if sizes[c + 1] > sizes[c]]
    found = None
    for bits in itertools.product((0, 1), repeat=len(basis)):
        xx = np.zeros(n, np.int64)
        xx[basis] = bits
        if np.array_equal((a.astype(int) @ xx) % 2, s):
            assert found is None
            found = xx
    assert ok and found is not None
    assert np.array_equal(out, found)


def test_logical_failure_rank_test(oracle_lib):
    """Residuals in the row space of H_Z are harmless; a logical operator is a failure."""
    hx, hz = I.bb72()
    n = hx.shape[1]
    g = I.Xoshiro256ss(7, np.arange(n, dtype=np.uint64))
    coeffs = (g.uniform() < 0.5).astype(int)[: hz.shape[0]]
    stab = (coeffs @ hz.astype(int)) % 2
    # a logical: a kernel vector of H_X (column j plus the combination of basis columns
    # that reproduces it) that raises the rank of H_Z
    r_hz = oracle_lib.gf2_rank(hz)
    logical = None
    for j in range(n):
        others = hx.copy()
        others[:, j] = 0
        ok, x, _ = oracle_lib.gf2_solve(others, hx[:, j])
        if not ok:
            continue
        v = x.copy()
        v[j] ^= 1
        assert not np.any((hx.astype(int) @ v) % 2)
        if oracle_lib.gf2_rank(np.vstack([hz, v])) > r_hz:
            logical = v
            break
    assert logical is not None
    res = np.vstack([stab, logical, (stab + logical) % 2, np.zeros(n, np.uint8)]).astype(np.uint8)
    assert oracle_lib.logical_failures(hz, res).tolist() == [0, 1, 1, 0]
