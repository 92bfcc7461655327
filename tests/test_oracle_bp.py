"""Oracle BP pinned against exact inference on tree Tanner graphs and a closed form (no GPU).

* Sum-product on a tree gives the exact posterior LLRs ln P(x_j=0|s)/P(x_j=1|s), in double
  and, within its derived rounding bound, in the FP32 mirror.
* Min-sum with alpha = 1 on a tree gives exact min-marginal differences
  min_{x_j=1} cost(x) - min_{x_j=0} cost(x), cost(x) = sum_k lambda_k x_k.
* One check, one iteration: the scaled min-sum message (alpha = 0.625, Sec. 4.3).
"""
import numpy as np
import pytest

from paper_2406_18655_gb300 import inputs as I


def _tree_case(seed, nv):
    h = I.random_tree_tanner(seed, nv)
    g = I.Xoshiro256ss(1000 + seed, np.arange(nv + h.shape[0], dtype=np.uint64))
    u = g.uniform()
    p = 0.02 + 0.43 * u[:nv]
    s = (u[nv:] < 0.5).astype(np.uint8)
    return h, p, s


def _all_x(n):
    return ((np.arange(2 ** n)[:, None] >> np.arange(n)[None, :]) & 1).astype(np.int64)


def _consistent(h, s):
    xs = _all_x(h.shape[1])
    ok = np.all((xs @ h.T.astype(np.int64)) % 2 == s, axis=1)
    return xs[ok]


@pytest.mark.parametrize("seed", range(8))
def test_sum_product_exact_on_trees(oracle_lib, seed):
    h, p, s = _tree_case(seed, 8 + seed % 7)
    n = h.shape[1]
    xs = _consistent(h, s)
    logw = xs @ np.log(p) + (1 - xs) @ np.log(1 - p)
    w = np.exp(logw)
    exact = np.array([np.log(w[xs[:, j] == 0].sum() / w[xs[:, j] == 1].sum()) for j in range(n)])
    llr, hard, used, conv = oracle_lib.bp(h, p, s[None], iters=2 * n, method=1, early_exit=0)
    assert used[0] == 2 * n
    np.testing.assert_allclose(llr[0], exact, rtol=1e-9, atol=1e-9)


@pytest.mark.parametrize("seed", range(16))
def test_sum_product_fp32_mirror_exact_on_trees(oracle_lib, seed):
    """The FP32 mirror of sum-product against exact inference on the float-rounded
    probabilities.  Bound: each message is at most 14 tanh products and one atanh, each
    rounded to 2^-24 relative, amplified by atanh's condition number (<= 10 for products up
    to tanh(2) ~ 0.96) along a path of at most 14 edges, on LLRs of magnitude <= 5:
    14 * 10 * 2^-24 * 5 ~ 4e-5; a dropped term or a flipped sign is off by 0.1 or more."""
    h, p, s = _tree_case(seed, 8 + seed % 7)
    n = h.shape[1]
    p32 = p.astype(np.float32).astype(np.float64)
    xs = _consistent(h, s)
    w = np.exp(xs @ np.log(p32) + (1 - xs) @ np.log(1 - p32))
    exact = np.array([np.log(w[xs[:, j] == 0].sum() / w[xs[:, j] == 1].sum()) for j in range(n)])
    assert np.abs(exact).max() <= 5.5
    llr, hard, used, conv = oracle_lib.bp(h, p, s[None], iters=2 * n, method=1, early_exit=0,
                                          precision=1)
    np.testing.assert_allclose(llr[0], exact, rtol=0, atol=5e-5)


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 2e-5)])
@pytest.mark.parametrize("seed", range(8))
def test_min_sum_alpha1_exact_on_trees(oracle_lib, seed, precision, tol):
    h, p, s = _tree_case(50 + seed, 8 + seed % 7)
    n = h.shape[1]
    lam = np.log((1 - p) / p)
    xs = _consistent(h, s)
    cost = xs @ lam
    exact = np.array([cost[xs[:, j] == 1].min() - cost[xs[:, j] == 0].min() for j in range(n)])
    llr, *_ = oracle_lib.bp(h, p, s[None], iters=2 * n, alpha=1.0, method=0, early_exit=0,
                           precision=precision)
    np.testing.assert_allclose(llr[0], exact, rtol=tol, atol=tol)


@pytest.mark.parametrize("deg", [2, 3, 4, 6, 7])
@pytest.mark.parametrize("syn", [0, 1])
def test_single_check_closed_form(oracle_lib, deg, syn):
    g = I.Xoshiro256ss(77 + deg, np.arange(deg, dtype=np.uint64))
    p = 0.05 + 0.9 * g.uniform()  # both signs of lambda
    h = np.ones((1, deg), np.uint8)
    lam = np.log((1 - p) / p)
    exp = np.empty(deg)
    for j in range(deg):
        others = np.delete(lam, j)
        sign = (-1) ** syn * np.prod(np.where(others < 0, -1.0, 1.0))
        exp[j] = lam[j] + sign * 0.625 * np.abs(others).min()
    llr, *_ = oracle_lib.bp(h, p, np.array([[syn]]), iters=1, early_exit=0)
    np.testing.assert_allclose(llr[0], exp, rtol=1e-14, atol=1e-14)
    # FP32 mirror: one float multiply and one float add
    lam32 = lam.astype(np.float32)
    exp32 = np.empty(deg, np.float32)
    for j in range(deg):
        others = np.delete(lam32, j)
        neg = (syn + int((others < 0).sum())) % 2
        mag = np.float32(0.625) * np.abs(others).min()
        exp32[j] = lam32[j] + (np.float32(-mag) if neg else np.float32(mag))
    llr32, *_ = oracle_lib.bp(h, p, np.array([[syn]]), iters=1, early_exit=0, precision=1)
    assert np.array_equal(llr32[0].astype(np.float32), exp32)


def test_priors(oracle_lib):
    p = np.array([0.5, 0.25, 0.05, 1e-3])
    np.testing.assert_allclose(oracle_lib.priors(p), [0.0, np.log(3.0), np.log(19.0), np.log(999.0)],
                               rtol=1e-15)
    assert np.array_equal(oracle_lib.priors(p, 1), np.log((1 - p) / p).astype(np.float32))


def test_early_exit_and_convergence(oracle_lib):
    hx, _ = I.bb72()
    p = np.full(72, 0.05)
    s = np.zeros((1, 36), np.uint8)
    llr, hard, used, conv = oracle_lib.bp(hx, p, s, iters=30)
    assert used[0] == 1 and conv[0] == 1 and not hard.any()
    e = I.sample_errors(3, 200, p)
    syn = I.syndromes(hx, e)
    llr, hard, used, conv = oracle_lib.bp(hx, p, syn, iters=30, precision=1)
    sat = np.all((hard.astype(int) @ hx.T) % 2 == syn, axis=1)
    assert np.array_equal(sat, conv.astype(bool))
    assert np.all(used[conv == 0] == 30)
    assert np.array_equal(hard, (llr < 0).astype(np.uint8))


def test_fp32_mirror_tracks_double(oracle_lib):
    """Same iteration count -> the FP32 mirror is within float rounding of the double run."""
    hx, _ = I.bb144()
    p = np.full(144, 0.04)
    e = I.sample_errors(5, 300, p)
    syn = I.syndromes(hx, e)
    l64, _, u64, _ = oracle_lib.bp(hx, p, syn, iters=10, precision=0)
    l32, _, u32, _ = oracle_lib.bp(hx, p, syn, iters=10, precision=1)
    same = u64 == u32
    assert same.mean() > 0.9
    d = np.abs(l64[same] - l32[same]) / np.maximum(1.0, np.abs(l64[same]))
    assert d.max() < 1e-4
