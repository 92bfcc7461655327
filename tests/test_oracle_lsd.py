"""Oracle LSD pinned against worked examples, OSD-0, brute force and invariants (no GPU)."""
import itertools
import json
import os

import numpy as np
import pytest

from paper_2406_18655_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


@pytest.mark.parametrize("name", ["lsd_repetition_n5.json", "lsd_merge_into_valid.json"])
def test_worked_examples_lsd0(oracle_lib, name):
    d = _load(name)
    r = oracle_lib.lsd(np.array(d["H"]), np.array(d["syndrome"]), np.array(d["llr"]))
    assert r["status"][0] == 2
    assert r["corrections"][0].tolist() == d["correction"]
    assert (r["nu"][0], r["kappa"][0], r["steps"][0]) == (d["nu"], d["kappa"], d["steps"])


def test_worked_example_lsd_mu(oracle_lib):
    d = _load("lsd_mu1_repetition_n3.json")
    for order, key in ((0, "order0"), (1, "order1")):
        r = oracle_lib.lsd(np.array(d["H"]), np.array(d["syndrome"]), np.array(d["llr"]),
                           order=order, probs=d["channel_p"])
        exp = d[key]
        assert r["corrections"][0].tolist() == exp["correction"]
        assert (r["nu"][0], r["kappa"][0], r["steps"][0]) == (exp["nu"], exp["kappa"], exp["steps"])


def _bp_llrs(oracle_lib, h, p, shots, seed, iters=30):
    e = I.sample_errors(seed, shots, np.full(h.shape[1], p))
    s = I.syndromes(h, e)
    llr, hard, used, conv = oracle_lib.bp(h, p, s, iters=iters, precision=1)
    return e, s, llr, conv


@pytest.mark.parametrize("code,p", [("bb72", 0.04), ("bb72", 0.1), ("bb144", 0.06), ("bb144", 0.1)])
def test_lsd_invariants(oracle_lib, code, p):
    """Every correction satisfies H e = s (Eq. 2 with exact local solves); final clusters are
    detector-disjoint, closed (a fault's detectors lie in its cluster), valid (Def. 4.2), and
    nu / kappa count them."""
    h = getattr(I, code)()[0]
    e, s, llr, conv = _bp_llrs(oracle_lib, h, p, 120, seed=hash(code) % 1000 + int(p * 100))
    r = oracle_lib.lsd(h, s, llr, labels=True)
    assert np.all(r["status"] == 2)
    assert np.array_equal((r["corrections"].astype(int) @ h.T) % 2, s)
    for k in range(s.shape[0]):
        dl, fl = r["det_lab"][k], r["fault_lab"][k]
        assert np.all(dl[s[k] == 1] >= 0)  # every flipped detector is in a cluster
        labels = sorted(set(dl[dl >= 0].tolist()))
        assert len(labels) == r["nu"][k]
        sizes = [int((fl == c).sum()) for c in labels]
        assert max(sizes, default=0) == r["kappa"][k]
        corr = r["corrections"][k]
        assert np.all(fl[corr == 1] >= 0)
        for j in np.nonzero(fl >= 0)[0]:
            assert np.all(dl[np.nonzero(h[:, j])[0]] == fl[j])
        for c in labels:
            rows = np.nonzero(dl == c)[0]
            cols = np.nonzero(fl == c)[0]
            ok, _, _ = oracle_lib.gf2_solve(h[np.ix_(rows, cols)], s[k][rows])
            assert ok


@pytest.mark.parametrize("code,p,random_llr", [("bb72", 0.05, False), ("bb72", 0.08, True),
                                               ("bb144", 0.05, False), ("bb144", 0.03, True)])
def test_single_cluster_equals_osd0(oracle_lib, code, p, random_llr):
    """One cluster holding every detector grows in global reliability order and stops as soon
    as s is in the span: its solution is exactly OSD-0's (Sec. 2.2)."""
    h = getattr(I, code)()[0]
    e, s, llr, conv = _bp_llrs(oracle_lib, h, p, 40, seed=31)
    if random_llr:
        g = I.Xoshiro256ss(9, np.arange(llr.size, dtype=np.uint64))
        llr = np.round(g.uniform() * 6 - 1, 1).reshape(llr.shape)
    r = oracle_lib.lsd(h, s, llr, single_cluster=True)
    assert np.all(r["status"] == 2)
    for k in range(s.shape[0]):
        ok, out = oracle_lib.osd0(h, s[k], llr[k])
        assert ok
        assert np.array_equal(r["corrections"][k], out)


@pytest.mark.parametrize("order", [1, 6, 10])
def test_lsd_mu_never_worse_than_lsd0(oracle_lib, order):
    h = I.bb72()[0]
    p = 0.08
    e, s, llr, conv = _bp_llrs(oracle_lib, h, p, 80, seed=41)
    r0 = oracle_lib.lsd(h, s, llr, order=0)
    rm = oracle_lib.lsd(h, s, llr, order=order, probs=p)
    assert np.all(rm["status"] == 2)
    assert np.array_equal((rm["corrections"].astype(int) @ h.T) % 2, s)
    # uniform channel weights: cost is proportional to Hamming weight
    assert np.all(rm["corrections"].sum(1) <= r0["corrections"].sum(1))
    assert np.all(rm["kappa"] >= r0["kappa"])


def test_lsd_mu_exhaustive_on_small_clusters(oracle_lib):
    """When mu covers every non-pivot column of a cluster, OSD-E is the exact minimum-cost
    solution over the cluster's coset (brute force over all local corrections)."""
    h = I.bb72()[0]
    p = np.full(72, 0.03)
    g = I.Xoshiro256ss(123, np.arange(72, dtype=np.uint64))
    p = 0.01 + 0.08 * g.uniform()  # non-uniform channel, so costs differ from weights
    e = I.sample_errors(17, 200, p)
    s = I.syndromes(h, e)
    llr, hard, used, conv = oracle_lib.bp(h, p, s, iters=30, precision=1)
    w = np.round(np.log((1 - p) / p).astype(np.float32).astype(np.float64) * 2 ** 32)
    order = 10
    r = oracle_lib.lsd(h, s, llr, order=order, probs=p, labels=True)
    checked = 0
    for k in range(s.shape[0]):
        dl, fl = r["det_lab"][k], r["fault_lab"][k]
        for c in sorted(set(dl[dl >= 0].tolist())):
            rows = np.nonzero(dl == c)[0]
            cols = np.nonzero(fl == c)[0]
            sub = h[np.ix_(rows, cols)]
            nonpiv = len(cols) - oracle_lib.gf2_rank(sub)
            if nonpiv > order or len(cols) > 16:
                continue
            xs = ((np.arange(2 ** len(cols))[:, None] >> np.arange(len(cols))[None, :]) & 1)
            ok = np.all((xs @ sub.T.astype(np.int64)) % 2 == s[k][rows], axis=1)
            best = (xs[ok] @ w[cols]).min()
            got = r["corrections"][k][cols].astype(np.int64) @ w[cols]
            assert got == best
            checked += 1
    assert checked > 20


def _cs_patterns(nonpiv: int, w: int):
    """Combination sweep of order w over nonpiv ranked non-pivot columns: no flip, every single
    column, every pair among the first w (App. D, OSD-CS-w)."""
    pats = [()] + [(k,) for k in range(nonpiv)]
    return pats + list(itertools.combinations(range(min(w, nonpiv)), 2))


@pytest.mark.parametrize("w", [0, 2, 4, 7])
def test_osd_cs_brute_force_single_cluster(oracle_lib, w):
    """With one cluster grown over every column (mu >= n), the combination sweep returns the
    least-cost solution of H e = s among those whose non-pivot part is one of the sweep's
    patterns; pivots are the first independent columns in reliability order.  Brute force over
    all 2^n vectors, written from that definition alone."""
    g = I.Xoshiro256ss(77 + w, np.arange(4, dtype=np.uint64))
    checked = 0
    for trial in range(12):
        m, n = 6, 13
        rng = np.random.default_rng(1000 * w + trial)
        h = (rng.random((m, n)) < 0.35).astype(np.uint8)
        h[:, :m] |= np.eye(m, dtype=np.uint8)  # full row rank, every syndrome solvable
        h = h[:, rng.permutation(n)]
        zero = np.nonzero(h.sum(0) == 0)[0]  # a column on no detector never joins a cluster
        h[rng.integers(0, m, zero.size), zero] = 1
        p = rng.uniform(0.01, 0.2, n)
        wfix = np.round(np.log((1 - p) / p).astype(np.float32).astype(np.float64) * 2 ** 32)
        shots = 6
        s = rng.integers(0, 2, (shots, m)).astype(np.uint8)
        llr = np.round(rng.uniform(-2, 6, (shots, n)), 3)
        r = oracle_lib.lsd(h, s, llr, order=n, osd_cs=w, probs=p, single_cluster=True)
        assert np.all(r["status"] == 2)
        xs = ((np.arange(2 ** n)[:, None] >> np.arange(n)[None, :]) & 1).astype(np.int64)
        for k in range(shots):
            if not s[k].any():
                assert not r["corrections"][k].any()
                continue
            order = sorted(range(n), key=lambda j: (llr[k][j], j))
            piv, nonpiv = [], []
            for j in order:
                cand = piv + [j]
                if oracle_lib.gf2_rank(h[:, cand]) == len(cand):
                    piv.append(j)
                else:
                    nonpiv.append(j)
            ok = np.all((xs @ h.T.astype(np.int64)) % 2 == s[k], axis=1)
            best, best_x = None, None
            for pat in _cs_patterns(len(nonpiv), w):
                want = np.zeros(n, np.int64)
                want[[nonpiv[i] for i in pat]] = 1
                sel = ok & np.all(xs[:, nonpiv] == want[nonpiv], axis=1)
                assert sel.sum() == 1  # pivots form a basis of the column space
                x = xs[sel][0]
                cost = x @ wfix
                if best is None or cost < best:
                    best, best_x = cost, x
            assert np.array_equal(r["corrections"][k].astype(np.int64), best_x)
            checked += 1
    assert checked > 50


def _cost(corr, wfix):
    return corr.astype(np.int64) @ wfix.astype(np.int64)


def test_osd_cs_orders_nest(oracle_lib):
    """The sweeps nest: the patterns of OSD-CS-w contain those of OSD-CS-w' for w' < w, and at
    mu = 2 those of OSD-E-2, on the same clusters (growth does not depend on the local
    reprocessing), so the total cost can only fall along that chain."""
    h = I.bb72()[0]
    g = I.Xoshiro256ss(5, np.arange(72, dtype=np.uint64))
    g.uniform()
    p = 0.02 + 0.14 * g.uniform()
    e = I.sample_errors(23, 160, p)
    s = I.syndromes(h, e)
    llr, hard, used, conv = oracle_lib.bp(h, p, s, iters=30, precision=1)
    wfix = np.round(np.log((1 - p) / p).astype(np.float32).astype(np.float64) * 2 ** 32)
    runs = {}
    for key, kw in {"E2": dict(order=2), "CS0": dict(order=2, osd_cs=0),
                    "CS2": dict(order=2, osd_cs=2), "CS4": dict(order=2, osd_cs=4)}.items():
        r = oracle_lib.lsd(h, s, llr, probs=p, labels=True, **kw)
        assert np.all(r["status"] == 2)
        assert np.array_equal((r["corrections"].astype(int) @ h.T) % 2, s)
        runs[key] = r
    for a in ("CS0", "CS2", "CS4"):
        assert np.array_equal(runs[a]["fault_lab"], runs["E2"]["fault_lab"])
    cost = {k: np.array([_cost(c, wfix) for c in r["corrections"]]) for k, r in runs.items()}
    assert np.all(cost["CS2"] <= cost["E2"])
    assert np.all(cost["CS2"] <= cost["CS0"])
    assert np.all(cost["CS4"] <= cost["CS2"])
    assert np.any(cost["CS4"] < cost["E2"])  # the sweep reaches further than OSD-E-2


def test_osd_cs_without_mu_is_lsd0(oracle_lib):
    """mu = 0 means no reprocessing whatever the sweep order."""
    h = I.bb72()[0]
    e, s, llr, conv = _bp_llrs(oracle_lib, h, 0.08, 60, seed=3)
    r0 = oracle_lib.lsd(h, s, llr)
    r1 = oracle_lib.lsd(h, s, llr, osd_cs=4)
    assert np.array_equal(r0["corrections"], r1["corrections"])


def test_unsolvable_syndrome(oracle_lib):
    """s outside image(H): the cluster exhausts its component and LSD reports status 3."""
    h = np.array([[1, 1, 0], [1, 1, 0], [0, 0, 1]], np.uint8)  # rows 0 and 1 are equal
    s = np.array([1, 0, 0], np.uint8)
    llr = np.array([1.0, 2.0, 3.0])
    r = oracle_lib.lsd(h, s, llr)
    assert r["status"][0] == 3 and not r["corrections"].any()


def test_decode_pipeline(oracle_lib):
    """BP first; LSD only when BP's hard decision fails (App. C.4)."""
    h = I.bb144()[0]
    p = 0.06
    e = I.sample_errors(23, 300, np.full(144, p))
    s = I.syndromes(h, e)
    d = oracle_lib.decode(h, p, s, bp_iters=50, precision=1, want_llr=True)
    assert np.array_equal((d["corrections"].astype(int) @ h.T) % 2, s)
    bp_ok = d["status"] == 1
    assert bp_ok.any() and (~bp_ok).any()
    assert np.array_equal(d["corrections"][bp_ok], (d["llr"][bp_ok] < 0).astype(np.uint8))
    r = oracle_lib.lsd(h, s[~bp_ok], d["llr"][~bp_ok])
    assert np.array_equal(r["corrections"], d["corrections"][~bp_ok])
    assert np.all(d["bp_iters"][~bp_ok] == 50)
