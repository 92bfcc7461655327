"""Learned-prior oracle (float64 numpy) pinned by finite differences and closed forms (no GPU)."""
import json
import os

import numpy as np
import pytest

from oracle import prior as P
from paper_2406_18655_gb300.learned import init_params
from paper_2406_18655_gb300 import inputs as I


def _case(seed, shots=3, p=0.08):
    h = I.bb72()[0]
    e = I.sample_errors(seed, shots, np.full(72, p))
    s = I.syndromes(h, e)
    lam = np.full(72, np.log((1 - p) / p))
    theta = init_params(seed).astype(np.float64)
    rng = np.random.default_rng(seed + 1)
    pp = P.unflatten(theta)
    pp["w_o"] = rng.normal(0, 0.3, 32)
    pp["b_o"] = np.array([0.1])
    for d in ("cv", "vc"):
        pp["b1_" + d] = rng.normal(0, 0.1, 32)
        pp["b2_" + d] = rng.normal(0, 0.05, 32)
    return h, e, s, lam, P.flatten(pp)


def test_num_params():
    assert P.num_params(32) == 4 * 32 + 2 * (32 * 65 + 32 + 32 * 32 + 32) + 32 + 1


@pytest.mark.parametrize("seed", [1, 2])
def test_gradient_matches_finite_differences(seed):
    h, e, s, lam, theta = _case(seed)
    loss, grad, _ = P.loss_and_grad(h, theta, s, e, lam, rounds=4)
    rng = np.random.default_rng(100 + seed)
    # coordinates from every parameter group
    idx, off = [], 0
    for name, shp in P.param_shapes():
        k = int(np.prod(shp))
        idx += list(off + rng.choice(k, size=min(k, 4), replace=False))
        off += k
    eps = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += eps
        tm[i] -= eps
        lp = P.loss_and_grad(h, tp, s, e, lam)[0]
        lm = P.loss_and_grad(h, tm, s, e, lam)[0]
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - grad[i]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (i, fd, grad[i])


def test_untrained_output_is_the_channel_prior():
    h, e, s, lam, theta = _case(3)
    pp = P.unflatten(theta)
    pp["w_o"][:] = 0
    pp["b_o"][:] = 0
    llr, _ = P.forward(P.Graph(h), P.flatten(pp), s, lam)
    assert np.array_equal(llr, np.broadcast_to(lam, llr.shape))
    loss, _ = P.loss_and_dllr(llr, e)
    # mean binary cross-entropy of the prior: -[e log p + (1-e) log(1-p)]
    pr = 1 / (1 + np.exp(lam[0]))
    exp = -np.mean(e * np.log(pr) + (1 - e) * np.log(1 - pr))
    assert abs(loss - exp) < 1e-12


def test_zero_rounds_closed_form():
    h, e, s, lam, theta = _case(4)
    pp = P.unflatten(theta)
    llr, _ = P.forward(P.Graph(h), theta, s, lam, rounds=0)
    hv = np.maximum(lam[:, None] * pp["a0"] + pp["a1"], 0)
    exp = lam + hv @ pp["w_o"] + pp["b_o"][0]
    np.testing.assert_allclose(llr, np.broadcast_to(exp, llr.shape), rtol=1e-14)


def test_messages_follow_the_tanner_graph():
    """A check's syndrome only influences variables within 2R hops (R rounds of messages)."""
    h, e, s, lam, theta = _case(5, shots=1)
    s2 = s.copy()
    c = int(np.nonzero(s[0] == 0)[0][0])
    s2[0, c] = 1
    l1, _ = P.forward(P.Graph(h), theta, s, lam, rounds=1)
    l2, _ = P.forward(P.Graph(h), theta, s2, lam, rounds=1)
    changed = np.nonzero(np.abs(l1 - l2)[0] > 0)[0]
    # one round: check c reaches its own variables, and (through the var->check update of
    # round 1) nothing else yet reaches the output
    assert set(changed.tolist()) <= set(np.nonzero(h[c])[0].tolist())
    assert len(changed) > 0


def _golden_rounds():
    path = os.path.join(os.path.dirname(__file__), "golden", "prior_rounds_hand.json")
    with open(path) as f:
        return json.load(f)


@pytest.mark.parametrize("case", [0, 1])
@pytest.mark.parametrize("rounds", [1, 2])
def test_round_update_matches_hand_derivation(case, rounds):
    """One and two rounds of the model stated in include/lsd.h, worked out by hand with
    hidden width 2 (tests/golden/prior_rounds_hand.json holds the derivation): pins the
    order of the MLP input blocks, the h_v^{t+1} read of the check update, the biases, the
    orientation of W2 and the syndrome sign."""
    g = _golden_rounds()
    hd = g["hd"]
    theta = P.flatten({k: np.array(v, dtype=np.float64) for k, v in g["params"].items()}, hd)
    c = g["cases"][case]
    h = np.array(c["H"], np.uint8)
    llr, _ = P.forward(P.Graph(h), theta, np.array([c["syndrome"]], np.uint8),
                       np.array(c["lambda"], np.float64), rounds=rounds, hd=hd)
    # dyadic values throughout: float64 is exact
    assert np.array_equal(llr[0], np.array(c["llr"][str(rounds)], np.float64)), llr[0]
