"""Seeded workloads shared by the GPU tests (inputs only; no decoding arithmetic)."""
import numpy as np

from paper_2406_18655_gb300 import inputs as I

_CACHE = {}


def code(name):
    """Dense check matrix (uint8) of a named synthetic workload."""
    if name in _CACHE:
        return _CACHE[name]
    if name == "bb72":
        h = I.bb72()[0]
    elif name == "bb144":
        h = I.bb144()[0]
    elif name == "bb288":
        h = I.bb288()[0]
    elif name == "st_bb72_d6":
        h = I.space_time(I.bb72()[0], 6)
    elif name == "st_bb144_d12":
        h = I.space_time(I.bb144()[0], 12)
    elif name == "st_bb288_d18":
        h = I.space_time(I.bb288()[0], 18)
    elif name == "rep_boundary":
        # repetition-like code whose first check has degree 1 (min over an empty set in BP)
        n = 12
        h = np.zeros((n, n), np.uint8)
        h[0, 0] = 1
        for i in range(1, n):
            h[i, i - 1] = h[i, i] = 1
    elif name == "hgp":
        h = I.hgp_48x64()[0]
    elif name == "ldpc_96x192":
        # (3,6)-regular, girth >= 6: the 96-detector / 192-fault LSD class (shuffle ranks of
        # six keys per lane)
        h = I.random_regular_ldpc(96, 192, 3, 6, seed=3)
    elif name == "ldpc_480x960":
        # the largest dense LSD class (512 x 2048: bitonic sort, no candidate masks, 16-word
        # elimination rows)
        h = I.random_regular_ldpc(480, 960, 3, 6, seed=4)
    elif name == "irreg_37x61":
        # irregular degrees, sizes off the 16-row tiles: column j has weight 1 + j % 4
        rng = np.random.default_rng(5)
        h = np.zeros((37, 61), np.uint8)
        for j in range(61):
            h[rng.choice(37, 1 + j % 4, replace=False), j] = 1
    else:
        raise KeyError(name)
    _CACHE[name] = h
    return h


def logicals_hz(name):
    if name == "bb72":
        return I.bb72()[1]
    if name == "bb144":
        return I.bb144()[1]
    if name == "bb288":
        return I.bb288()[1]
    raise KeyError(name)


def sample(name, p, shots, seed):
    """(H, probs float32 [n], errors [shots][n], syndromes [shots][m])."""
    h = code(name)
    probs = np.full(h.shape[1], p, np.float32)
    e = I.sample_errors(seed, shots, probs.astype(np.float64))
    return h, probs, e, I.syndromes(h, e)
