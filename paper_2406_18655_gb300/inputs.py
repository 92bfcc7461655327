"""Seeded synthetic inputs: check matrices and i.i.d. fault samples.

This module is shared by the CPU oracle's tests and by the GPU path's tests and
benchmark.  It only *produces inputs* (codes, errors, syndromes); it holds none
of the decoder's arithmetic (no BP, no cluster growth, no GF(2) elimination).

Codes
-----
* Bivariate bicycle (BB) codes (the code family decoded in the paper's
  BB experiments, App. C.3): x = S_l (x) I_m, y = I_l (x) S_m with S the
  cyclic shift, A and B sums of three monomials, H_X = [A | B],
  H_Z = [B^T | A^T].
* Hypergraph product (HGP) of a seeded (3,4)-regular classical matrix with
  girth >= 6 (the random family of App. C.2).
* A phenomenological space-time matrix ("[H | I] stacked per round") with d
  noisy rounds and one noiseless final round.

Randomness
----------
splitmix64 seeds xoshiro256** (Blackman and Vigna, "Scrambled linear
pseudorandom number generators", 2018), one stream per shot, so any shot range
can be regenerated independently.  A Bernoulli(p) draw is
``u = (x >> 11) * 2**-53 < p`` evaluated in double precision.
"""
from __future__ import annotations

import numpy as np

_U64 = np.uint64
_GOLDEN = _U64(0x9E3779B97F4A7C15)
_SM_M1 = _U64(0xBF58476D1CE4E5B9)
_SM_M2 = _U64(0x94D049BB133111EB)
_STREAM_MIX = _U64(0xD1B54A32D192ED03)


def _rotl(x: np.ndarray, k: int) -> np.ndarray:
    return (x << _U64(k)) | (x >> _U64(64 - k))


class Xoshiro256ss:
    """Vectorised xoshiro256** with one independent stream per entry of ``stream_ids``."""

    def __init__(self, seed: int, stream_ids: np.ndarray):
        ids = np.asarray(stream_ids, dtype=np.uint64)
        x = _U64(seed & 0xFFFFFFFFFFFFFFFF) ^ ((ids + _U64(1)) * _STREAM_MIX)
        s = []
        for _ in range(4):
            x = x + _GOLDEN
            z = x
            z = (z ^ (z >> _U64(30))) * _SM_M1
            z = (z ^ (z >> _U64(27))) * _SM_M2
            s.append(z ^ (z >> _U64(31)))
        self.s0, self.s1, self.s2, self.s3 = s

    def next_u64(self) -> np.ndarray:
        result = _rotl(self.s1 * _U64(5), 7) * _U64(9)
        t = self.s1 << _U64(17)
        self.s2 ^= self.s0
        self.s3 ^= self.s1
        self.s1 ^= self.s2
        self.s0 ^= self.s3
        self.s2 ^= t
        self.s3 = _rotl(self.s3, 45)
        return result

    def uniform(self) -> np.ndarray:
        return (self.next_u64() >> _U64(11)).astype(np.float64) * (2.0 ** -53)


# ----------------------------------------------------------------------------
# Codes
# ----------------------------------------------------------------------------

def _shift(k: int) -> np.ndarray:
    s = np.zeros((k, k), dtype=np.uint8)
    s[np.arange(k), (np.arange(k) + 1) % k] = 1
    return s


def _mat_power(a: np.ndarray, e: int) -> np.ndarray:
    out = np.eye(a.shape[0], dtype=np.int64)
    for _ in range(e):
        out = (out @ a) % 2
    return out.astype(np.uint8)


def bb_code(l: int, m: int, a_terms, b_terms):
    """Bivariate bicycle code.  ``a_terms``/``b_terms`` are lists of ('x'|'y', power).

    Returns (H_X, H_Z) as dense uint8 arrays of shape (l*m, 2*l*m).
    """
    x = np.kron(_shift(l), np.eye(m, dtype=np.uint8))
    y = np.kron(np.eye(l, dtype=np.uint8), _shift(m))

    def poly(terms):
        acc = np.zeros((l * m, l * m), dtype=np.int64)
        for var, p in terms:
            acc += _mat_power(x if var == "x" else y, p)
        return (acc % 2).astype(np.uint8)

    a = poly(a_terms)
    b = poly(b_terms)
    hx = np.concatenate([a, b], axis=1)
    hz = np.concatenate([b.T, a.T], axis=1)
    return hx, hz


def bb72():
    """[[72,12,6]]: l=6, m=6, A = x^3 + y + y^2, B = y^3 + x + x^2."""
    return bb_code(6, 6, [("x", 3), ("y", 1), ("y", 2)], [("y", 3), ("x", 1), ("x", 2)])


def bb144():
    """[[144,12,12]]: l=12, m=6, A = x^3 + y + y^2, B = y^3 + x + x^2."""
    return bb_code(12, 6, [("x", 3), ("y", 1), ("y", 2)], [("y", 3), ("x", 1), ("x", 2)])


def bb288():
    """[[288,12,18]]: l=12, m=12, A = x^3 + y^2 + y^7, B = y^3 + x + x^2."""
    return bb_code(12, 12, [("x", 3), ("y", 2), ("y", 7)], [("y", 3), ("x", 1), ("x", 2)])


def random_regular_ldpc(rows: int, cols: int, col_w: int, row_w: int, seed: int,
                        max_attempts: int = 2000) -> np.ndarray:
    """Seeded (col_w, row_w)-regular matrix with no repeated edge and no 4-cycle (girth >= 6).

    Columns are placed one at a time; each column draws ``col_w`` distinct rows with
    spare capacity, never two rows that an earlier column already shares.  A dead
    end restarts the construction with the next draws of the same stream.
    """
    assert rows * row_w == cols * col_w
    gen = Xoshiro256ss(seed, np.array([0], dtype=np.uint64))

    def draw(k: int) -> int:
        return int(gen.next_u64()[0] % np.uint64(k))

    for _ in range(max_attempts):
        h = np.zeros((rows, cols), dtype=np.uint8)
        cap = [row_w] * rows
        # pair[r1][r2]: some earlier column already holds both rows (a second one
        # would close a 4-cycle)
        pair = [[False] * rows for _ in range(rows)]
        ok = True
        for c in range(cols):
            chosen: list[int] = []
            for _k in range(col_w):
                allowed = [r for r in range(rows)
                           if cap[r] > 0 and r not in chosen
                           and not any(pair[r][r2] for r2 in chosen)]
                if not allowed:
                    ok = False
                    break
                # weight by remaining capacity so the last columns do not starve
                weights = [cap[r] for r in allowed]
                pick = draw(sum(weights))
                acc = 0
                for r, w in zip(allowed, weights):
                    acc += w
                    if pick < acc:
                        chosen.append(r)
                        break
            if not ok:
                break
            for r in chosen:
                h[r, c] = 1
                cap[r] -= 1
            for r1 in chosen:
                for r2 in chosen:
                    if r1 != r2:
                        pair[r1][r2] = True
        if ok and all(v == 0 for v in cap):
            return h
    raise RuntimeError("random_regular_ldpc: no girth-6 instance found")


def hgp(h: np.ndarray):
    """Hypergraph product of ``h`` (r x c) with itself.

    H_X = [h (x) I_c | I_r (x) h^T]  ((r*c) x (c*c + r*r)),
    H_Z = [I_c (x) h | h^T (x) I_r].
    """
    r, c = h.shape
    hx = np.concatenate([np.kron(h, np.eye(c, dtype=np.uint8)),
                         np.kron(np.eye(r, dtype=np.uint8), h.T)], axis=1) % 2
    hz = np.concatenate([np.kron(np.eye(c, dtype=np.uint8), h),
                         np.kron(h.T, np.eye(r, dtype=np.uint8))], axis=1) % 2
    return hx.astype(np.uint8), hz.astype(np.uint8)


def hgp_coo(h: np.ndarray):
    """H_X of :func:`hgp` as a COO list, for products too large to hold densely:
    returns (m, n, rows, cols) with rows, cols int32 in row-major order."""
    h = np.asarray(h, dtype=np.uint8)
    r, c = h.shape
    hi, hj = np.nonzero(h)                       # block h (x) I_c
    t = np.arange(c)
    rows1 = (hi[:, None] * c + t[None, :]).ravel()
    cols1 = (hj[:, None] * c + t[None, :]).ravel()
    ta, tb = np.nonzero(h.T)                     # block I_r (x) h^T
    u = np.arange(r)
    rows2 = (u[:, None] * c + ta[None, :]).ravel()
    cols2 = (c * c + u[:, None] * r + tb[None, :]).ravel()
    rows = np.concatenate([rows1, rows2]).astype(np.int64)
    cols = np.concatenate([cols1, cols2]).astype(np.int64)
    order = np.lexsort((cols, rows))
    return r * c, c * c + r * r, rows[order].astype(np.int32), cols[order].astype(np.int32)


def coo_syndrome(m: int, rows: np.ndarray, cols: np.ndarray, errors: np.ndarray) -> np.ndarray:
    """s = H e (mod 2) of one error vector for H given as a COO list; uint8 [m]."""
    w = errors.astype(np.int64)[cols]
    return (np.bincount(rows, weights=w, minlength=m).astype(np.int64) & 1).astype(np.uint8)


def hgp_48x64(seed: int = 2406):
    """HGP of a seeded (3,4)-regular 48x64 matrix: H_X is 3072 x 6400, row weight 7."""
    return hgp(random_regular_ldpc(48, 64, 3, 4, seed))


def space_time(h: np.ndarray, d: int) -> np.ndarray:
    """Phenomenological space-time check matrix of ``d`` noisy rounds plus a noiseless one.

    Detector block t (t = 0..d) is the difference of syndrome rounds t and t-1.
    Fault columns of round t (t = 0..d-1): first the n data faults (they flip
    detector block t through ``h``), then the m measurement faults (they flip
    detector blocks t and t+1).  Shape: ((d+1)*m) x (d*(n+m)).
    """
    m, n = h.shape
    out = np.zeros(((d + 1) * m, d * (n + m)), dtype=np.uint8)
    eye = np.eye(m, dtype=np.uint8)
    for t in range(d):
        c0 = t * (n + m)
        out[t * m:(t + 1) * m, c0:c0 + n] = h
        out[t * m:(t + 1) * m, c0 + n:c0 + n + m] = eye
        out[(t + 1) * m:(t + 2) * m, c0 + n:c0 + n + m] = eye
    return out


def space_time_hooks(h: np.ndarray, d: int, seed: int):
    """Space-time matrix with mid-round data faults, a synthetic stand-in for a
    circuit-level detector error model: weight-2 and weight-3 hyperedges across rounds.

    Per round t (t = 0..d-1) the columns are [n data | m measurement | n hook]: data and
    measurement faults as in :func:`space_time`; hook fault j of round t flips qubit j
    between the measurements of its checks, so a seeded subset of column j's checks (at
    least one, not all) fires in block t and the rest in block t+1.  Block d is the
    noiseless final round.  Returns (H, split) with split[t][j] the number of checks of
    qubit j (in ascending row order) that fire in block t.
    """
    h = np.asarray(h, dtype=np.uint8)
    m, n = h.shape
    F = 2 * n + m
    out = np.zeros(((d + 1) * m, d * F), dtype=np.uint8)
    eye = np.eye(m, dtype=np.uint8)
    gen = Xoshiro256ss(seed, np.arange(d * n, dtype=np.uint64))
    u = gen.uniform().reshape(d, n)
    split = np.zeros((d, n), np.int64)
    for t in range(d):
        c0 = t * F
        out[t * m:(t + 1) * m, c0:c0 + n] = h
        out[t * m:(t + 1) * m, c0 + n:c0 + n + m] = eye
        out[(t + 1) * m:(t + 2) * m, c0 + n:c0 + n + m] = eye
        for j in range(n):
            rows = np.nonzero(h[:, j])[0]
            k = 1 + int(u[t, j] * (rows.size - 1)) if rows.size > 1 else 1
            split[t, j] = k
            out[t * m + rows[:k], c0 + n + m + j] = 1
            out[(t + 1) * m + rows[k:], c0 + n + m + j] = 1
    return out, split


def space_time_hooks_probs(n: int, m: int, d: int, p: float, seed: int) -> np.ndarray:
    """Non-uniform priors for :func:`space_time_hooks`: data p, measurement p and hook p / 2,
    each scaled by a seeded factor in [0.25, 1.75) per column."""
    base = np.tile(np.concatenate([np.full(n, p), np.full(m, p), np.full(n, p / 2)]), d)
    g = Xoshiro256ss(seed, np.arange(base.size, dtype=np.uint64))
    return base * (0.25 + 1.5 * g.uniform())


def space_time_hooks_data_residual(residual: np.ndarray, n: int, m: int, d: int) -> np.ndarray:
    """Net data flip per qubit of a residual of :func:`space_time_hooks`: data and hook faults
    of every round, summed mod 2."""
    r = residual.reshape(residual.shape[0], d, 2 * n + m)
    return ((r[:, :, :n].sum(axis=1) + r[:, :, n + m:].sum(axis=1)) % 2).astype(np.uint8)


def space_time_probs(n: int, m: int, d: int, p: float, q: float) -> np.ndarray:
    """Per-column fault probabilities of :func:`space_time`: p for data, q for measurement."""
    block = np.concatenate([np.full(n, p), np.full(m, q)])
    return np.tile(block, d)


def space_time_data_residual(residual: np.ndarray, n: int, m: int, d: int) -> np.ndarray:
    """Sum (mod 2) over rounds of the data part of a space-time residual ``[shots][d*(n+m)]``."""
    r = residual.reshape(residual.shape[0], d, n + m)[:, :, :n]
    return (r.sum(axis=1) % 2).astype(np.uint8)


# ----------------------------------------------------------------------------
# Samples
# ----------------------------------------------------------------------------

def sample_errors(seed: int, shots: int, probs, first_shot: int = 0) -> np.ndarray:
    """i.i.d. faults: column j of shot k is 1 with probability probs[j].

    Shot k uses stream ``first_shot + k``; its draws are taken in ascending column order.
    Returns uint8 [shots][n].
    """
    probs = np.asarray(probs, dtype=np.float64)
    n = probs.shape[0]
    gen = Xoshiro256ss(seed, np.arange(first_shot, first_shot + shots, dtype=np.uint64))
    out = np.empty((shots, n), dtype=np.uint8)
    for j in range(n):
        out[:, j] = gen.uniform() < probs[j]
    return out


def syndromes(h: np.ndarray, errors: np.ndarray) -> np.ndarray:
    """s = H e (mod 2) for each row of ``errors``; uint8 [shots][m].

    Computed as a float32 product (exact: every count is below 2^24), in chunks.
    """
    ht = h.T.astype(np.float32)
    out = np.empty((errors.shape[0], h.shape[0]), dtype=np.uint8)
    step = 1 << 16
    for a in range(0, errors.shape[0], step):
        prod = errors[a:a + step].astype(np.float32) @ ht
        out[a:a + step] = (prod.astype(np.int64) & 1).astype(np.uint8)
    return out


def coo(h: np.ndarray):
    """(rows, cols) int32 arrays of the nonzeros of a dense 0/1 matrix, row-major order."""
    r, c = np.nonzero(h)
    return r.astype(np.int32), c.astype(np.int32)


def random_tree_tanner(seed: int, n_vars: int, max_check_deg: int = 4):
    """Random Tanner graph whose bipartite graph is a tree (used for BP exactness checks).

    Starts from variable 0; each new check joins one existing variable and 1..max_check_deg-1
    new variables until ``n_vars`` variables exist.  Every check has degree >= 2.
    Returns a dense uint8 H (m x n_vars).
    """
    gen = Xoshiro256ss(seed, np.array([0], dtype=np.uint64))

    def draw(k: int) -> int:
        return int(gen.next_u64()[0] % np.uint64(k))

    rows: list[list[int]] = []
    nv = 1
    while nv < n_vars:
        anchor = draw(nv)
        k = 1 + draw(max_check_deg - 1)
        k = min(k, n_vars - nv)
        new = list(range(nv, nv + k))
        nv += k
        rows.append([anchor] + new)
    h = np.zeros((len(rows), n_vars), dtype=np.uint8)
    for i, r in enumerate(rows):
        h[i, r] = 1
    return h
