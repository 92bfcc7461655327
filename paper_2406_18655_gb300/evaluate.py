"""Logical-error evaluation of decoder outputs (not part of the decoding path).

A residual r = e + e_hat with H_X r = 0 is harmless iff it lies in the row space of
H_Z, whose orthogonal complement is ker(H_Z).  So r is a logical failure iff
K r != 0 (mod 2) for a basis K of ker(H_Z).  K is computed once on the host; the
per-shot test is a float32 matrix product on the GPU (exact: sums stay below 2^24).
"""
from __future__ import annotations

import numpy as np


def gf2_nullspace(a: np.ndarray) -> np.ndarray:
    """Basis (rows) of {x : a x = 0 mod 2} by Gauss-Jordan elimination over GF(2)."""
    a = (np.asarray(a, dtype=np.uint8) & 1).copy()
    m, n = a.shape
    pivots = []
    row = 0
    for col in range(n):
        if row >= m:
            break
        hit = np.nonzero(a[row:, col])[0]
        if hit.size == 0:
            continue
        r = row + hit[0]
        if r != row:
            a[[row, r]] = a[[r, row]]
        others = np.nonzero(a[:, col])[0]
        others = others[others != row]
        a[others] ^= a[row]
        pivots.append(col)
        row += 1
    free = [c for c in range(n) if c not in set(pivots)]
    basis = np.zeros((len(free), n), np.uint8)
    for k, f in enumerate(free):
        basis[k, f] = 1
        for i, pc in enumerate(pivots):
            basis[k, pc] = a[i, f]
    return basis


class LogicalChecker:
    """Counts logical failures of corrections on the GPU for a CSS code (H_X decodes)."""

    def __init__(self, hz: np.ndarray, device="cuda"):
        import torch
        k = gf2_nullspace(hz)
        self.k = torch.from_numpy(k.T.astype(np.float32)).to(device)

    def failures(self, errors, corrections):
        """errors, corrections: uint8 [shots][n] CUDA tensors -> bool [shots]."""
        import torch
        r = (errors ^ corrections).float()
        v = torch.remainder(r @ self.k, 2.0)
        return v.any(dim=1)
