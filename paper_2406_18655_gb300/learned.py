"""Training helpers of the learned prior (lsd_prior_* in include/lsd.h).

Host-side orchestration only: the parameters are initialised here, every training pair is
sampled on the device (lsd_sample) and every forward, backward and Adam step runs in the
library's kernels.
"""
from __future__ import annotations

import numpy as np

HIDDEN = 32

# Flat parameter order of the C ABI.
PARAM_SHAPES = [("a0", (HIDDEN,)), ("a1", (HIDDEN,)), ("u0", (HIDDEN,)), ("u1", (HIDDEN,)),
                ("W1_cv", (HIDDEN, 2 * HIDDEN + 1)), ("b1_cv", (HIDDEN,)),
                ("W2_cv", (HIDDEN, HIDDEN)), ("b2_cv", (HIDDEN,)),
                ("W1_vc", (HIDDEN, 2 * HIDDEN + 1)), ("b1_vc", (HIDDEN,)),
                ("W2_vc", (HIDDEN, HIDDEN)), ("b2_vc", (HIDDEN,)),
                ("w_o", (HIDDEN,)), ("b_o", (1,))]


def init_params(seed: int, scale2: float = 0.1, hd: int = HIDDEN) -> np.ndarray:
    """Seeded initialisation: fan-in uniform first layers, second layers scaled by `scale2`,
    zero output weights, so the untrained prior returns the channel prior exactly.

    Flat, in the C ABI's parameter order, float32.  `hd` other than 32 is for small CPU
    models only (the kernels are built for a hidden width of 32)."""
    rng = np.random.default_rng(seed)
    parts = {}
    din = 2 * hd + 1
    parts["a0"] = rng.uniform(-1, 1, hd)
    parts["a1"] = rng.uniform(0, 0.5, hd)
    parts["u0"] = rng.uniform(-1, 1, hd)
    parts["u1"] = rng.uniform(-0.1, 0.1, hd)
    for d in ("cv", "vc"):
        parts["W1_" + d] = rng.uniform(-1, 1, (hd, din)) / np.sqrt(din)
        parts["b1_" + d] = np.zeros(hd)
        parts["W2_" + d] = rng.uniform(-1, 1, (hd, hd)) / np.sqrt(hd) * scale2
        parts["b2_" + d] = np.zeros(hd)
    parts["w_o"] = np.zeros(hd)
    parts["b_o"] = np.zeros(1)
    return np.concatenate([parts[k].ravel() for k, _ in PARAM_SHAPES]).astype(np.float32)


def train(decoder, prior, pairs: int, batch: int = 4096, seed: int = 1, lr: float = 3e-3,
          log_every: int = 0):
    """Adam on `pairs` device-sampled (error, syndrome) pairs at the decoder's channel
    probabilities; learning rate lr for 70 % of the steps, lr/3 then lr/10.

    Returns dict(steps, pairs, seconds, pairs_per_s, losses) with the device time of the loop.
    """
    import torch
    steps = max(1, pairs // batch)
    losses = []
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    stream = decoder.stream
    start.record(stream)
    for k in range(steps):
        e, s = decoder.sample(seed, batch, first_shot=k * batch)
        frac = k / steps
        rate = lr if frac < 0.7 else (lr / 3 if frac < 0.9 else lr / 10)
        want = bool(log_every) and (k % log_every == 0 or k == steps - 1)
        loss = prior.train_step(s, e, rate, want_loss=want)
        if want:
            losses.append((k, loss))
    end.record(stream)
    end.synchronize()
    secs = start.elapsed_time(end) / 1000.0
    return {"steps": steps, "pairs": steps * batch, "seconds": secs,
            "pairs_per_s": steps * batch / secs, "losses": losses}
