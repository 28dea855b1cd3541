"""Training the subspace network on bases the method computes.

Orchestration only: every step (patch solves, inputs, targets, forward,
backward, Adam) runs in the library's kernels through the C ABI.  The
minibatch draws are passed in by the caller (``indices``), so that the
random numbers come from the caller's seeded generator.
"""
from __future__ import annotations

import math
import time
from typing import Callable, List, Sequence, Tuple

import numpy as np

from . import MLP, Mesh


def training_set(scenes: Sequence, chunk: int = 256, stream=None):
    """Network inputs and targets of every free vertex of ``scenes``.

    The meshes are processed ``chunk`` at a time as one disjoint union:
    colouring, computed k = 2 bases (Eq. 5 on the 2-ring, at rest), then
    inputs X [N, 264] (bfloat16) and targets T [N, 576] (float32), both on
    the GPU.  Returns (X, T, rows per scene)."""
    import torch
    Xs, Ts, counts = [], [], []
    for c0 in range(0, len(scenes), chunk):
        part = list(scenes[c0:c0 + chunk])
        m = Mesh.from_scenes(part, stream=stream)
        try:
            m.color()
            m.build_subspace(2)
            X, T = m.learned_inputs(targets=True)
        finally:
            m.close()
        Xs.append(X)
        Ts.append(T)
        counts += [int((sc.pinned == 0).sum()) for sc in part]
    return torch.cat(Xs), torch.cat(Ts), np.array(counts, dtype=np.int64)


def train(net: MLP, X, T, indices: Callable[[int, int, int, int], np.ndarray], steps: int, batch: int,
          lr: float = 1e-3, lr_final: float = 1e-5, chunk_steps: int = 250) -> Tuple[np.ndarray, float]:
    """``steps`` Adam steps with a cosine learning-rate schedule from ``lr`` to
    ``lr_final`` (constant within each chunk of ``chunk_steps`` steps).
    ``indices(step0, count, batch, n)`` returns the int32 sample indices
    [count, batch] of steps step0 .. step0 + count - 1.  Returns (losses,
    seconds)."""
    import torch
    n = X.shape[0]
    losses: List[np.ndarray] = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for s0 in range(0, steps, chunk_steps):
        cnt = min(chunk_steps, steps - s0)
        frac = (s0 + 0.5 * cnt) / max(steps, 1)
        lr_c = lr_final + 0.5 * (lr - lr_final) * (1.0 + math.cos(math.pi * frac))
        idx = torch.from_numpy(np.ascontiguousarray(indices(s0, cnt, batch, n), dtype=np.int32)).cuda()
        losses.append(net.train(X, T, idx, batch, lr=lr_c))
    torch.cuda.synchronize()
    return np.concatenate(losses) if losses else np.zeros(0), time.perf_counter() - t0


def evaluate(net: MLP, X, T) -> float:
    """Mean squared error of the network on (X, T) (forward only)."""
    Y = net.forward(X)
    return float(((Y - T) ** 2).mean().item())
