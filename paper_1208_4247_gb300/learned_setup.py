"""Setting up the learned smoother for a hierarchy: train weights on the
GPU, then keep them per level only where they measurably beat red-black
Gauss-Seidel (the fallback).

* ``train_weights`` -- the two-grid contraction training of the library
  (gmg_learned_train) on a 65^3 then a 129^3 grid, started from weighted
  Jacobi (omega = 6/7) weights.
* ``select_levels`` -- the library's per-level fallback on the target
  problem (gmg_smoother_select): level by level from the finest, the learned
  weights are kept if the measured V-cycle contraction (geometric mean over a
  few cycles) improves, else the level smooths with red-black GS.
"""
from __future__ import annotations

import numpy as np

from . import gmg


def train_weights(d=3, sizes=((64, 1000, 8), (128, 250, 8)), lr=2e-3, seed=100):
    """Returns ({n: weights}, {n: loss history}); sizes = (n, steps, batch)
    trained in order, each starting from the previous result."""
    w = gmg.jacobi_weights(d, 6.0 / 7.0)
    out, hist = {}, {}
    for i, (n, steps, batch) in enumerate(sizes):
        w, h = gmg.learned_train(d, n, steps, batch, w, lr=lr, seed=seed + i)
        out[n] = w.copy()
        hist[n] = h
    return out, hist


def contraction(S, f, u, cycles=8, skip=2):
    u.zero_()
    rel = S.cycles(f, u, cycles)
    return float((rel[-1] / rel[skip]) ** (1.0 / (cycles - 1 - skip)))


def select_levels(S, f, u, candidates, levels):
    """candidates: {level: weights}.  The library's fallback rule
    (gmg_smoother_select): sets the kept weights on S and returns (kept
    levels, contraction before, contraction after)."""
    del u, levels  # the library measures on its own work array, every level
    return S.smoother_select(f, candidates)
