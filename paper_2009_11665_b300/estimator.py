"""Alg. 1's outer loop: colourings in waves until the estimate converges.

Alg. 1 (Sec. 2.3.1) repeats N times: draw a uniformly random colouring, run
the counting DP, turn the colourful count into finalCount = total / (P alpha),
and outputs the average of the finalCounts.  The paper bounds N by
O(e^k log(1/delta) / eps^2) for a (1 +- eps) approximation with probability
1 - 2 delta (Alon et al.), without a constant.  This module runs the loop in
waves of colourings and stops either at that bound (constant 1, or one the
caller gives) or earlier, once the normal-approximation confidence interval
of the running mean has relative half-width <= eps at level 1 - 2 delta.

* Counting is injected: ``count_wave(colourings) -> finalCounts`` takes a
  [w, n] int8 array of colourings and returns [templates, w] float64
  estimates.  ``session_counter`` builds one from a library Session (the GPU
  path); tests pass other counters.
* Colourings come from ``colouring_fn(index) -> [n] int8``, keyed by a
  global colouring index, so a run can stop and resume and several ranks
  can split the indices without drawing the same colouring twice.
* Replicas over colourings: rank r of a torch.distributed group counts
  indices ``wave_no * wave * world + r * wave + [0, wave)`` and the ranks sum
  (count, sum, sum of squares) per template after every wave, so every rank
  holds the same state and takes the same stopping decision.
* Checkpoint/resume: after every wave rank 0 writes the state (JSON, written
  to a temporary file and renamed); a new run given the same file continues
  after the last completed wave.
"""
from __future__ import annotations

import dataclasses
import json
import math
import os
from statistics import NormalDist
from typing import Callable, Optional

import numpy as np


def paper_iterations(k: int, eps: float, delta: float, constant: float = 1.0) -> int:
    """N = constant * e^k * ln(1/delta) / eps^2 (Alg. 1's bound with the
    O() constant made explicit), rounded up."""
    if not (0 < eps and 0 < delta < 1):
        raise ValueError("need eps > 0 and 0 < delta < 1")
    return int(math.ceil(constant * math.exp(k) * math.log(1.0 / delta) / (eps * eps)))


def colouring_indices(rank: int, world: int, wave: int, wave_no: int) -> np.ndarray:
    """Global colouring indices of `rank`'s share of wave `wave_no`."""
    start = (wave_no * world + rank) * wave
    return np.arange(start, start + wave, dtype=np.int64)


@dataclasses.dataclass
class EstimateResult:
    estimate: np.ndarray        # [templates] mean of the finalCounts
    colourings: int             # colourings counted (all ranks)
    stderr: np.ndarray          # [templates] standard error of the mean
    half_width: np.ndarray      # [templates] confidence half-width at 1 - 2 delta
    converged: bool             # every template reached half_width <= eps * |estimate|
    bound: int                  # the paper's N for this k, eps, delta


class ColourCodingEstimator:
    def __init__(self, count_wave: Callable[[np.ndarray], np.ndarray], colouring_fn: Callable[[int], np.ndarray],
                 k: int, eps: float, delta: float, wave: int = 16, min_colourings: int = 32,
                 max_colourings: Optional[int] = None, bound_constant: float = 1.0,
                 checkpoint: Optional[str] = None, group=None):
        if wave < 1 or min_colourings < 2:
            raise ValueError("wave >= 1 and min_colourings >= 2 required")
        self.count_wave = count_wave
        self.colouring_fn = colouring_fn
        self.k, self.eps, self.delta = int(k), float(eps), float(delta)
        self.wave = int(wave)
        self.min_colourings = int(min_colourings)
        self.bound = paper_iterations(k, eps, delta, bound_constant)
        self.max_colourings = self.bound if max_colourings is None else int(max_colourings)
        self.checkpoint = checkpoint
        self.group = group
        self.z = NormalDist().inv_cdf(1.0 - self.delta)
        if group is not None:
            import torch.distributed as dist

            self.rank, self.world = dist.get_rank(group), dist.get_world_size(group)
        else:
            self.rank, self.world = 0, 1

    # -- state -------------------------------------------------------------
    def _fresh(self):
        return {"waves": 0, "count": 0, "sum": None, "sumsq": None, "wave": self.wave, "world": self.world}

    def _load(self):
        if not self.checkpoint or not os.path.exists(self.checkpoint):
            return self._fresh()
        with open(self.checkpoint) as f:
            st = json.load(f)
        if st.get("wave") != self.wave or st.get("world") != self.world:
            raise ValueError("checkpoint was written with another wave size or number of ranks")
        return st

    def _save(self, st):
        if not self.checkpoint or self.rank != 0:
            return
        tmp = self.checkpoint + ".tmp"
        with open(tmp, "w") as f:
            json.dump(st, f)
        os.replace(tmp, self.checkpoint)

    def _reduce(self, vec: np.ndarray) -> np.ndarray:
        if self.group is None:
            return vec
        import torch
        import torch.distributed as dist

        dev = "cuda" if dist.get_backend(self.group) == "nccl" else "cpu"
        t = torch.from_numpy(np.ascontiguousarray(vec, dtype=np.float64)).to(dev)
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=self.group)
        return t.cpu().numpy()

    def _summary(self, st) -> EstimateResult:
        n = st["count"]
        s = np.asarray(st["sum"], dtype=np.float64)
        ss = np.asarray(st["sumsq"], dtype=np.float64)
        mean = s / n
        var = np.maximum(ss / n - mean * mean, 0.0) * n / max(n - 1, 1)
        se = np.sqrt(var / n)
        hw = self.z * se
        conv = bool(n >= self.min_colourings and np.all(hw <= self.eps * np.abs(mean)))
        return EstimateResult(mean, n, se, hw, conv, self.bound)

    # -- loop --------------------------------------------------------------
    def run(self, max_waves: Optional[int] = None) -> EstimateResult:
        """Counts waves until convergence or max_colourings (or max_waves
        more waves, for callers that interleave other work)."""
        st = self._load()
        done_here = 0
        while True:
            if st["count"] > 0:
                res = self._summary(st)
                if res.converged or st["count"] >= self.max_colourings:
                    return res
            if max_waves is not None and done_here >= max_waves:
                return self._summary(st)
            idx = colouring_indices(self.rank, self.world, self.wave, st["waves"])
            cols = np.stack([np.asarray(self.colouring_fn(int(i)), dtype=np.int8) for i in idx])
            est = np.asarray(self.count_wave(cols), dtype=np.float64)
            if est.ndim == 1:
                est = est[None, :]
            local = np.concatenate([[est.shape[1]], est.sum(axis=1), (est * est).sum(axis=1)])
            tot = self._reduce(local)
            t = est.shape[0]
            st["count"] += int(round(tot[0]))
            st["sum"] = (np.zeros(t) if st["sum"] is None else np.asarray(st["sum"])) + tot[1:1 + t]
            st["sumsq"] = (np.zeros(t) if st["sumsq"] is None else np.asarray(st["sumsq"])) + tot[1 + t:]
            st["sum"], st["sumsq"] = list(map(float, st["sum"])), list(map(float, st["sumsq"]))
            st["waves"] += 1
            done_here += 1
            self._save(st)


def session_counter(session, stream=None) -> Callable[[np.ndarray], np.ndarray]:
    """count_wave for a library Session of B colourings: runs the session on
    the wave (w == B) and returns the estimates [templates, B] on the host."""
    P = len(session.plans)

    def count_wave(cols: np.ndarray) -> np.ndarray:
        if cols.shape[0] != session.B:
            raise ValueError("wave size must equal the session's batch")
        est = np.zeros((P, session.B))
        session.run(np.ascontiguousarray(cols, dtype=np.int8), None, est, None, stream)
        session.sync(stream)
        return est

    return count_wave
