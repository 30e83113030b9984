"""Adaptive cloning depths across processes, one GPU each.

Primaries are independent (Sec. 3: clients never talk to each other), so a
multi-process run gives every rank a contiguous block of each epoch's primary
ids and keeps each rank's clones on its own GPU.  The one exchange the method
has is the feedback of Sec. 2/3: before an enhanced epoch the ranks sum their
cumulative range histograms (FP64, n_bins + 3 in the reed_range_profile
layout) and every rank re-estimates the same depths d_k = S^-1(2^-k) from the
sum.  Weights are powers of two, so these sums are exact in FP64 and the
result of a run does not depend on how many ranks share it.

The driver is written against a small engine interface so that its host
logic can be exercised without a GPU:

    engine.local_profile()      -> this rank's cumulative histogram
    engine.update_depths(total) -> re-estimate the depths from a summed histogram
    engine.set_depths(d)        -> set the depths explicitly
    engine.depths()             -> the current depths (host array)
    engine.run(first, count, enhanced)
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class Epoch:
    first: int       # first primary id of the epoch
    count: int       # primaries in the epoch (all ranks)
    enhanced: bool   # cloning on
    update: bool     # re-estimate the depths before it


def epoch_plan(n_ions: int, epoch_size: int, n_initial: int) -> list:
    """n_initial unenhanced primaries, then epochs of epoch_size primaries;
    the depths are re-estimated before every enhanced epoch that has finished
    tracks behind it (the first one uses the initial guess when n_initial is
    0).  The same schedule as an adaptive reed_run."""
    if epoch_size < 1 or n_initial < 0 or n_ions < 0:
        raise ValueError("need epoch_size >= 1, n_initial >= 0, n_ions >= 0")
    plan, done = [], 0
    ninit = min(n_initial, n_ions)
    if ninit > 0:
        plan.append(Epoch(0, ninit, False, False))
        done = ninit
    while done < n_ions:
        m = min(epoch_size, n_ions - done)
        plan.append(Epoch(done, m, True, done > 0))
        done += m
    return plan


def rank_block(first: int, count: int, rank: int, world: int) -> tuple:
    """Contiguous share [lo, lo + n) of the ids [first, first + count) for a
    rank; the shares of all ranks partition the range in rank order."""
    lo = first + count * rank // world
    hi = first + count * (rank + 1) // world
    return lo, hi - lo


def run_adaptive(engine, n_ions: int, epoch_size: int, n_initial: int, initial_depths, rank: int = 0,
                 world: int = 1, allreduce=None) -> list:
    """Run the adaptive schedule on this rank; returns the depths used by each
    enhanced epoch.  allreduce(profile) must return the element-wise sum over
    ranks (it is called by every rank at the same points, also when world is
    1 if it is given)."""
    if world > 1 and allreduce is None:
        raise ValueError("several ranks need an allreduce")
    engine.set_depths(np.asarray(initial_depths, dtype=np.float64))
    history = []
    for ep in epoch_plan(n_ions, epoch_size, n_initial):
        if ep.enhanced:
            if ep.update:
                prof = engine.local_profile()
                engine.update_depths(allreduce(prof) if allreduce is not None else prof)
            history.append(np.array(engine.depths(), dtype=np.float64))
        first, count = rank_block(ep.first, ep.count, rank, world)
        engine.run(first, count, ep.enhanced)
    return history


class ReedShard:
    """Engine over a `reed.Reed` context on this process's GPU.  Profiles are
    float64 CUDA tensors, so a NCCL all_reduce can sum them in place."""

    def __init__(self, reed_ctx, seed: int, precision: int = 0, **run_kw):
        self.r = reed_ctx
        self.seed = seed
        self.precision = precision
        self.run_kw = run_kw
        self.nthr = len(reed_ctx.w["thresholds"])
        if self.nthr < 1:
            raise ValueError("the workload needs initial cloning depths")
        self.nb = int(reed_ctx.w["n_bins"])
        self.bw = float(reed_ctx.w["bin_w"])

    def local_profile(self):
        import torch
        from . import reed
        t = torch.zeros(self.nb + 3, dtype=torch.float64, device="cuda")
        if reed.reed_stats(self.r.ctx)["tracks"] > 0:
            torch.cuda.synchronize()
            p = t.data_ptr()
            reed._check(reed.lib().reed_range_profile(self.r.ctx, p, self.nb, p + 8 * self.nb), self.r.ctx)
        return t

    def update_depths(self, total):
        from . import reed
        import torch
        torch.cuda.synchronize()
        reed.reed_update_thresholds(self.r.ctx, self.nthr, total.data_ptr(), self.nb, self.bw)

    def set_depths(self, d):
        from . import reed
        reed.reed_update_thresholds(self.r.ctx, self.nthr, thresholds=d)

    def depths(self):
        from . import reed
        return reed.reed_get_thresholds(self.r.ctx)[:self.nthr]

    def run(self, first, count, enhanced):
        if count <= 0:
            return
        thr = list(self.r.w["thresholds"]) if enhanced else []
        self.r.run(n_ions=count, seed=self.seed, precision=self.precision, first_id=first, thresholds=thr,
                   device_thresholds=enhanced, **self.run_kw)
