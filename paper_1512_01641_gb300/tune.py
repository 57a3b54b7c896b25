"""Tuning of the classifier weights, gap penalty and acceptance threshold.

The paper tunes the threshold and the penalty with a script that tries random
parameter values and keeps those whose automatic alignment is most similar to
a human one (Section 5.2).  Three tuners are provided here, all on the GPU:

* ``random_search``: the paper's own tuner -- settings drawn at random, each
  scored by hard Needleman-Wunsch alignment of the training pairs against the
  gold links, the most similar kept;
* ``grid_search``: the exhaustive baseline -- every (gap, thr, b) setting of a
  7 x 7 x 7 grid is scored the same way, the best is kept;
* ``adam_tune``: gradient descent on the soft-alignment loss (softnw_fwd /
  softnw_bwd through ``miner.SoftAligner``) over all seven parameters.

The similarity of an automatic and a human alignment is read as
2 * matched / (automatic links + human links), where matched counts the links
that a Needleman-Wunsch alignment of the two link lists pairs up; both lists
are monotone (they lie on alignment paths), so matched is the number of
common links and the similarity is the links' micro-F1.  All tuners are then
evaluated identically: hard alignment of held-out pairs, micro-F1 of the kept
links against the gold links.  Counts are computed once per batch
(mine_count) and reused by every evaluation and every step.
"""
from __future__ import annotations

import itertools
import time
from dataclasses import dataclass

import numpy as np

from . import miner

GRID = {
    "gap": [0.05, 0.1, 0.2, 0.3, 0.4, 0.6, 0.8],
    "thr": [0.2, 0.3, 0.4, 0.5, 0.6, 0.7, 0.8],
    "b": [-6.0, -5.0, -4.0, -3.0, -2.0, -1.0, 0.0],
}
THETA0 = np.array([4.0, 4.0, -2.0, 1.0, -3.0, 0.3, 0.5])  # w0..w3, b, gap, thr
# ranges of the random search: those the grid spans (uniform draws)
RANDOM_RANGES = {"b": (-6.0, 0.0), "gap": (0.05, 0.8), "thr": (0.2, 0.8)}
_THETA_INDEX = {"b": 4, "gap": 5, "thr": 6}


class TuneData:
    """A batch on the GPU with its plan, cached counts and gold links."""

    def __init__(self, batch):
        import torch
        self.batch = batch
        self.plan = miner.Plan(miner.DeviceBatch.from_batch(batch))
        self.counts = self.plan.count()
        self.gold = torch.from_numpy(miner.gold_cells(batch, self.plan)).cuda()
        self.out = self.plan.new_output()

    def f1(self, params: miner.MineParams) -> dict:
        """Micro precision / recall / F1 of hard-NW links against gold."""
        self.plan.align(params, self.counts, self.out)
        tp, nl, ng = (int(x) for x in self.plan.link_gold_counts(self.out, self.gold).cpu().tolist())
        p = tp / nl if nl else 0.0
        r = tp / ng if ng else 0.0
        f = 2 * p * r / (p + r) if p + r > 0 else 0.0
        return {"precision": p, "recall": r, "f1": f, "links": nl, "gold": ng, "correct": tp}


@dataclass
class TuneResult:
    method: str
    theta: list
    train_f1: float | None
    eval: dict
    seconds: float
    extra: dict

    def as_dict(self):
        return {"method": self.method, "theta": [float(x) for x in self.theta], "train_f1": self.train_f1,
                "eval": self.eval, "seconds": self.seconds, **self.extra}


def grid_search(train: TuneData, held_out: TuneData, theta0=THETA0, grid=GRID) -> TuneResult:
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    best, best_f1 = None, -1.0
    for gap, thr, b in itertools.product(grid["gap"], grid["thr"], grid["b"]):
        th = theta0.copy()
        th[4], th[5], th[6] = b, gap, thr
        f = train.f1(miner.params_from_theta(th))["f1"]
        if f > best_f1:
            best, best_f1 = th, f
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    ev = held_out.f1(miner.params_from_theta(best))
    n = len(grid["gap"]) * len(grid["thr"]) * len(grid["b"])
    return TuneResult("grid", best.tolist(), best_f1, ev, secs, {"settings": n})


def random_draws(trials: int, seed: int = 0, theta0=THETA0, ranges=RANDOM_RANGES) -> list:
    """The settings random_search tries: theta0 with each parameter of ranges
    (b, gap, thr, in that order) drawn uniformly from its range."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(trials):
        th = np.array(theta0, np.float64)
        for k in ("b", "gap", "thr"):
            if k in ranges:
                lo, hi = ranges[k]
                th[_THETA_INDEX[k]] = rng.uniform(lo, hi)
        out.append(th)
    return out


def random_search(train: TuneData, held_out: TuneData, trials: int = 343, seed: int = 0, theta0=THETA0,
                  ranges=RANDOM_RANGES) -> TuneResult:
    """The paper's tuner (Section 5.2): parameter settings drawn at random,
    keeping the setting whose hard alignment of the training pairs is
    most similar to the gold alignment (micro-F1, see the module docstring).
    The default budget equals the grid's 343 settings; ranges may name a
    subset of b, gap, thr (the paper tunes thr and gap)."""
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    best, best_f1 = None, -1.0
    for th in random_draws(trials, seed, theta0, ranges):
        f = train.f1(miner.params_from_theta(th))["f1"]
        if f > best_f1:
            best, best_f1 = th, f
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    ev = held_out.f1(miner.params_from_theta(best))
    return TuneResult("random", best.tolist(), best_f1, ev, secs,
                      {"trials": trials, "seed": seed, "ranges": {k: list(v) for k, v in ranges.items()}})


def adam_tune(train: TuneData, held_out: TuneData, steps: int = 200, lr: float = 0.05, gamma: float = 0.1,
              tau: float = 0.05, betas=(0.9, 0.999), theta0=THETA0, batch_pairs: int | None = 1024,
              seed: int = 0) -> TuneResult:
    """Adam on the soft-alignment loss; every step is one softnw_fwd + softnw_bwd
    over a minibatch of batch_pairs training pairs drawn without replacement
    (reshuffled every pass over the data), or over all of them when
    batch_pairs is None."""
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    al = miner.SoftAligner(train.plan, train.counts, train.gold, gamma, tau)
    rng = np.random.default_rng(seed)
    n = train.plan.n_pairs
    use_mb = batch_pairs is not None and batch_pairs < n
    perm, pos = rng.permutation(n), 0
    theta = np.array(theta0, np.float64)
    m = np.zeros(7)
    v = np.zeros(7)
    losses = []
    for t in range(1, steps + 1):
        if use_mb:
            if pos + batch_pairs > n:
                perm, pos = rng.permutation(n), 0
            al.select(perm[pos:pos + batch_pairs])
            pos += batch_pairs
        params = miner.params_from_theta(theta)
        loss, _, _ = al.forward(params)
        g = al.backward(params).cpu().numpy().astype(np.float64)
        losses.append(float(loss[0]))
        m = betas[0] * m + (1 - betas[0]) * g
        v = betas[1] * v + (1 - betas[1]) * g * g
        mh = m / (1 - betas[0] ** t)
        vh = v / (1 - betas[1] ** t)
        theta = theta - lr * mh / (np.sqrt(vh) + 1e-8)
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    ev = held_out.f1(miner.params_from_theta(theta))
    if use_mb:
        al.select(None)
    train_f1 = train.f1(miner.params_from_theta(theta))["f1"]  # after the timed region
    return TuneResult("adam", theta.tolist(), train_f1, ev, secs,
                      {"steps": steps, "lr": lr, "gamma": gamma, "tau": tau,
                       "batch_pairs": batch_pairs if use_mb else n,
                       "loss_first": losses[0], "loss_last": losses[-1]})


def compare(train_batch, eval_batch, steps=200, grid=GRID, gamma=0.1, random_trials=343, theta0=THETA0) -> dict:
    """Grid search vs the paper's random search vs Adam on the same GPU, all
    started from theta0 (the grid and the random search keep its weights
    w) and evaluated on held-out pairs."""
    theta0 = np.asarray(theta0, np.float64)
    train, held = TuneData(train_batch), TuneData(eval_batch)
    base = held.f1(miner.params_from_theta(theta0))
    base_train = train.f1(miner.params_from_theta(theta0))["f1"]
    g = grid_search(train, held, theta0=theta0, grid=grid)
    r = random_search(train, held, trials=random_trials, theta0=theta0)
    a = adam_tune(train, held, steps=steps, gamma=gamma, theta0=theta0)
    return {"theta0": theta0.tolist(), "baseline_eval": base, "baseline_train_f1": base_train,
            "grid": g.as_dict(), "random": r.as_dict(), "adam": a.as_dict(),
            "f1_gap_points": 100 * (a.eval["f1"] - g.eval["f1"]),
            "speedup_vs_grid": g.seconds / a.seconds if a.seconds > 0 else None,
            "train_pairs": train_batch.n_pairs, "eval_pairs": eval_batch.n_pairs}
