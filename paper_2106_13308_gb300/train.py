"""Training and evaluation protocol of the paper's experiments (Sec. 5.1,
Tables 2 and 5), on top of the C ABI (``vqmc.VQMC``).

* Training: ``iters`` iterations of ``vqmc_step`` (Adam, the default
  optimiser, lr 1e-2) or ``vqmc_sr_step`` (SGD+SR, lambda 1e-3, lr 0.1), each
  with a fresh batch of exact samples.
* Evaluation (Sec. 5.1): a separate batch of ``eval_batch`` (1024) fresh
  samples from the trained model; the reported score is their mean energy.
  Evaluation draws its uniforms from Philox iteration counters
  ``EVAL_COUNTER_BASE + k``, disjoint from the training counters 0, 1, ...
* Time to target (Table 5): after every training update an evaluation batch
  is drawn and training stops once the evaluation score reaches the target;
  the recorded time covers the training updates only (device time from CUDA
  events around each update, and host wall time), not the evaluations.

For Max-Cut the score is the cut: with E(s) = sum_{i<j} w_ij s_i s_j (no
field), cut(s) = (W_tot - E(s)) / 2, W_tot = sum of the edge weights, so the
mean cut of a batch is (W_tot - mean E) / 2 and its best cut is
(W_tot - min E) / 2.  The score of the time-to-target run is the evaluation
batch's mean cut (the paper reports means of evaluation batches).

Every computation runs in the library; this module only sequences calls and
reads back the FP64 statistics.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

EVAL_COUNTER_BASE = 1 << 62


def total_weight(instance) -> float:
    """W_tot = sum over edges of w_ij for a sparse Max-Cut instance."""
    if instance.get("kind") == "dense":
        raise ValueError("the cut is defined here for sparse Max-Cut instances")
    if instance.get("field") is not None:
        raise ValueError("the cut mapping needs h = 0")
    return float(sum(float(w) for w in instance["w"]))


def evaluate(model, eval_batch: int, k: int):
    """FP64 {mean, var, min, max} of the energies of `eval_batch` fresh
    samples drawn with Philox counter EVAL_COUNTER_BASE + k."""
    s, _ = model.sample(eval_batch, None, iteration=EVAL_COUNTER_BASE + k)
    e = model.local_energy(s)
    stats, _ = model.energy_stats(e)
    return [float(x) for x in stats.cpu().tolist()]


@dataclass
class TrainResult:
    iterations: int = 0
    train_device_ms: float = 0.0
    train_wall_s: float = 0.0
    reached: bool = False
    history: list = field(default_factory=list)  # per iteration: (train mean E, eval stats or None)
    final_eval: list | None = None


def train(model, batch: int, iters: int = 300, optimizer: str = "adam", lr: float | None = None,
          lam: float = 1e-3, eval_batch: int = 1024, eval_every: int = 0, target=None, score=None):
    """Trains `model` (a vqmc.VQMC) for up to `iters` iterations of `batch`
    samples.  optimizer: "adam" (vqmc_step; the context's own Adam learning
    rate) or "sr" (vqmc_sr_step with lr, default 0.1, and lam).  With
    eval_every > 0 an evaluation batch follows every eval_every-th update;
    with `target` (and `score`, a function of the evaluation statistics, the
    default being minus the mean energy) an evaluation follows every update
    and training stops at the first whose score is >= target.  After
    training, one final evaluation batch gives `final_eval`."""
    import torch
    from .vqmc import StepStats

    if optimizer not in ("adam", "sr"):
        raise ValueError("optimizer must be 'adam' or 'sr'")
    if score is None:
        def score(st):
            return -st[0]
    sr_lr = 0.1 if lr is None else float(lr)
    res = TrainResult()
    out = StepStats()
    on_gpu = torch.cuda.is_available()
    every = 1 if target is not None else eval_every
    for it in range(iters):
        t0 = time.perf_counter()
        if on_gpu:
            stream = torch.cuda.current_stream()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
        if optimizer == "adam":
            model.step(batch, out)
        else:
            model.sr_step(batch, sr_lr, lam, out)
        if on_gpu:
            e1.record(stream)
            e1.synchronize()
            res.train_device_ms += e0.elapsed_time(e1)
        res.train_wall_s += time.perf_counter() - t0
        res.iterations = it + 1
        ev = None
        if every > 0 and (it + 1) % every == 0:
            ev = evaluate(model, eval_batch, it)
        res.history.append((float(out.mean), ev))
        if target is not None and ev is not None and score(ev) >= target:
            res.reached = True
            break
    res.final_eval = evaluate(model, eval_batch, iters + 1)
    return res


def maxcut_scores(stats, w_tot: float):
    """(mean cut, best cut) of a batch from its energy statistics."""
    return (w_tot - stats[0]) / 2.0, (w_tot - stats[2]) / 2.0


def compare_precisions(make_model, batch: int, seeds: int = 5, iters: int = 300, eval_batch: int = 1024,
                       precisions=("bf16", "fp32")):
    """Final energies of the same training run at several precisions (Sec. 5.1
    protocol: `iters` Adam iterations, then the mean energy of an evaluation
    batch of `eval_batch` fresh samples, averaged over `seeds` runs).

    make_model(precision, seed) must return a fresh vqmc.VQMC with the seed's
    initial parameters and Philox key, so that for each seed the precisions
    start from the same state and draw from the same uniform streams.  Also
    records the evaluation mean before training.  Returns a dict with the
    per-seed final means per precision, their averages, and the relative
    difference |mean_a - mean_b| / |mean_b| of the first two precisions."""
    import torch
    finals = {p: [] for p in precisions}
    initial = []
    for seed in range(seeds):
        for q, prec in enumerate(precisions):
            m = make_model(prec, seed)
            if q == 0:
                initial.append(evaluate(m, eval_batch, 0)[0])
            for _ in range(iters):
                m.step(batch)
            finals[prec].append(evaluate(m, eval_batch, iters + 1)[0])
            if m.check() != 0:
                raise RuntimeError(f"device error flags after the {prec} run of seed {seed}")
            m.close()
            del m
            torch.cuda.empty_cache()
    means = {p: sum(v) / len(v) for p, v in finals.items()}
    a, b = precisions[0], precisions[1]
    return {"seeds": seeds, "iters": iters, "eval_batch": eval_batch, "initial_mean": sum(initial) / len(initial),
            "final_means": finals, "mean": means, "rel_diff": abs(means[a] - means[b]) / abs(means[b])}
