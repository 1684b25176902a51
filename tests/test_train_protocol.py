"""Host logic of the training/evaluation protocol (Sec. 5.1, Tables 2 and 5)
with a scripted stand-in for the GPU model: evaluation counters disjoint from
training counters, the time-to-target stop rule, optimiser dispatch, and the
Max-Cut score mapping cut = (W_tot - E) / 2."""
import numpy as np
import pytest
import torch

from paper_2106_13308_gb300 import inputs, train


class ScriptedModel:
    """Energies fall by 1 per training update; evaluation batches report the
    current level.  Records every call."""

    def __init__(self, start=0.0):
        self.level = start
        self.calls = []

    def step(self, B, out):
        self.calls.append(("adam", B))
        out.mean = self.level
        self.level -= 1.0

    def sr_step(self, B, lr, lam, out):
        self.calls.append(("sr", B, lr, lam))
        out.mean = self.level
        self.level -= 1.0

    def sample(self, B, u, iteration):
        self.calls.append(("sample", B, iteration))
        return torch.zeros((B, 3), dtype=torch.int8), torch.zeros(B)

    def local_energy(self, s):
        return torch.full((s.shape[0],), self.level, dtype=torch.float64)

    def energy_stats(self, e):
        x = e.numpy()
        return torch.tensor([x.mean(), x.var(), x.min(), x.max()], dtype=torch.float64), None


def test_evaluation_uses_counters_disjoint_from_training():
    m = ScriptedModel()
    res = train.train(m, batch=8, iters=5, eval_every=2, eval_batch=16)
    evals = [c for c in m.calls if c[0] == "sample"]
    assert [c[2] for c in evals] == [train.EVAL_COUNTER_BASE + 1, train.EVAL_COUNTER_BASE + 3,
                                     train.EVAL_COUNTER_BASE + 6]
    assert all(c[1] == 16 for c in evals)
    assert res.iterations == 5 and not res.reached
    assert [h[1] is not None for h in res.history] == [False, True, False, True, False]
    assert res.final_eval[0] == -5.0


def test_time_to_target_stops_at_the_first_evaluation_reaching_it():
    m = ScriptedModel(start=0.0)
    # score = -mean E; after update k the level is -k
    res = train.train(m, batch=4, iters=100, target=7.0)
    assert res.reached and res.iterations == 7
    assert sum(1 for c in m.calls if c[0] == "adam") == 7
    res2 = train.train(ScriptedModel(), batch=4, iters=3, target=50.0)
    assert not res2.reached and res2.iterations == 3


def test_optimizer_dispatch_and_defaults():
    m = ScriptedModel()
    train.train(m, batch=4, iters=2, optimizer="sr")
    assert [c for c in m.calls if c[0] == "sr"] == [("sr", 4, 0.1, 1e-3)] * 2
    with pytest.raises(ValueError):
        train.train(ScriptedModel(), batch=4, iters=1, optimizer="sgd")


def test_maxcut_score_mapping():
    n = 12
    e = inputs.erdos_renyi(n, 0.5, 3)
    w = inputs.int_weights(len(e), 1, 10, 4)
    inst = inputs.to_csr(n, e, w)
    wt = train.total_weight(inst)
    assert wt == float(np.sum(w))
    rng = np.random.default_rng(0)
    s = rng.choice([-1, 1], size=n)
    E = sum(int(wi) * s[i] * s[j] for (i, j), wi in zip(e, w))
    cut = sum(int(wi) for (i, j), wi in zip(e, w) if s[i] != s[j])
    mean_cut, best_cut = train.maxcut_scores([E, 0.0, E, E], wt)
    assert mean_cut == cut and best_cut == cut
    with pytest.raises(ValueError):
        train.total_weight(inputs.sk(5, 1))
