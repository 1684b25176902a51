"""The paper's training protocol on the GPU (Sec. 5.1, Tables 2 and 5):
SGD+SR time to a target cut on a 20-spin Max-Cut instance of the paper's
generator, and 50 Adam iterations on G(20, 0.5) with sigmoid hidden units
(BF16 model).  The brute-force optimum of the oracle bounds every cut."""
import numpy as np
import pytest

import oracle
from gpu_helpers import build_lib, make_model
from paper_2106_13308_gb300 import inputs, train

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build_lib()


def test_sr_reaches_a_target_cut():
    n, h, B = 20, 40, 1024
    e = inputs.paper_maxcut(n, 1)
    inst = inputs.to_csr(n, e, np.ones(len(e), dtype=np.int32))
    opt = oracle.maxcut_bruteforce(inst)
    wt = train.total_weight(inst)
    m = make_model(n, h, B, inst, act="relu", precision="fp32", theta=inputs.made_params(n, h, 2), seed=9)
    res = train.train(m, B, iters=60, optimizer="sr", target=opt - 2,
                      score=lambda st: train.maxcut_scores(st, wt)[0])
    assert res.reached, f"mean cut {train.maxcut_scores(res.final_eval, wt)[0]} after {res.iterations}"
    assert res.train_device_ms > 0 and res.train_wall_s > 0
    mean_cut, best_cut = train.maxcut_scores(res.final_eval, wt)
    assert best_cut <= opt
    assert mean_cut >= opt - 3
    assert m.check() == 0


def test_adam_improves_the_c1_workload():
    cfg = inputs.config("maxcut_er20")
    inst = inputs.make_instance(cfg)
    opt = oracle.maxcut_bruteforce(inst)
    wt = train.total_weight(inst)
    m = make_model(cfg["n"], cfg["h"], cfg["B"], inst, act=cfg["act"], precision="bf16",
                   theta=inputs.made_params(cfg["n"], cfg["h"], cfg["param_seed"], w_std=cfg["w_std"]), seed=3)
    first = train.evaluate(m, 1024, 0)
    res = train.train(m, cfg["B"], iters=50, eval_every=10)
    assert res.iterations == 50 and sum(ev is not None for _, ev in res.history) == 5
    assert res.final_eval[0] < first[0] - 5
    assert train.maxcut_scores(res.final_eval, wt)[1] <= opt
    assert m.check() == 0
