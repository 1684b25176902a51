"""GPU tests of vqmc_batch_*: members stepped together give exactly what
the same problems stepped one by one give, and a batch of instances of
uneven size (the many-instances configuration) runs."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2106_13308_gb300 import inputs

from gpu_helpers import build_lib, er_instance, make_model

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build_lib()


PROBLEMS = [
    # n, h, B, act, precision (tensor-core sampler, FP32, CUDA-core BF16)
    (150, 60, 64, "relu", "bf16"),
    (90, 90, 50, "sigmoid", "fp32"),
    (300, 200, 40, "relu", "bf16"),
    (2300, 2300, 20, "relu", "bf16"),  # more than 2048 hidden units
]


def test_batch_members_match_single_contexts():
    from paper_2106_13308_gb300.vqmc import StepStats, VQMCBatch
    probs, singles = [], []
    for q, (n, h, B, act, prec) in enumerate(PROBLEMS):
        inst = er_instance(n, 0.05, 200 + q)
        theta = inputs.lively_params(n, h, 300 + q)
        probs.append(dict(n=n, h=h, max_batch=B, instance=inst, act=act, precision=prec, seed=400 + q, lr=1e-3))
        singles.append(make_model(n, h, B, inst, act=act, precision=prec, theta=theta, seed=400 + q, lr=1e-3))
    batch = VQMCBatch(probs)
    for q, (n, h, B, act, prec) in enumerate(PROBLEMS):
        batch.members[q].set_params(torch.from_numpy(inputs.lively_params(n, h, 300 + q)))
    outs = (StepStats * len(PROBLEMS))()
    for it in range(3):
        batch.step([p[2] for p in PROBLEMS], outs)
        torch.cuda.synchronize()
        for q, (n, h, B, act, prec) in enumerate(PROBLEMS):
            ref = StepStats()
            singles[q].step(B, ref)
            torch.cuda.synchronize()
            assert (outs[q].mean, outs[q].var, outs[q].min, outs[q].max) == (ref.mean, ref.var, ref.min, ref.max)
            assert outs[q].iteration == ref.iteration == it
    for q in range(len(PROBLEMS)):
        assert torch.equal(batch.members[q].get_params(), singles[q].get_params())
        assert batch.members[q].check() == 0
    batch.close()


def test_many_instances_of_uneven_size():
    """A smaller instance of the many-instances configuration: 8 instances,
    n ~ U{100..600}, G(n, 6/(n-1)), weights +-1, h = n, 512 samples each."""
    from paper_2106_13308_gb300.vqmc import StepStats, VQMCBatch
    cfgs = inputs.batched_configs(count=8, n_hi=600)
    probs = [dict(n=c["n"], h=c["h"], max_batch=c["B"], instance=inputs.make_instance(c), act=c["act"],
                  precision="bf16", seed=c["graph_seed"]) for c in cfgs]
    batch = VQMCBatch(probs)
    for m, c in zip(batch.members, cfgs):
        m.set_params(torch.from_numpy(inputs.made_params(c["n"], c["h"], c["param_seed"], w_std=c["w_std"])))
    outs = (StepStats * len(cfgs))()
    first = None
    for it in range(5):
        batch.step(512, outs)
        torch.cuda.synchronize()
        if first is None:
            first = [o.mean for o in outs]
    for o, c in zip(outs, cfgs):
        assert np.isfinite(o.mean) and o.error_flags == 0 and o.iteration == 4
        # every energy is a sum of +-1 couplings: |E| <= number of edges
        assert abs(o.min) <= len(inputs.make_instance(c)["col"])
    assert all(m.check() == 0 for m in batch.members)
    batch.close()
