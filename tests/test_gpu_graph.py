"""Captured iterations on the GPU: a CUDA graph of vqmc_step (or
vqmc_sr_step) calls, replayed, gives bit for bit what the same number of
eager calls gives (the kernels read the iteration counter and the Adam
factors from device memory the iterations advance); the same for a batch of
problems, including after the schedule autotuner has picked its streams."""
import numpy as np
import pytest
import torch

from paper_2106_13308_gb300 import inputs

from gpu_helpers import build_lib, er_instance, make_model

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build_lib()


def _twins(n, h, B, act, prec, seed, **kw):
    inst = er_instance(n, 0.05 if n > 100 else 0.2, seed)
    theta = inputs.lively_params(n, h, seed + 1)
    return [make_model(n, h, B, inst, act=act, precision=prec, theta=theta, seed=seed + 2, **kw) for _ in range(2)]


# tensor-core sampler (BF16, h < n), CUDA-core BF16 (h = n) and FP32
CASES = [(300, 100, 96, "relu", "bf16"), (120, 120, 64, "sigmoid", "bf16"), (90, 70, 80, "relu", "fp32")]


@pytest.mark.parametrize("n,h,B,act,prec", CASES)
def test_graph_replays_equal_eager_steps(n, h, B, act, prec):
    from paper_2106_13308_gb300.vqmc import StepStats
    eager, graphed = _twins(n, h, B, act, prec, 40)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        eager.step(B)  # one eager step first: the graph continues from iteration 1
        graphed.step(B)
        graphed.graph_capture(B, steps=2)
        assert graphed.iteration == 1
        a, b = StepStats(), StepStats()
        for _ in range(4):
            eager.step(B, a)
        for _ in range(2):
            graphed.graph_launch(b)
        stream.synchronize()
    assert graphed.iteration == eager.iteration == 5
    assert (a.mean, a.var, a.min, a.max, a.iteration) == (b.mean, b.var, b.min, b.max, b.iteration)
    assert b.iteration == 4
    assert torch.equal(eager.get_params(), graphed.get_params())
    se, _ = eager.last_batch(B)
    sg, _ = graphed.last_batch(B)
    assert torch.equal(se, sg)
    # eager steps after the replays continue the same sequence
    with torch.cuda.stream(stream):
        eager.step(B, a)
        graphed.step(B, b)
        stream.synchronize()
    assert (a.mean, a.iteration) == (b.mean, b.iteration) == (a.mean, 5)
    assert torch.equal(eager.get_params(), graphed.get_params())
    assert eager.check() == 0 and graphed.check() == 0


def test_sr_graph_equals_eager_sr_steps():
    from paper_2106_13308_gb300.vqmc import StepStats
    n, h, B = 40, 50, 128
    eager, graphed = _twins(n, h, B, "relu", "fp32", 60)
    stream = torch.cuda.Stream()
    a, b = StepStats(), StepStats()
    with torch.cuda.stream(stream):
        graphed.graph_capture(B, steps=3, optimizer="sr", sr_lr=0.1, sr_lambda=1e-3)
        for _ in range(3):
            eager.sr_step(B, 0.1, 1e-3, a)
        graphed.graph_launch(b)
        stream.synchronize()
    assert (a.mean, a.var, a.iteration) == (b.mean, b.var, b.iteration)
    assert torch.equal(eager.get_params(), graphed.get_params())


def test_capture_errors():
    from paper_2106_13308_gb300.vqmc import VQMCError, VQMC_ERR_INVALID_ARG, vqmc_graph_capture, vqmc_graph_launch
    m, _ = _twins(50, 30, 16, "relu", "bf16", 70)
    with pytest.raises(VQMCError) as ei:
        vqmc_graph_launch(m.ctx)
    assert ei.value.status == VQMC_ERR_INVALID_ARG
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        for bad in (dict(B=0, steps=1), dict(B=16, steps=0), dict(B=17, steps=1)):
            with pytest.raises(VQMCError) as ei:
                vqmc_graph_capture(m.ctx, bad["B"], bad["steps"])
            assert ei.value.status == VQMC_ERR_INVALID_ARG
    assert m.iteration == 0 and m.check() == 0


def _batch_problems():
    cfgs = inputs.batched_configs(count=6, n_lo=100, n_hi=700)
    probs = [dict(n=c["n"], h=c["h"] if q % 2 else c["n"] // 3, max_batch=128, instance=inputs.make_instance(c),
                  act=c["act"], precision="bf16", seed=c["graph_seed"]) for q, c in enumerate(cfgs)]
    return cfgs, probs


def _make_batch(cfgs, probs):
    from paper_2106_13308_gb300.vqmc import VQMCBatch
    batch = VQMCBatch(probs)
    for m, c, p in zip(batch.members, cfgs, probs):
        m.set_params(torch.from_numpy(inputs.made_params(c["n"], p["h"], c["param_seed"], w_std=0.3)))
    return batch


def test_batch_graph_and_autotuned_schedule_equal_eager_batches():
    """After the autotuner has chosen each member's sampler layout and the
    schedule, replays of its graph equal eager batched steps of twins with
    the same samplers, started from the tuned members' state (checkpoints)."""
    import os
    import tempfile
    from paper_2106_13308_gb300.vqmc import StepStats
    cfgs, probs = _batch_problems()
    B = [p["max_batch"] for p in probs]
    tuned = _make_batch(cfgs, probs)
    stream = torch.cuda.Stream()
    outs_t = (StepStats * len(probs))()
    outs_e = (StepStats * len(probs))()
    with torch.cuda.stream(stream):
        streams, ms = tuned.autotune(B)
        stream.synchronize()
    assert 1 <= streams <= 6 and ms > 0
    steps_done = tuned.members[0].iteration
    assert all(m.iteration == steps_done for m in tuned.members)
    used, mstream, samplers, alone = tuned.schedule()
    assert used == streams and len(mstream) == len(probs) and all(0 <= q < used for q in mstream)
    assert all(a > 0 for a in alone)
    # h < n/2 members use the tensor-core sampler; the others one of the two CUDA-core layouts
    for p, smp in zip(probs, samplers):
        assert smp == "tensor_core" if p["h"] <= p["n"] // 3 else smp in ("cuda_core", "cuda_core_wide")
    eager = _make_batch(cfgs, [dict(p, sampler=smp) for p, smp in zip(probs, samplers)])
    with tempfile.TemporaryDirectory() as d:
        for q in range(len(probs)):
            path = os.path.join(d, f"m{q}.ckpt")
            tuned.members[q].save(path)
            eager.members[q].load(path)
    with torch.cuda.stream(stream):
        for _ in range(2):
            tuned.graph_launch(outs_t)
        for _ in range(2):
            eager.step(B, outs_e)
        stream.synchronize()
    for q in range(len(probs)):
        assert tuned.members[q].iteration == eager.members[q].iteration == steps_done + 2
        assert (outs_t[q].mean, outs_t[q].var, outs_t[q].iteration) == (outs_e[q].mean, outs_e[q].var,
                                                                         outs_e[q].iteration)
        assert torch.equal(tuned.members[q].get_params(), eager.members[q].get_params())
        assert tuned.members[q].check() == 0
    # a graph of several batched iterations
    with torch.cuda.stream(stream):
        tuned.graph_capture(B, steps=3)
        tuned.graph_launch(outs_t)
        for _ in range(3):
            eager.step(B, outs_e)
        stream.synchronize()
    for q in range(len(probs)):
        assert torch.equal(tuned.members[q].get_params(), eager.members[q].get_params())
    tuned.close()
    eager.close()
