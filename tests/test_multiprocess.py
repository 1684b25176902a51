"""World-size-2 host tests of the multi-GPU pieces, on CPU with gloo.

* The benchmark's replica aggregation: the job's time is the slowest rank's
  and the units done are the sum over ranks.
* The exchange step the path would need to shard one batch over GPUs (the
  paper's data parallelism, Sec. 4): every rank forms, on its own shard,
  sum_b E_b g_b, sum_b g_b (g_b = grad log pi(s_b)), sum_b E_b and B; one
  all-reduce of these gives every rank the gradient of the global-baseline
  estimator, which must equal the full-batch gradient (oracle, FP64).
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _init(rank, world, port):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)


def _replica_worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    _init(rank, world, port)
    ms, value = bench._replica_rate([40.0, 50.0][rank], 10, world, "cpu")
    out[rank] = (ms, value)
    dist.destroy_process_group()


def test_replica_rate_takes_slowest_rank_and_sums_units():
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_replica_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for r in (0, 1):
        ms, value = res[r]
        assert ms == 50.0
        assert value == pytest.approx(2 * 10 / 0.050)


def _shard_worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import oracle
    from paper_2106_13308_gb300 import inputs
    _init(rank, world, port)
    n, h, B = 12, 9, 40
    edges = inputs.erdos_renyi(n, 0.4, 3)
    inst = inputs.to_csr(n, edges, inputs.int_weights(len(edges), 1, 10, 4))
    P = oracle.theta_to_made(inputs.lively_params(n, h, 5), n, h)
    S = inputs.spins(B, n, 6)
    lo, hi = rank * B // world, (rank + 1) * B // world
    Sk = S[lo:hi]
    E = oracle.energy(inst, Sk)
    # per-sample gradients g_b through the oracle's batch gradient with one-hot coefficients
    gs = []
    for b in range(Sk.shape[0]):
        c = np.zeros(Sk.shape[0])
        c[b] = 1.0
        gs.append(oracle.made_to_theta(*oracle.logprob_grad(P, Sk, c)))
    G = np.stack(gs)
    part = np.concatenate([(E[:, None] * G).sum(0), G.sum(0), [E.sum(), float(Sk.shape[0])]])
    t = torch.from_numpy(part)
    dist.all_reduce(t)
    tot = t.numpy()
    d = G.shape[1]
    s_eg, s_g, s_e, bt = tot[:d], tot[d:2 * d], tot[2 * d], tot[2 * d + 1]
    mean = s_e / bt
    g_global = (s_eg - mean * s_g) / bt  # sum_b (E_b - mean) g_b / B
    (dW1, db1, dW2, db2), st, _ = oracle.vqmc_grad(P, inst, S)
    g_full = oracle.made_to_theta(dW1, db1, dW2, db2)
    out[rank] = (float(np.max(np.abs(g_global - g_full))), float(np.max(np.abs(g_full))), abs(mean - st[0]))
    dist.destroy_process_group()


def test_sharded_global_baseline_gradient_equals_full_batch():
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_shard_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for r in (0, 1):
        err, scale, dmean = res[r]
        assert scale > 0
        assert err <= 1e-12 * max(1.0, scale) * 40
        assert dmean <= 1e-12
