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


class _OracleShard:
    """The library's shard calls (vqmc_set_sample_offset, vqmc_shard_sums,
    vqmc_shard_apply) restated on the FP64 oracle, so that the host protocol
    of paper_2106_13308_gb300.sharded runs on CPU ranks."""

    def __init__(self, n, h, inst, theta, seed):
        import oracle
        self.o = oracle
        self.n, self.h, self.inst, self.seed = n, h, inst, seed
        self.theta = np.asarray(theta, np.float64).copy()
        self.m = np.zeros_like(self.theta)
        self.v = np.zeros_like(self.theta)
        self.t = 0
        self.iter = 0
        self.b0 = 0
        self.last_grad = None

    def set_sample_offset(self, b0):
        self.b0 = int(b0)

    def shard_sums(self, B, shift):
        o = self.o
        P = o.theta_to_made(self.theta, self.n, self.h)
        U = o.uniforms(self.b0 + B, self.n, self.seed, self.iter)[self.b0:]
        S, _ = o.sample(P, U)
        E = o.energy(self.inst, S)
        c1 = E - shift
        S1 = o.made_to_theta(*o.logprob_grad(P, S, c1))
        S0 = o.made_to_theta(*o.logprob_grad(P, S, np.ones(B)))
        return torch.from_numpy(np.concatenate([S1, S0])), torch.tensor([c1.sum(), (c1 * c1).sum(), float(B)],
                                                                         dtype=torch.float64)

    def shard_apply(self, sums, scal, shift):
        d = self.theta.size
        s = sums.numpy()
        bt = float(scal[2])
        mm = float(scal[0]) / bt
        g = (s[:d] - mm * s[d:]) / bt
        self.t += 1
        self.o.adam(self.theta, self.m, self.v, g, self.t)
        self.iter += 1
        self.last_grad = g
        return torch.from_numpy(g), torch.tensor([shift + mm, float(scal[1]) / bt - mm * mm], dtype=torch.float64)


def _sharded_problem():
    from paper_2106_13308_gb300 import inputs
    n, h = 12, 9
    edges = inputs.erdos_renyi(n, 0.4, 3)
    inst = inputs.to_csr(n, edges, inputs.int_weights(len(edges), 1, 10, 4))
    return n, h, inst, inputs.lively_params(n, h, 5)


def _sharded_run_worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    from paper_2106_13308_gb300.sharded import ShardedRun
    _init(rank, world, port)
    n, h, inst, theta = _sharded_problem()
    model = _OracleShard(n, h, inst, theta, seed=77)
    run = ShardedRun(model, 20)
    grads, stats = [], []
    for _ in range(4):
        st = run.step()
        grads.append(model.last_grad.copy())
        stats.append(st.numpy().copy())
    out[rank] = (model.theta.copy(), grads, stats, run.batch_total)
    dist.destroy_process_group()


def test_sharded_run_protocol_equals_full_batch_run():
    """Two gloo ranks of 20 samples each through ShardedRun (sample offsets,
    one all-reduce of the shard sums, global-baseline gradient, Adam) end
    with bit-identical parameters, which equal a single-process run of the
    same protocol on the full batch of 40; the first iteration's gradient
    equals the oracle's full-batch estimator on the same 40 samples."""
    import oracle
    from paper_2106_13308_gb300.sharded import ShardedRun
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_sharded_run_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    th0, g0, st0, bt = res[0]
    th1, g1, st1, _ = res[1]
    assert bt == 40
    assert np.array_equal(th0, th1)
    n, h, inst, theta = _sharded_problem()
    full = _OracleShard(n, h, inst, theta, seed=77)
    run = ShardedRun(full, 40)
    gf = []
    for _ in range(4):
        run.step()
        gf.append(full.last_grad.copy())
    scale = max(np.abs(gf[0]).max(), 1e-30)
    for k in range(4):
        assert np.max(np.abs(g0[k] - gf[k])) <= 1e-12 * scale * 40, k
    assert np.max(np.abs(th0 - full.theta)) <= 1e-12
    # iteration 0 (shift 0) against the oracle's own estimator on the full batch
    P = oracle.theta_to_made(np.asarray(theta, np.float64), n, h)
    S, _ = oracle.sample(P, oracle.uniforms(40, n, 77, 0))
    (dW1, db1, dW2, db2), sto, _ = oracle.vqmc_grad(P, inst, S)
    ref = oracle.made_to_theta(dW1, db1, dW2, db2)
    assert np.max(np.abs(g0[0] - ref)) <= 1e-12 * scale * 40
    assert abs(st0[0][0] - sto[0]) <= 1e-12 * abs(sto[0])
