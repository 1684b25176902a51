"""GPU tests of sampling parallelism (Sec. 4): K contexts on one GPU stand in
for K ranks, each drawing its shard of one batch (vqmc_set_sample_offset),
writing its shard sums (vqmc_shard_sums) and applying the update from the
sums added over the shards (vqmc_shard_apply); the host adds the sums in
place of the all-reduce.  No kernel waits on another context's kernels.

Checked against the full batch drawn by one context and against the oracle:
  * the shards' samples, concatenated, equal the full batch's bit for bit
    (same Philox counters);
  * the combined gradient equals the oracle's score-function gradient of the
    full batch (relative 1e-4 with FP32 weights, 3e-2 with BF16 weights, as
    the parity tests), for a shift of 0 and a shift near the mean;
  * every shard ends with bit-identical parameters, and the next iteration's
    shards again equal the full batch drawn from those parameters.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2106_13308_gb300 import inputs

from conftest import report
from gpu_helpers import act_code, build_lib, er_instance, make_model, oracle_params, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build_lib()
    assert torch.cuda.is_available()


CASES = [
    # n, h, shard batch, shards, precision, sampler
    (300, 200, 64, 3, "fp32", "auto"),      # CUDA-core sampler, FP32 GEMMs
    (1500, 300, 48, 2, "bf16", "auto"),     # tensor-core sampler, tcgen05 GEMMs
    (257, 130, 40, 4, "bf16", "cuda_core"),
]


@pytest.mark.parametrize("n,h,Bl,K,prec,sampler", CASES)
@pytest.mark.parametrize("near_mean", [False, True])
def test_virtual_shards_equal_the_full_batch(n, h, Bl, K, prec, sampler, near_mean):
    inst = er_instance(n, 0.02, 5)
    theta = inputs.lively_params(n, h, 6)
    seed = 9001
    Bt = Bl * K
    full = make_model(n, h, Bt, inst, precision=prec, theta=theta, seed=seed, sampler=sampler)
    shards = [make_model(n, h, Bl, inst, precision=prec, theta=theta, seed=seed, sampler=sampler) for _ in range(K)]
    for k, m in enumerate(shards):
        m.set_sample_offset(k * Bl)
    Sf, _ = full.sample(Bt, None, iteration=0)
    Ef = full.local_energy(Sf)
    shift = float(Ef.double().mean().item()) + 0.37 if near_mean else 0.0

    sums, scal = None, None
    for m in shards:
        s, c = m.shard_sums(Bl, shift)
        sums = s.clone() if sums is None else sums + s
        scal = c.clone() if scal is None else scal + c
    # the shards drew exactly the full batch's samples and energies
    Ss = torch.cat([m.last_batch(Bl)[0] for m in shards])
    Es = torch.cat([m.last_batch(Bl)[1] for m in shards])
    assert torch.equal(Ss, Sf) and torch.equal(Es, Ef)

    outs = [m.shard_apply(sums, scal, shift) for m in shards]
    g = outs[0][0].cpu().numpy()
    for gk, _ in outs[1:]:
        assert np.array_equal(gk.cpu().numpy(), g)
    P = oracle_params(theta, n, h, prec)
    code = act_code("relu", prec)
    (dW1, db1, dW2, db2), sto, _ = oracle.vqmc_grad(P, inst, Sf.cpu().numpy(), code)
    go = oracle.made_to_theta(dW1, db1, dW2, db2)
    err = rel_err(g, go)
    st = outs[0][1].cpu().numpy()
    report(f"shards {prec} n={n} h={h} {K}x{Bl} shift={'near mean' if near_mean else 0}", grad_rel=err,
           mean=float(st[0]), mean_ref=float(sto[0]))
    assert err <= (1e-4 if prec == "fp32" else 3e-2)
    assert abs(st[0] - sto[0]) <= 1e-12 * abs(sto[0]) + 1e-9
    assert abs(st[1] - sto[1]) <= 1e-9 * abs(sto[1]) + 1e-6

    # identical replicas; the next iteration's shards are the full batch of the new parameters
    th = shards[0].get_params().numpy()
    for m in shards[1:]:
        assert np.array_equal(m.get_params().numpy(), th)
        assert m.iteration == 1
    full.set_params(torch.from_numpy(th))
    Sf1, _ = full.sample(Bt, None, iteration=1)
    S1 = []
    for m in shards:
        m.shard_sums(Bl, shift)
        S1.append(m.last_batch(Bl)[0].clone())
    assert torch.equal(torch.cat(S1), Sf1)
    for m in shards:
        assert m.check() == 0
        m.close()
    full.close()


def test_shard_calls_reject_bad_arguments():
    from paper_2106_13308_gb300 import vqmc
    n, h, B = 40, 16, 8
    m = make_model(n, h, B, er_instance(n, 0.2, 7))
    sums = torch.zeros(2 * m.d, dtype=torch.float32, device="cuda")
    scal = torch.zeros(3, dtype=torch.float64, device="cuda")
    S = torch.ones((B, n), dtype=torch.int8, device="cuda")
    with pytest.raises(vqmc.VQMCError):  # samples without energies
        vqmc.vqmc_shard_sums(m.ctx, B, S, None, 0.0, sums, scal)
    with pytest.raises(vqmc.VQMCError):  # non-finite shift
        vqmc.vqmc_shard_sums(m.ctx, B, None, None, float("nan"), sums, scal)
    with pytest.raises(vqmc.VQMCError):  # batch above max_batch
        vqmc.vqmc_shard_sums(m.ctx, B + 1, None, None, 0.0, sums, scal)
    # B = 0 writes zeros
    sums.fill_(1.0)
    vqmc.vqmc_shard_sums(m.ctx, 0, None, None, 0.0, sums, scal)
    assert float(sums.abs().sum()) == 0.0 and float(scal.abs().sum()) == 0.0
    # a zero total count gives a zero gradient and the non-finite flag
    g, _ = m.shard_apply(sums, scal, 0.0)
    assert float(g.abs().sum()) == 0.0
    assert m.check() != 0
