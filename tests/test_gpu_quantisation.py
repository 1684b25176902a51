"""The BF16 path against the exact model of the FP32 master weights.

The parity tests compare the BF16 path with the oracle's BF16 model (the same
BF16-rounded weights, bfloat16 hidden activations).  These tests state how far
that model, as the kernels compute it, lies from the exact model: the oracle in
FP64 with the FP32 master weights unrounded and exact hidden activations.  At
the two sparse benchmark workloads (G(10000, 8/9999) with h = 2000, and the
random 3-regular graph with n = h = 1000) they measure and report

  * log pi of seeded configurations (vqmc_logprob, BF16 GEMMs): relative error
    per sample;
  * the logits on the samples' own prefixes, and the fraction of draws whose
    decision [u < p_i] the rounding flips (teacher-forced against the exact
    model's conditionals), and the rows that differ from the exact model's
    free-running samples on the same uniforms;
  * the score-function gradient of a sub-batch with its energies (vqmc_grad):
    ||g - g_exact|| / ||g_exact|| and per parameter block.

Asserted bounds are the stated BF16 tolerance for log pi (relative 2e-2) and a
loose sanity bound on the gradient (5e-2: BF16 keeps 8 significant bits, a
relative rounding of at most 2^-9 per weight and per GEMM operand); the
measured values are reported in the end-of-run summary.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2106_13308_gb300 import inputs

from conftest import report
from gpu_helpers import act_code, build_lib, grad_blocks, make_model, oracle_params, rel_err, sigmoid

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build_lib()
    assert torch.cuda.is_available()


@pytest.mark.parametrize("name,rows,gsub", [("maxcut_er10000", 16, 256), ("maxcut_3reg1000", 64, 512)])
def test_bf16_error_against_exact_model(name, rows, gsub):
    cfg = inputs.config(name)
    inst = inputs.make_instance(cfg)
    n, h, B = cfg["n"], cfg["h"], cfg["B"]
    theta = inputs.lively_params(n, h, cfg["param_seed"])
    seed = 4242
    m = make_model(n, h, B, inst, precision="bf16", theta=theta, seed=seed)
    exact = oracle_params(theta, n, h, "fp32")      # masked FP32 master, promoted to FP64
    bf16 = oracle_params(theta, n, h, "bf16")       # the BF16 model
    code_exact, code_bf16 = act_code("relu", "fp32"), act_code("relu", "bf16")

    # log pi of seeded configurations
    Sc = inputs.spins(64, n, 91)
    lp = m.logprob(torch.from_numpy(Sc).cuda()).cpu().numpy().astype(np.float64)
    lpo = oracle.logprob(exact, Sc, code_exact)
    lrel = np.abs(lp - lpo) / np.abs(lpo)

    # samples: the BF16 sampler (internal Philox) on the exact model's conditionals
    S, _ = m.sample(B, None, iteration=0)
    Sn = S.cpu().numpy()[:rows]
    U = oracle.uniforms(B, n, seed, 0)[:rows]
    Ze = oracle.logits(exact, Sn, code_exact)
    Zb = oracle.logits(bf16, Sn, code_bf16)
    flips = (Sn == 1) != (U.astype(np.float64) < sigmoid(Ze))
    So, _ = oracle.sample(exact, U, code_exact)
    differ = ~(Sn == So).all(axis=1)
    first = [int(np.argmax(Sn[r] != So[r])) for r in range(rows) if differ[r]]

    # gradient of a sub-batch with its energies
    Sg = S[:gsub].contiguous()
    Eg = m.local_energy(Sg)
    g, _ = m.grad(Sg, Eg)
    g = g.cpu().numpy()
    (dW1, db1, dW2, db2), _, _ = oracle.vqmc_grad(exact, inst, Sg.cpu().numpy(), code_exact)
    go = oracle.made_to_theta(dW1, db1, dW2, db2)
    grel = rel_err(g, go)
    blocks = {k: rel_err(v, grad_blocks(go, n, h)[k]) for k, v in grad_blocks(g, n, h).items()}

    report(f"bf16 vs exact model {name}",
           logp_rel_max=float(lrel.max()), logp_rel_median=float(np.median(lrel)),
           logit_abs_max=float(np.abs(Zb - Ze).max()), logit_abs_rms=float(np.sqrt(np.mean((Zb - Ze) ** 2))),
           draws=int(Sn.size), draws_flipped=int(flips.sum()), flip_rate=float(flips.mean()),
           rows=rows, rows_differing=int(differ.sum()),
           first_divergence_median=(float(np.median(first)) if first else None),
           grad_samples=gsub, grad_rel=grel, grad_rel_blocks=blocks)
    assert lrel.max() <= 2e-2
    assert grel <= 5e-2
    assert m.check() == 0
