"""Pins for the oracle's stochastic reconfiguration (natural-gradient) step,
Sec. 2.1: the Fisher estimate and gradient of the paper's population forms
and the regularised solve, checked against the push-through (Woodbury) form
on the B x B Gram matrix, the large-lambda limit, the linear system's
residual, and the batch gradient pinned elsewhere."""
import numpy as np
import pytest

import oracle
from paper_2106_13308_gb300 import inputs


def _case(n=14, h=9, B=24, seed=3, act=oracle.SIGMOID):
    inst = inputs.tim(n, seed)
    theta = inputs.lively_params(n, h, seed + 1)
    P = oracle.theta_to_made(theta, n, h)
    S = inputs.spins(B, n, seed + 2)
    return inst, P, S, act


def test_per_sample_gradients_sum_to_the_batch_gradient():
    inst, P, S, act = _case()
    O = oracle.per_sample_grads(P, S, act)
    c = np.random.default_rng(5).standard_normal(S.shape[0])
    g = oracle.made_to_theta(*oracle.logprob_grad(P, S, c, act))
    assert np.allclose(O.T @ c, g, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("lam", [1e-3, 0.1])
def test_sr_direction_equals_the_gram_form(lam):
    """(I + lam)^-1 g with I = O^T O / B, g = O^T eps / B equals
    O^T (O O^T + lam B)^-1 eps, eps = E - mean E (B x B instead of d x d)."""
    inst, P, S, act = _case()
    delta, st = oracle.sr_direction(P, inst, S, lam, act)
    O = oracle.per_sample_grads(P, S, act)
    eps = oracle.local_energy(P, inst, S, act) - st[0]
    B = S.shape[0]
    dual = O.T @ np.linalg.solve(O @ O.T + lam * B * np.eye(B), eps)
    assert np.allclose(delta, dual, rtol=1e-8, atol=1e-10 * np.abs(dual).max())


def test_sr_direction_solves_the_regularised_system_and_tends_to_the_gradient():
    inst, P, S, act = _case()
    O = oracle.per_sample_grads(P, S, act)
    B = S.shape[0]
    eps = oracle.local_energy(P, inst, S, act)
    eps = eps - eps.mean()
    g = O.T @ eps / B
    for lam in (1e-2, 1.0):
        delta, _ = oracle.sr_direction(P, inst, S, lam, act)
        r = (O.T @ (O @ delta)) / B + lam * delta - g
        assert np.linalg.norm(r) <= 1e-9 * np.linalg.norm(g)
    # a large lambda turns SR into plain gradient descent with step 1/lambda
    lam = 1e8
    delta, _ = oracle.sr_direction(P, inst, S, lam, act)
    assert np.allclose(lam * delta, g, rtol=1e-5, atol=1e-12)
