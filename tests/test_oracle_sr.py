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


def test_per_sample_gradient_against_central_differences():
    """O[b] against central differences of log pi(s_b) (FP64, eps = 1e-6) on
    random parameters of every block (sigmoid hidden units: no kinks)."""
    n, h = 9, 7
    theta = inputs.lively_params(n, h, 21).astype(np.float64)
    S = inputs.spins(5, n, 22)
    act = oracle.SIGMOID
    P = oracle.theta_to_made(theta, n, h)
    deg = oracle.degrees(n, h)
    O = oracle.per_sample_grads(P, S, act)
    rng = np.random.default_rng(23)
    d = theta.size
    eps = 1e-6
    for p in rng.choice(d, 40, replace=False):
        tp, tm = theta.copy(), theta.copy()
        tp[p] += eps
        tm[p] -= eps
        fd = (oracle.logprob(oracle.theta_to_made(tp, n, h), S, act)
              - oracle.logprob(oracle.theta_to_made(tm, n, h), S, act)) / (2 * eps)
        # entries outside the MADE masks are not parameters of the model
        if p < n * h:
            j, k = divmod(p, h)
            if not deg[k] >= j + 1:
                assert np.all(O[:, p] == 0)
                continue
        elif n * h + h <= p < 2 * n * h + h:
            i, k = divmod(p - n * h - h, h)
            if not i + 1 > deg[k]:
                assert np.all(O[:, p] == 0)
                continue
        assert np.allclose(O[:, p], fd, rtol=1e-6, atol=1e-8)


def test_sr_gram_is_the_matrix_of_inner_products():
    inst, P, S, act = _case()
    O = oracle.per_sample_grads(P, S, act)
    G = oracle.sr_gram(P, S, act)
    assert np.allclose(G, G.T, rtol=0, atol=0)
    assert np.allclose(np.diag(G), (O * O).sum(axis=1), rtol=1e-12)
    assert np.linalg.eigvalsh(G).min() > -1e-9 * np.abs(G).max()
