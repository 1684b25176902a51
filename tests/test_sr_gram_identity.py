"""The identity behind the GPU's stochastic-reconfiguration Gram kernel
(Sec. 2.1 Fisher form), checked on CPU against the oracle's explicit
per-sample score vectors O_b = grad log pi(s_b):

    O O^T = sum_i (delta_i delta_i^T) o P_i + sum_k (GA_k GA_k^T) o Q_{m(k)},
    P_i = 1 + sum_{k: m(k) < i} H_k H_k^T,   Q_t = 1 + sum_{j <= t} s_j s_j^T,

evaluated in the kernel's order (spin t, then the hidden units of degree t).
delta (the b2 block of O), GA (the b1 block) and H (the last output row of
the W2 block divided by delta, that output sees every unit) are read off the
oracle's O, so a wrong mask boundary or event order in the recurrence shows
as a mismatch."""
import numpy as np
import pytest

import oracle
from paper_2106_13308_gb300 import inputs


def _recurrence(S, delta, GA, H, n, h):
    B = S.shape[0]
    deg = oracle.degrees(n, h)
    G = np.zeros((B, B))
    P = np.ones((B, B))
    Q = np.ones((B, B))
    k = 0
    for t in range(n):  # spin t + 1 (1-based), then the units of degree t + 1
        Q += np.outer(S[:, t], S[:, t])
        G += np.outer(delta[:, t], delta[:, t]) * P
        while k < h and deg[k] == t + 1:
            G += np.outer(GA[:, k], GA[:, k]) * Q
            P += np.outer(H[:, k], H[:, k])
            k += 1
    assert k == h
    return G


@pytest.mark.parametrize("n,h,act", [(9, 14, oracle.SIGMOID), (12, 5, oracle.RELU), (7, 7, oracle.SIGMOID)])
def test_degree_ordered_recurrence_equals_the_gram_matrix(n, h, act):
    B = 40
    theta = inputs.lively_params(n, h, 50 + n)
    P = oracle.theta_to_made(theta, n, h)
    S = inputs.spins(B, n, 60 + n).astype(np.float64)
    O = oracle.per_sample_grads(P, S.astype(np.int8), act)
    nh = n * h
    delta = O[:, 2 * nh + h:]
    GA = O[:, nh:nh + h]
    last = O[:, nh + h + (n - 1) * h: nh + h + n * h]  # dW2 of output n: delta_n H_k for every unit
    H = last / delta[:, n - 1:n]
    G = _recurrence(S, delta, GA, H, n, h)
    ref = O @ O.T
    assert np.allclose(G, ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max())


def test_recurrence_detects_a_shifted_mask():
    """Adding the units of degree t before spin t's output term (one step
    early) changes the result: the test above would catch that mistake."""
    n, h, B = 8, 12, 24
    theta = inputs.lively_params(n, h, 7)
    P = oracle.theta_to_made(theta, n, h)
    S = inputs.spins(B, n, 8).astype(np.float64)
    O = oracle.per_sample_grads(P, S.astype(np.int8), oracle.SIGMOID)
    nh = n * h
    delta, GA = O[:, 2 * nh + h:], O[:, nh:nh + h]
    H = O[:, nh + h + (n - 1) * h:] / delta[:, n - 1:n]
    deg = oracle.degrees(n, h)
    G = np.zeros((B, B))
    Pm, Qm = np.ones((B, B)), np.ones((B, B))
    k = 0
    for t in range(n):
        Qm += np.outer(S[:, t], S[:, t])
        while k < h and deg[k] == t + 1:  # wrong order: units before the output term
            G += np.outer(GA[:, k], GA[:, k]) * Qm
            Pm += np.outer(H[:, k], H[:, k])
            k += 1
        G += np.outer(delta[:, t], delta[:, t]) * Pm
    assert not np.allclose(G, O @ O.T, rtol=1e-6)
