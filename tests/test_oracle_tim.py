"""Pins for the oracle's transverse-field Ising local energy (Eq. (hamiltonian),
matrix entries Eq. (e:tim)) against the Hamiltonian built as an explicit
2^n x 2^n matrix from Kronecker products of the Pauli matrices, the
variational principle, and the gradient identity behind the score-function
estimator (Sec. 2.1) checked by finite differences."""
import itertools

import numpy as np
import pytest

import oracle
from paper_2106_13308_gb300 import inputs

I2 = np.eye(2)
X2 = np.array([[0.0, 1.0], [1.0, 0.0]])
Z2 = np.array([[1.0, 0.0], [0.0, -1.0]])


def _op(n, i, P):
    """I^(i) (x) P (x) I^(n-i-1): P on spin i (0-based), spin 0 the most
    significant bit of the row index, as in Eq. (hamiltonian)."""
    M = np.ones((1, 1))
    for q in range(n):
        M = np.kron(M, P if q == i else I2)
    return M


def _hamiltonian(inst):
    """H = -sum_i (alpha_i X_i + beta_i Z_i) - sum_{i<j} beta_ij Z_i Z_j with
    beta = -J, beta_i = -h_i (the instance's Ising form)."""
    n = inst["n"]
    J = np.asarray(inst["J"], np.float64)
    f = np.asarray(inst["field"], np.float64)
    a = np.asarray(inst["alpha"], np.float64)
    H = np.zeros((2 ** n, 2 ** n))
    for i in range(n):
        H -= a[i] * _op(n, i, X2) + (-f[i]) * _op(n, i, Z2)
        for j in range(i + 1, n):
            H -= (-J[i, j]) * (_op(n, i, Z2) @ _op(n, j, Z2))
    return H


def _all_states(n):
    """Every configuration in row-index order: x = sum_i 2^(n-1-i) x_i,
    spin s_i = 1 - 2 x_i (Z eigenvalue of bit x_i)."""
    X = np.array(list(itertools.product([0, 1], repeat=n)), dtype=np.int64)
    return (1 - 2 * X).astype(np.int8)


def _case(n, h, seed, act):
    inst = inputs.tim(n, seed)
    theta = inputs.lively_params(n, h, seed + 1)
    P = oracle.theta_to_made(_masked(theta, n, h), n, h)
    return inst, theta, P


def _masked(theta, n, h):
    t = np.array(theta, dtype=np.float64, copy=True)
    m = oracle.degrees(n, h)
    W1t = t[: n * h].reshape(n, h)
    W2 = t[n * h + h: 2 * n * h + h].reshape(n, h)
    r = np.arange(n)[:, None]
    W1t[~(r < m[None, :])] = 0
    W2[~(m[None, :] <= r)] = 0
    return t


@pytest.mark.parametrize("act", [oracle.RELU, oracle.SIGMOID])
@pytest.mark.parametrize("n,h", [(4, 6), (5, 3)])
def test_tim_local_energy_equals_h_psi_over_psi(n, h, act):
    """E_loc(x) = (H psi)(x) / psi(x) with psi = sqrt(pi), for every x."""
    inst, _, P = _case(n, h, 30 + n, act)
    S = _all_states(n)
    pi = np.exp(oracle.logprob(P, S, act))
    assert abs(pi.sum() - 1.0) < 1e-12
    psi = np.sqrt(pi)
    want = (_hamiltonian(inst) @ psi) / psi
    got = oracle.local_energy(P, inst, S, act)
    assert np.allclose(got, want, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_tim_variational_bound(seed):
    """sum_x pi(x) E_loc(x) = <psi|H|psi> >= lowest eigenvalue of H."""
    n, h = 6, 5
    inst, _, P = _case(n, h, 50 + seed, oracle.RELU)
    S = _all_states(n)
    pi = np.exp(oracle.logprob(P, S))
    E = oracle.local_energy(P, inst, S)
    H = _hamiltonian(inst)
    psi = np.sqrt(pi)
    energy = float(pi @ E)
    assert abs(energy - float(psi @ H @ psi)) < 1e-11
    assert energy >= np.linalg.eigvalsh(H)[0] - 1e-12


def test_tim_score_function_gradient_is_the_gradient_of_the_energy():
    """d<H>/dtheta = sum_x pi(x) (E_loc(x) - <H>) d log pi(x)/dtheta although
    E_loc itself depends on theta (H is symmetric and psi = sqrt(pi) is real):
    the estimator's expectation against central finite differences of the
    exact <H>."""
    n, h = 5, 4
    inst, theta, P = _case(n, h, 70, oracle.SIGMOID)
    S = _all_states(n)

    def exact_energy(t):
        Q = oracle.theta_to_made(_masked(t, n, h), n, h)
        pi = np.exp(oracle.logprob(Q, S, oracle.SIGMOID))
        return float(pi @ oracle.local_energy(Q, inst, S, oracle.SIGMOID))

    pi = np.exp(oracle.logprob(P, S, oracle.SIGMOID))
    E = oracle.local_energy(P, inst, S, oracle.SIGMOID)
    L = float(pi @ E)
    g = oracle.made_to_theta(*oracle.logprob_grad(P, S, pi * (E - L), oracle.SIGMOID))
    t0 = _masked(theta, n, h)
    keep = _masked(np.ones_like(theta), n, h) != 0
    idx = np.random.default_rng(71).choice(np.flatnonzero(keep), size=12, replace=False)
    eps = 1e-5
    for k in idx:
        tp, tm = t0.copy(), t0.copy()
        tp[k] += eps
        tm[k] -= eps
        fd = (exact_energy(tp) - exact_energy(tm)) / (2 * eps)
        assert abs(fd - g[k]) <= 1e-7 + 1e-6 * abs(g[k]), (k, fd, g[k])


def test_tim_without_transverse_field_is_the_ising_energy():
    n, h = 12, 9
    inst, _, P = _case(n, h, 90, oracle.RELU)
    inst = dict(inst, alpha=np.zeros(n, dtype=np.float32))
    S = inputs.spins(64, n, 91)
    assert np.array_equal(oracle.local_energy(P, inst, S), oracle.energy(inst, S))
    assert np.array_equal(oracle.energy_tim_offdiag(P, S, inst["alpha"]), np.zeros(64))
