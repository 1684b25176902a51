"""Pins for the oracle's local energies, Max-Cut mapping, statistics and Adam."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2106_13308_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _graph(family, n, a=None, b=None):
    if family == "complete":
        e = [(i, j) for i in range(n) for j in range(i + 1, n)]
    elif family == "cycle":
        e = [(min(i, (i + 1) % n), max(i, (i + 1) % n)) for i in range(n)]
    elif family == "bipartite":
        e = [(i, a + j) for i in range(a) for j in range(b)]
    elif family == "petersen":
        outer = [(i, (i + 1) % 5) for i in range(5)]
        spokes = [(i, i + 5) for i in range(5)]
        inner = [(5 + i, 5 + (i + 2) % 5) for i in range(5)]
        e = [(min(p), max(p)) for p in outer + spokes + inner]
    else:
        raise ValueError(family)
    e = np.array(sorted(set(e)), dtype=np.int64)
    return inputs.to_csr(n, e, np.ones(len(e), dtype=np.int32))


def test_bruteforce_maxcut_textbook_graphs():
    gold = json.load(open(os.path.join(GOLD, "maxcut_small_graphs.json")))
    for g in gold["graphs"]:
        inst = _graph(g["family"], g["n"], g.get("a"), g.get("b"))
        assert oracle.maxcut_bruteforce(inst) == g["maxcut"], g["name"]


def test_cut_equals_ising_mapping():
    """Max-Cut special case of Eq. (hamiltonian): with E(s) = sum_{i<j} w_ij s_i s_j
    and h = 0, cut(s) = (W_tot - E(s)) / 2 exactly, for integer weights."""
    for n, seed in [(30, 1), (200, 2)]:
        e = inputs.erdos_renyi(n, 0.3, seed)
        w = inputs.int_weights(len(e), -5, 9, seed + 7)
        inst = inputs.to_csr(n, e, w)
        S = inputs.spins(100, n, seed + 3)
        E = oracle.energy(inst, S)
        c = oracle.cut(inst, S)
        assert np.array_equal(c, (w.sum() - E) / 2)
        assert np.all(E == np.round(E))


def test_dense_and_sparse_energies_agree_and_match_quadratic_form():
    n = 40
    e = inputs.erdos_renyi(n, 0.4, 5)
    w = inputs.int_weights(len(e), -3, 3, 6)
    field = inputs.int_weights(n, -2, 2, 8)
    inst = inputs.to_csr(n, e, w, field=field)
    J = inputs.dense_from_sparse(inst)
    S = inputs.spins(64, n, 7)
    Es = oracle.energy(inst, S)
    Ed = oracle.energy_dense(J, S, field)
    assert np.array_equal(Es, Ed)
    # library routine: E = 1/2 s^T J s + h.s
    Sf = S.astype(np.float64)
    ref = 0.5 * np.einsum("bi,ij,bj->b", Sf, J, Sf) + Sf @ field
    assert np.allclose(Ed, ref, rtol=0, atol=1e-9)
    sk = inputs.sk(50, 9)
    S2 = inputs.spins(16, 50, 10).astype(np.float64)
    E2 = oracle.energy_dense(sk["J"], S2)
    ref2 = 0.5 * np.einsum("bi,ij,bj->b", S2, sk["J"].astype(np.float64), S2)
    assert np.allclose(E2, ref2, rtol=1e-12, atol=1e-12)


def test_bruteforce_bounds_variational_and_enumeration():
    """Enumerated <E> is >= the ground energy (variational inequality,
    Sec. 2.1), and the ground energy is W_tot - 2 * maxcut."""
    n, h = 12, 18
    e = inputs.erdos_renyi(n, 0.5, 11)
    w = np.ones(len(e), dtype=np.int32)
    inst = inputs.to_csr(n, e, w)
    mc = oracle.maxcut_bruteforce(inst)
    th = inputs.lively_params(n, h, 12)
    out = oracle.enumerate_exact(oracle.theta_to_made(th, n, h), inst)
    Emin = w.sum() - 2 * mc
    assert out[1] >= Emin - 1e-12
    # enumeration of E over all states reaches exactly Emin
    states = np.array([[1 - 2 * ((x >> i) & 1) for i in range(n)] for x in range(1 << n)], dtype=np.int8)
    assert oracle.energy(inst, states).min() == Emin


def test_paper_generator_density_matches_table2_random_row():
    """The reading 'round half to even' of the paper's Max-Cut generator
    (Sec. 5.1) gives edge density 1/4, which the Table 2 Random row fixes:
    2 * E[random cut] / (n(n-1)/2) ~ 1/4."""
    gold = json.load(open(os.path.join(GOLD, "paper_table2_random_cut.json")))
    for n, rc in zip(gold["n"], gold["random_cut_mean"]):
        pairs = n * (n - 1) / 2
        printed_density = 2 * rc / pairs
        m = len(inputs.paper_maxcut(n, 100 + n))
        ours = m / pairs
        tol = 0.05 if n <= 20 else 0.02
        assert abs(printed_density - 0.25) < tol + 0.04 * (n <= 20)
        assert abs(ours - 0.25) < tol
        # a random partition cuts half the edges in expectation
        inst = inputs.to_csr(n, inputs.paper_maxcut(n, 100 + n), np.ones(m, dtype=np.int32))
        S = inputs.spins(400, n, 7)
        assert abs(oracle.cut(inst, S).mean() / m - 0.5) < 0.03


def test_stats_known_values():
    E = np.array([1.0, 2.0, 3.0, 6.0])
    st, coef = oracle.stats(E)
    assert st.tolist() == [3.0, 3.5, 1.0, 6.0]
    assert coef.tolist() == [-0.5, -0.25, 0.0, 0.75]
    assert abs(coef.sum()) == 0.0


def test_adam_closed_form_constant_gradient():
    """With a constant gradient the bias-corrected moments are m^ = g and
    v^ = g^2 at every step, so each Adam step moves lr * g / (|g| + eps)."""
    rng = np.random.default_rng(3)
    d = 50
    theta0 = rng.standard_normal(d)
    g = rng.standard_normal(d)
    theta, m, v = theta0.copy(), np.zeros(d), np.zeros(d)
    for t in range(1, 6):
        oracle.adam(theta, m, v, g, t, lr=1e-2)
        ref = theta0 - t * 1e-2 * g / (np.abs(g) + 1e-8)
        assert np.allclose(theta, ref, rtol=0, atol=1e-12)
    # zero gradient leaves parameters unchanged
    th2, m2, v2 = theta0.copy(), np.zeros(d), np.zeros(d)
    oracle.adam(th2, m2, v2, np.zeros(d), 1)
    assert np.array_equal(th2, theta0)


def test_vqmc_gradient_estimator_is_unbiased_on_tiny_n():
    """Averaged over many batches, sum_b c_b grad log pi(s_b) approaches the
    enumerated exact gradient (the estimator of Sec. 2.1 with the batch-mean
    baseline is consistent; its bias is O(1/B))."""
    n, h, B, R = 6, 8, 4096, 6
    P = oracle.theta_to_made(inputs.lively_params(n, h, 30), n, h)
    e = inputs.erdos_renyi(n, 0.7, 31)
    inst = inputs.to_csr(n, e, inputs.int_weights(len(e), -2, 3, 32))
    _, gex = oracle.enumerate_exact(P, inst, grad=True)
    gex = oracle.made_to_theta(*gex)
    acc = np.zeros_like(gex)
    for r in range(R):
        U = inputs.uniforms(B, n, 40 + r)
        S, _ = oracle.sample(P, U)
        g, _, _ = oracle.vqmc_grad(P, inst, S)
        acc += oracle.made_to_theta(*g)
    acc /= R
    rel = np.linalg.norm(acc - gex) / np.linalg.norm(gex)
    assert rel < 0.1, rel
