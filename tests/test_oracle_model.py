"""Pins for the oracle's MADE model, sampler, generator and gradient.

Each test checks the FP64 oracle against something other than itself: a
published known-answer vector, a closed form, an invariant of the
autoregressive construction, exhaustive enumeration, or central finite
differences.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2106_13308_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _params(n, h, seed, scale=1.0):
    th = inputs.made_params(n, h, seed, w_std=scale * 1.5 / math.sqrt(n), v_std=scale * 3.0 / math.sqrt(h),
                            bias_std=0.5)
    return oracle.theta_to_made(th, n, h)


def _small_instance(n, seed, p=0.5, weights="int"):
    e = inputs.erdos_renyi(n, p, seed)
    if weights == "int":
        w = inputs.int_weights(len(e), -3, 5, seed + 1)
    else:
        w = np.random.default_rng(seed).standard_normal(len(e)).astype(np.float32)
    inst = inputs.to_csr(n, e, w)
    return inst


# ------------------------------------------------------------ generator

def test_philox_known_answers():
    """Philox4x32-10 matches the generator's published known-answer vectors."""
    kat = json.load(open(os.path.join(GOLD, "philox4x32_10_kat.json")))
    for v in kat["vectors"]:
        ctr = [int(x, 16) for x in v["ctr"]]
        key = [int(x, 16) for x in v["key"]]
        out = [int(x, 16) for x in v["out"]]
        assert list(oracle.philox4x32_10(ctr, key)) == out


def test_uniform_grid_and_moments():
    u = oracle.uniforms(64, 257, seed=12345, it=7)
    assert u.dtype == np.float32 and u.min() >= 0.0 and u.max() < 1.0
    assert np.all((u.astype(np.float64) * (1 << 24)) % 1.0 == 0.0)
    assert abs(u.mean() - 0.5) < 0.01 and abs(u.var() - 1 / 12) < 0.005
    # distinct iterations and seeds give distinct streams
    assert not np.array_equal(u, oracle.uniforms(64, 257, seed=12345, it=8))
    assert not np.array_equal(u, oracle.uniforms(64, 257, seed=12346, it=7))
    # word (i mod 4) of counter (i/4, b, it): spot-check one entry against the raw generator
    w = oracle.philox4x32_10([5, 3, 7, 0], [12345, 0])
    assert u[3, 22] == np.float32((int(w[2]) >> 8) / float(1 << 24))


# ----------------------------------------------------------------- model

def test_degrees_sorted_and_in_range():
    for n, h in [(20, 40), (1000, 1000), (10000, 2000), (7, 3), (2, 5)]:
        m = oracle.degrees(n, h)
        assert m[0] == 1 and np.all(np.diff(m) >= 0) and m.max() <= max(n - 1, 1)


BF16_RELU = oracle.RELU | oracle.HIDDEN_BF16
BF16_SIGMOID = oracle.SIGMOID | oracle.HIDDEN_BF16


@pytest.mark.parametrize("act", [oracle.RELU, oracle.SIGMOID, BF16_RELU, BF16_SIGMOID])
def test_autoregressive_property(act):
    """z_i depends only on s_<i: changing s_i..s_n leaves z_i unchanged."""
    n, h = 13, 29
    P = _params(n, h, 3)
    rng = np.random.default_rng(0)
    s = inputs.spins(1, n, 4)[0]
    _, z = oracle.forward(P, s, act)
    assert z[0] == P[3][0]  # p(s_1) = sigma(c_1)
    for i in range(n):
        for _ in range(4):
            t = s.copy()
            t[i:] = np.where(rng.random(n - i) < 0.5, 1, -1)
            _, z2 = oracle.forward(P, t, act)
            assert np.array_equal(z2[: i + 1], z[: i + 1])
    # with h >= n - 1 every degree 1..n-1 is used, so z_i depends on s_{i-1}
    # for every i >= 2 (M1 uses m(k) >= j, M2 uses i > m(k): maximal
    # connectivity).  Checked with the sigmoid, which has no dead units.
    if act & 1 != oracle.SIGMOID:
        return
    for i in range(1, n):
        t = s.copy()
        t[i - 1] = -t[i - 1]
        _, z3 = oracle.forward(P, t, act)
        assert z3[i] != z[i], i


@pytest.mark.parametrize("n,h,act", [(12, 20, oracle.RELU), (12, 20, oracle.SIGMOID), (20, 40, oracle.SIGMOID),
                                     (12, 20, BF16_RELU), (14, 9, BF16_SIGMOID)])
def test_normalisation_by_enumeration(n, h, act):
    """sum_s pi(s) = 1 (autoregressive normalisation, Sec. 2.3)."""
    P = _params(n, h, 5)
    inst = _small_instance(n, 6)
    out = oracle.enumerate_exact(P, inst, act)
    assert abs(out[0] - 1.0) < 1e-12


# ------------------------------------------------ bfloat16 hidden layer

def test_round_bf16_matches_library_conversion():
    """vo_round_bf16 on binary32 inputs equals the library's float -> bfloat16
    conversion (round to nearest, ties to even): random magnitudes, exact
    halfway cases with even and odd kept significands, subnormals, signs."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(31)
    x = (rng.standard_normal(3000) * np.exp2(rng.integers(-40, 40, 3000))).astype(np.float32)
    bits = rng.integers(0, 1 << 16, 400, dtype=np.uint32) << 16
    halfway = ((bits | 0x8000) & 0x7F7FFFFF).view(np.float32)  # exactly between two bf16 values
    sub = (rng.integers(1, 1 << 23, 200, dtype=np.uint32)).view(np.float32)  # binary32 subnormals
    vals = np.concatenate([x, -x[:500], halfway, -halfway[:100], sub, np.float32([0.0, 1.0, -2.5, 3.0e38])])
    ref = torch.from_numpy(vals).to(torch.bfloat16).to(torch.float64).numpy()
    got = oracle.round_bf16(vals.astype(np.float64))
    assert np.array_equal(got, ref)


def test_hidden_bf16_is_identity_on_representable_activations():
    """With integer weights and biases every ReLU activation is a small
    integer, exactly representable in bfloat16, so the BF16 hidden layer
    gives the same logits as the exact one."""
    n, h = 9, 14
    rng = np.random.default_rng(33)
    th = oracle.made_to_theta(rng.integers(-3, 4, (h, n)).astype(np.float64), rng.integers(-2, 3, h).astype(np.float64),
                              rng.integers(-3, 4, (n, h)).astype(np.float64), rng.integers(-2, 3, n).astype(np.float64))
    P = oracle.theta_to_made(th, n, h)
    S = inputs.spins(16, n, 34)
    assert np.array_equal(oracle.logits(P, S, oracle.RELU), oracle.logits(P, S, BF16_RELU))


@pytest.mark.parametrize("act", [oracle.RELU, oracle.SIGMOID])
def test_hidden_bf16_logit_shift_within_rounding_bound(act):
    """Rounding each g1_k to 8 significant bits moves z_i by at most
    sum_k |W2_ik| |g1_k| 2^-8 (relative rounding error of bfloat16 <= 2^-9,
    doubled for slack), and it does move some logits."""
    n, h = 30, 45
    P = _params(n, h, 35)
    S = inputs.spins(8, n, 36)
    W1, b1, W2, b2 = P
    Z = oracle.logits(P, S, act)
    Zq = oracle.logits(P, S, act | oracle.HIDDEN_BF16)
    m = oracle.degrees(n, h)
    for b in range(S.shape[0]):
        a, _ = oracle.forward(P, S[b], act)
        g = np.maximum(a, 0) if act == oracle.RELU else 1 / (1 + np.exp(-a))
        M2 = (np.arange(1, n + 1)[:, None] > m[None, :])
        bound = (np.abs(W2) * M2) @ np.abs(g) * 2.0 ** -8
        assert np.all(np.abs(Zq[b] - Z[b]) <= bound + 1e-15)
    assert np.any(Zq != Z)


def test_independent_spins_closed_forms():
    """W2 = 0 makes the spins independent with pi_i(+1) = sigma(c_i):
    log pi(s) = sum log sigma(s_i c_i), = -n ln 2 at c = 0, and
    <E> = sum_{i<j} J_ij mu_i mu_j + sum h_i mu_i with mu = tanh(c/2)."""
    n, h = 10, 15
    W1, b1, W2, b2 = _params(n, h, 7)
    W2 = np.zeros_like(W2)
    S = inputs.spins(50, n, 8)
    lp = oracle.logprob((W1, b1, W2, b2), S)
    ref = np.array([sum(math.log(1 / (1 + math.exp(-s[i] * b2[i]))) for i in range(n)) for s in S])
    assert np.allclose(lp, ref, rtol=0, atol=1e-12)
    lp0 = oracle.logprob((W1, b1, W2, np.zeros(n)), S)
    assert np.allclose(lp0, -n * math.log(2.0), rtol=0, atol=1e-12)

    e = inputs.erdos_renyi(n, 0.6, 9)
    w = inputs.int_weights(len(e), -4, 4, 10)
    field = inputs.int_weights(n, -2, 2, 11)
    inst = inputs.to_csr(n, e, w, field=field)
    mu = np.tanh(b2 / 2)
    J = inputs.dense_from_sparse(inst)
    L_ref = 0.5 * mu @ J @ mu + field @ mu
    out, g = oracle.enumerate_exact((W1, b1, W2, b2), inst, grad=True)
    assert abs(out[1] - L_ref) < 1e-11
    # d<E>/dc_k = 1/2 (1 - mu_k^2) (sum_j J_kj mu_j + h_k)
    dc_ref = 0.5 * (1 - mu ** 2) * (J @ mu + field)
    assert np.allclose(g[3], dc_ref, rtol=0, atol=1e-11)
    # no dependence on W1, b1 when W2 = 0
    assert np.all(g[0] == 0) and np.all(g[1] == 0)


@pytest.mark.parametrize("act", [oracle.SIGMOID, oracle.RELU])
def test_exact_gradient_two_routes(act):
    """The enumerated score-function gradient sum_s p (E - L) grad log p equals
    central differences of the enumerated L(theta) (Sec. 2.1)."""
    n, h = 8, 11
    P = _params(n, h, 12)
    inst = _small_instance(n, 13)
    _, g = oracle.enumerate_exact(P, inst, act, grad=True)
    theta = oracle.made_to_theta(*P)
    gflat = oracle.made_to_theta(*g)
    m = oracle.degrees(n, h)
    rng = np.random.default_rng(14)
    # masked W1/W2 entries have zero gradient
    W1mask = np.array([[m[k] >= j for j in range(1, n + 1)] for k in range(h)])
    W2mask = np.array([[i > m[k] for k in range(h)] for i in range(1, n + 1)])
    assert np.all(g[0][~W1mask] == 0) and np.all(g[2][~W2mask] == 0)
    idx = list(rng.choice(theta.size, 40, replace=False)) + list(range(2 * n * h, 2 * n * h + h + n, 3))
    eps = 1e-5
    for q in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[q] += eps
        tm[q] -= eps
        Lp = oracle.enumerate_exact(oracle.theta_to_made(tp, n, h), inst, act)[1]
        Lm = oracle.enumerate_exact(oracle.theta_to_made(tm, n, h), inst, act)[1]
        fd = (Lp - Lm) / (2 * eps)
        # theta index q maps to flat position; made_to_theta(g) uses the same layout
        assert abs(fd - gflat[q]) <= 1e-7 + 1e-6 * abs(fd), (q, fd, gflat[q])


def test_batch_gradient_finite_differences():
    """sum_b c_b grad log pi(s_b) against central differences (eps = 1e-3,
    FP64) of sum_b c_b log pi(s_b) at the random 3-regular workload's model
    size (n = h = 1000, the sizes of the C2 configuration), on 32 random
    parameters inside the MADE masks (8 from each of W1, b1, W2, b2) and 16
    configurations.  A parameter whose +-eps move flips the sign of a hidden
    pre-activation (a ReLU kink) is excluded; entries outside the masks get
    exactly zero."""
    cfg = inputs.config("maxcut_3reg1000")
    n, h, B = cfg["n"], cfg["h"], 16
    P = _params(n, h, 15)
    S = inputs.spins(B, n, 16)
    coef = np.random.default_rng(17).standard_normal(B) / B
    g = oracle.made_to_theta(*oracle.logprob_grad(P, S, coef))
    theta = oracle.made_to_theta(*P)
    m = oracle.degrees(n, h)
    rng = np.random.default_rng(18)
    nh = n * h
    # parameters inside the masks: W1^T entry [j][k] (input j+1 feeds unit k iff m(k) >= j+1), b1[k],
    # W2 entry [i][k] (unit k feeds output i+1 iff i+1 > m(k)), b2[i]
    jj, kk = np.nonzero(np.arange(1, n + 1)[:, None] <= m[None, :])
    w1 = rng.choice(jj.size, 8, replace=False)
    ii, k2 = np.nonzero(np.arange(1, n + 1)[:, None] > m[None, :])
    w2 = rng.choice(ii.size, 8, replace=False)
    idx = np.concatenate([jj[w1] * h + kk[w1], nh + rng.choice(h, 8, replace=False),
                          nh + h + ii[w2] * h + k2[w2], 2 * nh + h + rng.choice(n, 8, replace=False)])
    # hidden pre-activations of the B configurations (to detect ReLU kinks)
    W1, b1 = P[0], P[1]
    mask1 = (np.arange(1, n + 1)[None, :] <= m[:, None])
    A = S.astype(np.float64) @ (W1 * mask1).T + b1
    eps = 1e-3
    checked = 0
    for q in idx:
        if q < nh:
            j, k = divmod(int(q), h)
            if np.any(np.sign(A[:, k] + eps * S[:, j]) != np.sign(A[:, k] - eps * S[:, j])):
                continue
        elif q < nh + h:
            k = int(q) - nh
            if np.any(np.sign(A[:, k] + eps) != np.sign(A[:, k] - eps)):
                continue
        tp, tm = theta.copy(), theta.copy()
        tp[q] += eps
        tm[q] -= eps
        fp = coef @ oracle.logprob(oracle.theta_to_made(tp, n, h), S)
        fm = coef @ oracle.logprob(oracle.theta_to_made(tm, n, h), S)
        fd = (fp - fm) / (2 * eps)
        assert abs(fd - g[q]) <= 1e-8 + 1e-5 * abs(g[q]), (q, fd, g[q])
        checked += 1
    assert checked >= 24
    # entries outside the masks get exactly zero
    W1g = g[: nh].reshape(n, h)  # W1^T layout: [j][k]
    assert np.all(W1g[~(np.arange(1, n + 1)[:, None] <= m[None, :])] == 0)
    W2g = g[nh + h: 2 * nh + h].reshape(n, h)
    assert np.all(W2g[~(np.arange(1, n + 1)[:, None] > m[None, :])] == 0)


# --------------------------------------------------------------- sampling

@pytest.mark.parametrize("n,h,act", [(40, 60, oracle.RELU), (40, 17, oracle.SIGMOID), (25, 25, oracle.RELU),
                                     (40, 60, BF16_RELU), (40, 17, BF16_SIGMOID)])
def test_literal_and_incremental_samplers_agree(n, h, act):
    """Algorithm 1 taken literally and its incremental form give the same
    samples on shared uniforms (barring near-ties) and the same log pi."""
    P = _params(n, h, 19)
    U = inputs.uniforms(48, n, 20)
    S1, lp1 = oracle.sample(P, U, act, literal=True)
    S2, lp2 = oracle.sample(P, U, act, literal=False)
    Z = oracle.logits(P, S1, act)
    near = np.abs(U.astype(np.float64) - 1 / (1 + np.exp(-Z))) < 1e-12
    rows = ~near.any(axis=1)
    assert rows.sum() >= 40
    assert np.array_equal(S1[rows], S2[rows])
    assert np.allclose(lp1, oracle.logprob(P, S1, act), rtol=0, atol=1e-10)
    assert np.allclose(lp2, oracle.logprob(P, S2, act), rtol=0, atol=1e-10)


def test_sampler_teacher_forced_rule():
    """Each drawn spin is +1 exactly when u < pi_i(+1 | s_<i) on its own prefix."""
    n, h = 50, 70
    P = _params(n, h, 21)
    U = inputs.uniforms(32, n, 22)
    S, _ = oracle.sample(P, U)
    p = 1 / (1 + np.exp(-oracle.logits(P, S)))
    assert np.array_equal(S == 1, U.astype(np.float64) < p)


def test_sampler_is_exact_chi_square():
    """Empirical frequencies of 2^n states match pi(s) (exact sampling claim
    of Sec. 2.3 / Sec. 4), chi-square at n = 5."""
    n, h = 5, 9
    P = _params(n, h, 23, scale=2.0)
    N = 60000
    U = inputs.uniforms(N, n, 24)
    S, _ = oracle.sample(P, U)
    idx = ((S == -1).astype(np.int64) << np.arange(n)).sum(axis=1)
    counts = np.bincount(idx, minlength=1 << n)
    states = np.array([[1 - 2 * ((x >> i) & 1) for i in range(n)] for x in range(1 << n)], dtype=np.int8)
    p = np.exp(oracle.logprob(P, states))
    assert abs(p.sum() - 1) < 1e-12
    exp_c = N * p
    chi2 = ((counts - exp_c) ** 2 / exp_c).sum()
    from scipy.stats import chi2 as chi2d
    assert chi2d.sf(chi2, (1 << n) - 1) > 1e-3, chi2
