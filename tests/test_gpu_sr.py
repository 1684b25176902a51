"""GPU parity of stochastic reconfiguration (Sec. 2.1; SGD+SR of Sec. 5.1)
against the FP64 oracle, which forms the per-sample score vectors explicitly
and solves the d x d system: the Gram matrix of the score vectors, the SR
direction, and one SGD+SR iteration; plus a training run on the C1-sized
Max-Cut instance that must approach the brute-force optimum.

Tolerances follow the FP32 arithmetic of the CUDA path.  A Gram entry sums
about n + h outer-product events in FP32, each with its own rounding, so
|G - G_ref| <= 4 (n + h + 2) 2^-24 sqrt(G_bb G_cc) (the Cauchy-Schwarz scale
of the entry).  The direction solves (G/B + lambda) x = c in FP32 with a
backward error of a few units of 2^-24 relative to the matrix, so its
relative error is bounded by kappa times that: 1e-5 + 64 kappa 2^-24, with
kappa the condition number of G/B + lambda computed by the oracle."""
import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import act_code, build_lib, er_instance, make_model, oracle_params, rel_err, \
    rows_without_near_ties
from paper_2106_13308_gb300 import inputs

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build_lib()


def _gram_tol(n, h, Gr):
    d = np.sqrt(np.maximum(np.diag(Gr), 0.0))
    return 4 * (n + h + 2) * U32 * np.outer(d, d) + 1e-30


# (n, h, B, act): several 64 x 64 tiles with ragged tails, one tile, one
# sample, a single spin, h > n and h < n
GRAM_CASES = [(37, 50, 150, "relu"), (64, 48, 96, "sigmoid"), (20, 45, 200, "relu"), (130, 70, 65, "sigmoid"),
              (5, 3, 1, "relu"), (1, 4, 7, "sigmoid")]


@pytest.mark.parametrize("n,h,B,act", GRAM_CASES)
def test_sr_gram_matches_oracle(n, h, B, act):
    inst = er_instance(n, 0.3, 7)
    theta = inputs.lively_params(n, h, 11)
    m = make_model(n, h, B, inst, act=act, precision="fp32", theta=theta)
    S = inputs.spins(B, n, 13)
    G = m.sr_gram(torch.from_numpy(S).cuda()).cpu().numpy().astype(np.float64)
    Gr = oracle.sr_gram(oracle_params(theta, n, h, "fp32"), S, act_code(act))
    assert G.shape == (B, B)
    assert np.array_equal(G, G.T)
    err = np.abs(G - Gr)
    tol = _gram_tol(n, h, Gr)
    assert np.all(err <= tol), f"max err/tol {np.max(err / tol):.3g}"


def _kappa(P, S, lam, code):
    O = oracle.per_sample_grads(P, S, code)
    B = S.shape[0]
    ev = np.linalg.eigvalsh(O @ O.T / B + lam * np.eye(B))
    return ev[-1] / ev[0]


def _zero_outside_masks(g, n, h):
    deg = oracle.degrees(n, h)
    W1t = np.asarray(g[: n * h]).reshape(n, h)
    W2 = np.asarray(g[n * h + h: 2 * n * h + h]).reshape(n, h)
    j = np.arange(1, n + 1)[:, None]
    return np.all(W1t[~(deg[None, :] >= j)] == 0) and np.all(W2[~(j > deg[None, :])] == 0)


# (n, h, B, act, lambda, instance): the paper's lambda = 1e-3 and a larger
# one; the transverse-field model (float energies with the off-diagonal part)
# and integer Max-Cut
DIR_CASES = [(37, 50, 150, "relu", 1e-3, "tim"), (20, 45, 200, "sigmoid", 1e-3, "tim"),
             (30, 40, 130, "relu", 0.1, "maxcut"), (64, 33, 64, "sigmoid", 1e-3, "maxcut"),
             (12, 10, 1, "relu", 1e-3, "tim")]


@pytest.mark.parametrize("n,h,B,act,lam,kind", DIR_CASES)
def test_sr_direction_matches_oracle(n, h, B, act, lam, kind):
    inst = inputs.tim(n, 3) if kind == "tim" else er_instance(n, 0.25, 5)
    theta = inputs.lively_params(n, h, 4)
    m = make_model(n, h, B, inst, act=act, precision="fp32", theta=theta)
    S = inputs.spins(B, n, 6)
    Sd = torch.from_numpy(S).cuda()
    E = m.local_energy(Sd)
    delta, st = m.sr_direction(Sd, E, lam)
    delta = delta.cpu().numpy()
    P = oracle_params(theta, n, h, "fp32")
    code = act_code(act)
    dref, stref = oracle.sr_direction(P, inst, S, lam, code)
    kappa = _kappa(P, S, lam, code)
    tol = 1e-5 + 64 * kappa * U32
    err = rel_err(delta, dref)
    assert err <= tol, f"rel err {err:.3g} > {tol:.3g} (kappa {kappa:.3g})"
    assert _zero_outside_masks(delta, n, h)
    # FP64 statistics: identical for integer energies; for the float energies
    # of the transverse field within what the energies' own difference dE
    # moves them (mean, min, max by dE, the variance by 4 dE sd + 4 dE^2)
    st = st.cpu().numpy()
    dE = float(np.max(np.abs(E.cpu().numpy().astype(np.float64) - oracle.local_energy(P, inst, S, code))))
    if kind == "maxcut":
        assert dE == 0 and np.allclose(st, stref, rtol=1e-12)
    else:
        slack = 1e-12 * np.abs(stref)
        assert np.all(np.abs(st[[0, 2, 3]] - stref[[0, 2, 3]]) <= dE + slack[[0, 2, 3]])
        assert abs(st[1] - stref[1]) <= 4 * dE * np.sqrt(stref[1]) + 4 * dE ** 2 + slack[1]
    assert m.check() == 0


def test_sr_direction_at_the_maximum_batch():
    """B = 16384, the largest SR batch: a 256 x 256-block Cholesky (more
    panel blocks than SMs) and a 256-block solve.  A small model keeps the
    oracle's d x d solve cheap; with B > d the smallest eigenvalue of
    O O^T / B + lambda is lambda, so kappa = (largest eigenvalue of
    O^T O / B + lambda) / lambda.  One sample more is rejected."""
    from paper_2106_13308_gb300.vqmc import VQMCError, VQMC_ERR_UNSUPPORTED
    n, h, B, lam = 12, 6, 16384, 1e-2
    inst = er_instance(n, 0.4, 31)
    theta = inputs.lively_params(n, h, 32)
    m = make_model(n, h, B, inst, act="relu", precision="fp32", theta=theta)
    S = inputs.spins(B, n, 33)
    Sd = torch.from_numpy(S).cuda()
    delta, _ = m.sr_direction(Sd, m.local_energy(Sd), lam)
    P = oracle_params(theta, n, h, "fp32")
    code = act_code("relu")
    dref, _ = oracle.sr_direction(P, inst, S, lam, code)
    O = oracle.per_sample_grads(P, S, code)
    kappa = np.linalg.eigvalsh(O.T @ O / B + lam * np.eye(O.shape[1]))[-1] / lam
    tol = 1e-5 + 64 * kappa * U32
    err = rel_err(delta.cpu().numpy(), dref)
    assert err <= tol, f"rel err {err:.3g} > {tol:.3g} (kappa {kappa:.3g})"
    assert m.check() == 0
    del m
    big = make_model(n, h, B + 1, inst, act="relu", precision="fp32", theta=theta)
    with pytest.raises(VQMCError) as ei:
        big.sr_gram(torch.from_numpy(inputs.spins(B + 1, n, 34)).cuda())
    assert ei.value.status == VQMC_ERR_UNSUPPORTED


def test_sr_direction_tends_to_the_gradient_for_large_lambda():
    """(I + lambda) delta = g: lambda delta -> g, the vqmc_grad result."""
    n, h, B = 40, 30, 256
    inst = er_instance(n, 0.2, 8)
    m = make_model(n, h, B, inst, act="relu", precision="fp32", theta=inputs.lively_params(n, h, 9))
    Sd = torch.from_numpy(inputs.spins(B, n, 10)).cuda()
    E = m.local_energy(Sd)
    lam = 1e5
    delta, _ = m.sr_direction(Sd, E, lam)
    g, _ = m.grad(Sd, E)
    assert rel_err(lam * delta.cpu().numpy(), g.cpu().numpy()) < 1e-3


def test_sr_edge_cases_and_errors():
    from paper_2106_13308_gb300.vqmc import VQMCError, VQMC_ERR_INVALID_ARG, VQMC_ERR_UNSUPPORTED
    n, h, B = 16, 12, 32
    inst = er_instance(n, 0.3, 3)
    m = make_model(n, h, B, inst, precision="fp32", theta=inputs.lively_params(n, h, 2))
    S = torch.from_numpy(inputs.spins(B, n, 4)).cuda()
    E = m.local_energy(S)
    d0, _ = m.sr_direction(S[:0], E[:0], 1e-3)
    assert torch.count_nonzero(d0).item() == 0
    for lam in (0.0, -1.0, float("nan"), float("inf")):
        with pytest.raises(VQMCError) as ei:
            m.sr_direction(S, E, lam)
        assert ei.value.status == VQMC_ERR_INVALID_ARG
    mb = make_model(n, h, B, inst, precision="bf16", theta=inputs.lively_params(n, h, 2))
    with pytest.raises(VQMCError) as ei:
        mb.sr_gram(S)
    assert ei.value.status == VQMC_ERR_UNSUPPORTED
    with pytest.raises(VQMCError) as ei:
        mb.sr_step(B)
    assert ei.value.status == VQMC_ERR_UNSUPPORTED


def test_sr_failed_factorisation_sets_the_error_word():
    """A Cholesky pivot that is not positive is reported, not hidden: with
    B = 128 samples and d = 22 parameters the Gram matrix has rank <= 22, and
    lambda = 1e-30 leaves the remaining 106 pivots to FP32 rounding noise of
    either sign.  The call completes (no fault, no wait), the direction is
    not finite and vqmc_check reports VQMC_DEVERR_NONFINITE."""
    from paper_2106_13308_gb300.vqmc import DEVERR_NONFINITE
    n, h, B = 4, 2, 128
    inst = er_instance(n, 0.9, 3)
    m = make_model(n, h, B, inst, precision="fp32", theta=inputs.lively_params(n, h, 2))
    assert m.d == 22
    S = torch.from_numpy(inputs.spins(B, n, 5)).cuda()
    delta, _ = m.sr_direction(S, m.local_energy(S), 1e-30)
    torch.cuda.synchronize()
    assert not torch.isfinite(delta).all()
    assert m.check() & DEVERR_NONFINITE
    assert m.check() == 0  # the word was read and cleared


def test_sr_step_is_sgd_on_the_sr_direction():
    """One vqmc_sr_step: the oracle draws the same samples from its own
    Philox uniforms (no near-ties for these seeds) and its direction gives
    theta_1 = theta_0 - lr delta."""
    from paper_2106_13308_gb300.vqmc import StepStats
    n, h, B, seed, lr, lam = 24, 30, 128, 77, 0.1, 1e-3
    inst = er_instance(n, 0.3, 9)
    theta = inputs.lively_params(n, h, 12)
    m = make_model(n, h, B, inst, act="relu", precision="fp32", theta=theta, seed=seed)
    th0 = m.get_params().numpy().astype(np.float64)
    out = StepStats()
    m.sr_step(B, lr, lam, out)
    torch.cuda.synchronize()
    th1 = m.get_params().numpy().astype(np.float64)
    P = oracle_params(theta, n, h, "fp32")
    code = act_code("relu")
    U = oracle.uniforms(B, n, seed, 0)
    So, _ = oracle.sample(P, U, code)
    assert rows_without_near_ties(P, So, U, "relu").all()
    s_gpu, _ = m.last_batch(B)
    assert np.array_equal(s_gpu.cpu().numpy(), So)
    dref, st = oracle.sr_direction(P, inst, So, lam, code)
    tol = 1e-5 + 64 * _kappa(P, So, lam, code) * U32
    resid = np.linalg.norm(th1 - (th0 - lr * dref))
    assert resid <= tol * lr * np.linalg.norm(dref) + 2 * U32 * np.linalg.norm(th0)
    assert np.allclose([out.mean, out.var, out.min, out.max], st, rtol=1e-12)
    assert out.iteration == 0 and m.iteration == 1 and out.error_flags == 0


def test_sr_training_reaches_the_max_cut():
    """SGD+SR with the paper's lambda = 1e-3 and lr = 0.1 on Max-Cut of
    G(20, 0.5) (unit weights; init std 0.01): within 40 iterations the mean
    energy falls far below its start and the batch holds a cut within 1 of
    the brute-force optimum (the oracle's SR run on the same instance
    reaches the optimum in about 15 iterations)."""
    from paper_2106_13308_gb300.vqmc import StepStats
    n, h, B = 20, 40, 256
    e = inputs.erdos_renyi(n, 0.5, 1)
    inst = inputs.to_csr(n, e, np.ones(len(e), dtype=np.int32))
    opt = oracle.maxcut_bruteforce(inst)
    wtot = float(len(e))
    m = make_model(n, h, B, inst, act="relu", precision="fp32", theta=inputs.made_params(n, h, 2), seed=9)
    out = StepStats()
    means = []
    for _ in range(40):
        m.sr_step(B, 0.1, 1e-3, out)
        torch.cuda.synchronize()
        means.append(out.mean)
    assert m.check() == 0
    assert np.mean(means[-5:]) < means[0] - 20
    best_cut = (wtot - out.min) / 2
    assert best_cut >= opt - 1
