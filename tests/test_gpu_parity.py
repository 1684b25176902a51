"""GPU parity: every step of the hot path through the C ABI against the FP64
oracle, element by element, on seeded inputs.

Tolerances:
  * uniforms, samples on shared uniforms, integer energies: bit-exact.
    Samples are checked teacher-forced: every draw with |u - p_i| >= 1e-6
    must equal [u < p_i] of the oracle's conditional on the sample's own
    prefix.  For the BF16 model a draw is also exempt when a hidden unit that
    feeds its logit has an FP32 pre-activation within FP32 rounding of a
    bfloat16 rounding boundary (the kernel's g1_k may then be one bfloat16
    step from the oracle's) and that step, times |W2_ik|, can carry z_i
    across logit(u) (gpu_helpers.bf16_logit_shift).  Exempt draws are counted
    and reported, with the draws in 1e-6 <= |u - p_i| < 1e-4 and the rows that
    differ from the free-running oracle;
  * the sampler's log pi: relative 1e-5 with FP32 weights; BF16: within the
    sum over draws of that logit shift plus 1e-5 relative;
  * log pi: relative error <= 1e-5 with FP32 weights and <= 2e-2 with BF16
    weights (the oracle then runs the BF16 model: the same BF16-rounded
    weights and bfloat16-rounded hidden activations);
  * gradients: ||g - g_ref|| / ||g_ref|| <= 1e-4 (FP32), <= 3e-2 (BF16: the
    GEMM operands H, delta and the hidden adjoint are BF16, 2^-9 relative
    each, through three GEMMs), each parameter block within 3x that;
  * FP64 statistics given identical energies: relative 1e-12.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2106_13308_gb300 import inputs

from conftest import report
from gpu_helpers import (ACT_ORACLE, act_code, bf16_sample_check, build_lib, grad_blocks, logp_rel, make_model, masked,
                         oracle_params, rel_err, rows_without_near_ties, teacher_forced, er_instance)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build_lib()
    assert torch.cuda.is_available()


CASES = [
    # n, h, B, act, precision, graph p
    (20, 40, 1024, "sigmoid", "fp32", 0.5),
    (20, 40, 1024, "sigmoid", "bf16", 0.5),
    (300, 200, 300, "relu", "fp32", 0.02),
    (257, 130, 77, "relu", "bf16", 0.03),
    (129, 500, 33, "relu", "fp32", 0.05),
    (1000, 1000, 64, "relu", "bf16", 0.003),
    # more than 2048 hidden units: the CUDA-core sampler's four-warp groups, 4 samples per CTA (ragged)
    (2600, 2600, 13, "relu", "bf16", 0.002),
    (2200, 2500, 9, "relu", "fp32", 0.002),
]


# ---------------------------------------------------------------- uniforms

def test_uniforms_match_oracle_philox():
    n, h, B = 37, 16, 50
    m = make_model(n, h, B, er_instance(n, 0.2, 1), seed=0xDEADBEEF12345)
    for it in (0, 1, 2**33 + 5):
        u = m.uniforms(B, it).cpu().numpy()
        assert np.array_equal(u, oracle.uniforms(B, n, 0xDEADBEEF12345, it))


# ----------------------------------------------------------------- sampler

@pytest.mark.parametrize("n,h,B,act,prec,p", CASES)
def test_sampler_matches_oracle(n, h, B, act, prec, p):
    inst = er_instance(n, p, 2)
    theta = inputs.lively_params(n, h, 3)
    m = make_model(n, h, B, inst, act=act, precision=prec, theta=theta)
    P = oracle_params(theta, n, h, prec)
    U = inputs.uniforms(B, n, 4)
    S, lp = m.sample(B, torch.from_numpy(U).cuda())
    S, lp = S.cpu().numpy(), lp.cpu().numpy()
    assert set(np.unique(S)) <= {-1, 1}
    # teacher-forced: each spin decided by the oracle's conditional on its own prefix
    _check_samples(P, S, lp, U, act_code(act, prec), prec, f"n={n} h={h} B={B} {act}")


def _check_samples(P, S, lp, U, code, prec, label=""):
    if prec == "fp32":
        mism, ties = teacher_forced(P, S, U, code, 1e-6)
        assert mism == 0, (mism, ties)
        # free-running oracle on the same uniforms: identical rows (barring near-ties)
        So, lpo = oracle.sample(P, U, code)
        rows = rows_without_near_ties(P, So, U, code, 1e-6)
        B = S.shape[0]
        assert rows.sum() >= B - 2, (rows.sum(), B)
        assert np.array_equal(S[rows], So[rows])
        assert logp_rel(lp[rows], lpo[rows]) <= 1e-5
        report(f"samples fp32 {label}", draws=int(S.size), near_ties_1e6=ties, rows=int(B),
               rows_equal_free_running=int((S == So).all(axis=1).sum()))
        return
    c = bf16_sample_check(P, S, U, code, lp=lp)
    report(f"samples bf16 {label}", **c)
    assert c["unflagged_mismatches"] == 0, c
    assert c["clean_rows_equal"], c
    assert c["logp_within_bound"], c

# Models where the tensor-core sampler applies (at most 32 hidden units
# completing within a block of 128, or of 64, steps): ragged n and B.
TC_CASES = [
    # n, h, B, act, graph p
    (1500, 300, 48, "relu", 0.01),      # blocks of 128, ~26 recent units
    (700, 160, 37, "sigmoid", 0.02),    # blocks of 128
    (513, 200, 20, "relu", 0.03),       # blocks of 64
    (130, 33, 16, "relu", 0.05),        # n close to one block, h below one unit tile
]


@pytest.mark.parametrize("n,h,B,act,p", TC_CASES)
def test_tensor_core_sampler_matches_oracle(n, h, B, act, p):
    inst = er_instance(n, p, 12)
    theta = inputs.lively_params(n, h, 13)
    m = make_model(n, h, B, inst, act=act, precision="bf16", theta=theta, sampler="tensor_core")
    P = oracle_params(theta, n, h, "bf16")
    U = inputs.uniforms(B, n, 14)
    S, lp = m.sample(B, torch.from_numpy(U).cuda())
    S, lp = S.cpu().numpy(), lp.cpu().numpy()
    assert set(np.unique(S)) <= {-1, 1}
    _check_samples(P, S, lp, U, act_code(act, "bf16"), "bf16", f"tensor-core n={n} h={h} B={B} {act}")
    assert m.check() == 0
    # the CUDA-core sampler runs the same model: the same check, and the rows
    # of the two samplers compared
    c = make_model(n, h, B, inst, act=act, precision="bf16", theta=theta, sampler="cuda_core")
    S2, lp2 = c.sample(B, torch.from_numpy(U).cuda())
    S2, lp2 = S2.cpu().numpy(), lp2.cpu().numpy()
    _check_samples(P, S2, lp2, U, act_code(act, "bf16"), "bf16", f"cuda-core n={n} h={h} B={B} {act}")
    report(f"tensor-core vs cuda-core rows n={n} h={h} B={B}", rows=int(B),
           rows_equal=int((S2 == S).all(axis=1).sum()))


def test_tensor_core_sampler_internal_philox_and_steps():
    """Internal Philox uniforms through the tensor-core sampler, and
    vqmc_step on it: samples equal the oracle's on the same uniforms."""
    n, h, B, seed = 900, 150, 64, 99
    inst = er_instance(n, 0.01, 15)
    theta = inputs.lively_params(n, h, 16)
    m = make_model(n, h, B, inst, precision="bf16", theta=theta, seed=seed, sampler="tensor_core")
    P = oracle_params(theta, n, h, "bf16")
    code = act_code("relu", "bf16")
    for it in (0, 3):
        S, lp = m.sample(B, None, iteration=it)
        U = oracle.uniforms(B, n, seed, it)
        _check_samples(P, S.cpu().numpy(), lp.cpu().numpy(), U, code, "bf16", f"tensor-core Philox it={it}")
    assert m.check() == 0


def test_tensor_core_sampler_rejected_where_it_does_not_apply():
    from paper_2106_13308_gb300.vqmc import VQMCError
    inst = er_instance(200, 0.05, 17)
    with pytest.raises(VQMCError):  # FP32 model
        make_model(200, 64, 8, inst, precision="fp32", sampler="tensor_core")
    with pytest.raises(VQMCError):  # h > n/2: more than 32 units complete within 64 steps
        make_model(200, 150, 8, inst, precision="bf16", sampler="tensor_core")


def test_sampler_internal_philox_matches_oracle():
    n, h, B, seed = 150, 90, 200, 777
    inst = er_instance(n, 0.05, 5)
    theta = inputs.lively_params(n, h, 6)
    m = make_model(n, h, B, inst, theta=theta, seed=seed)
    P = oracle_params(theta, n, h, "fp32")
    for it in (0, 9):
        S, lp = m.sample(B, None, iteration=it)
        S = S.cpu().numpy()
        U = oracle.uniforms(B, n, seed, it)
        So, lpo = oracle.sample(P, U)
        rows = rows_without_near_ties(P, So, U, "relu")
        assert rows.sum() >= B - 2
        assert np.array_equal(S[rows], So[rows])


def test_sampler_edge_sizes():
    # B = 1, B = 0 (no-op), n = 1 (a single conditional sigma(c_1)), h = 1
    for n, h, B in [(1, 1, 5), (2, 1, 17), (5, 64, 1), (64, 3, 40)]:
        inst = er_instance(n, 0.5, 7) if n > 1 else inputs.to_csr(1, np.zeros((0, 2), np.int64), np.zeros(0, np.int32))
        theta = inputs.lively_params(n, h, 8)
        m = make_model(n, h, B, inst, theta=theta)
        P = oracle_params(theta, n, h, "fp32")
        U = inputs.uniforms(B, n, 9)
        S, lp = m.sample(B, torch.from_numpy(U).cuda())
        So, lpo = oracle.sample(P, U)
        rows = rows_without_near_ties(P, So, U, "relu")
        assert np.array_equal(S.cpu().numpy()[rows], So[rows])
        assert logp_rel(lp.cpu().numpy()[rows], lpo[rows]) <= 1e-5
        s0 = torch.empty((0, n), dtype=torch.int8, device="cuda")
        from paper_2106_13308_gb300 import vqmc
        vqmc.vqmc_sample(m.ctx, 0, None, 0, s0)


# ----------------------------------------------------------- local energy

def test_sparse_energy_bit_exact():
    for n, p, B, seed in [(300, 0.02, 300, 11), (10000, 8 / 9999, 97, 12), (64, 0.9, 1000, 13)]:
        inst = er_instance(n, p, seed)
        m = make_model(n, 8, B, inst)
        S = inputs.spins(B, n, seed + 100)
        E = m.local_energy(torch.from_numpy(S).cuda()).cpu().numpy()
        Eo = oracle.energy(inst, S)
        assert E.dtype == np.int32 and np.array_equal(E.astype(np.float64), Eo)
        # Max-Cut mapping: cut = (W_tot - E)/2
        assert np.array_equal((inst["w"].sum() - E) // 2, oracle.cut(inst, S).astype(np.int64))


@pytest.mark.parametrize("lo,hi", [(-1, 1), (0, 0), (-15, 15), (1, 10), (-255, 255), (-256, 256), (-70000, 70000)])
def test_sparse_energy_weight_widths(lo, hi):
    """Integer weights of every width the energy kernels distinguish (|J| < 2,
    16, 256: bit-sliced counters of 6, 9 or 13 planes; wider: one sample per
    lane), on rows long enough that each thread adds many runs of 15 edges
    (n = 2000, p = 0.1: about 2e5 edges, 10 row slices for B = 1024) and a
    ragged last word of samples: bit-exact against the oracle."""
    n, B = 2000, 1000
    e = inputs.erdos_renyi(n, 0.1, 41)
    inst = inputs.to_csr(n, e, inputs.int_weights(len(e), lo, hi, 42))
    m = make_model(n, 8, 1024, inst)
    S = inputs.spins(B, n, 43)
    E = m.local_energy(torch.from_numpy(S).cuda()).cpu().numpy()
    assert E.dtype == np.int32 and np.array_equal(E.astype(np.float64), oracle.energy(inst, S))
    m.close()


def test_sparse_energy_with_field_and_pm1_weights():
    n, B = 1000, 130
    e = inputs.random_regular(n, 3, 21)
    inst = inputs.to_csr(n, e, inputs.pm1_weights(len(e), 22), field=inputs.int_weights(n, -3, 3, 23))
    m = make_model(n, 16, B, inst)
    S = inputs.spins(B, n, 24)
    E = m.local_energy(torch.from_numpy(S).cuda()).cpu().numpy()
    assert np.array_equal(E.astype(np.float64), oracle.energy(inst, S))


def test_sparse_float_energy():
    n, B = 500, 64
    e = inputs.erdos_renyi(n, 0.01, 31)
    w = np.random.default_rng(32).standard_normal(len(e)).astype(np.float32)
    inst = inputs.to_csr(n, e, w)
    m = make_model(n, 16, B, inst)
    S = inputs.spins(B, n, 33)
    E = m.local_energy(torch.from_numpy(S).cuda()).cpu().numpy()
    Eo = oracle.energy(inst, S)
    # FP32 accumulation of m terms of size O(1): |err| <= m * 2^-24 * max|partial|
    assert np.max(np.abs(E - Eo)) <= len(e) * 2.0 ** -23 * (np.abs(w).sum())


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_dense_energy(prec):
    n, B = 300, 200
    inst = inputs.sk(n, 41)
    m = make_model(n, 16, B, inst, precision=prec)
    S = inputs.spins(B, n, 42)
    E = m.local_energy(torch.from_numpy(S).cuda()).cpu().numpy()
    Eo = oracle.energy(inst, S)
    scale = np.sqrt(np.sum(inst["J"].astype(np.float64) ** 2))  # ~ ||J||_F
    err = np.max(np.abs(E - Eo))
    # FP32 products are exact for s = +-1; BF16 hi/lo keeps 16 mantissa bits of J
    bound = (n * n * 2.0 ** -23 if prec == "fp32" else n * n * 2.0 ** -16) * np.abs(inst["J"]).max()
    assert err <= bound, (err, bound, scale)


# ------------------------------------------------------------- statistics

def test_energy_stats_fp64():
    n, B = 100, 777
    inst = er_instance(n, 0.1, 51)
    m = make_model(n, 8, B, inst)
    S = inputs.spins(B, n, 52)
    E = m.local_energy(torch.from_numpy(S).cuda())
    st, coef = m.energy_stats(E)
    sto, coefo = oracle.stats(oracle.energy(inst, S))
    assert np.allclose(st.cpu().numpy(), sto, rtol=1e-12, atol=0)
    assert np.allclose(coef.cpu().numpy(), coefo, rtol=1e-6, atol=1e-12)


# ---------------------------------------------------------------- log prob

@pytest.mark.parametrize("n,h,B,act,prec,p", CASES)
def test_logprob_gemm_matches_oracle(n, h, B, act, prec, p):
    inst = er_instance(n, p, 61)
    theta = inputs.lively_params(n, h, 62)
    m = make_model(n, h, B, inst, act=act, precision=prec, theta=theta)
    P = oracle_params(theta, n, h, prec)
    S = inputs.spins(B, n, 63)
    lp = m.logprob(torch.from_numpy(S).cuda()).cpu().numpy()
    lpo = oracle.logprob(P, S, act_code(act, prec))
    tol = 1e-5 if prec == "fp32" else 2e-2
    assert logp_rel(lp, lpo) <= tol


# ---------------------------------------------------------------- gradient

@pytest.mark.parametrize("n,h,B,act,prec,p", CASES)
def test_gradient_matches_oracle(n, h, B, act, prec, p):
    inst = er_instance(n, p, 71)
    theta = inputs.lively_params(n, h, 72)
    m = make_model(n, h, B, inst, act=act, precision=prec, theta=theta)
    P = oracle_params(theta, n, h, prec)
    S = inputs.spins(B, n, 73)
    St = torch.from_numpy(S).cuda()
    E = m.local_energy(St)
    g, st = m.grad(St, E)
    (dW1, db1, dW2, db2), sto, Eo = oracle.vqmc_grad(P, inst, S, act_code(act, prec))
    go = oracle.made_to_theta(dW1, db1, dW2, db2)
    g = g.cpu().numpy()
    tol = 1e-4 if prec == "fp32" else 3e-2
    assert rel_err(g, go) <= tol
    for k, blk in grad_blocks(g, n, h).items():
        ref = grad_blocks(go, n, h)[k]
        if np.linalg.norm(ref) > 1e-8 * np.linalg.norm(go):
            assert rel_err(blk, ref) <= 3 * tol, k
    # outside the masks the gradient is exactly zero
    mask_zero = masked(np.ones_like(theta), n, h) == 0
    assert np.all(g[mask_zero] == 0)
    assert np.allclose(st.cpu().numpy(), sto, rtol=1e-12)


def test_logprob_backward_arbitrary_weights_and_autograd():
    from paper_2106_13308_gb300.vqmc import LogProb
    n, h, B = 90, 70, 45
    inst = er_instance(n, 0.05, 81)
    theta = inputs.lively_params(n, h, 82)
    m = make_model(n, h, B, inst, theta=theta)
    P = oracle_params(theta, n, h, "fp32")
    S = inputs.spins(B, n, 83)
    gout = np.random.default_rng(84).standard_normal(B).astype(np.float32)
    go = oracle.made_to_theta(*oracle.logprob_grad(P, S, gout.astype(np.float64)))
    St = torch.from_numpy(S).cuda()
    g = m.logprob_backward(St, torch.from_numpy(gout).cuda()).cpu().numpy()
    assert rel_err(g, go) <= 1e-4
    th = m.params_view().requires_grad_(True)
    lp = LogProb.apply(th, St, m)
    assert logp_rel(lp.detach().cpu().numpy(), oracle.logprob(P, S)) <= 1e-5
    lp.backward(torch.from_numpy(gout).cuda())
    assert rel_err(th.grad.cpu().numpy(), go) <= 1e-4


# -------------------------------------------------------------------- adam

@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("h", [30, 32])  # scalar path, and the 16-byte path (h % 4 == 0)
def test_adam_matches_oracle(h, prec):
    """Three Adam steps (Sec. 5.1) equal the oracle's.  The device gets a
    gradient that is non-zero outside the MADE masks too: only entries inside
    the masks are updated (the oracle gets the masked gradient), so the
    masked weights stay exactly zero."""
    n = 40
    inst = er_instance(n, 0.2, 91)
    theta = inputs.lively_params(n, h, 92)
    m = make_model(n, h, 4, inst, precision=prec, theta=theta)
    t0 = masked(theta, n, h).astype(np.float64)
    mo, vo = np.zeros_like(t0), np.zeros_like(t0)
    rng = np.random.default_rng(93)
    keep = masked(np.ones_like(theta), n, h)
    for t in range(1, 4):
        g = rng.standard_normal(t0.size).astype(np.float32)
        m.adam(torch.from_numpy(g).cuda())
        oracle.adam(t0, mo, vo, (g * keep).astype(np.float64), t)
    got = m.get_params().numpy()
    assert np.allclose(got, t0, rtol=0, atol=2e-6)
    assert np.all(got[keep == 0] == 0)


@pytest.mark.parametrize("n,h,B,act,prec", [(257, 130, 77, "relu", "bf16"), (300, 200, 30, "relu", "fp32"),
                                           (20, 40, 64, "sigmoid", "bf16"), (1000, 1000, 9, "relu", "bf16")])
def test_wide_cuda_core_layout_matches_oracle(n, h, B, act, prec):
    """The CUDA-core sampler's wide layout (groups of four warps splitting the
    hidden units, 4 samples per CTA), which the batch autotuner may choose
    for any member, draws the model's exact samples as the default layout."""
    inst = er_instance(n, 0.05, 22)
    theta = inputs.lively_params(n, h, 23)
    m = make_model(n, h, B, inst, act=act, precision=prec, theta=theta, sampler="cuda_core_wide")
    P = oracle_params(theta, n, h, prec)
    U = inputs.uniforms(B, n, 24)
    S, lp = m.sample(B, torch.from_numpy(U).cuda())
    S, lp = S.cpu().numpy(), lp.cpu().numpy()
    _check_samples(P, S, lp, U, act_code(act, prec), prec, f"wide layout n={n} h={h} B={B} {act}")
    assert m.check() == 0
