"""Shared helpers for the GPU parity tests (CUDA path vs the FP64 oracle).

Both sides receive only seeded inputs from paper_2106_13308_gb300.inputs;
BF16 comparisons round the same seeded theta to BF16 on the CPU (torch) and
give the oracle those values promoted to FP64."""
import math

import numpy as np
import torch

import oracle
from paper_2106_13308_gb300 import inputs

ACT_ORACLE = {"relu": oracle.RELU, "sigmoid": oracle.SIGMOID}


def act_code(act, precision="fp32"):
    """Oracle activation code of the model a precision runs: the BF16 model
    rounds hidden activations to bfloat16 (weights via oracle_params)."""
    code = ACT_ORACLE[act] if isinstance(act, str) else int(act)
    return code | (oracle.HIDDEN_BF16 if precision == "bf16" else 0)


def build_lib():
    from paper_2106_13308_gb300 import build
    build.build()


def bf16_round(theta: np.ndarray) -> np.ndarray:
    return torch.from_numpy(np.asarray(theta, dtype=np.float32)).to(torch.bfloat16).float().numpy()


def masked(theta: np.ndarray, n: int, h: int) -> np.ndarray:
    """theta with the entries outside the MADE masks set to zero (test-side,
    from the oracle's degrees)."""
    t = np.array(theta, dtype=np.float32, copy=True)
    m = oracle.degrees(n, h)
    W1t = t[: n * h].reshape(n, h)
    W2 = t[n * h + h: 2 * n * h + h].reshape(n, h)
    r = np.arange(n)[:, None]
    W1t[~(r < m[None, :])] = 0
    W2[~(m[None, :] <= r)] = 0
    return t


def oracle_params(theta, n, h, precision):
    t = masked(theta, n, h)
    if precision == "bf16":
        # W1, W2 are used in BF16 by the kernels; biases stay FP32
        tb = bf16_round(t)
        t = t.copy()
        t[: n * h] = tb[: n * h]
        t[n * h + h: 2 * n * h + h] = tb[n * h + h: 2 * n * h + h]
    return oracle.theta_to_made(t, n, h)


def sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def teacher_forced(P, S, U, act, tol=1e-6):
    """(mismatches, near_ties): every spin with |u - p_i| >= tol must equal
    [u < p_i] where p_i is the oracle's conditional on the sample's own prefix."""
    Z = oracle.logits(P, S, act_code(act))
    p = sigmoid(Z)
    U = np.asarray(U, dtype=np.float64)
    decided = np.abs(U - p) >= tol
    mism = decided & ((S == 1) != (U < p))
    return int(mism.sum()), int((~decided).sum())


def _act64(A, act):
    return np.maximum(A, 0.0) if (act & 1) == oracle.RELU else 1.0 / (1.0 + np.exp(-A))


def _to_bf16(x):
    """FP64 values rounded as the kernels round an FP32 activation: to FP32,
    then to the nearest bfloat16 (ties to even; torch's conversion)."""
    f = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32))
    return f.to(torch.bfloat16).to(torch.float64).numpy()


def bf16_logit_shift(P, S, code):
    """How far FP32 arithmetic may move the BF16 model's logits from the FP64
    oracle's, per draw, on the samples S (the oracle's BF16 model P: masked,
    BF16-valued weights).

    The kernels accumulate each hidden pre-activation a_k in FP32 and round
    g1_k = act(a_k) to bfloat16.  Where a_k lies within FP32 rounding of the
    point at which that rounding changes, the kernel's g1_k may be one
    bfloat16 step away from the oracle's (an "ambiguous" unit), and every
    later logit z_i moves by |W2_ik| times that step.  FP32 rounding of a_k is
    taken as 8 * 2^-24 * sqrt(m(k) + 1) * ||(b1_k, W1_k)||_2 (six standard
    deviations of the rounding noise of an (m(k) + 1)-term sum with terms of
    mixed sign, plus margin); a sigmoid evaluated in FP32 adds 2^-20 relative.
    Returns (shift (B, n), ambiguous units per sample (B,))."""
    W1, b1, W2, b2 = (np.asarray(x, np.float64) for x in P)
    h, n = W1.shape
    act = code & 1
    deg = oracle.degrees(n, h).astype(np.float64)
    A = np.asarray(S, np.float64) @ W1.T + b1
    epsA = 8.0 * 2.0 ** -24 * np.sqrt(deg + 1.0) * np.sqrt(np.sum(W1 * W1, axis=1) + b1 * b1)
    with np.errstate(over="ignore"):
        lo, hi = _act64(A - epsA, act), _act64(A + epsA, act)
    if act == oracle.SIGMOID:
        lo, hi = lo * (1.0 - 2.0 ** -20), hi * (1.0 + 2.0 ** -20)
    dG = np.abs(_to_bf16(hi) - _to_bf16(lo))
    return dG @ np.abs(W2).T, (dG > 0).sum(axis=1)


def bf16_sample_check(P, S, U, code, lp=None, tie=1e-6):
    """Teacher-forced check of BF16-model samples S (the GPU's) against the
    oracle on the same uniforms U.

    A draw is "flagged" when |u - p_i| < tie or when the logit shift of
    bf16_logit_shift can carry z_i across logit(u).  Every unflagged draw must
    equal [u < p_i] of the oracle's conditional on the sample's own prefix;
    flagged draws may go either way and are counted.  Rows in which every
    draw agrees with the oracle's conditional must equal the free-running
    oracle's rows on the same uniforms (induction over the steps).  With lp
    (the sampler's own log pi), every row must lie within sum_i shift_i +
    1e-5 |log pi| of the oracle's log pi of that row (|d log sigma(s z)/dz| <= 1,
    plus FP32 accumulation over n terms).  Returns a dict of counts."""
    S = np.asarray(S)
    Ud = np.asarray(U, np.float64)
    Z = oracle.logits(P, S, code)
    p = sigmoid(Z)
    shift, namb = bf16_logit_shift(P, S, code)
    with np.errstate(divide="ignore"):
        lg = np.log(Ud) - np.log1p(-Ud)
    near = np.abs(Ud - p) < tie
    flagged = near | (np.abs(lg - Z) <= shift)
    wrong = (S == 1) != (Ud < p)
    out = {
        "draws": int(S.size),
        "near_ties_1e-6": int(near.sum()),
        "band_1e-6_1e-4": int(((np.abs(Ud - p) >= tie) & (np.abs(Ud - p) < 1e-4)).sum()),
        "ambiguous_units_mean": float(namb.mean()) if namb.size else 0.0,
        "flagged": int(flagged.sum()),
        "flagged_other_way": int((wrong & flagged).sum()),
        "unflagged_mismatches": int((wrong & ~flagged).sum()),
    }
    clean = ~wrong.any(axis=1)
    So, _ = oracle.sample(P, Ud.astype(np.float32), code)
    out["rows"] = int(S.shape[0])
    out["rows_equal_free_running"] = int((S == So).all(axis=1).sum())
    out["rows_with_flagged_other_way"] = int((~clean).sum())
    out["clean_rows_equal"] = bool(np.array_equal(S[clean], So[clean]))
    if lp is not None:
        lpo = oracle.logprob(P, S, code)
        bound = shift.sum(axis=1) + 1e-5 * np.abs(lpo)
        err = np.abs(np.asarray(lp, np.float64) - lpo)
        out["logp_within_bound"] = bool(np.all(err <= bound))
        out["logp_max_rel"] = float(np.max(err / np.maximum(np.abs(lpo), 1e-30)))
    return out


def rows_without_near_ties(P, S_oracle, U, act, tol=1e-6):
    Z = oracle.logits(P, S_oracle, act_code(act))
    return ~(np.abs(np.asarray(U, np.float64) - sigmoid(Z)) < tol).any(axis=1)


def rel_err(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (den if den > 0 else 1.0))


def make_model(n, h, B, inst, act="relu", precision="fp32", theta=None, seed=123, lr=1e-2, sampler="auto"):
    from paper_2106_13308_gb300.vqmc import VQMC
    m = VQMC(n, h, B, inst, act=act, precision=precision, seed=seed, lr=lr, sampler=sampler)
    if theta is not None:
        m.set_params(torch.from_numpy(np.asarray(theta, dtype=np.float32)))
    return m


def er_instance(n, p, seed, lo=1, hi=10):
    e = inputs.erdos_renyi(n, p, seed)
    return inputs.to_csr(n, e, inputs.int_weights(len(e), lo, hi, seed + 1))


def grad_blocks(g, n, h):
    g = np.asarray(g, np.float64)
    return {"W1": g[: n * h], "b1": g[n * h: n * h + h], "W2": g[n * h + h: 2 * n * h + h],
            "b2": g[2 * n * h + h:]}


def logp_rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-30)))


__all__ = [name for name in dir() if not name.startswith("_")] + ["math"]
