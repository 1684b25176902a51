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
