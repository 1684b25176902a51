"""FP64 CPU oracle for the VQMC hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never calls it and the
two share no code; they meet only through the seeded inputs of
``paper_2106_13308_gb300.inputs`` (which hold none of the method's arithmetic).

The arithmetic lives in ``vqmc_oracle.c`` (plain C, IEEE double, OpenMP over
samples).  This module compiles it with gcc on first use and exposes it with
NumPy arguments, using the paper's parameter shapes (Sec. 2.3):

    W1 (h, n), b1 (h,), W2 (n, h), b2 (n,)      z = (M2.W2) act((M1.W1) s + b1) + b2

``theta_to_made`` / ``made_to_theta`` convert from/to the flat layout the CUDA
library uses, theta = [W1^T (n x h) | b1 (h) | W2 (n x h) | b2 (n)] (Sec. 4:
d = 2hn + h + n parameters).

Every function that has a pin in ``tests/test_oracle_*.py`` is listed there;
none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vqmc_oracle.c")
_LIB = os.path.join(_HERE, "libvqmc_oracle.so")
_lock = threading.Lock()
_lib = None

RELU, SIGMOID = 0, 1
# OR into an activation code: hidden activations rounded to bfloat16 (the BF16 model)
HIDDEN_BF16 = 2


def build(force: bool = False) -> str:
    """Compile the oracle shared library in place (gcc, -O2, OpenMP, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-fno-fast-math",
               "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            I = ctypes.c_int
            D = ctypes.c_double
            lib.vo_round_bf16.restype = D
            lib.vo_round_bf16.argtypes = [D]
            lib.vo_degree.restype = ctypes.c_long
            lib.vo_degree.argtypes = [ctypes.c_long] * 3
            lib.vo_num_threads.restype = I
            lib.vo_philox4x32_10.argtypes = [P, P, P]
            lib.vo_uniforms.argtypes = [I, I, ctypes.c_uint64, ctypes.c_uint64, P]
            lib.vo_forward.argtypes = [I, I, I, P, P, P, P, P, P, P]
            lib.vo_logprob.argtypes = [I, I, I, I, P, P, P, P, P, P]
            lib.vo_logits.argtypes = [I, I, I, I, P, P, P, P, P, P]
            lib.vo_sample_literal.argtypes = [I, I, I, I, P, P, P, P, P, P, P]
            lib.vo_sample_incremental.argtypes = [I, I, I, I, P, P, P, P, P, P, P]
            lib.vo_energy_sparse.argtypes = [I, I, P, P, P, P, P, P]
            lib.vo_energy_dense.argtypes = [I, I, P, P, P, P]
            lib.vo_energy_tim_offdiag.argtypes = [I, I, I, I, P, P, P, P, P, P, P]
            lib.vo_cut.argtypes = [I, I, P, P, P, P, P]
            lib.vo_maxcut_bruteforce.restype = D
            lib.vo_maxcut_bruteforce.argtypes = [I, P, P, P]
            lib.vo_stats.argtypes = [I, P, P, P]
            lib.vo_logprob_grad.argtypes = [I, I, I, I, P, P, P, P, P, P, P, P, P, P]
            lib.vo_adam.argtypes = [ctypes.c_long, P, P, P, P, I, D, D, D, D]
            lib.vo_enumerate.argtypes = [I, I, I, P, P, P, P, P, P, P, P, P, P]
            _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def _i8(a):
    return np.ascontiguousarray(a, dtype=np.int8)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def round_bf16(x) -> np.ndarray:
    """Each value rounded to the nearest bfloat16 (ties to even), as float64."""
    lib = _load()
    flat = np.asarray(x, dtype=np.float64).ravel()
    return np.array([lib.vo_round_bf16(float(v)) for v in flat], dtype=np.float64).reshape(np.shape(x))


def num_threads() -> int:
    return int(_load().vo_num_threads())


# ------------------------------------------------------------------ layout

def degrees(n: int, h: int) -> np.ndarray:
    """m(k) = 1 + floor(k (n-1) / h), k = 0..h-1 (MADE degree rule)."""
    lib = _load()
    return np.array([lib.vo_degree(k, n, h) for k in range(h)], dtype=np.int64)


def theta_to_made(theta, n: int, h: int):
    """Split the flat theta = [W1^T | b1 | W2 | b2] into FP64 (W1, b1, W2, b2)."""
    t = np.asarray(theta, dtype=np.float64).reshape(-1)
    assert t.size == 2 * n * h + h + n
    W1t = t[: n * h].reshape(n, h)
    b1 = t[n * h: n * h + h]
    W2 = t[n * h + h: 2 * n * h + h].reshape(n, h)
    b2 = t[2 * n * h + h:]
    return (np.ascontiguousarray(W1t.T), b1.copy(), np.ascontiguousarray(W2), b2.copy())


def made_to_theta(W1, b1, W2, b2) -> np.ndarray:
    """Inverse of theta_to_made."""
    return np.concatenate([np.asarray(W1).T.reshape(-1), np.asarray(b1).reshape(-1),
                           np.asarray(W2).reshape(-1), np.asarray(b2).reshape(-1)]).astype(np.float64)


# --------------------------------------------------------------- generator

def philox4x32_10(ctr, key) -> np.ndarray:
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.vo_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def uniforms(B: int, n: int, seed: int, it: int) -> np.ndarray:
    lib = _load()
    u = np.zeros((B, n), dtype=np.float32)
    lib.vo_uniforms(B, n, seed, it, _p(u))
    return u


# ------------------------------------------------------------------ model

def _made(params):
    W1, b1, W2, b2 = params
    return _f64(W1), _f64(b1), _f64(W2), _f64(b2)


def forward(params, s, act=RELU):
    """(a, z) of one sample: pre-activations (h,) and logits (n,)."""
    lib = _load()
    W1, b1, W2, b2 = _made(params)
    h, n = W1.shape
    s = _i8(s)
    a = np.zeros(h)
    z = np.zeros(n)
    lib.vo_forward(n, h, act, _p(W1), _p(b1), _p(W2), _p(b2), _p(s), _p(a), _p(z))
    return a, z


def logprob(params, S, act=RELU) -> np.ndarray:
    lib = _load()
    W1, b1, W2, b2 = _made(params)
    h, n = W1.shape
    S = _i8(S).reshape(-1, n)
    out = np.zeros(S.shape[0])
    lib.vo_logprob(S.shape[0], n, h, act, _p(W1), _p(b1), _p(W2), _p(b2), _p(S), _p(out))
    return out


def logits(params, S, act=RELU) -> np.ndarray:
    lib = _load()
    W1, b1, W2, b2 = _made(params)
    h, n = W1.shape
    S = _i8(S).reshape(-1, n)
    Z = np.zeros(S.shape, dtype=np.float64)
    lib.vo_logits(S.shape[0], n, h, act, _p(W1), _p(b1), _p(W2), _p(b2), _p(S), _p(Z))
    return Z


def sample(params, U, act=RELU, literal=False):
    """Algorithm 1 on the given uniforms U (B, n) float32 -> (S int8, logp)."""
    lib = _load()
    W1, b1, W2, b2 = _made(params)
    h, n = W1.shape
    U = np.ascontiguousarray(U, dtype=np.float32).reshape(-1, n)
    B = U.shape[0]
    S = np.zeros((B, n), dtype=np.int8)
    lp = np.zeros(B)
    fn = lib.vo_sample_literal if literal else lib.vo_sample_incremental
    fn(B, n, h, act, _p(W1), _p(b1), _p(W2), _p(b2), _p(U), _p(S), _p(lp))
    return S, lp


# ---------------------------------------------------------------- energies

def energy_sparse(inst, S) -> np.ndarray:
    lib = _load()
    n = inst["n"]
    rp, col = _i32(inst["row_ptr"]), _i32(inst["col"])
    w = _f64(inst["w"])
    f = _f64(inst.get("field"))
    S = _i8(S).reshape(-1, n)
    E = np.zeros(S.shape[0])
    lib.vo_energy_sparse(S.shape[0], n, _p(rp), _p(col), _p(w), _p(f), _p(S), _p(E))
    return E


def energy_dense(J, S, field=None) -> np.ndarray:
    lib = _load()
    J = _f64(J)
    n = J.shape[0]
    S = _i8(S).reshape(-1, n)
    E = np.zeros(S.shape[0])
    lib.vo_energy_dense(S.shape[0], n, _p(J), _p(_f64(field)), _p(S), _p(E))
    return E


def energy(inst, S) -> np.ndarray:
    """Diagonal (Ising) part of the local energy."""
    if inst["kind"] == "dense":
        return energy_dense(inst["J"], S, inst.get("field"))
    return energy_sparse(inst, S)


def energy_tim_offdiag(params, S, alpha, act=RELU) -> np.ndarray:
    """-sum_i alpha_i sqrt(pi(s^(i)) / pi(s)) for each sample (transverse field
    of Eq. (hamiltonian), psi = sqrt(pi)); n + 1 forward passes per sample."""
    lib = _load()
    W1, b1, W2, b2 = _made(params)
    h, n = W1.shape
    S = _i8(S).reshape(-1, n)
    alpha = _f64(alpha).reshape(-1)
    assert alpha.size == n
    E = np.zeros(S.shape[0])
    lib.vo_energy_tim_offdiag(S.shape[0], n, h, act, _p(W1), _p(b1), _p(W2), _p(b2), _p(alpha), _p(S), _p(E))
    return E


def local_energy(params, inst, S, act=RELU) -> np.ndarray:
    """Local energy of each sample: the diagonal energy, plus the transverse
    field's off-diagonal part when the instance has "alpha" (the model's
    parameters are needed only then)."""
    E = energy(inst, S)
    if inst.get("alpha") is not None:
        E = E + energy_tim_offdiag(params, S, inst["alpha"], act)
    return E


def cut(inst, S) -> np.ndarray:
    lib = _load()
    n = inst["n"]
    rp, col = _i32(inst["row_ptr"]), _i32(inst["col"])
    w = _f64(inst["w"])
    S = _i8(S).reshape(-1, n)
    c = np.zeros(S.shape[0])
    lib.vo_cut(S.shape[0], n, _p(rp), _p(col), _p(w), _p(S), _p(c))
    return c


def maxcut_bruteforce(inst) -> float:
    lib = _load()
    rp, col = _i32(inst["row_ptr"]), _i32(inst["col"])
    w = _f64(inst["w"])
    return float(lib.vo_maxcut_bruteforce(inst["n"], _p(rp), _p(col), _p(w)))


# ------------------------------------------------------------------ stats

def stats(E):
    """({mean, var, min, max}, coef) with coef_b = (E_b - mean) / B."""
    lib = _load()
    E = _f64(E).reshape(-1)
    out = np.zeros(4)
    coef = np.zeros(E.size)
    lib.vo_stats(E.size, _p(E), _p(out), _p(coef))
    return out, coef


# --------------------------------------------------------------- gradient

def logprob_grad(params, S, coef, act=RELU):
    """sum_b coef_b grad log pi(s_b) as (dW1, db1, dW2, db2)."""
    lib = _load()
    W1, b1, W2, b2 = _made(params)
    h, n = W1.shape
    S = _i8(S).reshape(-1, n)
    coef = _f64(coef).reshape(-1)
    assert coef.size == S.shape[0]
    dW1 = np.zeros((h, n))
    db1 = np.zeros(h)
    dW2 = np.zeros((n, h))
    db2 = np.zeros(n)
    lib.vo_logprob_grad(S.shape[0], n, h, act, _p(W1), _p(b1), _p(W2), _p(b2), _p(S), _p(coef),
                        _p(dW1), _p(db1), _p(dW2), _p(db2))
    return dW1, db1, dW2, db2


def vqmc_grad(params, inst, S, act=RELU):
    """Score-function gradient of one batch: stats of E, then sum_b c_b grad log pi."""
    E = local_energy(params, inst, S, act)
    st, coef = stats(E)
    return logprob_grad(params, S, coef, act), st, E


def per_sample_grads(params, S, act=RELU) -> np.ndarray:
    """O[b] = grad_theta log pi(s_b) in the flat theta layout, (B, d) FP64:
    the chain-rule gradient of one sample at a time."""
    W1, b1, W2, b2 = _made(params)
    S = _i8(S).reshape(-1, W1.shape[1])
    rows = [made_to_theta(*logprob_grad(params, S[b:b + 1], np.ones(1), act)) for b in range(S.shape[0])]
    return np.stack(rows)


def sr_gram(params, S, act=RELU) -> np.ndarray:
    """G[b][c] = O_b . O_c, the (B, B) Gram matrix of the per-sample score
    vectors (Sec. 2.1): B I with I the batch estimate of the Fisher form."""
    O = per_sample_grads(params, S, act)
    return O @ O.T


def sr_direction(params, inst, S, lam, act=RELU):
    """Stochastic reconfiguration (Sec. 2.1): with the batch estimates of the
    paper's population forms,
        g = (1/B) sum_b (E_b - mean E) O_b,   I = (1/B) sum_b O_b O_b^T,
    the natural-gradient direction solves (I + lam 1) delta = g; the update
    is theta <- theta - lr delta.  The d x d matrix is formed and solved
    directly (FP64), so this is for small models.  Returns (delta, stats)."""
    E = local_energy(params, inst, S, act)
    st, coef = stats(E)
    O = per_sample_grads(params, S, act)
    B, d = O.shape
    g = O.T @ (E - st[0]) / B
    I = O.T @ O / B
    delta = np.linalg.solve(I + lam * np.eye(d), g)
    return delta, st


def adam(theta, m, v, g, t, lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-8):
    """In-place Adam step on FP64 arrays."""
    lib = _load()
    for a in (theta, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    g = _f64(g)
    lib.vo_adam(theta.size, _p(theta), _p(m), _p(v), _p(g), t, lr, beta1, beta2, eps)


# ------------------------------------------------------------ enumeration

def enumerate_exact(params, inst, act=RELU, grad=False):
    """Exact (sum p, <E>, var E[, grad <E>]) by summing over all 2^n states."""
    lib = _load()
    W1, b1, W2, b2 = _made(params)
    h, n = W1.shape
    assert n <= 24
    rp, col = _i32(inst["row_ptr"]), _i32(inst["col"])
    w = _f64(inst["w"])
    f = _f64(inst.get("field"))
    out = np.zeros(3)
    g = np.zeros(2 * n * h + h + n) if grad else None
    lib.vo_enumerate(n, h, act, _p(W1), _p(b1), _p(W2), _p(b2), _p(rp), _p(col), _p(w), _p(f),
                     _p(out), _p(g))
    if not grad:
        return out
    nW = h * n
    return out, (g[:nW].reshape(h, n), g[nW:nW + h], g[nW + h:nW + h + n * h].reshape(n, h),
                 g[nW + h + n * h:])
