"""Seeded synthetic inputs for the VQMC hot path.

This module is the only thing the CUDA path and the FP64 oracle share: it
draws problem instances, initial parameters and explicit uniforms as plain
data.  It holds none of the method's arithmetic (no masks, no forward pass, no
energies): each side applies the MADE masks and evaluates everything itself.

Instances follow the paper's workloads (Sec. 5.1) and the benchmark
configurations used throughout the repository:

* ``paper_maxcut``: adjacency from (B + B^T)/2, B_ij ~ Bernoulli(0.5), rounded
  half-to-even and with a zero diagonal, i.e. an edge iff B_ij = B_ji = 1.
* ``erdos_renyi``: G(n, p) by geometric skipping over the strict upper
  triangle (Batagelj and Brandes 2005), so large sparse graphs cost O(n + m).
* ``random_regular``: the configuration (pairing) model with rejection of
  loops and multi-edges.
* ``sk``: Sherrington-Kirkpatrick couplings J_ij = J_ji ~ N(0, 1/n), zero
  diagonal, as a dense float32 matrix.
* ``tim``: the transverse-field Ising model of Eq. (hamiltonian) with the
  paper's disorder (Sec. 5): beta_i, beta_ij ~ U(-1, 1), alpha_i ~ U(0, 1),
  drawn once.  Stored as the library's Ising form E = sum_{i<j} J_ij s_i s_j
  + sum_i h_i s_i with J = -beta, h = -beta_i (dense), plus ``alpha``.

Sparse instances are stored as the strict upper triangle in CSR form
(``row_ptr`` int32 [n+1], ``col`` int32 [m] with col > row, ``w`` int32 or
float32 [m]) plus an optional field ``h`` (here always absent, h = 0).
"""
from __future__ import annotations

import numpy as np

# --------------------------------------------------------------- graphs


def _rng(seed) -> np.random.Generator:
    return np.random.default_rng(np.random.SeedSequence(int(seed)))


def erdos_renyi(n: int, p: float, seed: int) -> np.ndarray:
    """Edges (m, 2) int64 of G(n, p), i < j, in row-major order."""
    rng = _rng(seed)
    total = n * (n - 1) // 2
    if total == 0 or p <= 0:
        return np.zeros((0, 2), dtype=np.int64)
    if p >= 1:
        idx = np.arange(total, dtype=np.int64)
    else:
        # gaps between successive edges are Geometric(p) over the linear index
        est = int(total * p + 10 * np.sqrt(total * p + 1) + 16)
        chunks, pos = [], -1
        while True:
            gaps = rng.geometric(p, size=est)
            cand = pos + np.cumsum(gaps, dtype=np.int64)
            keep = cand[cand < total]
            chunks.append(keep)
            if keep.size < cand.size:
                break
            pos = int(cand[-1])
        idx = np.concatenate(chunks)
    return _unrank_upper(n, idx)


def _unrank_upper(n: int, idx: np.ndarray) -> np.ndarray:
    """Row-major linear index over {(i, j): 0 <= i < j < n} -> (i, j)."""
    idx = np.asarray(idx, dtype=np.int64)
    # start(i) = i*(2n - i - 1)/2 ; find the largest i with start(i) <= idx
    fi = np.floor(((2 * n - 1) - np.sqrt((2.0 * n - 1) ** 2 - 8.0 * idx)) / 2.0).astype(np.int64)
    fi = np.clip(fi, 0, n - 2)

    def start(i):
        return i * (2 * n - i - 1) // 2

    for _ in range(3):  # fix float rounding at the boundaries
        fi = np.where(start(fi) > idx, fi - 1, fi)
        fi = np.where(start(fi + 1) <= idx, fi + 1, fi)
    j = idx - start(fi) + fi + 1
    return np.stack([fi, j], axis=1)


def random_regular(n: int, d: int, seed: int, max_tries: int = 10000) -> np.ndarray:
    """Simple d-regular graph on n vertices by the pairing model with rejection."""
    assert (n * d) % 2 == 0 and d < n
    rng = _rng(seed)
    for _ in range(max_tries):
        pts = np.repeat(np.arange(n, dtype=np.int64), d)
        rng.shuffle(pts)
        e = pts.reshape(-1, 2)
        if np.any(e[:, 0] == e[:, 1]):
            continue
        e = np.sort(e, axis=1)
        key = e[:, 0] * n + e[:, 1]
        if np.unique(key).size != key.size:
            continue
        order = np.argsort(key)
        return e[order]
    raise RuntimeError("random_regular: no simple graph found")


def paper_maxcut(n: int, seed: int) -> np.ndarray:
    """(B + B^T)/2 with B_ij ~ Bernoulli(0.5), rounded half-to-even, zero
    diagonal (Sec. 5.1): an edge iff B_ij = B_ji = 1 (edge density 1/4)."""
    rng = _rng(seed)
    Bm = rng.integers(0, 2, size=(n, n))
    A = np.rint((Bm + Bm.T) / 2.0).astype(np.int64)
    np.fill_diagonal(A, 0)
    i, j = np.nonzero(np.triu(A, 1))
    return np.stack([i, j], axis=1).astype(np.int64)


# ---------------------------------------------------------------- weights

def int_weights(m: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """Integer weights uniform in {lo, ..., hi}."""
    return _rng(seed).integers(lo, hi + 1, size=m).astype(np.int32)


def pm1_weights(m: int, seed: int) -> np.ndarray:
    """Weights uniform in {-1, +1}."""
    return (2 * _rng(seed).integers(0, 2, size=m) - 1).astype(np.int32)


def to_csr(n: int, edges: np.ndarray, w: np.ndarray, field=None) -> dict:
    """CSR of the strict upper triangle; w int32 -> kind 'sparse_i32',
    float -> 'sparse_f32'."""
    edges = np.asarray(edges, dtype=np.int64).reshape(-1, 2)
    w = np.asarray(w)
    assert np.all(edges[:, 0] < edges[:, 1])
    order = np.lexsort((edges[:, 1], edges[:, 0]))
    edges, w = edges[order], w[order]
    counts = np.bincount(edges[:, 0], minlength=n)
    row_ptr = np.zeros(n + 1, dtype=np.int32)
    row_ptr[1:] = np.cumsum(counts)
    is_int = np.issubdtype(w.dtype, np.integer)
    inst = {
        "kind": "sparse_i32" if is_int else "sparse_f32",
        "n": int(n),
        "row_ptr": row_ptr,
        "col": edges[:, 1].astype(np.int32),
        "w": w.astype(np.int32 if is_int else np.float32),
        "field": None if field is None else np.asarray(field, dtype=np.int32 if is_int else np.float32),
    }
    return inst


def sk(n: int, seed: int) -> dict:
    """Dense SK couplings J_ij = J_ji ~ N(0, 1/n), zero diagonal, float32."""
    rng = _rng(seed)
    G = rng.standard_normal((n, n)) / np.sqrt(n)
    J = np.triu(G, 1)
    J = J + J.T
    return {"kind": "dense", "n": int(n), "J": J.astype(np.float32), "field": None}


def tim(n: int, seed: int) -> dict:
    """Transverse-field Ising instance (Eq. (hamiltonian), disorder of Sec. 5):
    dense J = -beta (beta_ij = beta_ji ~ U(-1, 1), zero diagonal), field
    h = -beta_i (beta_i ~ U(-1, 1)), alpha_i ~ U(0, 1), all float32."""
    rng = _rng(seed)
    beta2 = np.triu(rng.uniform(-1.0, 1.0, size=(n, n)), 1)
    beta2 = beta2 + beta2.T
    beta1 = rng.uniform(-1.0, 1.0, size=n)
    alpha = rng.uniform(0.0, 1.0, size=n)
    return {"kind": "dense", "n": int(n), "J": (-beta2).astype(np.float32), "field": (-beta1).astype(np.float32),
            "alpha": alpha.astype(np.float32)}


def dense_from_sparse(inst: dict) -> np.ndarray:
    """The same couplings as a dense symmetric float64 matrix."""
    n = inst["n"]
    J = np.zeros((n, n))
    rp, col, w = inst["row_ptr"], inst["col"], inst["w"]
    for i in range(n):
        for p in range(rp[i], rp[i + 1]):
            J[i, col[p]] = w[p]
            J[col[p], i] = w[p]
    return J


# ------------------------------------------------------------- parameters

def made_params(n: int, h: int, seed: int, w_std: float = 0.01, v_std: float | None = None,
                bias_std: float = 0.0) -> np.ndarray:
    """Flat float32 theta = [W1^T (n x h) | b1 (h) | W2 (n x h) | b2 (n)] with
    W1, W2 entries ~ N(0, std^2) and biases ~ N(0, bias_std^2).  No masks are
    applied here; each side applies the MADE masks itself."""
    rng = _rng(seed)
    v_std = w_std if v_std is None else v_std
    W1t = rng.standard_normal((n, h)) * w_std
    b1 = rng.standard_normal(h) * bias_std
    W2 = rng.standard_normal((n, h)) * v_std
    b2 = rng.standard_normal(n) * bias_std
    return np.concatenate([W1t.ravel(), b1, W2.ravel(), b2]).astype(np.float32)


def lively_params(n: int, h: int, seed: int) -> np.ndarray:
    """Parameters whose conditionals spread over (0, 1) rather than sitting at
    1/2: used by parity tests so that every branch of the sampler is hit."""
    return made_params(n, h, seed, w_std=1.5 / np.sqrt(max(n, 1)), v_std=3.0 / np.sqrt(max(h, 1)),
                       bias_std=0.5)


def uniforms(B: int, n: int, seed: int) -> np.ndarray:
    """Explicit uniforms on the 2^-24 grid in [0, 1), float32 (B, n)."""
    return (_rng(seed).integers(0, 1 << 24, size=(B, n)) * (1.0 / (1 << 24))).astype(np.float32)


def spins(B: int, n: int, seed: int) -> np.ndarray:
    """Uniformly random spin configurations in {-1, +1}, int8 (B, n)."""
    return (2 * _rng(seed).integers(0, 2, size=(B, n)) - 1).astype(np.int8)


# ------------------------------------------------------ named workloads

def config(name: str) -> dict:
    """The benchmark workloads, as plain descriptions (sizes, seeds)."""
    table = {
        # G(20, 0.5), unit weights, sigmoid hidden units, h = 40, B = 1024
        "maxcut_er20": dict(n=20, h=40, B=1024, act="sigmoid", graph="er", p=0.5, weights="unit",
                            graph_seed=1, param_seed=2, w_std=0.01),
        # random 3-regular, n = 1000, weights +-1, h = 1000, B = 4096
        "maxcut_3reg1000": dict(n=1000, h=1000, B=4096, act="relu", graph="regular", d=3,
                                weights="pm1", graph_seed=3, param_seed=4, w_std=0.01),
        # G(10000, 8/9999), weights uniform in {1..10}, h = 2000, B = 2048
        "maxcut_er10000": dict(n=10000, h=2000, B=2048, act="relu", graph="er", p=8.0 / 9999.0,
                               weights="int1_10", graph_seed=5, param_seed=6, w_std=0.01),
        # SK n = 2000 dense J ~ N(0, 1/n), h = 2000, B = 8192
        "sk2000": dict(n=2000, h=2000, B=8192, act="relu", graph="sk", graph_seed=7,
                       param_seed=8, w_std=0.01),
        # transverse-field Ising, n = 500 (the paper's largest TIM size, Tables 1 and 2),
        # h = 5 (ln n)^2 = 193 (Sec. 5), B = 1024
        "tim500": dict(n=500, h=193, B=1024, act="relu", graph="tim", graph_seed=9,
                       param_seed=10, w_std=0.01),
    }
    return dict(table[name], name=name)


def make_instance(cfg: dict) -> dict:
    n, g = cfg["n"], cfg["graph"]
    if g == "sk":
        return sk(n, cfg["graph_seed"])
    if g == "tim":
        return tim(n, cfg["graph_seed"])
    if g == "er":
        e = erdos_renyi(n, cfg["p"], cfg["graph_seed"])
    elif g == "regular":
        e = random_regular(n, cfg["d"], cfg["graph_seed"])
    elif g == "paper":
        e = paper_maxcut(n, cfg["graph_seed"])
    else:
        raise ValueError(g)
    wk = cfg["weights"]
    if wk == "unit":
        w = np.ones(len(e), dtype=np.int32)
    elif wk == "pm1":
        w = pm1_weights(len(e), cfg["graph_seed"] + 1000)
    elif wk == "int1_10":
        w = int_weights(len(e), 1, 10, cfg["graph_seed"] + 1000)
    else:
        raise ValueError(wk)
    return to_csr(n, e, w)


def batched_configs(count: int = 64, n_lo: int = 100, n_hi: int = 5000, avg_deg: float = 6.0,
                    seed: int = 6) -> list:
    """Many independent Max-Cut instances of uneven size: n ~ U{n_lo..n_hi},
    G(n, avg_deg/(n-1)), weights +-1, hidden = n, 512 samples each."""
    rng = _rng(seed)
    ns = rng.integers(n_lo, n_hi + 1, size=count)
    out = []
    for q, n in enumerate(ns):
        out.append(dict(n=int(n), h=int(n), B=512, act="relu", graph="er",
                        p=avg_deg / (int(n) - 1), weights="pm1", graph_seed=10_000 + q,
                        param_seed=20_000 + q, w_std=0.01, name=f"batched_{q}"))
    return out
