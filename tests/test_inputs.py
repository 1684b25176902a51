"""The seeded synthetic workloads (the paper's instances are not published):
structural properties of every generator, so that the recipes stated for the
benchmark configurations hold - G(n, p) edges unique, in the strict upper
triangle and Binomial in number; 3-regular graphs simple with every degree 3;
SK and transverse-field couplings symmetric with zero diagonal and the
stated distributions; the many-instances configuration; weights and spins in
range; the N = 10,000 benchmark graph's edge count."""
import numpy as np
import pytest

from paper_2106_13308_gb300 import inputs


def _check_simple_upper(e, n):
    assert e.ndim == 2 and e.shape[1] == 2
    assert np.all(e[:, 0] < e[:, 1]) and e.min(initial=0) >= 0 and e.max(initial=0) < n
    key = e[:, 0] * n + e[:, 1]
    assert np.unique(key).size == key.size


@pytest.mark.parametrize("n,p,seed", [(2000, 0.004, 1), (300, 0.3, 2), (50, 0.9, 3)])
def test_erdos_renyi_edges(n, p, seed):
    e = inputs.erdos_renyi(n, p, seed)
    _check_simple_upper(e, n)
    pairs = n * (n - 1) // 2
    mean, sd = pairs * p, np.sqrt(pairs * p * (1 - p))
    assert abs(len(e) - mean) <= 5 * sd
    assert np.array_equal(e, inputs.erdos_renyi(n, p, seed))  # seeded


def test_erdos_renyi_edge_cases():
    assert inputs.erdos_renyi(1, 0.5, 1).shape == (0, 2)
    assert inputs.erdos_renyi(10, 0.0, 1).shape == (0, 2)
    assert len(inputs.erdos_renyi(10, 1.0, 1)) == 45


def test_erdos_renyi_covers_pairs_uniformly():
    """Every pair is an edge with probability p: the edge frequency of each
    pair over 400 seeds of G(12, 0.3) stays within 5 standard deviations."""
    n, p, reps = 12, 0.3, 400
    cnt = np.zeros((n, n))
    for s in range(reps):
        e = inputs.erdos_renyi(n, p, 1000 + s)
        cnt[e[:, 0], e[:, 1]] += 1
    iu = np.triu_indices(n, 1)
    sd = np.sqrt(reps * p * (1 - p))
    assert np.all(np.abs(cnt[iu] - reps * p) <= 5 * sd)


def test_benchmark_graph_edge_count():
    cfg = inputs.config("maxcut_er10000")
    inst = inputs.make_instance(cfg)
    assert inst["n"] == 10000 and len(inst["col"]) == 40328  # the count stated for the workload
    w = inst["w"]
    assert w.dtype == np.int32 and w.min() >= 1 and w.max() <= 10


@pytest.mark.parametrize("n,d", [(1000, 3), (20, 3), (9, 4)])
def test_random_regular_is_simple_and_regular(n, d):
    e = inputs.random_regular(n, d, 7)
    _check_simple_upper(e, n)
    deg = np.bincount(e.ravel(), minlength=n)
    assert np.all(deg == d) and len(e) == n * d // 2


def test_csr_holds_the_edges_and_weights():
    n = 40
    e = inputs.erdos_renyi(n, 0.2, 5)
    w = inputs.int_weights(len(e), -3, 7, 6)
    inst = inputs.to_csr(n, e[::-1], w[::-1])  # any input order
    rp, col = inst["row_ptr"], inst["col"]
    assert rp[0] == 0 and rp[-1] == len(e) and np.all(np.diff(rp) >= 0)
    got = {(i, int(col[q])): int(inst["w"][q]) for i in range(n) for q in range(rp[i], rp[i + 1])}
    assert got == {(int(a), int(b)): int(x) for (a, b), x in zip(e, w)}
    J = inputs.dense_from_sparse(inst)
    assert np.array_equal(J, J.T) and np.all(np.diag(J) == 0)


def test_weights_and_spins_in_range():
    w = inputs.int_weights(10000, 1, 10, 1)
    assert w.min() == 1 and w.max() == 10
    pm = inputs.pm1_weights(10000, 2)
    assert set(np.unique(pm)) == {-1, 1} and abs(pm.mean()) < 0.05
    S = inputs.spins(100, 37, 3)
    assert S.dtype == np.int8 and S.shape == (100, 37) and set(np.unique(S)) <= {-1, 1}


def test_sk_couplings():
    n = 400
    inst = inputs.sk(n, 7)
    J = inst["J"].astype(np.float64)
    assert inst["kind"] == "dense" and inst["J"].dtype == np.float32
    assert np.array_equal(J, J.T) and np.all(np.diag(J) == 0)
    iu = np.triu_indices(n, 1)
    assert abs(J[iu].var() * n - 1.0) < 0.02 and abs(J[iu].mean()) < 5 / n


def test_transverse_field_instance():
    n = 300
    inst = inputs.tim(n, 9)
    J, hf, a = inst["J"], inst["field"], inst["alpha"]
    assert np.array_equal(J, J.T) and np.all(np.diag(J) == 0)
    iu = np.triu_indices(n, 1)
    assert J[iu].min() >= -1 and J[iu].max() <= 1 and abs(J[iu].var() - 1 / 3) < 0.01
    assert hf.min() >= -1 and hf.max() <= 1
    assert a.min() >= 0 and a.max() < 1


def test_many_instances_configuration():
    cfgs = inputs.batched_configs()
    assert len(cfgs) == 64
    for c in cfgs:
        assert 100 <= c["n"] <= 5000 and c["h"] == c["n"] and c["B"] == 512
        assert abs(c["p"] * (c["n"] - 1) - 6.0) < 1e-9 and c["weights"] == "pm1"
    assert len({c["graph_seed"] for c in cfgs}) == 64


def test_parameters_layout():
    n, h = 13, 7
    th = inputs.made_params(n, h, 3, w_std=0.01)
    assert th.dtype == np.float32 and th.size == 2 * n * h + h + n
    assert np.all(th[n * h: n * h + h] == 0) and np.all(th[2 * n * h + h:] == 0)  # biases zero
    assert abs(th[: n * h].std() - 0.01) < 0.004
