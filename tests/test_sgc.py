"""Native camera graph and stochastic graph clustering (Sec. 4.4) against the oracle.  Host-only calls of the
C ABI: no GPU is needed."""
import itertools
import math

import numpy as np
import pytest

import scenes
from oracle import sgc
from paper_2008_00446_gb300 import stba


def random_obs(m, n, seed, lo=2, hi=5):
    rng = np.random.default_rng(seed)
    oc, op = [], []
    for i in range(n):
        for j in rng.choice(m, size=int(rng.integers(lo, hi)), replace=False):
            oc.append(int(j))
            op.append(i)
    return np.array(oc, np.int32), np.array(op, np.int32)


def edge_dict(g):
    i, j, w = stba.stba_graph_edges(g)
    assert np.all(i < j)
    return {(int(a), int(b)): int(c) for a, b, c in zip(i, j, w)}


def test_camera_graph_equals_oracle():
    oc, op = random_obs(12, 200, 1)
    g = stba.stba_graph_create(12, 200, oc, op)
    assert edge_dict(g) == sgc.camera_graph(oc, op, 12)
    s = scenes.make_config("c0_ring")
    g = stba.stba_graph_create(s.m, s.n, s.obs_cam, s.obs_pt)
    assert edge_dict(g) == sgc.camera_graph(s.obs_cam, s.obs_pt, s.m)


def connected(w, members):
    members = set(members)
    start = next(iter(members))
    seen, stack = {start}, [start]
    adj = {}
    for (i, j) in w:
        adj.setdefault(i, []).append(j)
        adj.setdefault(j, []).append(i)
    while stack:
        a = stack.pop()
        for b in adj.get(a, []):
            if b in members and b not in seen:
                seen.add(b)
                stack.append(b)
    return seen == members


def check_clustering(w, m, gamma, lab, l):
    lab = [int(x) for x in lab]
    assert max(lab) + 1 == l and sorted(set(lab)) == list(range(l))
    firsts = [lab.index(c) for c in range(l)]
    assert firsts == sorted(firsts)
    sizes = np.bincount(lab, minlength=l)
    assert sizes.max() <= gamma
    for c in range(l):
        assert connected(w, [i for i in range(m) if lab[i] == c])
    for (i, j) in w:
        if lab[i] != lab[j]:
            assert sizes[lab[i]] + sizes[lab[j]] > gamma


@pytest.mark.parametrize("gamma", [1, 2, 5, 10, 30])
def test_clusterings_are_maximal_connected_and_capped(gamma):
    s = scenes.make_config("c0_ring")
    g = stba.stba_graph_create(s.m, s.n, s.obs_cam, s.obs_pt)
    w = edge_dict(g)
    labs, ls = stba.stba_graph_cluster_batch(g, 8, gamma=gamma, beta=10.0, seed=3)
    for lab, l in zip(labs, ls):
        check_clustering(w, s.m, gamma, lab, l)
    if gamma == 1:
        assert np.all(labs == np.arange(s.m))


def test_frequencies_follow_the_exact_distribution():
    # a small graph whose joins differ enough in dQ for Eq. 16 to be far from uniform
    m = 6
    w = {(0, 1): 6, (1, 2): 1, (2, 3): 5, (3, 4): 1, (4, 5): 4, (0, 5): 1, (1, 4): 2}
    oc, op, p = [], [], 0
    for (a, b), c in w.items():
        for _ in range(c):
            oc += [a, b]
            op += [p, p]
            p += 1
    g = stba.stba_graph_create(m, p, oc, op)
    assert edge_dict(g) == w
    gamma, beta = 3, 10.0
    dist = sgc.final_distribution(w, m, gamma, beta)
    N = 20000
    labs, _ = stba.stba_graph_cluster_batch(g, N, gamma=gamma, beta=beta, seed=100)
    counts = {}
    for lab in map(tuple, labs.tolist()):
        counts[lab] = counts.get(lab, 0) + 1
    assert set(counts) <= set(dist)
    assert max(dist.values()) < 0.9 and len(dist) >= 4
    for lab, pr in dist.items():
        sd = math.sqrt(pr * (1 - pr) / N)
        assert abs(counts.get(lab, 0) / N - pr) < 5 * sd + 1e-9, (lab, counts.get(lab, 0) / N, pr)


def test_large_beta_is_the_greedy_join():
    w = {(0, 1): 5, (1, 2): 5, (0, 2): 5, (3, 4): 5, (4, 5): 5, (3, 5): 5, (2, 3): 1}
    oc, op, p = [], [], 0
    for (a, b), c in w.items():
        for _ in range(c):
            oc += [a, b]
            op += [p, p]
            p += 1
    g = stba.stba_graph_create(6, p, oc, op)
    for seed in range(5):
        lab, l = stba.stba_graph_cluster(g, gamma=3, beta=1e5, seed=seed)
        assert list(lab) == sgc.greedy(w, 6, 3) and l == 2


def test_seeds_are_reproducible_and_batches_match_single_draws():
    oc, op = random_obs(40, 400, 7)
    g = stba.stba_graph_create(40, 400, oc, op)
    labs, ls = stba.stba_graph_cluster_batch(g, 5, gamma=8, beta=10.0, seed=21)
    for t in range(5):
        lab, l = stba.stba_graph_cluster(g, gamma=8, beta=10.0, seed=21 + t)
        assert np.array_equal(lab, labs[t]) and l == ls[t]
    assert len({tuple(x) for x in labs.tolist()}) > 1


def test_invalid_arguments():
    oc, op = random_obs(5, 20, 2)
    g = stba.stba_graph_create(5, 20, oc, op)
    for gamma, beta in ((0, 10.0), (5, -1.0), (5, float("nan")), (5, float("inf"))):
        with pytest.raises(stba.StbaError):
            stba.stba_graph_cluster(g, gamma=gamma, beta=beta)
    with pytest.raises(stba.StbaError):
        stba.stba_graph_create(5, 20, np.append(oc, 7), np.append(op, 0))
    with pytest.raises(stba.StbaError):
        stba.stba_graph_create(5, 20, np.append(oc, oc[0]), np.append(op, op[0]))


def test_dense_graph_draws_are_valid():
    # 300 cameras, about 8k camera edges: many records move and merge, and the moved-pair table rehashes
    oc, op = random_obs(300, 6000, 9, lo=2, hi=9)
    g = stba.stba_graph_create(300, 6000, oc, op)
    w = edge_dict(g)
    for gamma in (10, 40):
        labs, ls = stba.stba_graph_cluster_batch(g, 4, gamma=gamma, beta=10.0, seed=2)
        for lab, l in zip(labs, ls):
            check_clustering(w, 300, gamma, lab, l)


@pytest.mark.parametrize("m, n, seed", [(24, 150, 5), (60, 500, 6)])
def test_greedy_limit_on_larger_graphs(m, n, seed):
    # beta so large that every join is the one with the largest dQ: the merged pair sums (W, P) decide
    # every step, so a wrong merge of two records changes the result
    oc, op = random_obs(m, n, seed)
    g = stba.stba_graph_create(m, n, oc, op)
    w = edge_dict(g)
    expect = sgc.greedy(w, m, 6)
    for s in range(3):
        lab, l = stba.stba_graph_cluster(g, gamma=6, beta=1e12, seed=s)
        assert list(lab) == expect


def binom_two_sided(k, n, p):
    """P(X: pmf(X) <= pmf(k)), X ~ Binomial(n, p): the exact two-sided binomial test."""
    logpmf = [math.lgamma(n + 1) - math.lgamma(j + 1) - math.lgamma(n - j + 1) + j * math.log(p)
              + (n - j) * math.log1p(-p) for j in range(n + 1)]
    ref = logpmf[k] + 1e-9 * abs(logpmf[k]) + 1e-12   # outcomes as likely as k, up to rounding, count
    return min(1.0, sum(math.exp(v) for v in logpmf if v <= ref))


def test_binomial_test_helper():
    # hand values: fair coin, 10 tosses, 2 heads -> P(X <= 2 or X >= 8) = 112 / 1024
    assert binom_two_sided(2, 10, 0.5) == pytest.approx(112 / 1024, rel=1e-9)
    assert binom_two_sided(5, 10, 0.5) == pytest.approx(1.0)
    assert binom_two_sided(0, 300, 1e-4) == pytest.approx(1.0)


def test_co_clustering_frequencies_match_the_oracle_sampler():
    # 24 cameras on a banded ring: the probability that two cameras end in one cluster, native draws
    # against the oracle's sampler (Eq. 16 step by step), for every camera pair
    m = 24
    rng = np.random.default_rng(3)
    oc, op = [], []
    for i in range(150):   # banded ring: a point is seen by a camera and 1..3 of its successors
        c0 = int(rng.integers(m))
        for d in range(int(rng.integers(2, 5))):
            oc.append((c0 + d) % m)
            op.append(i)
    oc, op = np.array(oc, np.int32), np.array(op, np.int32)
    g = stba.stba_graph_create(m, 150, oc, op)
    w = edge_dict(g)
    rng = np.random.default_rng(4)
    n_or, n_nat = 300, 6000
    co_or = np.zeros((m, m))
    for _ in range(n_or):
        lab = np.asarray(sgc.sample(w, m, 5, 10.0, rng.random(m)))
        co_or += lab[:, None] == lab[None, :]
    labs, _ = stba.stba_graph_cluster_batch(g, n_nat, gamma=5, beta=10.0, seed=77)
    co_nat = np.zeros((m, m))
    for lab in labs:
        co_nat += lab[:, None] == lab[None, :]
    p_or, p_nat = co_or / n_or, co_nat / n_nat
    p = (co_or + co_nat) / (n_or + n_nat)
    iu = np.triu_indices(m, 1)
    # per camera pair, the exact two-sided binomial test of the oracle's count among its draws against the
    # native frequency (20 times as many draws), Bonferroni-corrected over the pairs: many pairs are rare
    # (counts of 0..2 among the oracle's draws), where a normal approximation overstates the deviation
    pmin = min(binom_two_sided(int(k), n_or, min(max(q, 0.5 / n_nat), 1 - 0.5 / n_nat))
               for k, q in zip(co_or[iu], p_nat[iu]))
    assert pmin * len(iu[0]) > 1e-3, pmin
    assert np.max(np.abs(p_or - p_nat)[iu]) < 0.12
    assert np.ptp(p[iu]) > 0.3   # near cameras share clusters, far ones never: the statistic is not flat
