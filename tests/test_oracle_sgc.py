"""Pins of the stochastic-graph-clustering oracle (Sec. 4.4, Eq. 16) against hand-computed values, closed
forms, identities and brute force."""
import itertools
import math

import numpy as np
import pytest

from oracle import sgc


def test_camera_graph_matches_pairwise_intersections():
    rng = np.random.default_rng(3)
    m, n = 7, 40
    obs_cam, obs_pt = [], []
    for i in range(n):
        for j in rng.choice(m, size=rng.integers(2, 5), replace=False):
            obs_cam.append(int(j))
            obs_pt.append(i)
    w = sgc.camera_graph(obs_cam, obs_pt, m)
    seen = [set(p for c, p in zip(obs_cam, obs_pt) if c == j) for j in range(m)]
    for a, b in itertools.combinations(range(m), 2):
        common = len(seen[a] & seen[b])
        assert w.get((a, b), 0) == common


# edges (0,1):3, (1,2):1, (2,3):2, (0,2):1 -> s = 7, k = (4, 4, 4, 2)
W4 = {(0, 1): 3, (1, 2): 1, (2, 3): 2, (0, 2): 1}


def test_modularity_hand_values():
    assert sgc.modularity(W4, 4, [0, 0, 1, 1]) == pytest.approx(23.0 / 98.0, rel=1e-15)
    assert sgc.modularity(W4, 4, [0, 1, 2, 3]) == 0.0
    assert sgc.modularity(W4, 4, [0, 0, 0, 0]) == pytest.approx(3.0 / 14.0, rel=1e-15)


def test_delta_q_is_the_modularity_increase():
    rng = np.random.default_rng(5)
    m = 9
    for trial in range(20):
        w = {}
        for a, b in itertools.combinations(range(m), 2):
            if rng.random() < 0.4:
                w[(a, b)] = int(rng.integers(1, 20))
        lab = list(rng.integers(0, 4, size=m))
        X = [i for i in range(m) if lab[i] == 0]
        Y = [i for i in range(m) if lab[i] == 1]
        if not X or not Y:
            continue
        after = [0 if lab[i] == 1 else lab[i] for i in range(m)]
        d = sgc.modularity(w, m, after) - sgc.modularity(w, m, lab)
        assert sgc.delta_q(w, m, X, Y) == pytest.approx(d, abs=1e-14)


def test_symmetric_path_joins_are_equally_likely():
    w = {(0, 1): 1, (1, 2): 1}
    dist = sgc.final_distribution(w, 3, 2, 10.0)
    assert dist == pytest.approx({(0, 0, 1): 0.5, (0, 1, 1): 0.5}, rel=1e-15)
    assert sgc.final_distribution(w, 3, 3, 10.0) == pytest.approx({(0, 0, 0): 1.0})


def test_eq16_probability_on_an_unequal_path():
    # w_ab = 2, w_bc = 1: s = 3, k = (2, 3, 1); dQ(a,b) = (2 - 6/6)/6 = 1/6, dQ(b,c) = (1 - 3/6)/6 = 1/12
    w = {(0, 1): 2, (1, 2): 1}
    for beta in (0.0, 1.0, 10.0, 40.0):
        p_ab = math.exp(beta / 6) / (math.exp(beta / 6) + math.exp(beta / 12))
        dist = sgc.final_distribution(w, 3, 2, beta)
        assert dist[(0, 0, 1)] == pytest.approx(p_ab, rel=1e-14)
        assert dist[(0, 1, 1)] == pytest.approx(1 - p_ab, rel=1e-14)


def _connected(w, members):
    members = set(members)
    if len(members) == 1:
        return True
    start = next(iter(members))
    seen, stack = {start}, [start]
    while stack:
        a = stack.pop()
        for (i, j) in w:
            for x, y in ((i, j), (j, i)):
                if x == a and y in members and y not in seen:
                    seen.add(y)
                    stack.append(y)
    return seen == members


def _check_final(w, m, gamma, lab):
    l = max(lab) + 1
    assert sorted(set(lab)) == list(range(l))
    firsts = [min(i for i in range(m) if lab[i] == c) for c in range(l)]
    assert firsts == sorted(firsts)   # numbered by smallest camera
    sizes = [lab.count(c) for c in range(l)]
    assert max(sizes) <= gamma
    for c in range(l):
        assert _connected(w, [i for i in range(m) if lab[i] == c])
    for (i, j) in w:   # maximal: no allowed join left
        if lab[i] != lab[j]:
            assert sizes[lab[i]] + sizes[lab[j]] > gamma


def test_final_distribution_is_a_distribution_over_maximal_clusterings():
    rng = np.random.default_rng(11)
    m = 6
    w = {}
    for a, b in itertools.combinations(range(m), 2):
        if rng.random() < 0.6:
            w[(a, b)] = int(rng.integers(1, 6))
    for gamma in (1, 2, 3, 6):
        dist = sgc.final_distribution(w, m, gamma, 10.0)
        assert sum(dist.values()) == pytest.approx(1.0, abs=1e-13)
        for lab in dist:
            _check_final(w, m, gamma, list(lab))
    assert sgc.final_distribution(w, m, 1, 10.0) == {tuple(range(m)): 1.0}


def test_sampler_frequencies_follow_the_enumeration():
    w = {(0, 1): 1, (1, 2): 4, (2, 3): 1, (0, 3): 2, (1, 3): 1}
    m, gamma, beta = 4, 2, 10.0
    dist = sgc.final_distribution(w, m, gamma, beta)
    rng = np.random.default_rng(17)
    N = 4000
    counts = {}
    for _ in range(N):
        lab = tuple(sgc.sample(w, m, gamma, beta, rng.random(m)))
        counts[lab] = counts.get(lab, 0) + 1
    assert set(counts) <= set(dist)
    for lab, p in dist.items():
        sd = math.sqrt(p * (1 - p) / N)
        assert abs(counts.get(lab, 0) / N - p) < 5 * sd + 1e-12


def test_greedy_splits_two_triangles():
    w = {(0, 1): 5, (1, 2): 5, (0, 2): 5, (3, 4): 5, (4, 5): 5, (3, 5): 5, (2, 3): 1}
    assert sgc.greedy(w, 6, 3) == [0, 0, 0, 1, 1, 1]
    # a large beta concentrates Eq. 16 on the largest increase
    dist = sgc.final_distribution(w, 6, 3, 2000.0)
    assert dist[(0, 0, 0, 1, 1, 1)] > 0.999
