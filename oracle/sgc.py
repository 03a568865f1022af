"""Stochastic graph clustering (Sec. 4.4, Eq. 16) -- plain reference implementation.

TEST INFRASTRUCTURE ONLY (see the package docstring): the product path never imports this module.

The camera graph joins two cameras when they observe a common point; the weight w_ij of edge (i, j) is
the number of points both observe.  Clusters start as single cameras and are joined one pair at a time,
bottom-up.  A join of two neighbouring clusters N_x, N_y (at least one camera edge between them) is
drawn with probability proportional to exp(beta * dQ(N_x, N_y)) (Eq. 16), where dQ is the increase of
the modularity

    Q = 1/(2s) * sum over edges e_ij of delta(nu_i, nu_j) * (w_ij - k_i k_j / (2s)),

s = sum of all edge weights (each edge once), k_i = sum of the weights of the edges at camera i.  The
sum runs over the edges of the graph, as the paper writes it (not over all ordered pairs of cameras as in
the textbook modularity).  Joining N_x and N_y therefore adds exactly the terms of the edges between
them:

    dQ(N_x, N_y) = 1/(2s) * sum over edges e_ij, i in N_x, j in N_y, of (w_ij - k_i k_j / (2s)).

Readings where the paper is silent (listed in the design notes as well):
  * a join is allowed when the joined cluster has at most Gamma cameras ("we stop joining clusters if
    their sizes exceed Gamma"); the normalisation of Eq. 16 runs over the allowed joins;
  * the process ends when no allowed join is left (every pair of neighbouring clusters would exceed
    Gamma); a join is allowed whatever the sign of dQ;
  * the final clusters are numbered 0..l-1 in the order of their smallest camera index.

Functions:
  camera_graph           -- edge weights from the observations (plain loops)
  modularity, delta_q    -- Q and dQ by their definitions
  allowed_joins          -- the allowed joins of a partition with their Eq. 16 probabilities
  sample                 -- one clustering, drawing each join by inverse CDF from given uniforms
  final_distribution     -- exact probability of every final clustering (tiny graphs: enumerates all
                            join sequences)
  greedy                 -- the limit beta -> infinity: always the join with the largest dQ
"""
from __future__ import annotations

import math
from functools import lru_cache


def camera_graph(obs_cam, obs_pt, m):
    """{(i, j): w_ij} with i < j: the number of points observed by both cameras."""
    tracks = {}
    for j, i in zip(obs_cam, obs_pt):
        tracks.setdefault(int(i), set()).add(int(j))
    w = {}
    for cams in tracks.values():
        cs = sorted(cams)
        for a in range(len(cs)):
            for b in range(a + 1, len(cs)):
                w[(cs[a], cs[b])] = w.get((cs[a], cs[b]), 0) + 1
    return w


def strengths(w, m):
    """s and k_i."""
    k = [0.0] * m
    s = 0.0
    for (i, j), x in w.items():
        k[i] += x
        k[j] += x
        s += x
    return s, k


def modularity(w, m, label):
    """Q of the partition given by label[i] (cluster of camera i), summed over the edges."""
    s, k = strengths(w, m)
    q = 0.0
    for (i, j), x in w.items():
        if label[i] == label[j]:
            q += x - k[i] * k[j] / (2.0 * s)
    return q / (2.0 * s)


def delta_q(w, m, X, Y):
    """dQ of joining the camera sets X and Y."""
    s, k = strengths(w, m)
    X, Y = set(X), set(Y)
    d = 0.0
    for (i, j), x in w.items():
        if (i in X and j in Y) or (i in Y and j in X):
            d += x - k[i] * k[j] / (2.0 * s)
    return d / (2.0 * s)


def _neighbours(w, part):
    """Pairs (a, b), a < b, of indices into the tuple of clusters `part` joined by at least one edge."""
    where = {}
    for c, cl in enumerate(part):
        for i in cl:
            where[i] = c
    nb = set()
    for (i, j) in w:
        a, b = where[i], where[j]
        if a != b:
            nb.add((min(a, b), max(a, b)))
    return sorted(nb)


def allowed_joins(w, m, part, gamma, beta):
    """[(a, b, probability)] over the allowed joins of the clusters part[a], part[b] (Eq. 16)."""
    joins = [(a, b) for a, b in _neighbours(w, part) if len(part[a]) + len(part[b]) <= gamma]
    if not joins:
        return []
    e = [math.exp(beta * delta_q(w, m, part[a], part[b])) for a, b in joins]
    t = sum(e)
    return [(a, b, x / t) for (a, b), x in zip(joins, e)]


def _join(part, a, b):
    rest = [cl for c, cl in enumerate(part) if c not in (a, b)]
    return tuple(sorted(rest + [tuple(sorted(part[a] + part[b]))]))


def labels(part, m):
    """Cluster ids 0..l-1 in the order of the clusters' smallest camera."""
    lab = [0] * m
    for c, cl in enumerate(sorted(part, key=min)):
        for i in cl:
            lab[i] = c
    return lab


def sample(w, m, gamma, beta, uniforms):
    """One clustering.  The t-th join takes the t-th number of `uniforms` (in [0, 1)) and picks the join
    whose cumulative probability, in the order of allowed_joins, first exceeds it."""
    part = tuple((i,) for i in range(m))
    t = 0
    while True:
        joins = allowed_joins(w, m, part, gamma, beta)
        if not joins:
            return labels(part, m)
        u = uniforms[t]
        t += 1
        acc = 0.0
        pick = joins[-1]
        for jn in joins:
            acc += jn[2]
            if u < acc:
                pick = jn
                break
        part = _join(part, pick[0], pick[1])


def final_distribution(w, m, gamma, beta):
    """{tuple(labels): probability} over all final clusterings (exhaustive; tiny graphs only)."""
    edges = tuple(sorted(w.items()))

    @lru_cache(maxsize=None)
    def go(part):
        joins = allowed_joins(dict(edges), m, part, gamma, beta)
        if not joins:
            return {tuple(labels(part, m)): 1.0}
        out = {}
        for a, b, p in joins:
            for key, q in go(_join(part, a, b)).items():
                out[key] = out.get(key, 0.0) + p * q
        return out

    return go(tuple((i,) for i in range(m)))


def greedy(w, m, gamma):
    """beta -> infinity: every step takes the allowed join with the largest dQ."""
    part = tuple((i,) for i in range(m))
    while True:
        joins = [(a, b) for a, b in _neighbours(w, part) if len(part[a]) + len(part[b]) <= gamma]
        if not joins:
            return labels(part, m)
        a, b = max(joins, key=lambda ab: delta_q(w, m, part[ab[0]], part[ab[1]]))
        part = _join(part, a, b)
