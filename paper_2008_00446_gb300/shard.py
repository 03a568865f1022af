"""Cluster sharding of the STBA iteration over several GPUs (one process per GPU): the host-side plan.

After point splitting and binding (Sec. 4.1-4.2) the clusters share no virtual point, so the cluster
systems S'_k Delta c_k = b'_k of Eq. 13 and their factorisations are independent.  A rank therefore owns
whole clusters: their cameras, the observations those cameras make, the virtual points of those
observations and the points they see.  The residuals and Jacobians (Algorithm 1, first step), the
virtual-point blocks (Eq. 10), S'_k, b'_k and the cluster solves are local.  What sums over all the clusters
that see one physical point is exchanged, and only for the boundary points (seen by cameras of two or more
ranks):

  1. the steepest-descent correction (Sec. 4.3; taken when lambda >= 0.1): per point and coordinate, the
     sums over its virtual copies of w' and of the diagonal of H_lambda -- 6 values per boundary point,
     before b'_k is formed;
  2. the point update (Eq. 15, equal to Eq. 6): the physical damped C_i (6 values of the symmetric 3 x 3)
     and w_i (3 values), which do not depend on Delta c and can be summed while the clusters factorise,
     then the partial sums of W_o^T Delta c_cam(o) over each rank's own observations (3 values) once the
     cluster solves are done, so the point update needs no other rank's Delta c;
  3. the LM control (Algorithm 1): F(x + Delta x), the gradient max-norm and the two norms of the stop
     tests, four scalars;
  4. on an accepted step, the update itself: Algorithm 1 draws a new clustering every iteration, so cameras
     move between ranks from one iteration to the next.  Every rank therefore keeps the whole problem
     resident (observations and parameters: far below one GPU's memory even for 25M observations) and
     works on its owned part only; the owner of each camera contributes its Delta c and the lowest rank
     that sees each point its Delta p, and every rank applies the gathered update (9 m + 3 n values).  A
     rejected step exchanges nothing more.

Clusters go to ranks longest-processing-time first, by a cost model of one iteration per cluster: the
factorisation, (9 n_k)^3 / 3 flops, plus a per-observation term for the linearisation and the system
build.  Points seen by several ranks are counted in the norms by the lowest of them.

This module is host logic only (NumPy); it runs no arithmetic of the method."""
from __future__ import annotations

import dataclasses

import numpy as np

OBS_COST = 2000.0   # flop-equivalents per observation (Jacobian, virtual-point blocks, camera-pair sums)


@dataclasses.dataclass
class ShardPlan:
    rank: int
    world: int
    clusters: np.ndarray       # owned cluster ids, ascending
    cameras: np.ndarray        # owned camera ids, ascending
    obs: np.ndarray            # indices of the observations made by owned cameras, ascending
    points: np.ndarray         # points seen by owned cameras, ascending
    boundary: np.ndarray       # boundary point ids, ascending (the same array on every rank)
    boundary_slot: np.ndarray  # per entry of `points`: its position in `boundary`, or -1
    counts_point: np.ndarray   # per entry of `points`: True where this rank is the lowest that sees it
    load: float                # the cost model's total over the owned clusters
    m: int                     # cameras of the whole problem
    n: int                     # points of the whole problem

    @property
    def local_boundary(self) -> np.ndarray:
        """Positions in `points` of the boundary points this rank sees."""
        return np.flatnonzero(self.boundary_slot >= 0)


def cluster_costs(clusters, obs_cam, obs_cost=OBS_COST) -> np.ndarray:
    """Per-cluster cost of one iteration: (9 n_k)^3 / 3 + obs_cost x (observations of cluster k)."""
    clusters = np.asarray(clusters)
    l = int(clusters.max()) + 1
    n_k = np.bincount(clusters, minlength=l).astype(np.float64)
    q_k = np.bincount(clusters[np.asarray(obs_cam)], minlength=l).astype(np.float64)
    return (9.0 * n_k) ** 3 / 3.0 + obs_cost * q_k


def assign_clusters(costs, world) -> np.ndarray:
    """Rank of every cluster: longest processing time first (ties: lower cluster id first, then lower rank),
    which keeps the largest load within 4/3 of the best possible."""
    costs = np.asarray(costs, dtype=np.float64)
    order = sorted(range(len(costs)), key=lambda k: (-costs[k], k))
    load = np.zeros(world)
    owner = np.empty(len(costs), dtype=np.int32)
    for k in order:
        r = int(np.argmin(load))
        owner[k] = r
        load[r] += costs[k]
    return owner


def plan_shards(clusters, obs_cam, obs_pt, n, world, obs_cost=OBS_COST) -> list[ShardPlan]:
    """The plan of every rank for one cluster assignment (cameras 0..m-1, points 0..n-1)."""
    clusters = np.asarray(clusters, dtype=np.int64)
    obs_cam = np.asarray(obs_cam, dtype=np.int64)
    obs_pt = np.asarray(obs_pt, dtype=np.int64)
    m = len(clusters)
    if world < 1:
        raise ValueError("world must be at least 1")
    if len(obs_cam) != len(obs_pt):
        raise ValueError("obs_cam and obs_pt differ in length")
    if m == 0 or clusters.min() < 0:
        raise ValueError("cluster ids must be 0..l-1")
    l = int(clusters.max()) + 1
    if np.any(np.bincount(clusters, minlength=l) == 0):
        raise ValueError("every cluster id 0..l-1 needs at least one camera")
    if len(obs_cam) and (obs_cam.min() < 0 or obs_cam.max() >= m or obs_pt.min() < 0 or obs_pt.max() >= n):
        raise ValueError("observation index out of range")
    costs = cluster_costs(clusters, obs_cam, obs_cost)
    owner = assign_clusters(costs, world)
    cam_rank = owner[clusters]
    obs_rank = cam_rank[obs_cam]
    # ranks that see each point: a (point, rank) incidence, deduplicated
    pr = np.unique(obs_pt * world + obs_rank)
    p_of, r_of = pr // world, pr % world
    nranks = np.bincount(p_of, minlength=n)
    boundary = np.flatnonzero(nranks >= 2)
    first_rank = np.full(n, world, dtype=np.int64)
    np.minimum.at(first_rank, p_of, r_of)
    slot = np.full(n, -1, dtype=np.int64)
    slot[boundary] = np.arange(len(boundary))
    plans = []
    for r in range(world):
        pts_r = p_of[r_of == r]
        plans.append(ShardPlan(rank=r, world=world, clusters=np.flatnonzero(owner == r),
                               cameras=np.flatnonzero(cam_rank == r), obs=np.flatnonzero(obs_rank == r),
                               points=pts_r, boundary=boundary, boundary_slot=slot[pts_r],
                               counts_point=first_rank[pts_r] == r, load=float(costs[owner == r].sum()),
                               m=m, n=n))
    return plans


def exchange_values(plans, corrected: bool, accepted: bool) -> dict:
    """Values exchanged in one iteration (payload, before the collectives' own traffic): 6 per boundary
    point for the correction when it is taken, 9 before and 3 after the cluster solves for the point
    update, 4 scalars, and the gathered update (9 m + 3 n) when the step is accepted."""
    p = plans[0]
    nb = len(p.boundary)
    return {"boundary_points": nb, "correction": 6 * nb if corrected else 0, "point_blocks": 9 * nb,
            "point_rhs": 3 * nb, "scalars": 4, "update": 9 * p.m + 3 * p.n if accepted else 0}
