"""The cluster-sharded iteration (one rank per GPU, each owning whole clusters) checked on CPU ranks.

The plan of `paper_2008_00446_gb300.shard` is checked for what it promises (a partition of clusters,
cameras and observations; the boundary points; load balance).  Then 2 and 3 `gloo` ranks run LM iterations
of Algorithm 1 each over its own clusters only, with the oracle's building blocks for the local arithmetic
and the plan's exchanges as all-reduces over the boundary points and four scalars, and the result must
equal the single-process oracle: every rank's Delta c and Delta p, F(x + Delta x), the accept decisions and
lambda, over iterations with and without the steepest-descent correction (Sec. 4.3), and with the Huber
loss on a scene with gross outliers (the robust weights are per observation, so local).  The bars are those of
the FP64 parity tests (steps 1e-6 in norm, F 1e-8): the summation order differs between the ranks and the
single process, and the nearly gauge-free systems at small lambda amplify that rounding.  This checks the
exchange plan of the sharded design; no GPU is involved."""
import os
import socket

import numpy as np
import pytest

import scenes
from oracle import sgc
from oracle import stba as ostba
from paper_2008_00446_gb300 import shard


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def ring_scene(huber):
    """The ring scene; with a robust loss, 2 % of its observations moved by gross errors (seeded)."""
    s = scenes.make_config("c0_ring")
    if huber > 0:
        rng = np.random.default_rng(21)
        uv = s.obs_uv.copy()
        bad = rng.choice(len(uv), size=len(uv) // 50, replace=False)
        uv[bad] += rng.normal(0.0, 30.0, size=(len(bad), 2))
        s.obs_uv = uv
    return s


def ring_with_sgc(gamma, seed, iters):
    s = ring_scene(0.0)
    w = sgc.camera_graph(s.obs_cam, s.obs_pt, s.m)
    rng = np.random.default_rng(seed)
    seq = np.array([sgc.sample(w, s.m, gamma, 10.0, rng.random(s.m)) for _ in range(iters)], np.int32)
    return s, seq


# ------------------------------------------------------------------------------------------------------
# the plan
# ------------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("world", [1, 2, 3, 5, 40])
def test_plan_partitions_the_problem(world):
    s, seq = ring_with_sgc(6, 3, 1)
    cl = seq[0]
    plans = shard.plan_shards(cl, s.obs_cam, s.obs_pt, s.n, world)
    assert len(plans) == world
    l = cl.max() + 1
    assert np.array_equal(np.sort(np.concatenate([p.clusters for p in plans])), np.arange(l))
    assert np.array_equal(np.sort(np.concatenate([p.cameras for p in plans])), np.arange(s.m))
    assert np.array_equal(np.sort(np.concatenate([p.obs for p in plans])), np.arange(len(s.obs_cam)))
    ranks_of_point = [set() for _ in range(s.n)]
    for p in plans:
        assert np.array_equal(p.cameras, np.flatnonzero(np.isin(cl, p.clusters)))
        assert np.array_equal(p.obs, np.flatnonzero(np.isin(s.obs_cam, p.cameras)))
        assert np.array_equal(p.points, np.unique(s.obs_pt[p.obs]))
        for i in p.points:
            ranks_of_point[i].add(p.rank)
    boundary = np.array([i for i in range(s.n) if len(ranks_of_point[i]) >= 2], dtype=np.int64)
    total = 0
    for p in plans:
        assert np.array_equal(p.boundary, boundary)
        assert np.array_equal(p.boundary_slot >= 0, np.isin(p.points, boundary))
        assert np.array_equal(p.boundary[p.boundary_slot[p.boundary_slot >= 0]], p.points[p.boundary_slot >= 0])
        assert np.array_equal(p.counts_point, [min(ranks_of_point[i]) == p.rank for i in p.points])
        total += p.counts_point.sum()
    assert total == s.n   # every point counted once in the norms
    costs = shard.cluster_costs(cl, s.obs_cam)
    loads = [p.load for p in plans]
    assert sum(loads) == pytest.approx(costs.sum(), rel=1e-12)
    assert max(loads) <= costs.sum() / world + costs.max() + 1e-6   # list-scheduling bound
    if world == 1:
        assert len(boundary) == 0


def test_lpt_assignment_by_hand():
    # costs 7, 5, 4, 3, 3 on two ranks: 7 -> r0, 5 -> r1, 4 -> r1 (9), 3 -> r0 (10), 3 -> r1 (12)
    owner = shard.assign_clusters([5.0, 3.0, 7.0, 4.0, 3.0], 2)
    assert list(owner) == [1, 0, 0, 1, 1]


def test_exchange_values():
    # cameras 0,1 | 2 in two clusters; point 0 seen by both ranks, point 1 by rank 0 only
    plans = shard.plan_shards(np.array([0, 0, 1]), [0, 1, 2, 0, 1], [0, 0, 0, 1, 1], 2, 2)
    assert list(plans[0].boundary) == [0]
    ex = shard.exchange_values(plans, corrected=True, accepted=True)
    assert ex == {"boundary_points": 1, "correction": 6, "point_blocks": 9, "point_rhs": 3, "scalars": 4,
                  "update": 9 * 3 + 3 * 2}
    ex = shard.exchange_values(plans, corrected=False, accepted=False)
    assert ex["correction"] == 0 and ex["update"] == 0


def test_plan_rejects_bad_input():
    with pytest.raises(ValueError):
        shard.plan_shards(np.array([0, 2]), [0, 1], [0, 0], 1, 2)        # cluster 1 empty
    with pytest.raises(ValueError):
        shard.plan_shards(np.array([0, 1]), [0, 2], [0, 0], 1, 2)        # camera out of range
    with pytest.raises(ValueError):
        shard.plan_shards(np.array([0, 1]), [0, 1], [0, 0], 1, 0)        # no ranks


# ------------------------------------------------------------------------------------------------------
# the sharded iteration on gloo ranks
# ------------------------------------------------------------------------------------------------------
def _sum(torch, dist, a):
    t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64))
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t.numpy()


def _max(torch, dist, x):
    t = torch.tensor([float(x)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sharded_iteration(torch, dist, plan, s, cl, cams, pts, lam, F, opt):
    """One iteration of Algorithm 1 on this rank's clusters; returns the new state and the step."""
    m, n = len(cams), len(pts)
    o = plan.obs
    oc, op, uv = s.obs_cam[o], s.obs_pt[o], s.obs_uv[o]
    lin = ostba.linearise(cams, pts, oc, op, uv, opt.huber)   # the rows of this rank's observations
    vp_of_obs, vp_point, _ = ostba.virtual_points(op, oc, cl)   # all of them belong to owned clusters
    nv = len(vp_point)
    J_pv = ostba.point_jacobian(lin.Jp, vp_of_obs, nv)
    B = ostba.damped(lin.J_c.T @ lin.J_c, lam)
    Cv = ostba.damped(J_pv.T @ J_pv, lam)
    Ev = (lin.J_c.T @ J_pv).tocsr()
    v1 = -(lin.J_c.T @ lin.f)
    w1 = -(J_pv.T @ lin.f)
    bslot = np.full(n, -1, np.int64)
    bslot[plan.points] = plan.boundary_slot
    nb = len(plan.boundary)
    if opt.correction and lam >= opt.correction_lambda:
        # exchange 1: per point and coordinate, the sums over all its virtual copies of w' and diag(H_lambda)
        h = (1.0 + lam) * np.asarray(J_pv.multiply(J_pv).sum(axis=0)).ravel().reshape(nv, 3)
        g3 = w1.reshape(nv, 3)
        sg, sh = np.zeros((n, 3)), np.zeros((n, 3))
        np.add.at(sg, vp_point, g3)
        np.add.at(sh, vp_point, h)
        ex = np.zeros((nb, 6))
        loc = plan.points[plan.boundary_slot >= 0]
        ex[bslot[loc], :3] = sg[loc]
        ex[bslot[loc], 3:] = sh[loc]
        ex = _sum(torch, dist, ex)
        sg[loc], sh[loc] = ex[bslot[loc], :3], ex[bslot[loc], 3:]
        w1 = (h * (sg / np.where(sh > 0, sh, 1.0))[vp_point]).ravel()
    Cv_inv = ostba.block_diag_inverse(Cv)
    Sp = (B - Ev @ Cv_inv @ Ev.T).tocsr()
    bp = v1 - Ev @ (Cv_inv @ w1)
    dc = np.zeros(9 * m)
    ok = 1.0
    for k in plan.clusters:
        _, idx = ostba.cluster_camera_indices(cl, k)
        xk = ostba.cholesky_solve(Sp[idx][:, idx].toarray(), bp[idx])
        if xk is None:
            ok = 0.0
        else:
            dc[idx] = xk
    ok = -_max(torch, dist, -ok)   # every rank's clusters factorised
    # exchange 2: physical damped C_i and w_i over the ranks that see the point, then the W^T Delta c sums
    _, C, E, v, w = ostba.physical_blocks(lin, lam)
    Cc = C.tocoo()
    Cb = np.zeros((n, 3, 3))
    np.add.at(Cb, (Cc.row // 3, Cc.row % 3, Cc.col % 3), Cc.data)   # C is block diagonal
    loc = plan.points[plan.boundary_slot >= 0]
    ex = np.zeros((nb, 12))
    ex[bslot[loc], :9] = Cb[loc].reshape(-1, 9)
    ex[bslot[loc], 9:] = w.reshape(n, 3)[loc]
    ex = _sum(torch, dist, ex)
    Cb[loc] = ex[bslot[loc], :9].reshape(-1, 3, 3)
    w = w.reshape(n, 3).copy()
    w[loc] = ex[bslot[loc], 9:]
    e = (E.T @ dc).reshape(n, 3)
    ex = np.zeros((nb, 3))
    ex[bslot[loc]] = e[loc]
    ex = _sum(torch, dist, ex)
    e[loc] = ex[bslot[loc]]
    dp = np.zeros((n, 3))
    for i in plan.points:
        dp[i] = np.linalg.solve(Cb[i], w[i] - e[i])
    # exchange 3: the cost of the candidate and the quantities of the stop tests; this rank's observations
    # touch only its own cameras and points, whose new values it has
    dc = dc.reshape(m, 9)
    F_part = ostba.robust_cost(cams + dc, pts + dp, oc, op, uv, opt.huber) if ok else 0.0
    pc = plan.points[plan.counts_point]
    F_new = _sum(torch, dist, np.array([F_part]))[0] if ok else np.inf
    grad_inf = _max(torch, dist, max(np.max(np.abs(v), initial=0.0), np.max(np.abs(w[plan.points]), initial=0.0)))
    sq = _sum(torch, dist, np.array([np.sum(dc[plan.cameras] ** 2) + np.sum(dp[pc] ** 2),
                                      np.sum(cams[plan.cameras] ** 2) + np.sum(pts[pc] ** 2)]))
    stop = ostba.stop_tests(F, F_new, grad_inf, float(np.sqrt(sq[0])), float(np.sqrt(sq[1])), opt)
    accepted = bool(np.isfinite(F_new) and F_new < F)
    rec = dict(dc=dc[plan.cameras], dp=dp[plan.points], F_after=F_new, accepted=accepted, stop=stop)
    if accepted:
        # exchange 4: the gathered update (each camera from its owner, each point from one rank that sees it)
        mask = np.zeros(n, bool)
        mask[pc] = True
        upd = _sum(torch, dist, np.concatenate([dc.ravel(), np.where(mask[:, None], dp, 0.0).ravel()]))
        cams = cams + upd[: 9 * m].reshape(m, 9)
        pts = pts + upd[9 * m:].reshape(n, 3)
        F, lam_new = F_new, max(lam / 3.0, opt.lambda_min)
    else:
        lam_new = lam * 3.0
    rec["lam"] = lam_new
    return cams, pts, lam_new, F, rec


def _worker(rank, world, port, seq, lambda0, huber, out_dir):
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        s = ring_scene(huber)
        opt = ostba.Options(lambda0=lambda0, ftol=1e-6, gtol=1e-6, xtol=1e-6, huber=huber)
        cams, pts, lam = s.cameras.copy(), s.points.copy(), lambda0
        F = ostba.robust_cost(cams, pts, s.obs_cam, s.obs_pt, s.obs_uv, opt.huber)
        recs = {}
        for t, cl in enumerate(seq):
            plan = shard.plan_shards(cl, s.obs_cam, s.obs_pt, s.n, world)[rank]
            cams, pts, lam, F, rec = sharded_iteration(torch, dist, plan, s, cl, cams, pts, lam, F, opt)
            recs[f"cams{t}"] = plan.cameras
            recs[f"points{t}"] = plan.points
            for key in ("dc", "dp"):
                recs[f"{key}{t}"] = rec[key]
            recs[f"scal{t}"] = np.array([rec["F_after"], float(rec["accepted"]), rec["lam"], float(rec["stop"])])
        recs["cams_end"], recs["pts_end"] = cams, pts
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), **recs)
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as so:
        so.bind(("127.0.0.1", 0))
        return so.getsockname()[1]


@pytest.mark.parametrize("world, gamma, lambda0, huber", [(2, 10, 1e-4, 0.0), (2, 6, 0.5, 0.0), (3, 5, 0.5, 0.0),
                                                           (2, 6, 1e-4, 0.5)])
def test_sharded_iterations_equal_the_oracle(tmp_path, world, gamma, lambda0, huber):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as tmp_mp
    s, seq = ring_with_sgc(gamma, 11 + world, 4)
    port = _free_port()
    tmp_mp.start_processes(_worker, args=(world, port, seq, lambda0, huber, str(tmp_path)), nprocs=world,
                           start_method="spawn", join=True)
    s = ring_scene(huber)
    opt = ostba.Options(lambda0=lambda0, ftol=1e-6, gtol=1e-6, xtol=1e-6, huber=huber)
    cams, pts, lam = s.cameras.copy(), s.points.copy(), lambda0
    F = ostba.robust_cost(cams, pts, s.obs_cam, s.obs_pt, s.obs_uv, opt.huber)
    res = [np.load(tmp_path / f"rank{r}.npz") for r in range(world)]
    corrected = 0
    for t, cl in enumerate(seq):
        cams, pts, lam, F, rec = ostba.lm_iteration(cams, pts, s.obs_cam, s.obs_pt, s.obs_uv, cl, lam, F, opt)
        corrected += rec["corrected"]
        for r in range(world):
            z = res[r]
            dc = rec["dc"][z[f"cams{t}"]]
            dp = rec["dp"][z[f"points{t}"]]
            assert rel(z[f"dc{t}"], dc) < 1e-6 and rel(z[f"dp{t}"], dp) < 1e-6
            F_after, acc, lam_r, stop = z[f"scal{t}"]
            assert F_after == pytest.approx(rec["F_after"], rel=1e-8)
            assert bool(acc) == rec["accepted"] and lam_r == lam and bool(stop) == rec["stop"]
        assert sum(len(res[r][f"cams{t}"]) for r in range(world)) == s.m
    for r in range(world):   # every rank holds the whole, identical state
        assert rel(res[r]["cams_end"], cams) < 1e-8 and rel(res[r]["pts_end"], pts) < 1e-8
    if lambda0 >= 0.1:
        assert corrected >= 1   # the exchange of the correction was exercised
