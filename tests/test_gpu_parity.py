"""Parity of the CUDA LM iteration (through the C ABI) with the FP64 CPU oracle.

Every comparison is element-wise (tests/elementwise.py): each camera's 9 values, each point's 3 and each
9 x 9 camera block of a cluster system against the largest reference value of that row or block.
Tolerances: FP64 mode, step and parameters <= 1e-6 (the stated bar).  The cluster systems S'_k, b_k agree
to 1e-8: both sides round in FP64, and b' = v' - E' C'^-1 w' cancels by a factor up to 1/lambda (1e4) for
virtual points with one observation (the CUDA path evaluates that case in the cancellation-free Woodbury
form).  F(x + dx) agrees to 1e-8 relative: with steps equal to 1e-6, F moves by at most
|grad F(x + dx)| |d dx|.  Mixed mode: every element of the step within 1e-3 of its parameter kind's largest
reference value (elementwise.cols) and the final reprojection RMSE within 0.1 % of the oracle's."""
import numpy as np
import pytest

import scenes
from oracle import camera as ocam
from oracle import stba as ostba

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2008_00446_gb300 import stba  # noqa: E402
from elementwise import blocks, cols, rows  # noqa: E402


def oracle_first(s, clusters, lam=1e-4, correction=True):
    F0 = ocam.cost(s.cameras, s.points, s.obs_cam, s.obs_pt, s.obs_uv)
    opt = ostba.Options(lambda0=lam, correction=correction)
    return ostba.lm_iteration(s.cameras, s.points, s.obs_cam, s.obs_pt, s.obs_uv, clusters, lam, F0, opt, keep=True)


def make_ctx(s, clusters, device=False, **kw):
    if device:
        d = torch.device("cuda:0")
        args = [torch.tensor(a, device=d) for a in (s.cameras, s.points, s.obs_cam, s.obs_pt, s.obs_uv, clusters)]
    else:
        args = [s.cameras, s.points, s.obs_cam, s.obs_pt, s.obs_uv, clusters]
    return stba.stba_create(*args, **kw)


CASES = {
    "three_clusters": (dict(m=8, n=80, seed=5), [0, 0, 0, 1, 1, 1, 2, 2]),
    "one_cluster": (dict(m=7, n=60, seed=6), [0] * 7),
    "each_camera_own": (dict(m=6, n=50, seed=7), [0, 1, 2, 3, 4, 5]),
    "interleaved": (dict(m=9, n=90, seed=8), [2, 0, 1, 2, 0, 1, 2, 0, 1]),
    "ragged_many_tiles": (dict(m=37, n=400, seed=9, radius=12.0), list(np.arange(37) % 3)),
}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("lam", [1e-4, 0.5])
def test_first_iteration_fp64_matches_oracle(case, lam):
    kw, cl = CASES[case]
    s = scenes.make_tiny_scene(**kw)
    cl = np.asarray(cl, np.int32)
    c2, p2, lam2, F2, rec = oracle_first(s, cl, lam)
    ctx = make_ctx(s, cl, precision=stba.STBA_FP64, lambda0=lam)
    info = stba.stba_lm_iteration(ctx)
    st = rec["step"]
    assert info["corrected"] == rec["corrected"] == (lam >= 0.1)
    for k in range(int(cl.max()) + 1):
        S, b = stba.stba_get_cluster_system(ctx, k)
        assert blocks(S, st["S_blocks"][k]) < 1e-8, (k, blocks(S, st["S_blocks"][k]))
        assert rows(b, st["b_blocks"][k], 9) < 1e-8, (k, rows(b, st["b_blocks"][k], 9))
    dc, dp = stba.stba_last_step(ctx)
    assert rows(dc, rec["dc"], 9) < 1e-6, rows(dc, rec["dc"], 9)
    assert rows(dp, rec["dp"], 3) < 1e-6, rows(dp, rec["dp"], 3)
    assert abs(info["F_after"] - rec["F_after"]) <= 1e-8 * rec["F_after"]
    assert info["accepted"] == rec["accepted"]
    assert info["lambda"] == pytest.approx(rec["lam"], rel=1e-15)
    cams, pts = stba.stba_get_params(ctx)
    assert rows(cams, c2, 9) < 1e-9 and rows(pts, p2, 3) < 1e-9
    ctx.close()


def test_device_pointers_and_host_pointers_agree():
    kw, cl = CASES["three_clusters"]
    s = scenes.make_tiny_scene(**kw)
    cl = np.asarray(cl, np.int32)
    a = make_ctx(s, cl, device=False)
    b = make_ctx(s, cl, device=True)
    ia, ib = stba.stba_lm_iteration(a), stba.stba_lm_iteration(b)
    assert abs(ia["F_after"] - ib["F_after"]) <= 1e-12 * ia["F_after"]
    cams = torch.empty((s.m, 9), dtype=torch.float64, device="cuda:0")
    pts = torch.empty((s.n, 3), dtype=torch.float64, device="cuda:0")
    stba.stba_get_params(b, cams, pts)
    ca, pa = stba.stba_get_params(a)
    assert rows(cams.cpu().numpy(), ca, 9) < 1e-9 and rows(pts.cpu().numpy(), pa, 3) < 1e-9


def run_oracle(s, cl_seq, iters, **opt):
    return ostba.solve(s.cameras, s.points, s.obs_cam, s.obs_pt, s.obs_uv, cl_seq, iters, ostba.Options(**opt))


@pytest.fixture(scope="module")
def ring():
    return scenes.make_config("c0_ring")


@pytest.mark.parametrize("use_graph", [1, 0])
def test_ring_ten_iterations_fp64(ring, use_graph):
    """The 30-camera ring (3 clusters of 10), 10 LM iterations in FP64: identical accept / lambda sequence,
    per-iteration costs to 1e-10 and steps to 1e-6."""
    s = ring
    c, p, lam, F, hist = run_oracle(s, s.clusters, 10)
    ctx = make_ctx(s, s.clusters, precision=stba.STBA_FP64, use_graph=use_graph)
    errs = []
    for t, rec in enumerate(hist):
        info = stba.stba_lm_iteration(ctx)
        dc, dp = stba.stba_last_step(ctx)
        errs.append((t, rows(dc, rec["dc"], 9), rows(dp, rec["dp"], 3), abs(info["F_after"] / rec["F_after"] - 1)))
        assert info["accepted"] == rec["accepted"], errs
        assert info["lambda"] == pytest.approx(rec["lam"], rel=1e-14)
        assert abs(info["F_before"] - rec["F_before"]) <= 1e-8 * rec["F_before"], errs
        assert abs(info["F_after"] - rec["F_after"]) <= 1e-8 * rec["F_after"], errs
        assert errs[-1][1] < 1e-6 and errs[-1][2] < 1e-6, errs
    cams, pts = stba.stba_get_params(ctx)
    assert rows(cams, c, 9) < 1e-8 and rows(pts, p, 3) < 1e-8
    ctx.close()


def test_ring_cluster_sequence_with_set_clusters(ring):
    s = ring
    seq = scenes.cluster_sequence(s, 6, seed=1001)
    c, p, lam, F, hist = run_oracle(s, seq, 6)
    ctx = make_ctx(s, seq[0], precision=stba.STBA_FP64)
    for t, rec in enumerate(hist):
        stba.stba_set_clusters(ctx, seq[t])
        info = stba.stba_lm_iteration(ctx)
        assert info["accepted"] == rec["accepted"]
        assert abs(info["F_after"] - rec["F_after"]) <= 1e-8 * rec["F_after"], t
    cams, pts = stba.stba_get_params(ctx)
    assert rows(cams, c, 9) < 1e-8 and rows(pts, p, 3) < 1e-8


@pytest.mark.parametrize("precision", [stba.STBA_FP64, stba.STBA_MIXED])
def test_graph_structures_alternating_equal_the_oracle(ring, precision):
    """Clusterings whose factorisations have different numbers of tile steps, in turn (3 clusters of 10,
    one of 30, 2 of 15, and again): each new one is captured and either updates the executable graph kept
    for its launch structure or instantiates one.  Every iteration against the oracle run with the same
    sequence: FP64 every step 1e-6 per row, F(x + dx) 1e-8 and the accept decisions; mixed the first step
    within the mixed bar and the final RMSE within 0.1 %."""
    s = ring
    m = s.m
    shapes = [np.arange(m) // 10, np.zeros(m), np.arange(m) // 15]
    seq = np.array([shapes[t % 3] for t in range(7)], np.int32)
    c, p, lam, F, hist = run_oracle(s, seq, len(seq))
    ctx = make_ctx(s, seq[0], precision=precision)
    for t, rec in enumerate(hist):
        stba.stba_set_clusters(ctx, seq[t])
        info = stba.stba_lm_iteration(ctx)
        dc, dp = stba.stba_last_step(ctx)
        if precision == stba.STBA_FP64:
            assert info["accepted"] == rec["accepted"], t
            assert rows(dc, rec["dc"], 9) < 1e-6 and rows(dp, rec["dp"], 3) < 1e-6, t
            assert abs(info["F_after"] - rec["F_after"]) <= 1e-8 * rec["F_after"], t
        elif t == 0:
            assert cols(dc, rec["dc"], 9) < 1e-3 and cols(dp, rec["dp"], 3) < 1e-3
    if precision == stba.STBA_MIXED:
        _, Fg, _ = stba.stba_get_state(ctx)
        assert abs(ostba.rmse(Fg, s.q) - ostba.rmse(F, s.q)) <= 1e-3 * ostba.rmse(F, s.q)
    ctx.close()


def test_ring_sgc_draws_with_set_clusters(ring):
    """Per-iteration stochastic-graph-clustering draws (Gamma = 8, so several clusters of uneven size) applied
    with stba_set_clusters: the device re-ordering and the carried-over residuals give the oracle's
    iterations; the context's camera graph gives the same draws as a standalone graph."""
    s = ring
    g = stba.stba_graph_create(s.m, s.n, s.obs_cam, s.obs_pt)
    seq, ls = stba.stba_graph_cluster_batch(g, 6, gamma=8, beta=10.0, seed=77)
    assert ls.min() >= 4
    c, p, lam, F, hist = run_oracle(s, seq, 6)
    ctx = make_ctx(s, seq[0], precision=stba.STBA_FP64)
    seq2, _ = stba.stba_cluster_sgc(ctx, count=6, gamma=8, beta=10.0, seed=77)
    assert np.array_equal(seq, seq2)
    for t, rec in enumerate(hist):
        stba.stba_set_clusters(ctx, seq[t])
        info = stba.stba_lm_iteration(ctx)
        assert stba.stba_problem_info(ctx)["l"] == ls[t]
        assert info["accepted"] == rec["accepted"]
        assert abs(info["F_after"] - rec["F_after"]) <= 1e-8 * rec["F_after"], t
    cams, pts = stba.stba_get_params(ctx)
    assert rows(cams, c, 9) < 1e-8 and rows(pts, p, 3) < 1e-8


def test_ring_mixed_precision(ring):
    s = ring
    c, p, lam, F, hist = run_oracle(s, s.clusters, 10)
    ctx = make_ctx(s, s.clusters, precision=stba.STBA_MIXED)
    info = stba.stba_lm_iteration(ctx)
    dc, dp = stba.stba_last_step(ctx)
    assert cols(dc, hist[0]["dc"], 9) < 1e-3, cols(dc, hist[0]["dc"], 9)
    assert cols(dp, hist[0]["dp"], 3) < 1e-3, cols(dp, hist[0]["dp"], 3)
    for _ in range(9):
        stba.stba_lm_iteration(ctx)
    _, Fg, _ = stba.stba_get_state(ctx)
    rmse_o = ostba.rmse(F, s.q)
    rmse_g = ostba.rmse(Fg, s.q)
    assert abs(rmse_g - rmse_o) <= 1e-3 * rmse_o, (rmse_g, rmse_o)


def test_cost_and_state_roundtrip(ring):
    s = ring
    ctx = make_ctx(s, s.clusters)
    F = stba.stba_cost(ctx)
    assert F == pytest.approx(ocam.cost(s.cameras, s.points, s.obs_cam, s.obs_pt, s.obs_uv), rel=1e-12)
    stba.stba_lm_iteration(ctx)
    lam, F1, it = stba.stba_get_state(ctx)
    assert it == 1
    cams, pts = stba.stba_get_params(ctx)
    # resume into a fresh context from the checkpoint
    ctx2 = make_ctx(s, s.clusters)
    stba.stba_set_params(ctx2, cams, pts)
    stba.stba_set_state(ctx2, lam, -1.0, it)
    a, b = stba.stba_lm_iteration(ctx), stba.stba_lm_iteration(ctx2)
    assert a["F_after"] == pytest.approx(b["F_after"], rel=1e-12)
    assert a["iteration"] == b["iteration"] == 2


def test_solve_stops_on_function_tolerance(ring):
    s = ring
    ctx = make_ctx(s, s.clusters, ftol=0.5)
    info = stba.stba_solve(ctx, 20)
    assert info["stop"] and info["iteration"] < 20


def test_mixed_precision_cluster_systems_and_solve(ring):
    """Mixed mode, first iteration on the ring: the FP32-term / FP64-sum S'_k and b_k against the oracle,
    and the device solve against an FP64 solve of the device's own S'_k (isolates factorisation error)."""
    s = ring
    c, p, lam, F, hist = run_oracle(s, s.clusters, 1)
    st = ostba.lm_iteration(s.cameras, s.points, s.obs_cam, s.obs_pt, s.obs_uv, s.clusters, 1e-4,
                            ocam.cost(s.cameras, s.points, s.obs_cam, s.obs_pt, s.obs_uv), ostba.Options(),
                            keep=True)[4]["step"]
    ctx = make_ctx(s, s.clusters, precision=stba.STBA_MIXED)
    stba.stba_lm_iteration(ctx)
    dc, _ = stba.stba_last_step(ctx)
    errs = []
    for k in range(3):
        S, b = stba.stba_get_cluster_system(ctx, k)
        cams_k = np.flatnonzero(s.clusters == k)
        x_own = np.linalg.solve(S, b)
        x_dev = dc[cams_k].ravel()
        errs.append((k, blocks(S, st["S_blocks"][k]), rows(b, st["b_blocks"][k], 9), rows(x_dev, x_own, 9),
                     rows(x_own, np.linalg.solve(st["S_blocks"][k], st["b_blocks"][k]), 9)))
    print("mixed cluster systems (k, S err, b err, device-solve vs own-S FP64 solve, own-S solve vs oracle):", errs)
    for k, eS, eb, esolve, eown in errs:
        assert eS < 1e-5 and eb < 1e-5, errs
        assert esolve < 1e-4, errs
