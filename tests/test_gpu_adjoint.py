"""The CUDA adjoint (stba_record / stba_adjoint and the autograd function) against the oracle's FP64
reverse-mode derivative and against central differences of the CUDA forward map.

Loss: the sum of squared camera-centre errors to seeded targets (the differentiable configuration).  The
upstream gradient is computed once on the host and handed to both sides, so the comparison isolates the
adjoint.  Tolerances:
  - FP64 mode vs the oracle: 1e-6 of the largest gradient entry, element-wise (the FP64 bar for steps and
    parameters).  The oracle's second-derivative products are central differences with a relative step
    1e-6 (truncation ~1e-12, rounding ~1e-10 of the products); the rest of both sides rounds in FP64.
  - FP64 mode vs central differences of the CUDA forward map (step 1e-4): 1e-5 relative to
    |fd| + 1e-3 max|g|, as for the oracle's own pin.  The runs start at lambda0 = 0.03: at smaller damping
    the gauge directions of the camera-centre loss are nearly free and FP64 rounding of the forward map
    dominates a central difference.
  - Mixed mode vs the FP64 oracle: 1e-3 norm-wise, the bar of the mixed-mode forward step.  The adjoint's
    per-observation products (Jacobians and their dual-number derivatives) run in FP32 like the forward
    step's, its vectors and sums in FP64; it reuses the forward step's FP32 virtual-point, point and cluster
    factors (refined once in FP64); measured ~1.5e-5 on the sub-scene.
  - Full-size directional derivative (FP64): 1e-5 relative; measured ~3e-8 with an observation step 1e-3.
Runs that start at lambda0 >= 0.1 differentiate accepted steps taken with the steepest-descent correction
(Sec. 4.3) against the same bars."""
import numpy as np
import pytest

import scenes
from oracle import adjoint as oadj
from oracle import stba as ostba

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2008_00446_gb300 import stba  # noqa: E402

LAMBDA0 = 0.03


def targets_for(s, seed=11):
    rng = np.random.default_rng(seed)
    return oadj.camera_centres(s.cameras_true) + rng.normal(0, 0.1, (s.m, 3))


def run_gpu(s, seq, iters, precision=stba.STBA_FP64, lambda0=LAMBDA0, cams0=None, pts0=None, uv=None, **kw):
    seq = np.asarray(seq, np.int32)
    first = seq[0] if seq.ndim == 2 else seq
    ctx = stba.stba_create(s.cameras if cams0 is None else cams0, s.points if pts0 is None else pts0, s.obs_cam,
                           s.obs_pt, s.obs_uv if uv is None else uv, first, precision=precision, lambda0=lambda0, **kw)
    stba.stba_record(ctx, iters)
    infos = []
    for t in range(iters):
        if seq.ndim == 2 and t > 0:
            stba.stba_set_clusters(ctx, seq[t])
        infos.append(stba.stba_lm_iteration(ctx))
    cams, pts = stba.stba_get_params(ctx)
    return ctx, cams, pts, infos


def max_rel(g, ref):
    return float(np.max(np.abs(np.asarray(g) - ref)) / max(np.max(np.abs(ref)), 1e-300))


def tiny(seed=5, m=8, n=80):
    return scenes.make_tiny_scene(m=m, n=n, seed=seed, clusters=np.array([0, 0, 0, 1, 1, 1, 2, 2][:m], np.int32))


def c3_sub(n_cams=10, n_pts=200):
    """The 10-camera / 200-point sub-scene of the 500-camera differentiable configuration: the cameras
    closest to camera 0 (so that they share points), split into two clusters."""
    full = scenes.make_config("c3_diff")
    cen = oadj.camera_centres(full.cameras_true)
    keep = np.argsort(np.linalg.norm(cen - cen[0], axis=1))[:n_cams]
    s = scenes.subscene(full, keep, max_points=n_pts, seed=3)
    s.clusters = (np.arange(s.m) >= s.m // 2).astype(np.int32)
    return s


def random_sequence(m, iters, l, seed):
    rng = np.random.default_rng(seed)
    seq = []
    for _ in range(iters):
        base = np.arange(m) % l
        seq.append(rng.permutation(base))
    return np.asarray(seq, np.int32)


@pytest.mark.parametrize("kind", ["static", "resampled"])
@pytest.mark.parametrize("lambda0", [LAMBDA0, 0.5, 0.2])
def test_adjoint_fp64_matches_oracle(kind, lambda0):
    # lambda0 >= 0.1: accepted steps with the steepest-descent correction (Sec. 4.3); 0.2 mixes corrected and
    # uncorrected steps in one chain
    s = tiny()
    iters = 4
    seq = s.clusters if kind == "static" else random_sequence(s.m, iters, 3, seed=2)
    tg = targets_for(s)
    co, po, tape = oadj.forward(s.cameras, s.points, s.obs_cam, s.obs_pt, s.obs_uv, seq, iters,
                                ostba.Options(lambda0=lambda0))
    ctx, cams, pts, infos = run_gpu(s, seq, iters, lambda0=lambda0)
    assert [i["accepted"] for i in infos] == [t["accepted"] for t in tape]
    assert [i["corrected"] for i in infos] == [t["corrected"] for t in tape]
    if lambda0 >= 0.1:
        assert infos[0]["corrected"] and infos[0]["accepted"]
    assert np.max(np.abs(cams - co)) < 1e-8 * np.max(np.abs(co))
    a_c = oadj.centre_loss_grad(co, tg)
    a_p = np.random.default_rng(4).normal(0, 1e-3, po.shape)   # exercises the point upstream too
    gc_o, gp_o, gq_o = oadj.backward(tape, s.obs_cam, s.obs_pt, s.obs_uv, a_c, a_p)
    gq, gc, gp = stba.stba_adjoint(ctx, a_c, a_p)
    assert max_rel(gc, gc_o) < 1e-6, max_rel(gc, gc_o)
    assert max_rel(gp, gp_o) < 1e-6, max_rel(gp, gp_o)
    assert max_rel(gq, gq_o) < 1e-6, max_rel(gq, gq_o)
    ctx.close()


def test_adjoint_restores_state_and_repeats():
    s = tiny(seed=6)
    ctx, cams, pts, infos = run_gpu(s, s.clusters, 3)
    lam, F, it = stba.stba_get_state(ctx)
    a_c = oadj.centre_loss_grad(cams, targets_for(s))
    g1 = stba.stba_adjoint(ctx, a_c)
    c2, p2 = stba.stba_get_params(ctx)
    assert np.array_equal(c2, cams) and np.array_equal(p2, pts)
    assert stba.stba_get_state(ctx) == (lam, F, it)
    g2 = stba.stba_adjoint(ctx, a_c)
    for x, y in zip(g1, g2):
        assert max_rel(x, y) < 1e-12
    # the next iteration is the one a context without the adjoint takes
    twin, _, _, _ = run_gpu(s, s.clusters, 3)
    stba.stba_record(ctx, 0)
    stba.stba_record(twin, 0)
    i1 = stba.stba_lm_iteration(ctx)
    i2 = stba.stba_lm_iteration(twin)
    assert i1["F_after"] == pytest.approx(i2["F_after"], rel=1e-12)
    ctx.close()
    twin.close()


@pytest.mark.parametrize("lambda0", [LAMBDA0, 0.5])
def test_adjoint_vs_central_differences_c3_subscene(lambda0):
    s = c3_sub()
    iters = 5
    tg = targets_for(s)
    ctx, cams, pts, infos = run_gpu(s, s.clusters, iters, lambda0=lambda0)
    flags = [i["accepted"] for i in infos]
    assert any(i["corrected"] and i["accepted"] for i in infos) == (lambda0 >= 0.1)
    gq, gc, gp = stba.stba_adjoint(ctx, oadj.centre_loss_grad(cams, tg))
    ctx.close()
    h = 1e-4

    def L(**kw):
        c, cc, _, inf = run_gpu(s, s.clusters, iters, lambda0=lambda0, **kw)
        c.close()
        assert [i["accepted"] for i in inf] == flags
        return oadj.centre_loss(cc, tg)

    rng = np.random.default_rng(1)
    errs = []
    for o, k in zip(rng.integers(0, s.q, 5), rng.integers(0, 2, 5)):
        up, um = s.obs_uv.copy(), s.obs_uv.copy()
        up[o, k] += h
        um[o, k] -= h
        fd = (L(uv=up) - L(uv=um)) / (2 * h)
        errs.append(abs(fd - gq[o, k]) / (abs(fd) + 1e-3 * np.max(np.abs(gq))))
    for j, k in zip(rng.integers(0, s.m, 5), [0, 3, 5, 6, 8]):
        hk = h * max(1.0, abs(s.cameras[j, k]))
        cp, cm = s.cameras.copy(), s.cameras.copy()
        cp[j, k] += hk
        cm[j, k] -= hk
        fd = (L(cams0=cp) - L(cams0=cm)) / (2 * hk)
        errs.append(abs(fd - gc[j, k]) / (abs(fd) + 1e-3 * np.max(np.abs(gc))))
    assert max(errs) < 1e-5, errs


@pytest.mark.parametrize("lambda0", [LAMBDA0, 0.5])
def test_adjoint_mixed_precision_vs_fp64_oracle(lambda0):
    s = c3_sub()
    iters = 5
    tg = targets_for(s)
    co, po, tape = oadj.forward(s.cameras, s.points, s.obs_cam, s.obs_pt, s.obs_uv, s.clusters, iters,
                                ostba.Options(lambda0=lambda0))
    ctx, cams, pts, infos = run_gpu(s, s.clusters, iters, precision=stba.STBA_MIXED, lambda0=lambda0)
    assert [i["accepted"] for i in infos] == [t["accepted"] for t in tape]
    a_c = oadj.centre_loss_grad(co, tg)
    gc_o, gp_o, gq_o = oadj.backward(tape, s.obs_cam, s.obs_pt, s.obs_uv, a_c, np.zeros_like(po))
    gq, gc, gp = stba.stba_adjoint(ctx, a_c)
    nrel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))   # noqa: E731
    errs = (nrel(gc, gc_o), nrel(gp, gp_o), nrel(gq, gq_o))
    print("mixed-precision adjoint, norm-wise relative errors (cams0, pts0, obs):", errs)
    assert max(errs) < 1e-3, errs
    ctx.close()


def centres_torch(c):
    """-R(w)^T t per camera, R^T t = t - a (w x t) + b (w (w.t) - s t), in torch (differentiable)."""
    w, t = c[:, 0:3], c[:, 3:6]
    s = (w * w).sum(1, keepdim=True)
    th = torch.sqrt(s)
    a = torch.sin(th) / th
    b = (1 - torch.cos(th)) / s
    wt = (w * t).sum(1, keepdim=True)
    return -(t - a * torch.linalg.cross(w, t, dim=1) + b * (w * wt - s * t))


def test_autograd_function_matches_oracle():
    s = tiny(seed=8)
    iters = 3
    tg = targets_for(s)
    dev = torch.device("cuda:0")
    c0 = torch.tensor(s.cameras, device=dev, requires_grad=True)
    p0 = torch.tensor(s.points, device=dev, requires_grad=True)
    uv = torch.tensor(s.obs_uv, device=dev, requires_grad=True)
    cams, pts = stba.stba_differentiable(c0, p0, uv, torch.tensor(s.obs_cam, device=dev),
                                         torch.tensor(s.obs_pt, device=dev), s.clusters, iters,
                                         stba.stba_default_options(lambda0=LAMBDA0))
    cen = centres_torch(cams)
    assert np.allclose(cen.detach().cpu().numpy(), oadj.camera_centres(cams.detach().cpu().numpy()), atol=1e-12)
    loss = ((cen - torch.tensor(tg, device=dev)) ** 2).sum()
    loss.backward()
    co, po, tape = oadj.forward(s.cameras, s.points, s.obs_cam, s.obs_pt, s.obs_uv, s.clusters, iters,
                                ostba.Options(lambda0=LAMBDA0))
    gc_o, gp_o, gq_o = oadj.backward(tape, s.obs_cam, s.obs_pt, s.obs_uv, oadj.centre_loss_grad(co, tg),
                                     np.zeros_like(po))
    assert max_rel(c0.grad.cpu().numpy(), gc_o) < 1e-6
    assert max_rel(p0.grad.cpu().numpy(), gp_o) < 1e-6
    assert max_rel(uv.grad.cpu().numpy(), gq_o) < 1e-6


def test_adjoint_state_errors():
    s = tiny(seed=9)
    ctx = stba.stba_create(s.cameras, s.points, s.obs_cam, s.obs_pt, s.obs_uv, s.clusters, lambda0=LAMBDA0)
    a_c = np.zeros((s.m, 9))
    with pytest.raises(stba.StbaError) as e:
        stba.stba_adjoint(ctx, a_c)            # nothing recorded
    assert e.value.status == 7
    stba.stba_record(ctx, 1)
    stba.stba_lm_iteration(ctx)
    with pytest.raises(stba.StbaError) as e:
        stba.stba_lm_iteration(ctx)            # beyond the tape
    assert e.value.status == 7
    stba.stba_record(ctx, 2)
    stba.stba_lm_iteration(ctx)
    stba.stba_set_params(ctx, s.cameras, s.points)
    with pytest.raises(stba.StbaError) as e:
        stba.stba_adjoint(ctx, a_c)            # chain broken by replaced parameters
    assert e.value.status == 7
    ctx.close()
    # the FP64 factor option of mixed precision has no adjoint
    ctx = stba.stba_create(s.cameras, s.points, s.obs_cam, s.obs_pt, s.obs_uv, s.clusters, lambda0=LAMBDA0,
                           precision=stba.STBA_MIXED, factor_fp64=1)
    stba.stba_record(ctx, 1)
    stba.stba_lm_iteration(ctx)
    with pytest.raises(stba.StbaError) as e:
        stba.stba_adjoint(ctx, a_c)
    assert e.value.status == 7
    ctx.close()
    # an accepted step with the steepest-descent correction (lambda >= 0.1) is differentiated, not refused
    ctx = stba.stba_create(s.cameras, s.points, s.obs_cam, s.obs_pt, s.obs_uv, s.clusters, lambda0=0.5)
    stba.stba_record(ctx, 1)
    info = stba.stba_lm_iteration(ctx)
    assert info["corrected"]
    gq, gc, gp = stba.stba_adjoint(ctx, np.ones((s.m, 9)))
    assert np.isfinite(gq).all() and np.isfinite(gc).all() and np.isfinite(gp).all()
    ctx.close()


@pytest.mark.parametrize("lambda0", [LAMBDA0, 0.5])
def test_adjoint_directional_derivative_full_c3(lambda0):
    """Full 500-camera configuration (about 280k observations), FP64 forward and adjoint: the derivative
    along a random observation perturbation equals the central difference of the CUDA forward map; at
    lambda0 = 0.5 the accepted steps use the steepest-descent correction."""
    s = scenes.make_config("c3_diff")
    iters = 5
    tg = targets_for(s)
    ctx, cams, pts, infos = run_gpu(s, s.clusters, iters, lambda0=lambda0)
    flags = [i["accepted"] for i in infos]
    assert any(i["corrected"] and i["accepted"] for i in infos) == (lambda0 >= 0.1)
    gq, gc, gp = stba.stba_adjoint(ctx, oadj.centre_loss_grad(cams, tg))
    ctx.close()
    d = np.random.default_rng(5).normal(0, 1, s.obs_uv.shape)
    h = 1e-3
    vals = []
    for sgn in (1, -1):
        c, cc, _, inf = run_gpu(s, s.clusters, iters, lambda0=lambda0, uv=s.obs_uv + sgn * h * d)
        c.close()
        assert [i["accepted"] for i in inf] == flags
        vals.append(oadj.centre_loss(cc, tg))
    fd = (vals[0] - vals[1]) / (2 * h)
    ad = float(np.sum(gq * d))
    print("full-size directional derivative: adjoint", ad, "central difference", fd)
    assert abs(ad - fd) <= 1e-5 * abs(fd), (ad, fd)
