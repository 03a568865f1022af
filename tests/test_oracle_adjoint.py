"""Pins of the oracle's reverse-mode derivative of K STBA iterations against central finite differences of
the whole forward map (accept flags and clusters frozen; the test checks they do not flip under +-h).

The loss is the sum of squared camera-centre errors, which moves along the similarity-gauge directions;
at lambda ~ 1e-5 those are nearly free, the forward map's FP64 rounding noise there dominates a central
difference, and the comparison would test the noise.  The chained runs therefore start at lambda0 = 0.03
(below the correction threshold 0.1); at that damping the differences agree to ~1e-8.  Runs that start at
lambda0 = 0.5 or 0.2 take steps with the steepest-descent correction of Sec. 4.3 and pin its adjoint."""
import numpy as np
import pytest

import scenes
from oracle import adjoint, camera, stba


def setup(seed=3, m=6, n=40, clusters=(0, 0, 0, 1, 1, 1)):
    s = scenes.make_tiny_scene(m=m, n=n, seed=seed, clusters=np.asarray(clusters, np.int32))
    rng = np.random.default_rng(seed + 100)
    targets = adjoint.camera_centres(s.cameras_true) + rng.normal(0, 0.1, (s.m, 3))
    return s, targets


CHAIN_OPT = stba.Options(lambda0=0.03)


def run(s, cams0, pts0, uv, iters, opt=CHAIN_OPT):
    c, p, tape = adjoint.forward(cams0, pts0, s.obs_cam, s.obs_pt, uv, s.clusters, iters, opt)
    return c, p, tape


@pytest.mark.parametrize("iters,lambda0", [(1, 0.03), (3, 0.03), (1, 0.5), (3, 0.5), (3, 0.2)])
def test_adjoint_matches_central_differences(iters, lambda0):
    # lambda0 >= 0.1: the steps use the steepest-descent correction (Sec. 4.3); 0.2 corrects the first step
    # and, once an accepted step divides lambda by 3, not the later ones
    s, targets = setup()
    opt = stba.Options(lambda0=lambda0)
    c, p, tape = run(s, s.cameras, s.points, s.obs_uv, iters, opt)
    flags = [t["accepted"] for t in tape]
    if lambda0 >= 0.1:
        assert tape[0]["corrected"] and tape[0]["accepted"]
    if lambda0 == 0.2 and iters == 3:
        assert not all(t["corrected"] for t in tape)
    a_c = adjoint.centre_loss_grad(c, targets)
    gc, gp, gq = adjoint.backward(tape, s.obs_cam, s.obs_pt, s.obs_uv, a_c, np.zeros_like(p))
    rng = np.random.default_rng(0)
    h = 1e-4

    def L(cams0=None, pts0=None, uv=None):
        cc, _, tp = run(s, s.cameras if cams0 is None else cams0, s.points if pts0 is None else pts0,
                        s.obs_uv if uv is None else uv, iters, opt)
        assert [t["accepted"] for t in tp] == flags
        return adjoint.centre_loss(cc, targets)

    errs = []
    for o, k in zip(rng.integers(0, s.q, 6), rng.integers(0, 2, 6)):
        up, um = s.obs_uv.copy(), s.obs_uv.copy()
        up[o, k] += h
        um[o, k] -= h
        fd = (L(uv=up) - L(uv=um)) / (2 * h)
        errs.append(abs(fd - gq[o, k]) / (abs(fd) + 1e-3 * np.max(np.abs(gq))))
    for j, k in zip(rng.integers(0, s.m, 6), [0, 2, 4, 6, 7, 8]):
        hk = h * max(1.0, abs(s.cameras[j, k]))
        cp, cm = s.cameras.copy(), s.cameras.copy()
        cp[j, k] += hk
        cm[j, k] -= hk
        fd = (L(cams0=cp) - L(cams0=cm)) / (2 * hk)
        errs.append(abs(fd - gc[j, k]) / (abs(fd) + 1e-3 * np.max(np.abs(gc))))
    for i, k in zip(rng.integers(0, s.n, 4), [0, 1, 2, 1]):
        pp, pm = s.points.copy(), s.points.copy()
        pp[i, k] += h
        pm[i, k] -= h
        fd = (L(pts0=pp) - L(pts0=pm)) / (2 * h)
        errs.append(abs(fd - gp[i, k]) / (abs(fd) + 1e-3 * np.max(np.abs(gp))))
    assert max(errs) < 1e-5, errs


def test_rejected_step_passes_adjoint_through():
    s, targets = setup(seed=9)
    # a huge first step is rejected: start far away with a tiny damping
    opt = stba.Options(lambda0=1e-12)
    cams0 = s.cameras.copy()
    cams0[:, 3:6] += 0.5
    c, p, tape = run(s, cams0, s.points, s.obs_uv, 3, opt)
    a_c = adjoint.centre_loss_grad(c, targets)
    gc, gp, gq = adjoint.backward(tape, s.obs_cam, s.obs_pt, s.obs_uv, a_c, np.zeros_like(p))
    if all(t["accepted"] for t in tape):
        pytest.skip("no rejection occurred in this configuration")
    flags = [t["accepted"] for t in tape]
    h = 1e-4
    j, k = 1, 6
    cp, cm = cams0.copy(), cams0.copy()
    cp[j, k] += h * abs(cams0[j, k])
    cm[j, k] -= h * abs(cams0[j, k])
    outs = []
    for cc0 in (cp, cm):
        cc, _, tp = run(s, cc0, s.points, s.obs_uv, 3, opt)
        assert [t["accepted"] for t in tp] == flags
        outs.append(adjoint.centre_loss(cc, targets))
    fd = (outs[0] - outs[1]) / (2 * h * abs(cams0[j, k]))
    assert abs(fd - gc[j, k]) <= 2e-4 * (abs(fd) + 1e-3 * np.max(np.abs(gc)))


def test_centre_loss_gradient_closed_form():
    # translation part: centre = -R^T t, so d L / d t = -2 R (centre - target)
    s, targets = setup()
    g = adjoint.centre_loss_grad(s.cameras, targets)
    cen = adjoint.camera_centres(s.cameras)
    for j in range(s.m):
        R = camera.rotation_matrix(s.cameras[j, 0:3])
        np.testing.assert_allclose(g[j, 3:6], -2 * R @ (cen[j] - targets[j]), rtol=1e-10, atol=1e-12)
