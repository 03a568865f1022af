"""Pins of the oracle's Huber loss (Sec. 5.1, read as Ceres' HuberLoss(a) on ||f_o||^2): the loss by hand,
its derivative against finite differences, the plain-least-squares limit, and the gradient of the
robust objective against central differences of the objective itself (which fixes the sqrt(rho') scaling
of both the residual and the Jacobian rows)."""
import numpy as np
import pytest

import scenes
from oracle import camera
from oracle import stba as ostba


def test_rho_by_hand_and_continuity():
    a = 0.5
    assert ostba.huber_rho(0.16, a) == pytest.approx(0.16, rel=1e-15)
    assert ostba.huber_rho(1.0, a) == pytest.approx(0.75, rel=1e-15)          # 2 * 0.5 * 1 - 0.25
    assert ostba.huber_rho(4.0, a) == pytest.approx(1.75, rel=1e-15)          # 2 * 0.5 * 2 - 0.25
    eps = 1e-12
    assert ostba.huber_rho(0.25 - eps, a) == pytest.approx(ostba.huber_rho(0.25 + eps, a), abs=1e-11)
    assert ostba.huber_weight(0.25, a) == 1.0
    assert ostba.huber_weight(1.0, a) == pytest.approx(0.5, rel=1e-15)        # a / sqrt(s)
    assert ostba.huber_rho(3.0, 0.0) == 3.0 and ostba.huber_weight(3.0, 0.0) == 1.0


@pytest.mark.parametrize("s", [0.01, 0.2, 0.3, 1.0, 7.5, 100.0])
def test_weight_is_the_derivative_of_rho(s):
    a, h = 0.5, 1e-6
    d = (ostba.huber_rho(s + h, a) - ostba.huber_rho(s - h, a)) / (2 * h)
    assert ostba.huber_weight(s, a) == pytest.approx(float(d), rel=1e-7)


def outlier_scene(seed=3):
    s = scenes.make_tiny_scene(m=5, n=30, seed=seed)
    uv = s.obs_uv.copy()
    rng = np.random.default_rng(seed)
    bad = rng.choice(len(uv), size=6, replace=False)
    uv[bad] += rng.normal(0.0, 25.0, size=(6, 2))   # gross outliers next to N(0, 1) pixel noise
    return s, uv


def test_large_scale_is_plain_least_squares():
    s, uv = outlier_scene()
    F = camera.cost(s.cameras, s.points, s.obs_cam, s.obs_pt, uv)
    assert ostba.robust_cost(s.cameras, s.points, s.obs_cam, s.obs_pt, uv, 1e9) == F
    lin0 = ostba.linearise(s.cameras, s.points, s.obs_cam, s.obs_pt, uv)
    lin1 = ostba.linearise(s.cameras, s.points, s.obs_cam, s.obs_pt, uv, huber=1e9)
    assert np.array_equal(lin0.f, lin1.f) and np.array_equal(lin0.Jc, lin1.Jc)


def test_robust_gradient_matches_central_differences():
    s, uv = outlier_scene()
    a = 0.5
    f = camera.residuals(s.cameras, s.points, s.obs_cam, s.obs_pt, uv)
    sq = np.sum(f * f, axis=1)
    assert np.any(sq > a * a) and np.any(sq <= a * a)   # both branches of the loss are active
    lin = ostba.linearise(s.cameras, s.points, s.obs_cam, s.obs_pt, uv, huber=a)
    g_c = 2 * (lin.J_c.T @ lin.f)       # dF/dc = 2 J~_c^T f~
    g_p = 2 * (lin.J_p.T @ lin.f)
    x_c, x_p = s.cameras.copy(), s.points.copy()

    def F(c, p):
        return ostba.robust_cost(c, p, s.obs_cam, s.obs_pt, uv, a)

    rng = np.random.default_rng(1)
    for idx in rng.choice(x_c.size, size=12, replace=False):
        h = 1e-6 * max(1.0, abs(x_c.flat[idx]))
        cp, cm = x_c.copy(), x_c.copy()
        cp.flat[idx] += h
        cm.flat[idx] -= h
        d = (F(cp, x_p) - F(cm, x_p)) / (2 * h)
        assert g_c[idx] == pytest.approx(d, rel=2e-5, abs=1e-4 * np.abs(g_c).max())
    for idx in rng.choice(x_p.size, size=12, replace=False):
        h = 1e-6
        pp, pm = x_p.copy(), x_p.copy()
        pp.flat[idx] += h
        pm.flat[idx] -= h
        d = (F(x_c, pp) - F(x_c, pm)) / (2 * h)
        assert g_p[idx] == pytest.approx(d, rel=2e-5, abs=1e-4 * np.abs(g_p).max())


def test_huber_iterations_descend_and_resist_outliers():
    s, uv = outlier_scene(seed=4)
    opt_h = ostba.Options(huber=0.5)
    c_h, p_h, lam, F, hist = ostba.solve(s.cameras, s.points, s.obs_cam, s.obs_pt, uv, s.clusters, 15, opt_h)
    Fs = [h["F_before"] for h in hist] + [F]
    assert all(b <= a for a, b in zip(Fs, Fs[1:]))     # accepted steps never raise the robust cost
    c_l, p_l, _, _, _ = ostba.solve(s.cameras, s.points, s.obs_cam, s.obs_pt, uv, s.clusters, 15, ostba.Options())
    err_h = np.linalg.norm(p_h - s.points_true)
    err_l = np.linalg.norm(p_l - s.points_true)
    assert err_h < err_l
