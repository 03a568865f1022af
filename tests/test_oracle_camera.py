"""Pins of the oracle's reprojection error and Jacobian (Sec. 3) against things other than itself."""
import numpy as np
import pytest
import scipy.linalg
from scipy.spatial.transform import Rotation

import scenes
from oracle import camera


def hat(w):
    return np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]])


@pytest.mark.parametrize("scale", [3.0, 1.0, 1e-2, 1e-4, 3e-5, 1e-9, 0.0])
def test_rotation_matches_scipy_and_expm(scale):
    rng = np.random.default_rng(1)
    for _ in range(20):
        w = rng.normal(size=3)
        w *= scale / max(np.linalg.norm(w), 1e-300)
        R = camera.rotation_matrix(w)
        np.testing.assert_allclose(R, Rotation.from_rotvec(w).as_matrix(), rtol=0, atol=2e-15)
        np.testing.assert_allclose(R, scipy.linalg.expm(hat(w)), rtol=0, atol=4e-15)


def test_rotation_near_pi():
    for w in ([np.pi - 1e-7, 0, 0], [0, 0, -np.pi + 1e-9], [1.8, -1.9, 1.2]):
        w = np.array(w)
        np.testing.assert_allclose(camera.rotation_matrix(w), Rotation.from_rotvec(w).as_matrix(), atol=3e-15)


def test_projection_matches_generator_on_noise_free_scene():
    # the generator projects with SciPy rotations; the oracle has its own Rodrigues code
    s = scenes.make_tiny_scene(m=6, n=40, noise=0.0, seed=3)
    f = camera.residuals(s.cameras_true, s.points_true, s.obs_cam, s.obs_pt, s.obs_uv)
    assert np.max(np.abs(f)) < 1e-9
    s0 = scenes.make_ring_scene(m=12, n=100, noise=0.0, clusters=2, seed=5)
    f0 = camera.residuals(s0.cameras_true, s0.points_true, s0.obs_cam, s0.obs_pt, s0.obs_uv)
    assert np.max(np.abs(f0)) < 1e-9


def test_projection_closed_form_identity_camera():
    # identity rotation, zero translation, no distortion: pi = f (X/Z, Y/Z)
    cam = np.array([[0, 0, 0, 0, 0, 0, 800.0, 0, 0]])
    X = np.array([[0.3, -0.2, 2.0]])
    np.testing.assert_allclose(camera.project(cam, X), [[120.0, -80.0]], rtol=1e-15)
    # pure distortion: u = f (1 + k1 r2 + k2 r2^2) x
    cam2 = np.array([[0, 0, 0, 0, 0, 0, 1.0, 0.1, 0.01]])
    X2 = np.array([[1.0, 1.0, 1.0]])
    np.testing.assert_allclose(camera.project(cam2, X2), [[1.24, 1.24]], rtol=1e-15)


def central_fd(fun, x, h):
    J = np.empty((2, len(x)))
    for k in range(len(x)):
        xp, xm = x.copy(), x.copy()
        hk = h * max(1.0, abs(x[k]))
        xp[k] += hk
        xm[k] -= hk
        J[:, k] = (fun(xp) - fun(xm)) / (2 * hk)
    return J


@pytest.mark.parametrize("small_rotation", [False, True])
def test_jacobian_matches_central_differences(small_rotation):
    s = scenes.make_tiny_scene(m=5, n=25, seed=11)
    cams = s.cameras.copy()
    if small_rotation:
        cams[:, 0:3] *= 1e-6 / np.linalg.norm(cams[:, 0:3], axis=1, keepdims=True)
    Jc, Jp = camera.jacobians(cams, s.points, s.obs_cam, s.obs_pt)
    worst = 0.0
    for o in range(0, s.q, 3):
        c, p = cams[s.obs_cam[o]], s.points[s.obs_pt[o]]
        fc = lambda x: camera.project(x[None], p[None])[0]
        fp = lambda x: camera.project(c[None], x[None])[0]
        Jc_fd = central_fd(fc, c, 1e-6)
        Jp_fd = central_fd(fp, p, 1e-6)
        sc = np.max(np.abs(Jc[o])) + 1e-30
        worst = max(worst, np.max(np.abs(Jc[o] - Jc_fd)) / sc, np.max(np.abs(Jp[o] - Jp_fd)) / np.max(np.abs(Jp[o])))
    assert worst < 1e-7, worst


def test_jacobian_of_translation_is_projection_derivative():
    # d pi / d t equals d pi / d Xc; with w = 0 it also equals d pi / d p (closed-form chain rule)
    s = scenes.make_tiny_scene(m=4, n=10, seed=2)
    cams = s.cameras.copy()
    cams[:, 0:3] = 0.0
    Jc, Jp = camera.jacobians(cams, s.points, s.obs_cam, s.obs_pt)
    np.testing.assert_allclose(Jc[:, :, 3:6], Jp, rtol=1e-13, atol=1e-10)
    # d pi / d f = pi / f
    pi = camera.project(cams[s.obs_cam], s.points[s.obs_pt])
    np.testing.assert_allclose(Jc[:, :, 6], pi / cams[s.obs_cam, 6:7], rtol=1e-13)
