"""Reprojection error f(x) and its Jacobian J(x) (Sec. 3 of the paper).

Camera parameters c = [w (angle-axis, 3), t (3), f, k1, k2]; point p in R^3.
  Xc = R(w) p + t,  (x, y) = Xc.xy / Xc.z,  r2 = x^2 + y^2,
  pi(c, p) = f (1 + k1 r2 + k2 r2^2) (x, y),     residual  f_o = pi(c_j, p_i) - q_o.
R(w) is Rodrigues' formula R = I + a [w]x + b [w]x^2 with a = sin(th)/th, b = (1 - cos th)/th^2, th = |w|;
for th^2 < 1e-8 the Taylor series of a and b (to th^4) replaces the quotients.

The Jacobian is taken by complex-step differentiation (Squire & Trapp 1998): for an analytic g,
g'(x) = Im g(x + i h) / h exactly up to rounding for tiny h, with no subtraction error.  It is therefore a
differentiation method independent of the hand-derived formulas the CUDA path uses.
"""
import numpy as np

SMALL_TH2 = 1e-8
CS_STEP = 1e-30


def rodrigues_coeffs(th2):
    """a = sin(th)/th and b = (1-cos th)/th^2 as functions of th^2 (real or complex arrays)."""
    small = np.real(th2) < SMALL_TH2
    th2s = np.where(small, 1.0, th2)
    th = np.sqrt(th2s)
    a_big = np.sin(th) / th
    b_big = (1.0 - np.cos(th)) / th2s
    a_small = 1.0 - th2 / 6.0 + th2 * th2 / 120.0
    b_small = 0.5 - th2 / 24.0 + th2 * th2 / 720.0
    return np.where(small, a_small, a_big), np.where(small, b_small, b_big)


def rotate(w, X):
    """R(w) X for stacked w, X of shape (..., 3): X + a (w x X) + b (w (w.X) - th^2 X)."""
    th2 = np.sum(w * w, axis=-1)
    a, b = rodrigues_coeffs(th2)
    wx = np.cross(w, X)
    wdx = np.sum(w * X, axis=-1)
    return X + a[..., None] * wx + b[..., None] * (w * wdx[..., None] - th2[..., None] * X)


def rotation_matrix(w):
    """R(w) as a (3, 3) matrix, columns R e_k."""
    return np.stack([rotate(w, e) for e in np.eye(3)], axis=-1)


def project(cams, pts):
    """pi(c, p) for one camera per point: cams (k, 9), pts (k, 3) -> (k, 2).  Works on complex input."""
    Xc = rotate(cams[:, 0:3], pts) + cams[:, 3:6]
    x = Xc[:, 0] / Xc[:, 2]
    y = Xc[:, 1] / Xc[:, 2]
    r2 = x * x + y * y
    d = 1.0 + cams[:, 7] * r2 + cams[:, 8] * r2 * r2
    s = cams[:, 6] * d
    return np.stack([s * x, s * y], axis=1)


def depth(cams, pts):
    return (rotate(cams[:, 0:3], pts) + cams[:, 3:6])[:, 2]


def residuals(cams, pts, obs_cam, obs_pt, obs_uv):
    """f_o = pi(c_cam(o), p_pt(o)) - q_o, shape (q, 2)."""
    return project(cams[obs_cam], pts[obs_pt]) - obs_uv


def cost(cams, pts, obs_cam, obs_pt, obs_uv):
    """F(x) = ||f(x)||^2 (Sec. 3)."""
    f = residuals(cams, pts, obs_cam, obs_pt, obs_uv)
    return float(np.sum(f * f))


def jacobians(cams, pts, obs_cam, obs_pt):
    """Per-observation blocks d f_o / d c (q, 2, 9) and d f_o / d p (q, 2, 3) by complex step."""
    C = cams[obs_cam].astype(np.complex128)
    P = pts[obs_pt].astype(np.complex128)
    q = len(obs_cam)
    Jc = np.empty((q, 2, 9))
    Jp = np.empty((q, 2, 3))
    for k in range(9):
        Ck = C.copy()
        Ck[:, k] += 1j * CS_STEP
        Jc[:, :, k] = np.imag(project(Ck, P)) / CS_STEP
    for k in range(3):
        Pk = P.copy()
        Pk[:, k] += 1j * CS_STEP
        Jp[:, :, k] = np.imag(project(C, Pk)) / CS_STEP
    return Jc, Jp
