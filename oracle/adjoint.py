"""FP64 reverse-mode derivative of K STBA LM iterations (test infrastructure; see oracle/__init__.py).

The paper has no adjoint.  This follows the reading that the derivative is taken through the executed
LM steps, with the damping, the cluster assignments and the accept flags held at their forward values
(they are decisions, not smooth functions).  An accepted step is Delta = -M(J(x)) f(x, q): the camera part
is the camera part of the relaxed expanded solve H' dx' = -J'^T f (Eq. 10), the point part is Eq. 15,
Delta p = -C^-1 J_p^T (f + J_c Delta c).  For an upstream adjoint a = (a_c, a_p) of x_{t+1} = x_t + Delta:

  u   = C^-1 a_p                         a^_c = a_c - E u
  z_c = S'^-1 a^_c  (per cluster)        z_v  = -C'_v^-1 E'_v^T z_c   (z' = [z_c; z_v] = H'^-1 [a^_c; 0])
  q_bar_o += g_o = J_o (z'_o + [0; u])   (the observation enters through f = pi - q)
  x_bar    = a - sum_o [ J_o^T g_o + sum of Hessian-vector terms ]

where, with H_s the 12x12 Hessian of residual component s of observation o in its local parameters and
(alpha, beta) meaning sum_s alpha_s H_s beta, the terms are
  (f_o, z'_o) + (J_o dx'_o, z'_o) + (J_o z'_o, dx'_o) + sum_s H_s (2 lam J_o[s,:] o z'_o o dx'_o)
  + (J_o DP_o, U_o) + (J_o U_o, DP_o) + sum_s H_s (2 lam J_o[s,:] o U_o o DP_o) + (rho_o, U_o) + (J_o U_o, DC_o)
with dx' = [Delta c; Delta p'] the expanded step (virtual points), U = [0; u], DP = [0; Delta p],
DC = [Delta c; 0], rho = f + J_c Delta c.  A rejected step passes the adjoint through unchanged.
Hessian-vector products are central differences of the complex-step Jacobian along beta.

A step taken with the steepest-descent correction (Sec. 4.3, Algorithm 1: lambda >= the threshold) solves
H' dx' = g~' with the corrected right-hand side.  In closed form (the oracle's literal A-matrix correction
equals it, see the correction pins) w~'_v = (h_v / H_i) o w_i for every virtual point v of point i, with
h_v = diag(J'_v^T J'_v) (undamped), H_i = sum over the copies of h_v = diag(J_p^T J_p)_i and w_i the physical
w; Eq. 15 still takes the physical, uncorrected w.  Differentiating z'^T g~' then gives, besides the
expanded step dx' now built from w~':
  - in the terms that come from g (the f-Hessian term, J_o^T g_o and q_bar), z'_o is replaced by
    z~_o = [z_c; zeta_i], zeta_i = sum_v h_v o z_v / H_i (the h-weighted mean of the copies' z_v);
  - the derivative of h_v / H_i adds  - sum_s H_s [0; 2 kappa_v o J_p,o[s,:]]  with
    kappa_v = (z_v - zeta_i) o w_i / H_i;
the terms that come from H' keep the solved z'.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import camera, stba


def local_jacobians(C, P):
    """Complex-step Jacobian blocks for one camera (C, (k,9)) and point (P, (k,3)) per row."""
    k = len(C)
    Jc = np.empty((k, 2, 9))
    Jp = np.empty((k, 2, 3))
    Cc = C.astype(np.complex128)
    Pc = P.astype(np.complex128)
    for i in range(9):
        Ci = Cc.copy()
        Ci[:, i] += 1j * camera.CS_STEP
        Jc[:, :, i] = np.imag(camera.project(Ci, Pc)) / camera.CS_STEP
    for i in range(3):
        Pi = Pc.copy()
        Pi[:, i] += 1j * camera.CS_STEP
        Jp[:, :, i] = np.imag(camera.project(Cc, Pi)) / camera.CS_STEP
    return np.concatenate([Jc, Jp], axis=2)   # (k, 2, 12)


def hessian_vector(C, P, alpha, beta):
    """sum_s alpha[:, s] H_s beta per row: d/de [J(x + e beta)^T alpha] by a central difference."""
    scale = (np.linalg.norm(np.concatenate([C, P], 1), axis=1) + 1.0)
    bn = np.linalg.norm(beta, axis=1)
    h = np.where(bn > 0, 1e-6 * scale / np.maximum(bn, 1e-300), 0.0)
    Jp_ = local_jacobians(C + h[:, None] * beta[:, :9], P + h[:, None] * beta[:, 9:])
    Jm_ = local_jacobians(C - h[:, None] * beta[:, :9], P - h[:, None] * beta[:, 9:])
    dJ = np.where(bn[:, None, None] > 0, (Jp_ - Jm_) / np.where(h > 0, 2 * h, 1.0)[:, None, None], 0.0)
    return np.einsum('ks,ksj->kj', alpha, dJ)


def forward(cams, pts, obs_cam, obs_pt, obs_uv, cluster_seq, iters, opt: stba.Options = None):
    """K iterations of STBA with the record the adjoint needs."""
    opt = opt or stba.Options()
    cluster_seq = np.asarray(cluster_seq)
    lam = opt.lambda0
    F = camera.cost(cams, pts, obs_cam, obs_pt, obs_uv)
    tape = []
    for t in range(iters):
        cl = cluster_seq[t] if cluster_seq.ndim == 2 else cluster_seq
        c_new, p_new, lam_new, F, rec = stba.lm_iteration(cams, pts, obs_cam, obs_pt, obs_uv, cl, lam, F, opt)
        tape.append(dict(cams=cams, pts=pts, lam=lam, clusters=cl, accepted=rec["accepted"],
                         corrected=rec["corrected"]))
        cams, pts, lam = c_new, p_new, lam_new
    return cams, pts, tape


def step_adjoint(cams, pts, obs_cam, obs_pt, obs_uv, clusters, lam, a_c, a_p, corrected=False):
    """Adjoint of one accepted step at x = (cams, pts): returns (x_bar_cams, x_bar_pts, q_bar).
    corrected: the step used the steepest-descent correction (Sec. 4.3)."""
    m, n, q = len(cams), len(pts), len(obs_cam)
    lin = stba.linearise(cams, pts, obs_cam, obs_pt, obs_uv)
    f = lin.f.reshape(q, 2)
    # forward step quantities (Algorithm 1, uncorrected)
    vp_of_obs, vp_point, _ = stba.virtual_points(obs_pt, obs_cam, clusters)
    nv = len(vp_point)
    J_pv = stba.point_jacobian(lin.Jp, vp_of_obs, nv)
    B = stba.damped(lin.J_c.T @ lin.J_c, lam)
    Cv = stba.damped(J_pv.T @ J_pv, lam)
    Ev = (lin.J_c.T @ J_pv).tocsr()
    g = -(sp.hstack([lin.J_c, J_pv]).tocsr().T @ lin.f)
    v1, w1 = g[: 9 * m], g[9 * m:]
    if corrected:   # w~'_v = (h_v / H_i) o w_i, the closed form of the correction
        hv = np.asarray(J_pv.multiply(J_pv).sum(axis=0)).reshape(nv, 3)
        Hi = np.zeros((n, 3))
        np.add.at(Hi, vp_point, hv)
        wi = np.zeros((n, 3))
        np.add.at(wi, vp_point, w1.reshape(nv, 3))
        w1 = (hv / Hi[vp_point] * wi[vp_point]).reshape(-1)
    Cv_inv = stba.block_diag_inverse(Cv)
    Sp = (B - Ev @ Cv_inv @ Ev.T).tocsr()
    bp = v1 - Ev @ (Cv_inv @ w1)
    l = int(clusters.max()) + 1
    dc = np.zeros(9 * m)
    Sk = []
    for k in range(l):
        _, idx = stba.cluster_camera_indices(clusters, k)
        S_k = Sp[idx][:, idx].toarray()
        Sk.append((idx, S_k))
        dc[idx] = np.linalg.solve(S_k, bp[idx])
    dpv = Cv_inv @ (w1 - Ev.T @ dc)                        # expanded (virtual point) step
    _, C, E, v, w = stba.physical_blocks(lin, lam)
    Cinv = stba.block_diag_inverse(C)
    dp = Cinv @ (w - E.T @ dc)
    # adjoint
    u = Cinv @ a_p.reshape(-1)
    ahat = a_c.reshape(-1) - E @ u
    zc = np.zeros(9 * m)
    for idx, S_k in Sk:
        zc[idx] = np.linalg.solve(S_k, ahat[idx])
    zv = -(Cv_inv @ (Ev.T @ zc))
    # per-observation local vectors [camera 9; point 3]
    dcm, zcm = dc.reshape(m, 9), zc.reshape(m, 9)
    z_o = np.concatenate([zcm[obs_cam], zv.reshape(nv, 3)[vp_of_obs]], 1)
    zt_o = z_o   # z~_o: the z seen by the right-hand side g
    if corrected:
        zeta = np.zeros((n, 3))
        np.add.at(zeta, vp_point, hv * zv.reshape(nv, 3))
        zeta /= Hi
        kappa = (zv.reshape(nv, 3) - zeta[vp_point]) * wi[vp_point] / Hi[vp_point]
        zt_o = np.concatenate([zcm[obs_cam], zeta[obs_pt]], 1)
    dx_o = np.concatenate([dcm[obs_cam], dpv.reshape(nv, 3)[vp_of_obs]], 1)
    U_o = np.concatenate([np.zeros((q, 9)), u.reshape(n, 3)[obs_pt]], 1)
    DP_o = np.concatenate([np.zeros((q, 9)), dp.reshape(n, 3)[obs_pt]], 1)
    DC_o = np.concatenate([dcm[obs_cam], np.zeros((q, 3))], 1)
    J_o = np.concatenate([lin.Jc, lin.Jp], axis=2)         # (q, 2, 12)
    Jz, Jdx, JU, JDP, Jzt = (np.einsum('ksj,kj->ks', J_o, vv) for vv in (z_o, dx_o, U_o, DP_o, zt_o))
    rho = f + np.einsum('ksj,kj->ks', lin.Jc, dcm[obs_cam])
    g_o = Jzt + JU
    C_o, P_o = cams[obs_cam], pts[obs_pt]
    terms = np.einsum('ksj,ks->kj', J_o, g_o)
    if corrected:
        terms += hessian_vector(C_o, P_o, f, zt_o)
        terms += hessian_vector(C_o, P_o, Jdx, z_o)
        for s in range(2):
            es = np.zeros((q, 2))
            es[:, s] = 1.0
            beta = np.concatenate([np.zeros((q, 9)), -2.0 * kappa[vp_of_obs] * lin.Jp[:, s, :]], 1)
            terms += hessian_vector(C_o, P_o, es, beta)
    else:
        terms += hessian_vector(C_o, P_o, f + Jdx, z_o)
    terms += hessian_vector(C_o, P_o, Jz, dx_o)
    terms += hessian_vector(C_o, P_o, JDP + rho, U_o)
    terms += hessian_vector(C_o, P_o, JU, DP_o + DC_o)
    for s in range(2):
        es = np.zeros((q, 2))
        es[:, s] = 1.0
        terms += hessian_vector(C_o, P_o, es, 2 * lam * J_o[:, s, :] * z_o * dx_o)
        terms += hessian_vector(C_o, P_o, es, 2 * lam * J_o[:, s, :] * U_o * DP_o)
    xb_c = a_c.copy().reshape(m, 9)
    xb_p = a_p.copy().reshape(n, 3)
    np.add.at(xb_c, obs_cam, -terms[:, :9])
    np.add.at(xb_p, obs_pt, -terms[:, 9:])
    return xb_c, xb_p, g_o


def backward(tape, obs_cam, obs_pt, obs_uv, a_cams, a_pts):
    """Adjoint of the recorded iterations for upstream (a_cams, a_pts) of the final parameters.
    Returns (dL/d cams0, dL/d pts0, dL/d obs_uv)."""
    a_c, a_p = a_cams.copy(), a_pts.copy()
    qbar = np.zeros((len(obs_cam), 2))
    for rec in reversed(tape):
        if not rec["accepted"]:
            continue
        a_c, a_p, g_o = step_adjoint(rec["cams"], rec["pts"], obs_cam, obs_pt, obs_uv, rec["clusters"], rec["lam"],
                                     a_c, a_p, corrected=rec.get("corrected", False))
        qbar += g_o
    return a_c, a_p, qbar


def camera_centres(cams):
    """centre_j = -R(w_j)^T t_j."""
    R = np.stack([camera.rotation_matrix(w) for w in cams[:, 0:3]])
    return -np.einsum('kji,kj->ki', R, cams[:, 3:6])


def centre_loss(cams, targets):
    """L = sum_j |centre_j - target_j|^2 (the scalar loss of the differentiable configuration)."""
    d = camera_centres(cams) - targets
    return float(np.sum(d * d))


def centre_loss_grad(cams, targets):
    """dL/d cams by complex step through camera_centres (exact up to rounding)."""
    g = np.zeros_like(cams)
    for i in range(cams.shape[0]):
        for k in range(6):
            c = cams[i].astype(np.complex128).copy()
            c[k] += 1j * camera.CS_STEP
            R = camera.rotation_matrix(c[0:3])
            cen = -R.T @ c[3:6]
            d = cen - targets[i]
            g[i, k] = np.imag(np.sum(d * d)) / camera.CS_STEP
    return g
