"""One LM iteration of full-RCS LM and of STBA, written as the paper's sparse-matrix equations (FP64).

Notation follows the paper: x = [c; p], J = [J_c, J_p]; B, C, E, v, w of Eq. 4; S, Delta c, Delta p of
Eq. 5-6; virtual points, J' = [J_c, J'_p], D', A of Eq. 7-8; H_lambda and nu of Eq. 9; S', b' of Eq. 10;
the per-cluster systems S'_i Delta c_i = b_i of Eq. 13; and the unified point update of Eq. 15.

Readings where the paper is silent or garbled (also listed in the design notes):
  * w = -J_p^T f (Eq. 4); Algorithm 1 prints w = J_p^T f.  g = -J'^T f (Algorithm 1 prints -J' f).
  * Damping lambda D^T D = lambda diag(J^T J) with no clamping; a lower bound lambda_min is optional.
  * Virtual points are the distinct (point, cluster) pairs: after point binding, cameras in different
    clusters share no point, so each cluster owns one virtual copy of every point it sees (Sec. 4.2).
  * The correction (Sec. 4.3, Algorithm 1) runs when the current lambda >= 0.1, with
    H~ = diag(H_lambda); A ties the virtual copies of each point (one row per copy beyond the first and
    per coordinate).  It changes w' only, because A has no camera columns.
  * The point update uses the physical, uncorrected C, E, w (Algorithm 1, Eq. 15 = Eq. 6).
  * Acceptance is strict: F(x + Dx) < F(x) accepts and divides lambda by 3, anything else (including a
    non-finite cost or a failed Cholesky factorisation) rejects and multiplies it by 3.
  * Stop tests (Ceres definitions): |F - F_new| / F < ftol; ||J^T f||_inf < gtol;
    ||Dx|| < xtol (||x|| + xtol).  They are evaluated on the candidate step, and the acceptance rule
    still applies in that iteration.
  * Huber loss (Sec. 5.1, "scale factor 0.5"), optional: read as Ceres' HuberLoss(a), a = 0.5, on the
    squared norm s = ||f_o||^2 of each observation: rho(s) = s for s <= a^2, 2 a sqrt(s) - a^2 beyond.
    The objective becomes F = sum rho(s_o).  The normal equations take each observation's residual and
    Jacobian rows scaled by sqrt(rho'(s_o)) at the current x (rho' = 1, or a / sqrt(s) beyond a^2;
    rho'' <= 0 throughout, so this is Ceres' corrector for this loss: iteratively reweighted least
    squares); the method's equations are otherwise unchanged.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.linalg
import scipy.sparse as sp
import scipy.sparse.linalg

from . import camera


# ----------------------------------------------------------------------------------------------------------
# sparse Jacobians
# ----------------------------------------------------------------------------------------------------------
def camera_jacobian(Jc, obs_cam, m):
    """J_c as a sparse (2q, 9m) matrix: row 2o+s, column 9 cam(o) + k holds d f_{o,s} / d c_k."""
    q = len(obs_cam)
    rows = np.repeat(np.arange(2 * q), 9)
    cols = (9 * np.repeat(obs_cam, 2)[:, None] + np.arange(9)[None, :]).ravel()
    return sp.csr_matrix((Jc.reshape(-1), (rows, cols)), shape=(2 * q, 9 * m))


def point_jacobian(Jp, col_of_obs, ncols):
    """J_p (or J'_p) as a sparse (2q, 3 ncols) matrix; observation o owns columns 3 col_of_obs[o] + 0..2."""
    q = len(col_of_obs)
    rows = np.repeat(np.arange(2 * q), 3)
    cols = (3 * np.repeat(col_of_obs, 2)[:, None] + np.arange(3)[None, :]).ravel()
    return sp.csr_matrix((Jp.reshape(-1), (rows, cols)), shape=(2 * q, 3 * ncols))


def damped(M, lam):
    """M + lam diag(M) (Eq. 4, with D = diag(J^T J)^(1/2))."""
    return (M + lam * sp.diags(M.diagonal())).tocsr()


def block_diag_inverse(M, bs=3):
    """Inverse of a block-diagonal sparse matrix with bs x bs blocks (C and C' of Eq. 4 / Eq. 10)."""
    Mb = sp.bsr_matrix(M, blocksize=(bs, bs))
    Mb.sort_indices()
    nb = M.shape[0] // bs
    if not (len(Mb.indices) == nb and np.array_equal(Mb.indices, np.arange(nb))):
        raise ValueError("matrix is not block diagonal")
    inv = np.linalg.inv(Mb.data)
    return sp.bsr_matrix((inv, Mb.indices, Mb.indptr), shape=M.shape).tocsr()


# ----------------------------------------------------------------------------------------------------------
# point splitting / binding (Sec. 4.1-4.2)
# ----------------------------------------------------------------------------------------------------------
def virtual_points(obs_pt, obs_cam, clusters):
    """Virtual point of every observation: one per distinct (point, cluster of the observing camera).

    Returns vp_of_obs (q,), vp_point (nv,), vp_cluster (nv,); virtual points ordered by (point, cluster)."""
    key = np.stack([obs_pt, clusters[obs_cam]], axis=1)
    uniq, vp_of_obs = np.unique(key, axis=0, return_inverse=True)
    return vp_of_obs.reshape(-1), uniq[:, 0], uniq[:, 1]


def constraint_matrix(vp_point, m, basis="star"):
    """Equality-constraint matrix A of Eq. 8 over x' = [c (9m); p' (3 nv)].

    For a point with virtual copies p^(1..L), each row a_j = [0 .. 1 .. -1 .. 0] ties two copies in one
    coordinate.  `basis` = "star" ties every copy to the first, "chain" ties consecutive copies; both span
    the same constraint space (A full row rank, r' = 3 sum_i (L_i - 1) rows)."""
    nv = len(vp_point)
    rows, cols, vals = [], [], []
    r = 0
    starts = np.flatnonzero(np.r_[True, vp_point[1:] != vp_point[:-1]])
    ends = np.r_[starts[1:], nv]
    for s, e in zip(starts, ends):
        for j in range(s + 1, e):
            a = s if basis == "star" else j - 1
            for k in range(3):
                rows += [r, r]
                cols += [9 * m + 3 * a + k, 9 * m + 3 * j + k]
                vals += [1.0, -1.0]
                r += 1
    return sp.csr_matrix((vals, (rows, cols)), shape=(r, 9 * m + 3 * nv))


# ----------------------------------------------------------------------------------------------------------
# the linear step
# ----------------------------------------------------------------------------------------------------------
@dataclasses.dataclass
class Linearisation:
    f: np.ndarray      # (2q,) residual vector, row 2o+s
    Jc: np.ndarray     # (q, 2, 9)
    Jp: np.ndarray     # (q, 2, 3)
    J_c: sp.csr_matrix
    J_p: sp.csr_matrix


def huber_rho(s, a):
    """rho(s) of the Huber loss with scale a on the squared norm s (a <= 0: no robust loss, rho(s) = s)."""
    s = np.asarray(s, dtype=float)
    if a <= 0:
        return s
    return np.where(s <= a * a, s, 2.0 * a * np.sqrt(s) - a * a)


def huber_weight(s, a):
    """rho'(s): 1 inside a^2, a / sqrt(s) beyond."""
    s = np.asarray(s, dtype=float)
    if a <= 0:
        return np.ones_like(s)
    return np.where(s <= a * a, 1.0, a / np.sqrt(np.maximum(s, a * a)))


def robust_cost(cams, pts, obs_cam, obs_pt, obs_uv, a=0.0):
    """F(x) = sum over observations of rho(||f_o||^2) (rho(s) = s without a robust loss)."""
    f = camera.residuals(cams, pts, obs_cam, obs_pt, obs_uv)
    return float(np.sum(huber_rho(np.sum(f * f, axis=1), a)))


def linearise(cams, pts, obs_cam, obs_pt, obs_uv, huber=0.0):
    f = camera.residuals(cams, pts, obs_cam, obs_pt, obs_uv)
    Jc, Jp = camera.jacobians(cams, pts, obs_cam, obs_pt)
    if huber > 0:   # rows of observation o scaled by sqrt(rho'(||f_o||^2))
        sw = np.sqrt(huber_weight(np.sum(f * f, axis=1), huber))
        f = f * sw[:, None]
        Jc = Jc * sw[:, None, None]
        Jp = Jp * sw[:, None, None]
    f = f.reshape(-1)
    return Linearisation(f, Jc, Jp, camera_jacobian(Jc, obs_cam, len(cams)),
                         point_jacobian(Jp, obs_pt, len(pts)))


def physical_blocks(lin: Linearisation, lam):
    """B, C, E, v, w of Eq. 4."""
    B = damped(lin.J_c.T @ lin.J_c, lam)
    C = damped(lin.J_p.T @ lin.J_p, lam)
    E = (lin.J_c.T @ lin.J_p).tocsr()
    v = -(lin.J_c.T @ lin.f)
    w = -(lin.J_p.T @ lin.f)
    return B, C, E, v, w


def point_update(C, E, w, dc):
    """Delta p = C^-1 (w - E^T Delta c)  (Eq. 6; equal to Eq. 15)."""
    return block_diag_inverse(C) @ (w - E.T @ dc)


def cluster_camera_indices(clusters, k):
    cams_k = np.flatnonzero(clusters == k)
    return cams_k, (9 * cams_k[:, None] + np.arange(9)[None, :]).ravel()


def cholesky_solve(S, b):
    """Dense LL^T solve; returns None when S is not numerically positive definite."""
    try:
        cf = scipy.linalg.cho_factor(S, lower=True, check_finite=True)
    except (np.linalg.LinAlgError, ValueError):
        return None
    return scipy.linalg.cho_solve(cf, b)


def full_rcs_step(lin: Linearisation, lam):
    """Full-RCS LM step: S Delta c = v - E C^-1 w (Eq. 5), S = B - E C^-1 E^T, then Eq. 6."""
    B, C, E, v, w = physical_blocks(lin, lam)
    Cinv = block_diag_inverse(C)
    S = (B - E @ Cinv @ E.T).toarray()
    b = v - E @ (Cinv @ w)
    dc = cholesky_solve(S, b)
    ok = dc is not None
    if not ok:
        dc = np.zeros_like(b)
    dp = point_update(C, E, w, dc)
    return dict(dc=dc, dp=dp, S=S, b=b, v=v, w=w, spd=ok)


def correction(Jprime, g, A, lam):
    """Steepest-descent correction of Sec. 4.3 / Algorithm 1:
    H_lambda = J'^T J' + lambda D'^T D',  H~ = diag(H_lambda),
    nu = (A H~^-1 A^T)^-1 A H~^-1 g,  g <- g - A^T nu."""
    Hdiag = (1.0 + lam) * np.asarray(Jprime.multiply(Jprime).sum(axis=0)).ravel()
    Hinv = sp.diags(1.0 / Hdiag)
    M = (A @ Hinv @ A.T).tocsc()
    nu = scipy.sparse.linalg.spsolve(M, A @ (Hinv @ g))
    return g - A.T @ np.atleast_1d(nu)


def stba_step(lin: Linearisation, obs_cam, obs_pt, clusters, lam, use_correction=True, corr_lambda=0.1,
              keep=False):
    """The STBA step of Algorithm 1 for one cluster assignment.

    Builds J' = [J_c, J'_p] over the virtual points, B, C', E', g = [v'; w'] = -J'^T f, applies the
    correction when lam >= corr_lambda, forms S' = B - E' C'^-1 E'^T and b' = v' - E' C'^-1 w', solves
    S'_i Delta c_i = b_i for every cluster i (Eq. 13), and updates the points with Eq. 15."""
    m = lin.J_c.shape[1] // 9
    vp_of_obs, vp_point, vp_cluster = virtual_points(obs_pt, obs_cam, clusters)
    nv = len(vp_point)
    J_pv = point_jacobian(lin.Jp, vp_of_obs, nv)
    Jprime = sp.hstack([lin.J_c, J_pv]).tocsr()
    B = damped(lin.J_c.T @ lin.J_c, lam)
    Cv = damped(J_pv.T @ J_pv, lam)
    Ev = (lin.J_c.T @ J_pv).tocsr()
    g = -(Jprime.T @ lin.f)
    corrected = bool(use_correction and lam >= corr_lambda)
    if corrected:
        A = constraint_matrix(vp_point, m)
        if A.shape[0] > 0:
            g = correction(Jprime, g, A, lam)
    v1, w1 = g[: 9 * m], g[9 * m:]
    Cv_inv = block_diag_inverse(Cv)
    Sp = (B - Ev @ Cv_inv @ Ev.T).tocsr()
    bp = v1 - Ev @ (Cv_inv @ w1)
    dc = np.zeros(9 * m)
    l = int(clusters.max()) + 1
    spd = np.ones(l, dtype=bool)
    S_blocks, b_blocks = [], []
    for k in range(l):
        _, idx = cluster_camera_indices(clusters, k)
        Sk = Sp[idx][:, idx].toarray()
        bk = bp[idx]
        xk = cholesky_solve(Sk, bk)
        if xk is None:
            spd[k] = False
        else:
            dc[idx] = xk
        if keep:
            S_blocks.append(Sk)
            b_blocks.append(bk)
    _, C, E, v, w = physical_blocks(lin, lam)
    dp = point_update(C, E, w, dc)
    out = dict(dc=dc, dp=dp, spd=bool(spd.all()), spd_per_cluster=spd, corrected=corrected, v=v, w=w,
               nv=nv, vp_of_obs=vp_of_obs, vp_point=vp_point, vp_cluster=vp_cluster)
    if keep:
        out.update(S_blocks=S_blocks, b_blocks=b_blocks, S_prime=Sp, b_prime=bp, g=g)
    return out


# ----------------------------------------------------------------------------------------------------------
# brute force (tiny problems only)
# ----------------------------------------------------------------------------------------------------------
def brute_force_lm_step(lin: Linearisation, lam):
    """Dense solve of (J^T J + lam D^T D) Dx = -J^T f (Eq. 3)."""
    J = sp.hstack([lin.J_c, lin.J_p]).toarray()
    H = J.T @ J
    H = H + lam * np.diag(np.diag(H))
    return np.linalg.solve(H, -J.T @ lin.f)


def brute_force_expanded_step(lin: Linearisation, obs_cam, obs_pt, clusters, lam, nu_exact=False):
    """Dense solve over x' = [c; p'] (Eq. 7-9).  nu_exact=False drops every cross-cluster constraint
    (the relaxed problem STBA solves without correction); nu_exact=True uses the exact Lagrange
    multipliers of Eq. 9, which restores the full LM step."""
    m = lin.J_c.shape[1] // 9
    vp_of_obs, vp_point, _ = virtual_points(obs_pt, obs_cam, clusters)
    J_pv = point_jacobian(lin.Jp, vp_of_obs, len(vp_point))
    Jp_ = sp.hstack([lin.J_c, J_pv]).toarray()
    H = Jp_.T @ Jp_
    H = H + lam * np.diag(np.diag(H))
    rhs = -Jp_.T @ lin.f
    if nu_exact:
        A = constraint_matrix(vp_point, m).toarray()
        if A.shape[0]:
            Hi = np.linalg.inv(H)
            nu = -np.linalg.solve(A @ Hi @ A.T, A @ Hi @ (Jp_.T @ lin.f))
            rhs = rhs - A.T @ nu
    return np.linalg.solve(H, rhs), vp_of_obs, vp_point


# ----------------------------------------------------------------------------------------------------------
# LM control (Algorithm 1)
# ----------------------------------------------------------------------------------------------------------
@dataclasses.dataclass
class Options:
    lambda0: float = 1e-4
    lambda_min: float = 0.0
    correction: bool = True
    correction_lambda: float = 0.1
    ftol: float = -1.0
    gtol: float = -1.0
    xtol: float = -1.0
    huber: float = 0.0     # Huber scale a (0: plain least squares)


def stop_tests(F, F_new, grad_inf, dx_norm, x_norm, opt: Options):
    stop = False
    if opt.ftol > 0 and F > 0 and abs(F - F_new) / F < opt.ftol:
        stop = True
    if opt.gtol > 0 and grad_inf < opt.gtol:
        stop = True
    if opt.xtol > 0 and dx_norm < opt.xtol * (x_norm + opt.xtol):
        stop = True
    return stop


def lm_iteration(cams, pts, obs_cam, obs_pt, obs_uv, clusters, lam, F, opt: Options, method="stba",
                 keep=False):
    """One iteration of Algorithm 1 (method="stba") or of full-RCS LM (method="lm").

    Returns the new (cams, pts, lam, F) and a record of the step."""
    m, n = len(cams), len(pts)
    lin = linearise(cams, pts, obs_cam, obs_pt, obs_uv, opt.huber)
    if method == "lm":
        st = full_rcs_step(lin, lam)
    else:
        st = stba_step(lin, obs_cam, obs_pt, clusters, lam, opt.correction, opt.correction_lambda, keep=keep)
    dc = st["dc"].reshape(m, 9)
    dp = st["dp"].reshape(n, 3)
    cams_new = cams + dc
    pts_new = pts + dp
    if st["spd"]:
        F_new = robust_cost(cams_new, pts_new, obs_cam, obs_pt, obs_uv, opt.huber)
    else:
        F_new = np.inf
    grad_inf = max(np.max(np.abs(st["v"])), np.max(np.abs(st["w"])))
    dx_norm = float(np.sqrt(np.sum(dc * dc) + np.sum(dp * dp)))
    x_norm = float(np.sqrt(np.sum(cams * cams) + np.sum(pts * pts)))
    stop = stop_tests(F, F_new, grad_inf, dx_norm, x_norm, opt)
    accepted = bool(np.isfinite(F_new) and F_new < F)
    if accepted:
        lam_new = max(lam / 3.0, opt.lambda_min)
        cams, pts, F_out = cams_new, pts_new, F_new
    else:
        lam_new = lam * 3.0
        F_out = F
    rec = dict(F_before=F, F_after=F_new, lam_used=lam, lam=lam_new, accepted=accepted, stop=stop, dc=dc, dp=dp,
               spd=st["spd"], corrected=st.get("corrected", False), grad_inf=grad_inf, dx_norm=dx_norm,
               x_norm=x_norm)
    if keep:
        rec["step"] = st
    return cams, pts, lam_new, F_out, rec


def solve(cams, pts, obs_cam, obs_pt, obs_uv, cluster_seq, iters, opt: Options = None, method="stba",
          keep=False, stop_early=False):
    """Run `iters` iterations; cluster_seq is (iters, m) or (m,) (a fixed assignment)."""
    opt = opt or Options()
    cluster_seq = np.asarray(cluster_seq)
    lam = opt.lambda0
    F = robust_cost(cams, pts, obs_cam, obs_pt, obs_uv, opt.huber)
    hist = []
    for t in range(iters):
        cl = cluster_seq[t] if cluster_seq.ndim == 2 else cluster_seq
        cams, pts, lam, F, rec = lm_iteration(cams, pts, obs_cam, obs_pt, obs_uv, cl, lam, F, opt, method, keep)
        hist.append(rec)
        if stop_early and rec["stop"]:
            break
    return cams, pts, lam, F, hist


def rmse(F, q):
    """Per-coordinate reprojection RMS in pixels: sqrt(F / 2q)."""
    return float(np.sqrt(F / (2.0 * q)))
