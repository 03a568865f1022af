"""Pins of the oracle's LM / STBA step (Eq. 3-15, Algorithm 1) against brute force, closed forms and
the identities the paper states."""
import numpy as np
import pytest
import scipy.sparse as sp

import scenes
from oracle import camera, stba


def tiny(m=5, n=30, seed=7, clusters=None, **kw):
    s = scenes.make_tiny_scene(m=m, n=n, seed=seed, **kw)
    if clusters is not None:
        s.clusters = np.asarray(clusters, dtype=np.int32)
    return s


def lin_of(s, cams=None, pts=None):
    return stba.linearise(s.cameras if cams is None else cams, s.points if pts is None else pts,
                          s.obs_cam, s.obs_pt, s.obs_uv)


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("lam", [1e-4, 1e-1, 10.0])
def test_schur_step_equals_brute_force_normal_equations(lam):
    # Eq. 5-6 reproduce the dense solve of Eq. 3
    s = tiny()
    lin = lin_of(s)
    st = stba.full_rcs_step(lin, lam)
    dx = stba.brute_force_lm_step(lin, lam)
    assert rel(st["dc"], dx[: 9 * s.m]) < 1e-9
    assert rel(st["dp"], dx[9 * s.m:]) < 1e-9


@pytest.mark.parametrize("lam", [1e-4, 0.3])
def test_single_cluster_stba_is_lm(lam):
    # Gamma = infinity: one cluster, A empty, STBA is classic LM (Appendix B)
    s = tiny(m=6, n=40, seed=3)
    lin = lin_of(s)
    st = stba.stba_step(lin, s.obs_cam, s.obs_pt, np.zeros(s.m, np.int32), lam, use_correction=True)
    dx = stba.brute_force_lm_step(lin, lam)
    assert rel(st["dc"], dx[: 9 * s.m]) < 1e-9
    assert rel(st["dp"], dx[9 * s.m:]) < 1e-9


@pytest.mark.parametrize("clusters", [[0, 0, 1, 1, 2, 2], [0, 1, 0, 1, 0, 1], [0, 1, 2, 3, 4, 5]])
def test_stba_camera_step_equals_relaxed_expanded_solve(clusters):
    # without correction, S' Delta c = b' (Eq. 10, 13) is the camera part of the dense solve over the
    # virtual-point expansion with every cross-cluster constraint dropped
    s = tiny(m=6, n=40, seed=5, clusters=clusters)
    lin = lin_of(s)
    lam = 1e-3
    st = stba.stba_step(lin, s.obs_cam, s.obs_pt, s.clusters, lam, use_correction=False)
    dxv, _, _ = stba.brute_force_expanded_step(lin, s.obs_cam, s.obs_pt, s.clusters, lam)
    assert rel(st["dc"], dxv[: 9 * s.m]) < 1e-9


def test_point_update_is_damped_least_squares_of_eq15():
    # Eq. 15: Delta p minimises ||J_p Delta p + f + J_c Delta c||^2 + lam ||D_p Delta p||^2
    s = tiny(m=6, n=40, seed=8, clusters=[0, 0, 0, 1, 1, 1])
    lin = lin_of(s)
    lam = 1e-2
    st = stba.stba_step(lin, s.obs_cam, s.obs_pt, s.clusters, lam, use_correction=False)
    Jp = lin.J_p.toarray()
    Dp = np.sqrt(np.sum(Jp * Jp, axis=0))
    A = np.vstack([Jp, np.sqrt(lam) * np.diag(Dp)])
    rhs = np.concatenate([-lin.f - lin.J_c @ st["dc"], np.zeros(Jp.shape[1])])
    dp_ls = np.linalg.lstsq(A, rhs, rcond=None)[0]
    assert rel(st["dp"], dp_ls) < 1e-9


def test_exact_multipliers_restore_the_lm_step():
    # Eq. 9 with the exact nu enforces A Dx' = 0 and reproduces the LM step of Eq. 3
    s = tiny(m=5, n=30, seed=9, clusters=[0, 1, 1, 2, 0])
    lin = lin_of(s)
    lam = 1e-3
    dxv, vp_of_obs, vp_point = stba.brute_force_expanded_step(lin, s.obs_cam, s.obs_pt, s.clusters, lam,
                                                              nu_exact=True)
    dx = stba.brute_force_lm_step(lin, lam)
    assert rel(dxv[: 9 * s.m], dx[: 9 * s.m]) < 1e-8
    dpv = dxv[9 * s.m:].reshape(-1, 3)
    np.testing.assert_allclose(dpv, dx[9 * s.m:].reshape(-1, 3)[vp_point], rtol=1e-7, atol=1e-12)


def test_every_camera_its_own_cluster_gives_block_diagonal_rcs():
    # Gamma = 1 (Sec. 4.1): S' is block diagonal with 9x9 blocks; each block solve is independent
    s = tiny(m=5, n=30, seed=4, clusters=np.arange(5))
    lin = lin_of(s)
    lam = 1e-3
    st = stba.stba_step(lin, s.obs_cam, s.obs_pt, s.clusters, lam, use_correction=False, keep=True)
    Sp = st["S_prime"].toarray()
    for a in range(s.m):
        for b in range(s.m):
            if a != b:
                assert np.all(Sp[9 * a:9 * a + 9, 9 * b:9 * b + 9] == 0)
        blk = Sp[9 * a:9 * a + 9, 9 * a:9 * a + 9]
        np.testing.assert_allclose(st["dc"][9 * a:9 * a + 9], np.linalg.solve(blk, st["b_prime"][9 * a:9 * a + 9]),
                                   rtol=1e-9)


def test_cluster_diagonal_structure():
    s = tiny(m=6, n=40, seed=12, clusters=[1, 0, 1, 0, 2, 2])
    lin = lin_of(s)
    st = stba.stba_step(lin, s.obs_cam, s.obs_pt, s.clusters, 1e-3, keep=True)
    Sp = st["S_prime"].toarray()
    for a in range(s.m):
        for b in range(s.m):
            if s.clusters[a] != s.clusters[b]:
                assert np.all(Sp[9 * a:9 * a + 9, 9 * b:9 * b + 9] == 0)


def closed_form_correction(g, Hdiag, vp_point, m):
    # derived in closed form: H~-weighted projection of H~^-1 g onto equal steps of each point's copies
    out = g.copy()
    w, h = g[9 * m:].reshape(-1, 3), Hdiag[9 * m:].reshape(-1, 3)
    res = out[9 * m:].reshape(-1, 3)
    for i in np.unique(vp_point):
        sel = vp_point == i
        dbar = w[sel].sum(0) / h[sel].sum(0)
        res[sel] = h[sel] * dbar
    return out


@pytest.mark.parametrize("basis", ["star", "chain"])
def test_correction_matches_closed_form_and_invariants(basis):
    s = tiny(m=6, n=40, seed=13, clusters=[0, 1, 2, 0, 1, 2])
    lin = lin_of(s)
    lam = 0.5
    vp_of_obs, vp_point, _ = stba.virtual_points(s.obs_pt, s.obs_cam, s.clusters)
    Jpv = stba.point_jacobian(lin.Jp, vp_of_obs, len(vp_point))
    Jprime = sp.hstack([lin.J_c, Jpv]).tocsr()
    g = -(Jprime.T @ lin.f)
    A = stba.constraint_matrix(vp_point, s.m, basis=basis)
    gc = stba.correction(Jprime, g, A, lam)
    Hdiag = (1 + lam) * np.asarray(Jprime.multiply(Jprime).sum(0)).ravel()
    np.testing.assert_allclose(gc, closed_form_correction(g, Hdiag, vp_point, s.m), rtol=1e-10, atol=1e-9)
    # camera part unchanged; per-point sums of w' preserved; corrected steepest-descent step feasible
    np.testing.assert_array_equal(gc[: 9 * s.m], g[: 9 * s.m])
    wsum = np.zeros((s.n, 3))
    wsum_c = np.zeros((s.n, 3))
    np.add.at(wsum, vp_point, g[9 * s.m:].reshape(-1, 3))
    np.add.at(wsum_c, vp_point, gc[9 * s.m:].reshape(-1, 3))
    np.testing.assert_allclose(wsum_c, wsum, rtol=1e-10, atol=1e-8)
    assert np.max(np.abs(A @ (gc / Hdiag))) < 1e-10 * np.max(np.abs(g / Hdiag))


def test_correction_only_when_lambda_at_least_threshold():
    s = tiny(m=6, n=40, seed=14, clusters=[0, 1, 2, 0, 1, 2])
    lin = lin_of(s)
    lo = stba.stba_step(lin, s.obs_cam, s.obs_pt, s.clusters, 0.0999, use_correction=True)
    hi = stba.stba_step(lin, s.obs_cam, s.obs_pt, s.clusters, 0.1, use_correction=True)
    off = stba.stba_step(lin, s.obs_cam, s.obs_pt, s.clusters, 0.1, use_correction=False)
    assert not lo["corrected"] and hi["corrected"] and not off["corrected"]
    assert rel(hi["dc"], off["dc"]) > 1e-6


def test_lm_control_monotone_and_lambda_sequence():
    s = tiny(m=6, n=40, seed=15, clusters=[0, 0, 1, 1, 2, 2])
    c, p, lam, F, hist = stba.solve(s.cameras, s.points, s.obs_cam, s.obs_pt, s.obs_uv, s.clusters, 12)
    Fcur = camera.cost(s.cameras, s.points, s.obs_cam, s.obs_pt, s.obs_uv)
    lam_cur = 1e-4
    for r in hist:
        assert r["F_before"] == Fcur and r["lam_used"] == lam_cur
        if r["accepted"]:
            assert r["F_after"] < Fcur
            Fcur = r["F_after"]
            lam_cur = lam_cur / 3
        else:
            lam_cur = lam_cur * 3
        assert np.isclose(r["lam"], lam_cur, rtol=0, atol=0)
    assert F == Fcur


@pytest.mark.parametrize("method", ["lm", "stba"])
def test_noise_free_scene_converges_to_zero(method):
    s = scenes.make_tiny_scene(m=6, n=60, seed=21, noise=0.0, clusters=np.array([0, 0, 0, 1, 1, 1]))
    F0 = camera.cost(s.cameras, s.points, s.obs_cam, s.obs_pt, s.obs_uv)
    iters = 15 if method == "lm" else 60
    _, _, _, F, _ = stba.solve(s.cameras, s.points, s.obs_cam, s.obs_pt, s.obs_uv, s.clusters, iters,
                               method=method)
    assert F < 1e-10 * F0, (F, F0)


def test_noise_statistics_at_optimum():
    # with N(0,1) pixel noise, F* / (2q - dof) -> 1, dof = 9m + 3n - 7 (similarity gauge)
    s = scenes.make_ring_scene(m=12, n=300, clusters=2, seed=31)
    _, _, _, F, _ = stba.solve(s.cameras, s.points, s.obs_cam, s.obs_pt, s.obs_uv, s.clusters, 12, method="lm")
    dof = 9 * s.m + 3 * s.n - 7
    ratio = F / (2 * s.q - dof)
    assert 0.9 < ratio < 1.1, ratio


def test_stop_tests():
    opt = stba.Options(ftol=1e-6)
    assert stba.stop_tests(1.0, 1.0 - 1e-7, 1.0, 1.0, 1.0, opt)
    assert not stba.stop_tests(1.0, 0.9, 1.0, 1.0, 1.0, opt)
    assert stba.stop_tests(1.0, 0.9, 1e-7, 1.0, 1.0, stba.Options(gtol=1e-6))
    assert stba.stop_tests(1.0, 0.9, 1.0, 1e-7, 1.0, stba.Options(xtol=1e-6))
    assert not stba.stop_tests(1.0, 0.9, 1.0, 1e-5, 1.0, stba.Options(xtol=1e-6))


# ----------------------------------------------------------------------------------------------------------
# the corrected step (lambda >= 0.1): Alg. 1 feeds the corrected g' into b' of Eq. 10 and keeps the physical,
# uncorrected w for the point update of Eq. 15.  These pins rebuild J' densely in the test, so a mistake in
# either half of that composition (corrected w' summed into the point update through another route than its
# preserved per-point sums, the uncorrected w' in b', the virtual C' in Eq. 15) fails one of them.
# ----------------------------------------------------------------------------------------------------------
def dense_expanded_system(s, lin, lam):
    """J' = [J_c, J'_p] built densely from the per-observation blocks, H' = J'^T J' + lam diag(J'^T J'),
    g' = -J'^T f, and each virtual point's physical point (virtual points = distinct (point, cluster))."""
    key = s.obs_pt.astype(np.int64) * (int(s.clusters.max()) + 1) + s.clusters[s.obs_cam]
    uniq, vp = np.unique(key, return_inverse=True)
    vp_point = uniq // (int(s.clusters.max()) + 1)
    nv = len(uniq)
    Jd = np.zeros((2 * s.q, 9 * s.m + 3 * nv))
    for o in range(s.q):
        Jd[2 * o:2 * o + 2, 9 * s.obs_cam[o]:9 * s.obs_cam[o] + 9] = lin.Jc[o]
        Jd[2 * o:2 * o + 2, 9 * s.m + 3 * vp[o]:9 * s.m + 3 * vp[o] + 3] = lin.Jp[o]
    H = Jd.T @ Jd
    H = H + lam * np.diag(np.diag(H))
    return H, -Jd.T @ lin.f, vp_point


def corrected_rhs(g, Hdiag, vp_point, m):
    """Minimiser of sum_k (1/2 d^T H~_k d - g_k^T d) over equal d for every point's copies, per coordinate:
    d = sum_k g_k / sum_k H~_k, and the corrected g_k = H~_k d (the steepest-descent correction of Sec. 4.3
    with the multipliers of Eq. 9 eliminated by hand)."""
    out = g.copy()
    w = out[9 * m:].reshape(-1, 3)
    h = Hdiag[9 * m:].reshape(-1, 3)
    for i in np.unique(vp_point):
        sel = vp_point == i
        w[sel] = h[sel] * (w[sel].sum(0) / h[sel].sum(0))
    return out


@pytest.mark.parametrize("lam", [0.1, 0.5, 4.0])
@pytest.mark.parametrize("clusters", [[0, 1, 2, 0, 1, 2], [0, 0, 1, 1, 1, 0]])
def test_corrected_camera_step_solves_expanded_system_with_corrected_rhs(lam, clusters):
    # Alg. 1, correction branch: Delta c is the camera part of H'_lambda dx' = g'_corrected (Eq. 9 with nu
    # replaced by the correction), i.e. b' of Eq. 10 is formed from the corrected w'
    s = tiny(m=6, n=40, seed=17, clusters=clusters)
    lin = lin_of(s)
    st = stba.stba_step(lin, s.obs_cam, s.obs_pt, s.clusters, lam, use_correction=True)
    assert st["corrected"]
    H, g, vp_point = dense_expanded_system(s, lin, lam)
    gc = corrected_rhs(g, np.diag(H), vp_point, s.m)
    assert rel(gc, g) > 1e-6                      # the correction does change the right-hand side here
    dx_c = np.linalg.solve(H, gc)
    dx_u = np.linalg.solve(H, g)
    assert rel(st["dc"], dx_c[: 9 * s.m]) < 1e-9
    assert rel(st["dc"], dx_u[: 9 * s.m]) > 1e-6  # and it is not the uncorrected relaxed step


@pytest.mark.parametrize("lam", [0.1, 0.5, 4.0])
def test_corrected_point_update_is_eq15_with_physical_w(lam):
    # Eq. 15 (Alg. 1, last step): whatever Delta c the corrected system gives, Delta p minimises
    # ||J_p Delta p + f + J_c Delta c||^2 + lam ||D_p Delta p||^2 over the physical points, with the
    # physical (uncorrected) w = -J_p^T f and the physical damped C
    s = tiny(m=6, n=40, seed=19, clusters=[0, 1, 2, 0, 1, 2])
    lin = lin_of(s)
    st = stba.stba_step(lin, s.obs_cam, s.obs_pt, s.clusters, lam, use_correction=True)
    assert st["corrected"]
    Jp = np.zeros((2 * s.q, 3 * s.n))
    Jc = np.zeros((2 * s.q, 9 * s.m))
    for o in range(s.q):
        Jp[2 * o:2 * o + 2, 3 * s.obs_pt[o]:3 * s.obs_pt[o] + 3] = lin.Jp[o]
        Jc[2 * o:2 * o + 2, 9 * s.obs_cam[o]:9 * s.obs_cam[o] + 9] = lin.Jc[o]
    Dp = np.sqrt(np.sum(Jp * Jp, axis=0))
    A = np.vstack([Jp, np.sqrt(lam) * np.diag(Dp)])
    rhs = np.concatenate([-lin.f - Jc @ st["dc"], np.zeros(3 * s.n)])
    dp_ls = np.linalg.lstsq(A, rhs, rcond=None)[0]
    assert rel(st["dp"], dp_ls) < 1e-9
    # the per-cluster virtual-point steps of Eq. 14 (solved with the virtual C' and corrected w') differ
    H, g, vp_point = dense_expanded_system(s, lin, lam)
    dxv = np.linalg.solve(H, corrected_rhs(g, np.diag(H), vp_point, s.m))[9 * s.m:].reshape(-1, 3)
    first_copy = np.array([dxv[np.flatnonzero(vp_point == i)[0]] for i in range(s.n)])
    assert rel(first_copy.ravel(), st["dp"]) > 1e-6


def test_corrected_iteration_record_and_cost():
    # one full iteration with the correction: F(x + dx) is the cost at the corrected step, the record says
    # corrected, and lambda follows the x3 / /3 rule on that F
    s = tiny(m=6, n=40, seed=20, clusters=[0, 1, 2, 0, 1, 2])
    F0 = camera.cost(s.cameras, s.points, s.obs_cam, s.obs_pt, s.obs_uv)
    opt = stba.Options(lambda0=0.5)
    c, p, lam, F, rec = stba.lm_iteration(s.cameras, s.points, s.obs_cam, s.obs_pt, s.obs_uv, s.clusters, 0.5, F0,
                                          opt)
    assert rec["corrected"]
    F_new = camera.cost(s.cameras + rec["dc"], s.points + rec["dp"], s.obs_cam, s.obs_pt, s.obs_uv)
    assert rec["F_after"] == pytest.approx(F_new, rel=1e-12)
    assert lam == pytest.approx(0.5 / 3 if F_new < F0 else 1.5, rel=1e-15)
