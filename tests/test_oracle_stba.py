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
