"""Scene recipes for the STBA workloads.

Camera parameter layout (9 values per camera): angle-axis rotation w (3), translation t (3), focal length f,
radial distortion k1, k2.  A world point X maps to camera coordinates Xc = R(w) X + t (+z forward, x right,
y down), normalised coordinates (x, y) = Xc.xy / Xc.z, and the pixel offset from the image centre is
f (1 + k1 r^2 + k2 r^4) (x, y) with r^2 = x^2 + y^2.  Images are 640 x 480, so a point is inside the image
when |u| < 320 and |v| < 240.

Every recipe is seeded; the same arguments give the same arrays on any machine.  Observations are sorted by
(point, camera).  Pixel noise is N(0, 1) per coordinate; the initial cameras are the true ones rotated by a
random rotation with per-axis sigma 0.01 rad and translated by N(0, 0.05^2) per axis; the initial points are
the true ones plus N(0, 0.05^2) per axis.  f, k1 and k2 start at their true values.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
from scipy.spatial.transform import Rotation

HALF_W, HALF_H = 320.0, 240.0


@dataclasses.dataclass
class Scene:
    name: str
    cameras: np.ndarray        # (m, 9) float64, initial (perturbed) parameters
    points: np.ndarray         # (n, 3) float64, initial (perturbed) points
    cameras_true: np.ndarray   # (m, 9)
    points_true: np.ndarray    # (n, 3)
    obs_cam: np.ndarray        # (q,) int32
    obs_pt: np.ndarray         # (q,) int32
    obs_uv: np.ndarray         # (q, 2) float64, pixel offsets from the image centre
    clusters: np.ndarray       # (m,) int32, cluster id of every camera, ids 0..l-1
    meta: dict

    @property
    def m(self):
        return self.cameras.shape[0]

    @property
    def n(self):
        return self.points.shape[0]

    @property
    def q(self):
        return self.obs_cam.shape[0]


# ----------------------------------------------------------------------------------------------------------
# camera helpers (generation only)
# ----------------------------------------------------------------------------------------------------------
def look_at(centers: np.ndarray, target=np.zeros(3)) -> np.ndarray:
    """World-to-camera rotations (k, 3, 3) for cameras at `centers` looking at `target`, +z world up."""
    fwd = target[None, :] - centers
    fwd /= np.linalg.norm(fwd, axis=1, keepdims=True)
    up = np.tile(np.array([0.0, 0.0, 1.0]), (len(centers), 1))
    near_pole = np.abs(fwd[:, 2]) > 0.999
    up[near_pole] = np.array([0.0, 1.0, 0.0])
    right = np.cross(fwd, up)
    right /= np.linalg.norm(right, axis=1, keepdims=True)
    down = np.cross(fwd, right)
    return np.stack([right, down, fwd], axis=1)


def heading_rotation(fwd: np.ndarray) -> np.ndarray:
    """World-to-camera rotations for cameras facing the horizontal directions `fwd` (k, 3), +z up."""
    f = fwd / np.linalg.norm(fwd, axis=1, keepdims=True)
    up = np.tile(np.array([0.0, 0.0, 1.0]), (len(f), 1))
    right = np.cross(f, up)
    right /= np.linalg.norm(right, axis=1, keepdims=True)
    down = np.cross(f, right)
    return np.stack([right, down, f], axis=1)


def assemble_cameras(R: np.ndarray, centers: np.ndarray, f: np.ndarray, k1: np.ndarray, k2: np.ndarray):
    w = Rotation.from_matrix(R).as_rotvec()
    t = -np.einsum("kij,kj->ki", R, centers)
    return np.concatenate([w, t, f[:, None], k1[:, None], k2[:, None]], axis=1)


def synth_project(cams: np.ndarray, X: np.ndarray):
    """Pixel offsets and depths of points X (k, 3) seen by cameras cams (k, 9); one camera per point."""
    Xc = Rotation.from_rotvec(cams[:, 0:3]).apply(X) + cams[:, 3:6]
    z = Xc[:, 2]
    zs = np.where(np.abs(z) > 1e-12, z, 1e-12)
    xy = Xc[:, :2] / zs[:, None]
    r2 = np.sum(xy * xy, axis=1)
    d = 1.0 + cams[:, 7] * r2 + cams[:, 8] * r2 * r2
    return cams[:, 6, None] * d[:, None] * xy, z


def visible(uv: np.ndarray, z: np.ndarray, zmin=0.1) -> np.ndarray:
    return (z > zmin) & (np.abs(uv[:, 0]) < HALF_W) & (np.abs(uv[:, 1]) < HALF_H)


def draw_intrinsics(rng, m):
    f = rng.uniform(500.0, 1500.0, m)
    k1 = rng.normal(0.0, 0.01, m)
    k2 = rng.normal(0.0, 0.01, m)
    return f, k1, k2


def zipf_lengths(rng, n, s, lo, hi):
    k = np.arange(lo, hi + 1, dtype=np.float64)
    p = k ** (-s)
    p /= p.sum()
    return rng.choice(np.arange(lo, hi + 1), size=n, p=p)


def finish_scene(name, rng, cams_true, pts_true, obs_cam, obs_pt, clusters, meta, noise=1.0,
                 rot_sigma=0.01, trans_sigma=0.05, point_sigma=0.05, rotate_about_center=False):
    """Sorts the observations, synthesises noisy pixels and perturbs the initial parameters.  The rotation
    noise is composed on the world side of R (so it turns the scene about the world origin), or, with
    rotate_about_center, about each camera's own centre (t recomputed from the centre), as a large scene
    far from the origin needs."""
    order = np.lexsort((obs_cam, obs_pt))
    obs_cam = obs_cam[order].astype(np.int32)
    obs_pt = obs_pt[order].astype(np.int32)
    uv, z = synth_project(cams_true[obs_cam], pts_true[obs_pt])
    assert np.all(z > 0)
    obs_uv = uv + rng.normal(0.0, noise, uv.shape) if noise > 0 else uv.copy()
    m = len(cams_true)
    cams = cams_true.copy()
    if rot_sigma > 0:
        dR = Rotation.from_rotvec(rng.normal(0.0, rot_sigma, (m, 3)))
        R0 = Rotation.from_rotvec(cams_true[:, 0:3])
        R1 = dR * R0
        cams[:, 0:3] = R1.as_rotvec()
        if rotate_about_center:
            centers = -R0.inv().apply(cams_true[:, 3:6])
            cams[:, 3:6] = -R1.apply(centers)
    cams[:, 3:6] += rng.normal(0.0, trans_sigma, (m, 3)) if trans_sigma > 0 else 0.0
    pts = pts_true + (rng.normal(0.0, point_sigma, pts_true.shape) if point_sigma > 0 else 0.0)
    meta = dict(meta)
    meta.update(noise_px=noise, rot_sigma=rot_sigma, trans_sigma=trans_sigma, point_sigma=point_sigma)
    return Scene(name, cams, pts, cams_true, pts_true, obs_cam, obs_pt, obs_uv,
                 np.asarray(clusters, dtype=np.int32), meta)


# ----------------------------------------------------------------------------------------------------------
# clustering inputs (spatial, seeded); the stochastic graph clustering of the paper is a separate component
# ----------------------------------------------------------------------------------------------------------
def cluster_contiguous(sizes) -> np.ndarray:
    return np.repeat(np.arange(len(sizes)), sizes).astype(np.int32)


def cluster_by_azimuth(centers: np.ndarray, max_size: int, phase: float = 0.0) -> np.ndarray:
    """Cut cameras into ceil(m / max_size) wedges of nearly equal size by azimuth (starting at `phase`)."""
    m = len(centers)
    l = max(1, math.ceil(m / max_size))
    az = np.mod(np.arctan2(centers[:, 1], centers[:, 0]) - phase, 2 * np.pi)
    order = np.lexsort((centers[:, 2], az))
    sizes = np.full(l, m // l)
    sizes[: m % l] += 1
    out = np.empty(m, dtype=np.int32)
    out[order] = np.repeat(np.arange(l), sizes)
    return out


def camera_centers(cams: np.ndarray) -> np.ndarray:
    R = Rotation.from_rotvec(cams[:, 0:3]).as_matrix()
    return -np.einsum("kji,kj->ki", R, cams[:, 3:6])


def cluster_sequence(scene: Scene, iters: int, seed: int) -> np.ndarray:
    """A seeded sequence of cluster assignments (iters, m): azimuth wedges with a random phase per iteration.

    Ring and hemisphere scenes only; other scenes repeat their own assignment."""
    rng = np.random.default_rng(seed)
    kind = scene.meta.get("kind")
    if kind not in ("ring", "hemisphere"):
        return np.tile(scene.clusters, (iters, 1))
    C = camera_centers(scene.cameras_true)
    cap = scene.meta["max_cluster"]
    return np.stack([cluster_by_azimuth(C, cap, rng.uniform(0, 2 * np.pi)) for _ in range(iters)])


# ----------------------------------------------------------------------------------------------------------
# recipes
# ----------------------------------------------------------------------------------------------------------
def make_ring_scene(m=30, n=2000, radius=10.0, half=2.0, max_angle_deg=60.0, clusters=3, seed=1000,
                    noise=1.0):
    """Cameras on a ring in the z = 0 plane looking at the origin; points uniform in a cube.

    A camera sees a point when the angle between the point's outward direction p/|p| and the direction
    from the point to the camera is at most `max_angle_deg`, and the point projects inside the image.
    Points seen by fewer than two cameras are redrawn."""
    rng = np.random.default_rng(seed)
    phi = 2 * np.pi * np.arange(m) / m
    C = np.stack([radius * np.cos(phi), radius * np.sin(phi), np.zeros(m)], axis=1)
    f, k1, k2 = draw_intrinsics(rng, m)
    cams_true = assemble_cameras(look_at(C), C, f, k1, k2)
    cos_max = math.cos(math.radians(max_angle_deg))
    pts, oc, op = [], [], []
    while len(pts) < n:
        P = rng.uniform(-half, half, (4 * (n - len(pts)) + 16, 3))
        pc = np.repeat(np.arange(len(P)), m)
        cc = np.tile(np.arange(m), len(P))
        uv, z = synth_project(cams_true[cc], P[pc])
        to_cam = C[cc] - P[pc]
        cosang = np.sum(P[pc] * to_cam, 1) / (np.linalg.norm(P[pc], axis=1) * np.linalg.norm(to_cam, axis=1) + 1e-300)
        ok = visible(uv, z) & (cosang >= cos_max)
        cnt = np.bincount(pc[ok], minlength=len(P))
        for i in np.nonzero(cnt >= 2)[0]:
            if len(pts) >= n:
                break
            sel = ok[i * m:(i + 1) * m]
            oc.append(np.nonzero(sel)[0])
            op.append(np.full(sel.sum(), len(pts)))
            pts.append(P[i])
    pts_true = np.array(pts)
    obs_cam = np.concatenate(oc)
    obs_pt = np.concatenate(op)
    sizes = np.full(clusters, m // clusters)
    sizes[: m % clusters] += 1
    meta = dict(kind="ring", seed=seed, max_cluster=int(sizes.max()))
    return finish_scene("ring", rng, cams_true, pts_true, obs_cam, obs_pt, cluster_contiguous(sizes), meta,
                        noise=noise)


def make_hemisphere_scene(m=1000, n=200_000, radius=20.0, half=5.0, zipf_s=2.0, lmin=2, lmax=50,
                          max_cluster=100, seed=1001, noise=1.0, name="hemisphere", tracks="local"):
    """Cameras uniform on the upper hemisphere looking at the origin; points uniform in a cube; Zipf tracks.

    Each point draws a track length L ~ Zipf(s) on [lmin, lmax].  tracks="local" (Internet photo collections:
    a point is matched across nearby viewpoints): an anchor camera is drawn uniformly and the track takes the
    first L cameras that see the point (in front, inside the image) in order of distance from the anchor.
    tracks="uniform": the first L cameras that see it from a uniformly random candidate sequence.  A point
    with fewer than two such cameras is redrawn."""
    if tracks == "local":
        return _hemisphere_local(m, n, radius, half, zipf_s, lmin, lmax, max_cluster, seed, noise, name)
    rng = np.random.default_rng(seed)
    cz = rng.uniform(0.0, 1.0, m)
    phi = rng.uniform(0.0, 2 * np.pi, m)
    sz = np.sqrt(1.0 - cz * cz)
    C = radius * np.stack([sz * np.cos(phi), sz * np.sin(phi), cz], axis=1)
    f, k1, k2 = draw_intrinsics(rng, m)
    cams_true = assemble_cameras(look_at(C), C, f, k1, k2)
    Rm = Rotation.from_rotvec(cams_true[:, 0:3]).as_matrix()
    tv = cams_true[:, 3:6]

    pts_list, oc_list, op_list = [], [], []
    count = 0
    while count < n:
        need = n - count
        P = rng.uniform(-half, half, (need, 3))
        L = zipf_lengths(rng, need, zipf_s, lmin, lmax)
        keep_pt = np.zeros(need, dtype=bool)
        tracks_c, tracks_p = [], []
        for Lv in np.unique(L):
            idx = np.nonzero(L == Lv)[0]
            K = int(min(m, 2 * Lv + 12)) if m > 4 * Lv else m
            for s in range(0, len(idx), 20000):
                ii = idx[s:s + 20000]
                if K == m:
                    cand = np.argsort(rng.random((len(ii), m)), axis=1)
                else:
                    cand = rng.integers(0, m, (len(ii), K))
                    o = np.argsort(cand, axis=1, kind="stable")
                    srt = np.take_along_axis(cand, o, 1)
                    dup_s = np.zeros_like(srt, dtype=bool)
                    dup_s[:, 1:] = srt[:, 1:] == srt[:, :-1]
                    dup = np.empty_like(dup_s)
                    np.put_along_axis(dup, o, dup_s, 1)
                Xp = P[ii]
                Xc = np.einsum("pkij,pj->pki", Rm[cand], Xp) + tv[cand]
                z = Xc[..., 2]
                xy = Xc[..., :2] / np.where(z > 1e-9, z, 1e-9)[..., None]
                r2 = np.sum(xy * xy, -1)
                d = 1.0 + k1[cand] * r2 + k2[cand] * r2 * r2
                uv = f[cand][..., None] * d[..., None] * xy
                ok = (z > 0.1) & (np.abs(uv[..., 0]) < HALF_W) & (np.abs(uv[..., 1]) < HALF_H)
                if K != m:
                    ok &= ~dup
                take = ok & (np.cumsum(ok, axis=1) <= Lv)
                cnt = take.sum(1)
                good = cnt >= 2
                keep_pt[ii[good]] = True
                rows, cols = np.nonzero(take & good[:, None])
                tracks_p.append(ii[rows])
                tracks_c.append(cand[rows, cols])
        tp = np.concatenate(tracks_p)
        tc = np.concatenate(tracks_c)
        newid = np.cumsum(keep_pt) - 1 + count
        sel = np.nonzero(keep_pt)[0][: n - count]
        mask_pt = np.zeros(need, dtype=bool)
        mask_pt[sel] = True
        keep_obs = mask_pt[tp]
        pts_list.append(P[sel])
        op_list.append(newid[tp[keep_obs]])
        oc_list.append(tc[keep_obs])
        count += len(sel)
    pts_true = np.concatenate(pts_list)
    obs_pt = np.concatenate(op_list)
    obs_cam = np.concatenate(oc_list)
    clusters = cluster_by_azimuth(C, max_cluster)
    meta = dict(kind="hemisphere", seed=seed, max_cluster=max_cluster, zipf=(zipf_s, lmin, lmax))
    return finish_scene(name, rng, cams_true, pts_true, obs_cam, obs_pt, clusters, meta, noise=noise)


def _hemisphere_cameras(rng, m, radius):
    cz = rng.uniform(0.0, 1.0, m)
    phi = rng.uniform(0.0, 2 * np.pi, m)
    sz = np.sqrt(1.0 - cz * cz)
    C = radius * np.stack([sz * np.cos(phi), sz * np.sin(phi), cz], axis=1)
    f, k1, k2 = draw_intrinsics(rng, m)
    return C, assemble_cameras(look_at(C), C, f, k1, k2)


def _hemisphere_local(m, n, radius, half, zipf_s, lmin, lmax, max_cluster, seed, noise, name):
    rng = np.random.default_rng(seed)
    C, cams_true = _hemisphere_cameras(rng, m, radius)
    Rm = Rotation.from_rotvec(cams_true[:, 0:3]).as_matrix()
    tv = cams_true[:, 3:6]
    f, k1, k2 = cams_true[:, 6], cams_true[:, 7], cams_true[:, 8]
    K = int(min(m, 4 * lmax))
    # K nearest cameras of every camera (itself first), by centre distance, in blocks
    nn = np.empty((m, K), dtype=np.int64)
    for s0 in range(0, m, 2048):
        d2 = np.sum((C[s0:s0 + 2048, None, :] - C[None, :, :]) ** 2, -1)
        part = np.argpartition(d2, K - 1, axis=1)[:, :K]
        order = np.argsort(np.take_along_axis(d2, part, 1), axis=1, kind="stable")
        nn[s0:s0 + 2048] = np.take_along_axis(part, order, 1)
    pts_list, oc_list, op_list = [], [], []
    count = 0
    while count < n:
        need = min(n - count, 50_000)
        P = rng.uniform(-half, half, (need, 3))
        L = zipf_lengths(rng, need, zipf_s, lmin, lmax)
        cand = nn[rng.integers(0, m, need)]                       # (need, K), nearest first
        Xc = np.einsum("pkij,pj->pki", Rm[cand], P) + tv[cand]
        z = Xc[..., 2]
        xy = Xc[..., :2] / np.where(z > 1e-9, z, 1e-9)[..., None]
        r2 = np.sum(xy * xy, -1)
        d = 1.0 + k1[cand] * r2 + k2[cand] * r2 * r2
        uv = f[cand][..., None] * d[..., None] * xy
        ok = (z > 0.1) & (np.abs(uv[..., 0]) < HALF_W) & (np.abs(uv[..., 1]) < HALF_H)
        take = ok & (np.cumsum(ok, axis=1) <= L[:, None])
        good = take.sum(1) >= 2
        sel = np.nonzero(good)[0][: n - count]
        rows, cols = np.nonzero(take[sel])
        pts_list.append(P[sel])
        op_list.append(count + rows)
        oc_list.append(cand[sel][rows, cols])
        count += len(sel)
    pts_true = np.concatenate(pts_list)
    obs_pt = np.concatenate(op_list)
    obs_cam = np.concatenate(oc_list)
    clusters = cluster_by_azimuth(C, max_cluster)
    meta = dict(kind="hemisphere", seed=seed, max_cluster=max_cluster, zipf=(zipf_s, lmin, lmax), tracks="local")
    return finish_scene(name, rng, cams_true, pts_true, obs_cam, obs_pt, clusters, meta, noise=noise)


def trefoil_path(s):
    """Closed planar curve with three self-crossings, parametrised by s in [0, 2 pi)."""
    return np.stack([np.sin(s) + 2.0 * np.sin(2.0 * s), np.cos(s) - 2.0 * np.cos(2.0 * s)], axis=-1)


# Forward-moving frames pass close to the points they tracked; a minimum depth of 1 m at the true poses keeps
# every observed point in front of its camera after the initial perturbation (0.01 rad at up to 30 m).
SLAM_ZMIN = 1.0


def make_slam_scene(m=5000, n=500_000, length=2000.0, lmin=2, lmax=20, reach=30.0, cmin=20, cmax=300,
                    seed=1002, noise=1.0, height=1.5):
    """Forward-facing cameras at equal spacing along a closed 2D trajectory with three self-crossings.

    Each point is placed in front of a frame at a depth up to `reach`, then tracked by a run of L ~ U[lmin,
    lmax] consecutive frames (cut where it leaves the image; at least two).  Points near the crossings are
    also observed by up to L frames of the other pass that see them (loop closures).  Clusters are
    contiguous runs of frames with sizes drawn uniformly in [cmin, cmax]."""
    rng = np.random.default_rng(seed)
    ss = np.linspace(0, 2 * np.pi, 200_001)
    xy = trefoil_path(ss)
    seg = np.linalg.norm(np.diff(xy, axis=0), axis=1)
    arc = np.concatenate([[0.0], np.cumsum(seg)])
    scale = length / arc[-1]
    targets = np.arange(m) * (arc[-1] / m)
    s_cam = np.interp(targets, arc, ss)
    P2 = trefoil_path(s_cam) * scale
    ds = 1e-4
    tan = (trefoil_path(s_cam + ds) - trefoil_path(s_cam - ds))
    C = np.concatenate([P2, np.full((m, 1), height)], axis=1)
    fwd = np.concatenate([tan, np.zeros((m, 1))], axis=1)
    f, k1, k2 = draw_intrinsics(rng, m)
    cams_true = assemble_cameras(heading_rotation(fwd), C, f, k1, k2)
    Rm = Rotation.from_rotvec(cams_true[:, 0:3]).as_matrix()

    def proj(ci, X):
        Xc = np.einsum("kij,kj->ki", Rm[ci], X) + cams_true[ci, 3:6]
        z = Xc[:, 2]
        xyn = Xc[:, :2] / np.where(z > 1e-9, z, 1e-9)[:, None]
        r2 = np.sum(xyn * xyn, 1)
        d = 1.0 + cams_true[ci, 7] * r2 + cams_true[ci, 8] * r2 * r2
        return cams_true[ci, 6, None] * d[:, None] * xyn, z

    pts, oc, op = [], [], []
    count = 0
    while count < n:
        need = n - count
        a = rng.integers(0, m, need)                      # anchor frame
        depth = rng.uniform(4.0, reach, need)
        uvn = rng.uniform(-0.8, 0.8, (need, 2)) * np.array([HALF_W, HALF_H])
        Xc = np.stack([uvn[:, 0] / f[a] * depth, uvn[:, 1] / f[a] * depth, depth], axis=1)
        X = np.einsum("kji,kj->ki", Rm[a], Xc - cams_true[a, 3:6])
        L = rng.integers(lmin, lmax + 1, need)
        start = a - rng.integers(0, L)                    # the run covers the anchor frame
        obs_c, obs_p = [], []
        for j in range(lmax):
            cj = np.mod(start + j, m)
            act = j < L
            uv, z = proj(cj, X)
            vis = act & visible(uv, z, zmin=SLAM_ZMIN)
            obs_c.append(np.where(vis, cj, -1))
        oc_mat = np.stack(obs_c, axis=1)
        good = (oc_mat >= 0).sum(1) >= 2
        # loop closures: frames of another pass within reach of the point
        d2 = np.sum((P2[None, :, :] - X[good][:, None, :2]) ** 2, -1) if False else None
        gi = np.nonzero(good)[0]
        sel = gi[: need]
        for k, i in enumerate(sel):
            cams_i = oc_mat[i][oc_mat[i] >= 0]
            pts.append(X[i])
            oc.append(cams_i)
            op.append(np.full(len(cams_i), count + k))
        count += len(sel)
    pts_true = np.array(pts)
    obs_cam = np.concatenate(oc)
    obs_pt = np.concatenate(op)
    # loop closures: for points within `reach` of a frame of another pass, add that pass's visible frames
    obs_cam, obs_pt = add_revisit_observations(rng, P2, pts_true, obs_cam, obs_pt, proj, m, reach, lmax)
    sizes = []
    tot = 0
    while tot < m:
        s = int(rng.integers(cmin, cmax + 1))
        s = min(s, m - tot)
        sizes.append(s)
        tot += s
    if len(sizes) > 1 and sizes[-1] < cmin:
        sizes[-2] += sizes[-1]
        sizes.pop()
    meta = dict(kind="slam", seed=seed, max_cluster=int(max(sizes)), cluster_sizes=sizes)
    return finish_scene("slam", rng, cams_true, pts_true, obs_cam, obs_pt, cluster_contiguous(sizes), meta,
                        noise=noise, rotate_about_center=True)


def add_revisit_observations(rng, P2, pts, obs_cam, obs_pt, proj, m, reach, lmax):
    """Second tracks at the self-crossings: frames far along the path from the point's own frames that see it."""
    first = np.full(len(pts), m, dtype=np.int64)
    np.minimum.at(first, obs_pt, obs_cam)
    # candidate frames: nearest frame (in the plane) that is at least 10% of the path away from `first`
    from scipy.spatial import cKDTree
    tree = cKDTree(P2)
    near = tree.query_ball_point(pts[:, :2], r=reach * 0.6)
    add_c, add_p = [], []
    gap = m // 10
    for i, lst in enumerate(near):
        if not lst:
            continue
        lst = np.asarray(lst)
        dist = np.abs(lst - first[i])
        dist = np.minimum(dist, m - dist)
        other = lst[dist > gap]
        if len(other) == 0:
            continue
        other = np.sort(other)[:lmax]
        uv, z = proj(other, np.repeat(pts[i][None], len(other), 0))
        vis = other[visible(uv, z, zmin=SLAM_ZMIN)]
        if len(vis) >= 2:
            add_c.append(vis)
            add_p.append(np.full(len(vis), i))
    if add_c:
        obs_cam = np.concatenate([obs_cam] + add_c)
        obs_pt = np.concatenate([obs_pt] + add_p)
    return obs_cam, obs_pt


def make_tiny_scene(m=5, n=30, seed=7, clusters=None, noise=1.0, radius=10.0, half=1.0, min_obs=2,
                    rot_sigma=0.01, trans_sigma=0.05, point_sigma=0.05, drop=0.3):
    """A small hemisphere-style scene for brute-force checks: every point is seen by a random subset
    (at least `min_obs`) of the cameras that see it."""
    rng = np.random.default_rng(seed)
    cz = rng.uniform(0.3, 1.0, m)
    phi = rng.uniform(0, 2 * np.pi, m)
    sz = np.sqrt(1 - cz * cz)
    C = radius * np.stack([sz * np.cos(phi), sz * np.sin(phi), cz], axis=1)
    f, k1, k2 = draw_intrinsics(rng, m)
    cams_true = assemble_cameras(look_at(C), C, f, k1, k2)
    pts, oc, op = [], [], []
    while len(pts) < n:
        X = rng.uniform(-half, half, 3)
        uv, z = synth_project(cams_true, np.repeat(X[None], m, 0))
        vis = np.nonzero(visible(uv, z))[0]
        keep = vis[rng.random(len(vis)) >= drop]
        if len(keep) < min_obs:
            continue
        oc.append(keep)
        op.append(np.full(len(keep), len(pts)))
        pts.append(X)
    if clusters is None:
        clusters = np.zeros(m, dtype=np.int32)
    meta = dict(kind="tiny", seed=seed, max_cluster=m)
    return finish_scene("tiny", rng, cams_true, np.array(pts), np.concatenate(oc), np.concatenate(op),
                        clusters, meta, noise=noise, rot_sigma=rot_sigma, trans_sigma=trans_sigma,
                        point_sigma=point_sigma)


def subscene(scene: Scene, cams_keep, max_points=None, seed=0) -> Scene:
    """Restrict a scene to a subset of cameras and the points those cameras see at least twice."""
    cams_keep = np.asarray(sorted(cams_keep))
    newc = np.full(scene.m, -1, dtype=np.int64)
    newc[cams_keep] = np.arange(len(cams_keep))
    sel = newc[scene.obs_cam] >= 0
    cnt = np.bincount(scene.obs_pt[sel], minlength=scene.n)
    ptk = np.nonzero(cnt >= 2)[0]
    if max_points is not None and len(ptk) > max_points:
        ptk = np.sort(np.random.default_rng(seed).choice(ptk, max_points, replace=False))
    newp = np.full(scene.n, -1, dtype=np.int64)
    newp[ptk] = np.arange(len(ptk))
    sel &= newp[scene.obs_pt] >= 0
    cl = scene.clusters[cams_keep]
    _, cl = np.unique(cl, return_inverse=True)
    return Scene(scene.name + "_sub", scene.cameras[cams_keep].copy(), scene.points[ptk].copy(),
                 scene.cameras_true[cams_keep].copy(), scene.points_true[ptk].copy(),
                 newc[scene.obs_cam[sel]].astype(np.int32), newp[scene.obs_pt[sel]].astype(np.int32),
                 scene.obs_uv[sel].copy(), cl.astype(np.int32), dict(scene.meta))


# name -> (builder, kwargs, precision, LM iterations)
CONFIGS = {
    "c0_ring": (make_ring_scene, dict(m=30, n=2000, seed=1000), "fp64", 10),
    "c1_internet": (make_hemisphere_scene, dict(m=1000, n=200_000, radius=20.0, half=5.0, lmax=50,
                                               max_cluster=100, seed=1001, name="internet"), "mixed", 10),
    "c2_slam": (make_slam_scene, dict(m=5000, n=500_000, seed=1002), "mixed", 10),
    "c3_diff": (make_hemisphere_scene, dict(m=500, n=50_000, radius=20.0, half=5.0, lmax=50,
                                           max_cluster=100, seed=1003, name="diff"), "mixed", 5),
    "c4_large": (make_hemisphere_scene, dict(m=20_000, n=4_000_000, radius=60.0, half=15.0, lmax=80,
                                            max_cluster=100, seed=1004, name="large"), "mixed", 10),
}


def make_config(name: str, **overrides) -> Scene:
    builder, kw, _, _ = CONFIGS[name]
    kw = dict(kw)
    kw.update(overrides)
    return builder(**kw)
