"""Seeded synthetic bundle-adjustment scenes.

This module is the data recipe shared by the tests, the benchmark and the
oracle's tests.  It holds none of the solver's arithmetic: it draws ground-truth
cameras and points, decides which camera sees which point, synthesises the
pixel observations with a forward projection written in rotation-matrix form
(scipy's ``Rotation`` converts matrices to angle-axis), adds pixel noise and
perturbs the parameters to give the starting point of the optimisation.

The paper generates street-view scenes from a 3D city model (Section 4) that is
not available here; these generators stand in for them with the same kind of
visibility structure: a ring of cameras around an object, a street chain, a
city grid and a loop with cross links.  Camera parameters follow the
9-parameter angle-axis / translation / focal / k1 / k2 convention of the
Bundle Adjustment in the Large datasets (Section 4): a camera looks down its
-z axis, ``P = R X + t``, ``p = -P_xy / P_z``, ``pi = f (1 + k1 |p|^2 + k2 |p|^4) p``.

Observations come out in a shuffled order and points in a shuffled order, so
consumers cannot rely on any sortedness of the input.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
from scipy.spatial.transform import Rotation


@dataclass
class Scene:
    name: str
    n_cams: int
    n_pts: int
    n_obs: int
    cam_idx: np.ndarray      # int32 [n_obs]
    pt_idx: np.ndarray       # int32 [n_obs]
    obs: np.ndarray          # float64 [n_obs, 2] pixel observations
    cams: np.ndarray         # float64 [n_cams, 9] starting (perturbed) cameras
    pts: np.ndarray          # float64 [n_pts, 3] starting (perturbed) points
    cams_true: np.ndarray
    pts_true: np.ndarray
    lam: float               # LM damping of the first step
    rtol: float              # PCG relative-residual target


def _look_rotation(forward: np.ndarray, up=np.array([0.0, 0.0, 1.0])) -> np.ndarray:
    """World-to-camera rotations whose camera -z axis points along ``forward``.

    forward: [n, 3].  Rows of each returned matrix are the camera axes in world
    coordinates (x right, y up, z backwards)."""
    fwd = forward / np.linalg.norm(forward, axis=1, keepdims=True)
    z = -fwd
    x = np.cross(up[None, :], z)
    x /= np.linalg.norm(x, axis=1, keepdims=True)
    y = np.cross(z, x)
    return np.stack([x, y, z], axis=1)


def _forward_project(Rm, t, f, k1, k2, X):
    """Pixel coordinates and camera-frame depth of world points X (all [n, ...])."""
    P = np.einsum("nij,nj->ni", Rm, X) + t
    p = -P[:, :2] / P[:, 2:3]
    r2 = np.sum(p * p, axis=1)
    d = 1.0 + k1 * r2 + k2 * r2 * r2
    return (f * d)[:, None] * p, P[:, 2]


def _intrinsics(rng, n):
    f = rng.uniform(450.0, 550.0, n)
    k1 = rng.normal(0.0, 1e-3, n)
    k2 = rng.normal(0.0, 1e-3, n)
    return f, k1, k2


def _assemble(name, rng, Rm, centres, f, k1, k2, X, cam_idx, pt_idx, sigma,
              rel_pert, trans_pert, point_pert, lam, rtol, drift=None, outlier_frac=0.0,
              outlier_px=30.0) -> Scene:
    """Project, add noise, perturb, shuffle; returns a Scene.  outlier_frac > 0 gives that
    fraction of the observations an extra N(0, outlier_px^2) error (wrong correspondences,
    the outliers of Section 5's robust-loss experiment)."""
    n_c = Rm.shape[0]
    n_p = X.shape[0]
    t = -np.einsum("nij,nj->ni", Rm, centres)
    uv, depth = _forward_project(Rm[cam_idx], t[cam_idx], f[cam_idx], k1[cam_idx],
                                 k2[cam_idx], X[pt_idx])
    if np.any(depth >= -1e-3):
        raise ValueError("generator produced a point behind a camera")
    obs = uv + rng.normal(0.0, sigma, uv.shape)
    if outlier_frac > 0.0:
        orng = np.random.default_rng(int(rng.integers(2**62)))
        bad = orng.random(len(obs)) < outlier_frac
        obs[bad] += orng.normal(0.0, outlier_px, (int(bad.sum()), 2))
    rvec = Rotation.from_matrix(Rm).as_rotvec()
    cams_true = np.concatenate([rvec, t, f[:, None], k1[:, None], k2[:, None]], axis=1)

    # starting point: 1% multiplicative noise on rotations and intrinsics,
    # additive noise on camera centres and points, optional long-range drift
    c_pert = centres + trans_pert * rng.normal(size=centres.shape)
    X_pert = X + point_pert * rng.normal(size=X.shape)
    if drift is not None:
        c_pert = c_pert + drift(centres)
        X_pert = X_pert + drift(X)
    r_pert = rvec * (1.0 + rel_pert * rng.normal(size=rvec.shape))
    R_pert = Rotation.from_rotvec(r_pert).as_matrix()
    t_pert = -np.einsum("nij,nj->ni", R_pert, c_pert)
    intr = cams_true[:, 6:9] * (1.0 + rel_pert * rng.normal(size=(n_c, 3)))
    cams = np.concatenate([r_pert, t_pert, intr], axis=1)

    # shuffle point ids and observation order
    pperm = rng.permutation(n_p)            # new id of old point
    inv = np.empty(n_p, dtype=np.int64)
    inv[pperm] = np.arange(n_p)
    pts_true = np.empty_like(X)
    pts_true[pperm] = X
    pts = np.empty_like(X_pert)
    pts[pperm] = X_pert
    pt_new = pperm[pt_idx]
    operm = rng.permutation(len(cam_idx))
    return Scene(name=name, n_cams=n_c, n_pts=n_p, n_obs=len(cam_idx),
                 cam_idx=np.ascontiguousarray(cam_idx[operm], dtype=np.int32),
                 pt_idx=np.ascontiguousarray(pt_new[operm], dtype=np.int32),
                 obs=np.ascontiguousarray(obs[operm]),
                 cams=np.ascontiguousarray(cams), pts=np.ascontiguousarray(pts),
                 cams_true=cams_true, pts_true=pts_true, lam=lam, rtol=rtol)


def ring(seed=0, n_cams=32, n_pts=4000, kmin=4, kmax=8, radius=10.0, sigma=0.5,
         lam=1e-4, rtol=1e-8, outlier_frac=0.0) -> Scene:
    """Cameras on a ring of ``radius`` looking at points uniform in [-2, 2]^3;
    each point is seen by kmin..kmax random cameras (tiny plain FP64 scene)."""
    rng = np.random.default_rng(seed)
    ang = 2 * np.pi * np.arange(n_cams) / n_cams
    centres = np.stack([radius * np.cos(ang), radius * np.sin(ang),
                        0.5 * np.sin(3 * ang)], axis=1)
    Rm = _look_rotation(-centres)
    f, k1, k2 = _intrinsics(rng, n_cams)
    X = rng.uniform(-2.0, 2.0, (n_pts, 3))
    k = rng.integers(kmin, kmax + 1, n_pts)
    cam_idx, pt_idx = [], []
    for p in range(n_pts):
        cs = rng.choice(n_cams, size=k[p], replace=False)
        cam_idx.append(np.sort(cs))
        pt_idx.append(np.full(k[p], p))
    cam_idx = np.concatenate(cam_idx)
    pt_idx = np.concatenate(pt_idx)
    return _assemble("ring", rng, Rm, centres, f, k1, k2, X, cam_idx, pt_idx, sigma,
                     rel_pert=0.01, trans_pert=0.01 * radius, point_pert=0.01 * radius * 0.2,
                     lam=lam, rtol=rtol, outlier_frac=outlier_frac)


def _path(n, spacing, wiggle_amp, wiggle_len, rng):
    """A gently curving 2D polyline with ``n`` samples ``spacing`` apart."""
    s = np.arange(n) * spacing
    heading = wiggle_amp * np.sin(2 * np.pi * s / wiggle_len)
    d = np.stack([np.cos(heading), np.sin(heading)], axis=1)
    xy = np.concatenate([np.zeros((1, 2)), np.cumsum(d[:-1] * spacing, axis=0)])
    return xy, heading


def street_chain(seed=0, n_cams=2000, n_pts=300_000, sigma=1.0, lam=1e-4,
                 rtol=1e-6) -> Scene:
    """Forward-looking cameras along a 1D street; each facade point is seen by
    2..12 consecutive cameras (mean 5).  Poorly conditioned chain."""
    rng = np.random.default_rng(seed)
    xy, heading = _path(n_cams, 1.0, 0.25, 400.0, rng)
    yaw = heading + np.deg2rad(rng.uniform(-4, 4, n_cams))
    centres = np.concatenate([xy, np.full((n_cams, 1), 2.0)], axis=1)
    fwd = np.stack([np.cos(yaw), np.sin(yaw), np.zeros(n_cams)], axis=1)
    Rm = _look_rotation(fwd)
    f, k1, k2 = _intrinsics(rng, n_cams)
    k = np.clip(2 + rng.binomial(10, 0.3, n_pts), 2, 12)
    j0 = (rng.random(n_pts) * (n_cams - k + 1)).astype(np.int64)
    last = j0 + k - 1
    # point ahead of the last camera that sees it, on a facade on either side
    ahead = rng.uniform(6.0, 12.0, n_pts)
    side = np.where(rng.random(n_pts) < 0.5, -1.0, 1.0) * rng.uniform(4.5, 5.5, n_pts)
    hd = heading[last]
    tang = np.stack([np.cos(hd), np.sin(hd)], axis=1)
    left = np.stack([-np.sin(hd), np.cos(hd)], axis=1)
    pxy = xy[last] + ahead[:, None] * tang + side[:, None] * left
    X = np.concatenate([pxy, rng.uniform(0.2, 6.0, (n_pts, 1))], axis=1)
    cam_idx = (j0[:, None] + np.arange(12)[None, :])
    mask = np.arange(12)[None, :] < k[:, None]
    pt_idx = np.broadcast_to(np.arange(n_pts)[:, None], cam_idx.shape)
    cam_idx = cam_idx[mask]
    pt_idx = pt_idx[mask]
    return _assemble("street_chain", rng, Rm, centres, f, k1, k2, X, cam_idx, pt_idx,
                     sigma, rel_pert=0.01, trans_pert=0.05, point_pert=0.05,
                     lam=lam, rtol=rtol)


def city_grid(seed=0, rows=100, cols=200, n_pts=4_000_000, kmin=2, kmax=15,
              spacing=10.0, sigma=1.0, lam=1e-4, rtol=1e-6, batch=500_000) -> Scene:
    """One camera per street-grid node with a random heading; facade points near
    the streets, each seen by kmin..kmax nearby cameras.  Long-range drift that
    grows with distance from the origin plus a sine-wave component is added to
    the starting point (Section 4 and the scaling experiment of Section 5)."""
    rng = np.random.default_rng(seed)
    n_cams = rows * cols
    gy, gx = np.divmod(np.arange(n_cams), cols)
    centres = np.stack([gx * spacing, gy * spacing, np.full(n_cams, 2.0)], axis=1)
    yaw = rng.uniform(0, 2 * np.pi, n_cams)
    fwd = np.stack([np.cos(yaw), np.sin(yaw), np.zeros(n_cams)], axis=1)
    Rm = _look_rotation(fwd)
    f, k1, k2 = _intrinsics(rng, n_cams)
    t = -np.einsum("nij,nj->ni", Rm, centres)
    offs = np.array([(dy, dx) for dy in range(-2, 3) for dx in range(-2, 3)])
    Xs, cams_l, pts_l = [], [], []
    made = 0
    while made < n_pts:
        m = min(batch, n_pts - made) * 2
        # points near the street lines: either on an x-street or a y-street
        host = rng.integers(0, n_cams, m)
        hy, hx = np.divmod(host, cols)
        along = rng.uniform(-0.5, 0.5, m) * spacing
        across = np.where(rng.random(m) < 0.5, -1, 1) * rng.uniform(2.5, 3.5, m)
        horiz = rng.random(m) < 0.5
        px = hx * spacing + np.where(horiz, along, across)
        py = hy * spacing + np.where(horiz, across, along)
        pz = rng.uniform(0.5, 8.0, m)
        X = np.stack([px, py, pz], axis=1)
        cy = hy[:, None] + offs[None, :, 0]
        cx = hx[:, None] + offs[None, :, 1]
        valid = (cy >= 0) & (cy < rows) & (cx >= 0) & (cx < cols)
        cand = np.where(valid, cy * cols + cx, 0)
        P = np.einsum("mkij,mj->mki", Rm[cand], X) + t[cand]
        pz_c = P[..., 2]
        with np.errstate(divide="ignore", invalid="ignore"):
            u = -P[..., 0] / pz_c
            v = -P[..., 1] / pz_c
            dist = np.linalg.norm(X[:, None, :] - centres[cand], axis=2)
            vis = valid & (pz_c < -1.0) & (np.abs(u) < 1.2) & (np.abs(v) < 1.2) & (dist < 25.0)
        nvis = vis.sum(axis=1)
        want = np.clip(kmin + rng.binomial(kmax - kmin, 0.25, m), kmin, kmax)
        k = np.minimum(want, nvis)
        keep = k >= kmin
        X, vis, cand, k = X[keep], vis[keep], cand[keep], k[keep]
        take = min(len(X), n_pts - made)
        X, vis, cand, k = X[:take], vis[:take], cand[:take], k[:take]
        # choose k visible candidates at random: random keys, visible first
        key = np.where(vis, rng.random(vis.shape), 2.0)
        order = np.argsort(key, axis=1)
        sel = np.take_along_axis(cand, order, axis=1)
        mask = np.arange(sel.shape[1])[None, :] < k[:, None]
        cams_l.append(sel[mask])
        pts_l.append((made + np.broadcast_to(np.arange(take)[:, None], sel.shape))[mask])
        Xs.append(X)
        made += take
    X = np.concatenate(Xs)
    cam_idx = np.concatenate(cams_l)
    pt_idx = np.concatenate(pts_l)
    span = np.array([cols * spacing, rows * spacing, 1.0])
    drift_dir = np.array([0.6, 0.8, 0.0])

    def drift(Y):
        r = np.linalg.norm(Y[:, :2], axis=1) / np.linalg.norm(span[:2])
        wave = np.sin(2 * np.pi * Y[:, 0] / (span[0] / 3.0))
        return (0.5 * r)[:, None] * drift_dir + (0.2 * wave)[:, None] * np.array([0, 0, 1.0])

    return _assemble("city_grid", rng, Rm, centres, f, k1, k2, X, cam_idx, pt_idx, sigma,
                     rel_pert=0.01, trans_pert=0.05, point_pert=0.05, lam=lam, rtol=rtol,
                     drift=drift)


def loop_closure(seed=0, n_cams=10_000, n_pts=1_000_000, cross_frac=0.05, sigma=1.0,
                 lam=1e-4, rtol=1e-6) -> Scene:
    """A closed racetrack loop: cameras drive down one street and back along a
    parallel street 20 units away, all facing the median between them.  Most
    points are seen by consecutive cameras of one street; ``cross_frac`` of them
    are also seen from the other street, linking cameras far apart in loop order."""
    rng = np.random.default_rng(seed)
    half = n_cams // 2
    xA = np.arange(half, dtype=float)
    xB = np.arange(n_cams - half, dtype=float)[::-1]
    centres = np.concatenate([
        np.stack([xA, np.zeros(half), np.full(half, 2.0)], axis=1),
        np.stack([xB, np.full(n_cams - half, 20.0), np.full(n_cams - half, 2.0)], axis=1)])
    yaw = np.concatenate([np.full(half, np.pi / 2), np.full(n_cams - half, -np.pi / 2)])
    yaw = yaw + np.deg2rad(rng.uniform(-5, 5, n_cams))
    fwd = np.stack([np.cos(yaw), np.sin(yaw), np.zeros(n_cams)], axis=1)
    Rm = _look_rotation(fwd)
    f, k1, k2 = _intrinsics(rng, n_cams)
    k = np.clip(2 + rng.binomial(12, 0.5, n_pts), 2, 14)
    j0 = (rng.random(n_pts) * (half - k)).astype(np.int64)
    onB = rng.random(n_pts) < 0.5
    cross = rng.random(n_pts) < cross_frac
    xmid = j0 + (k - 1) / 2.0
    y = np.where(cross, rng.uniform(9.0, 11.0, n_pts),
                 np.where(onB, rng.uniform(13.0, 15.0, n_pts), rng.uniform(5.0, 7.0, n_pts)))
    X = np.stack([xmid + rng.uniform(-0.5, 0.5, n_pts), y, rng.uniform(0.5, 4.0, n_pts)], axis=1)
    cams_l, pts_l = [], []
    ar = np.arange(14)
    m = ar[None, :] < k[:, None]
    idxA = j0[:, None] + ar[None, :]                  # street A camera at x
    idxB = (n_cams - 1) - idxA                        # street B camera at the same x
    primary = np.where(onB[:, None] & ~cross[:, None], idxB, idxA)
    P = np.broadcast_to(np.arange(n_pts)[:, None], idxA.shape)
    cams_l.append(primary[m])
    pts_l.append(P[m])
    kc = np.clip(k // 2, 2, 14)
    mc = (ar[None, :] < kc[:, None]) & cross[:, None]
    cams_l.append(idxB[mc])
    pts_l.append(P[mc])
    cam_idx = np.concatenate(cams_l)
    pt_idx = np.concatenate(pts_l)
    return _assemble("loop_closure", rng, Rm, centres, f, k1, k2, X, cam_idx, pt_idx, sigma,
                     rel_pert=0.02, trans_pert=0.1, point_pert=0.1, lam=lam, rtol=rtol)


def subscene(scene: Scene, n_cams: int, n_pts: int, seed: int = 0) -> Scene:
    """The first ``n_cams`` cameras (in camera order) and up to ``n_pts`` of the
    points seen only by them, with their observations; ids are compacted."""
    rng = np.random.default_rng(seed)
    inside = scene.cam_idx < n_cams
    bad = np.zeros(scene.n_pts, dtype=bool)
    bad[scene.pt_idx[~inside]] = True
    cnt = np.bincount(scene.pt_idx[inside], minlength=scene.n_pts)
    good = np.flatnonzero(~bad & (cnt >= 2))
    good = np.sort(rng.choice(good, size=min(n_pts, len(good)), replace=False))
    newid = -np.ones(scene.n_pts, dtype=np.int64)
    newid[good] = np.arange(len(good))
    keep = inside & (newid[scene.pt_idx] >= 0)
    return Scene(name=scene.name + "_sub", n_cams=n_cams, n_pts=len(good), n_obs=int(keep.sum()),
                 cam_idx=scene.cam_idx[keep].astype(np.int32),
                 pt_idx=newid[scene.pt_idx[keep]].astype(np.int32),
                 obs=scene.obs[keep].copy(), cams=scene.cams[:n_cams].copy(),
                 pts=scene.pts[good].copy(), cams_true=scene.cams_true[:n_cams].copy(),
                 pts_true=scene.pts_true[good].copy(), lam=scene.lam, rtol=scene.rtol)


def rotated_start(scene: Scene, sigma: float, seed: int = 0) -> Scene:
    """The same scene with N(0, sigma^2) added to every angle-axis component of the
    starting cameras: a start far from the optimum whose Gauss-Newton steps overshoot
    (points cross the cameras' image planes), so that LM steps get rejected."""
    rng = np.random.default_rng(seed)
    cams = scene.cams.copy()
    cams[:, :3] += sigma * rng.normal(size=(scene.n_cams, 3))
    return Scene(name=scene.name + "_rot", n_cams=scene.n_cams, n_pts=scene.n_pts, n_obs=scene.n_obs,
                 cam_idx=scene.cam_idx, pt_idx=scene.pt_idx, obs=scene.obs, cams=cams,
                 pts=scene.pts.copy(), cams_true=scene.cams_true, pts_true=scene.pts_true,
                 lam=scene.lam, rtol=scene.rtol)


def tiny(seed=0, n_cams=6, n_pts=40, kmin=2, kmax=4) -> Scene:
    """A few-camera ring for brute-force and dense checks."""
    return ring(seed=seed, n_cams=n_cams, n_pts=n_pts, kmin=kmin, kmax=kmax)


CONFIGS = {
    "ring": ring,
    "street_chain": street_chain,
    "city_grid": city_grid,
    "loop_closure": loop_closure,
}
