"""Seeded synthetic inputs shaped like GS-LIVO's sliding windows.

This module only draws inputs: Gaussian parameters, camera poses, view layouts
and perturbations.  It holds none of the renderer's arithmetic (no projection,
compositing or gradients), so the FP64 oracle and the CUDA path can both be fed
from it without sharing any of the method's code.

The paper's windows are LiDAR-seeded planar Gaussians (Sec. II-B.1): a scale
matrix with one tiny "slice" axis (Eq. scaling_matrix) and a rotation whose
third column is the surface normal (the normal-to-rotation formula of
Sec. II-B.1).  Window sizes follow Sec. III (100k Gaussians at 640x480 on the
desktop, 20k at 256x216 on the Orin NX); the build's configurations scale those.

Parameters are returned as a dict of float32 numpy arrays:
  means [N,3] world metres, log_scales [N,3], quats [N,4] (w,x,y,z, not
  normalised), opacity [N] (logit), sh [N,K,3] with K = (degree+1)^2,
  plus the int 'sh_degree'.
Views are dicts: R [3,3] (camera-from-world rotation, rows are the camera
x-right / y-down / z-forward axes), t [3], fx, fy, cx, cy, W, H, g_begin, g_end.
"""
from __future__ import annotations

import math

import numpy as np

# Degree-0 colour range: the renderer maps a degree-0 coefficient k to
# colour k / (2 sqrt(pi)) + 0.5, so k uniform in (-sqrt(pi), sqrt(pi)) gives a
# colour uniform in (0, 1).  Stated here as an input distribution only.
SQRT_PI = math.sqrt(math.pi)


def _rng(seed):
    return np.random.default_rng(seed)


def lookat_view(eye, target, W, H, f, g_begin=0, g_end=0, up=(0.0, 0.0, 1.0)):
    """Pinhole camera at `eye` looking at `target`, world z up, image y down."""
    eye = np.asarray(eye, np.float64)
    fwd = np.asarray(target, np.float64) - eye
    fwd /= np.linalg.norm(fwd)
    right = np.cross(fwd, np.asarray(up, np.float64))
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    R = np.stack([right, down, fwd])  # rows: camera axes in world coordinates
    t = -R @ eye
    return dict(R=R.astype(np.float32), t=t.astype(np.float32), fx=float(f), fy=float(f),
                cx=W / 2.0, cy=H / 2.0, W=int(W), H=int(H), g_begin=int(g_begin), g_end=int(g_end))


def identity_view(W, H, f, g_begin=0, g_end=0):
    return dict(R=np.eye(3, dtype=np.float32), t=np.zeros(3, np.float32), fx=float(f), fy=float(f),
                cx=W / 2.0, cy=H / 2.0, W=int(W), H=int(H), g_begin=int(g_begin), g_end=int(g_end))


def random_quats(rng, n):
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q.astype(np.float32)


def frustum_scene(n=10_000, seed=0):
    """Plain single-view scene: means uniform in [-2,2]x[-2,2]x[2,8] (camera
    frame, identity pose), log-scales ~ N(-3, 0.5), random unit quaternions,
    opacity logit ~ N(0,1), degree-0 colour ~ U(0,1)."""
    rng = _rng(seed)
    means = np.stack([rng.uniform(-2, 2, n), rng.uniform(-2, 2, n), rng.uniform(2, 8, n)], 1)
    log_scales = rng.normal(-3.0, 0.5, (n, 3))
    quats = random_quats(rng, n)
    opacity = rng.normal(0.0, 1.0, n)
    sh = rng.uniform(-SQRT_PI, SQRT_PI, (n, 1, 3))
    return dict(means=means.astype(np.float32), log_scales=log_scales.astype(np.float32),
                quats=quats, opacity=opacity.astype(np.float32), sh=sh.astype(np.float32), sh_degree=0)


def _normal_frame(n):
    """Rotation with columns (e_x x n / |.|, n x that, n): the paper's
    normal-to-rotation initialisation (Sec. II-B.1); e_y replaces e_x where n
    is parallel to e_x."""
    ex = np.broadcast_to(np.array([1.0, 0.0, 0.0]), n.shape).copy()
    par = np.abs(n[:, 0]) > 0.999
    ex[par] = np.array([0.0, 1.0, 0.0])
    a = np.cross(ex, n)
    a /= np.linalg.norm(a, axis=1, keepdims=True)
    b = np.cross(n, a)
    return np.stack([a, b, n], axis=2)  # [N,3,3], columns a, b, n


def _rot_to_quat(R):
    """Unit quaternions (w,x,y,z) of a batch of rotation matrices (Shepperd's method)."""
    n = R.shape[0]
    q = np.empty((n, 4))
    tr = R[:, 0, 0] + R[:, 1, 1] + R[:, 2, 2]
    cand = np.stack([tr, R[:, 0, 0], R[:, 1, 1], R[:, 2, 2]], 1)
    k = np.argmax(cand, 1)
    m = R
    for case in range(4):
        sel = k == case
        if not np.any(sel):
            continue
        ms = m[sel]
        if case == 0:
            s = np.sqrt(np.maximum(tr[sel] + 1.0, 1e-300)) * 2
            q[sel] = np.stack([0.25 * s, (ms[:, 2, 1] - ms[:, 1, 2]) / s, (ms[:, 0, 2] - ms[:, 2, 0]) / s,
                               (ms[:, 1, 0] - ms[:, 0, 1]) / s], 1)
        elif case == 1:
            s = np.sqrt(np.maximum(1.0 + ms[:, 0, 0] - ms[:, 1, 1] - ms[:, 2, 2], 1e-300)) * 2
            q[sel] = np.stack([(ms[:, 2, 1] - ms[:, 1, 2]) / s, 0.25 * s, (ms[:, 0, 1] + ms[:, 1, 0]) / s,
                               (ms[:, 0, 2] + ms[:, 2, 0]) / s], 1)
        elif case == 2:
            s = np.sqrt(np.maximum(1.0 + ms[:, 1, 1] - ms[:, 0, 0] - ms[:, 2, 2], 1e-300)) * 2
            q[sel] = np.stack([(ms[:, 0, 2] - ms[:, 2, 0]) / s, (ms[:, 0, 1] + ms[:, 1, 0]) / s, 0.25 * s,
                               (ms[:, 1, 2] + ms[:, 2, 1]) / s], 1)
        else:
            s = np.sqrt(np.maximum(1.0 + ms[:, 2, 2] - ms[:, 0, 0] - ms[:, 1, 1], 1e-300)) * 2
            q[sel] = np.stack([(ms[:, 1, 0] - ms[:, 0, 1]) / s, (ms[:, 0, 2] + ms[:, 2, 0]) / s,
                               (ms[:, 1, 2] + ms[:, 2, 1]) / s, 0.25 * s], 1)
    return q


def _box_room_surfaces(scale=1.0):
    """Floor of a (6 s) x (6 s) room plus three axis-aligned boxes standing on
    it.  Returns a list of rectangles (origin, edge_u, edge_v, normal)."""
    s = scale
    rects = [(np.array([-3 * s, -3 * s, 0.0]), np.array([6 * s, 0, 0]), np.array([0, 6 * s, 0]),
              np.array([0, 0, 1.0]))]
    boxes = [((-1.5 * s, -1.0 * s), (1.0 * s, 1.0 * s), 1.0 * s),
             ((1.2 * s, 0.8 * s), (1.2 * s, 0.8 * s), 1.5 * s),
             ((0.3 * s, -1.9 * s), (1.6 * s, 0.6 * s), 0.6 * s)]
    for (bx, by), (sx, sy), h in boxes:
        x0, x1, y0, y1 = bx - sx / 2, bx + sx / 2, by - sy / 2, by + sy / 2
        rects += [
            (np.array([x0, y0, h]), np.array([sx, 0, 0]), np.array([0, sy, 0]), np.array([0, 0, 1.0])),
            (np.array([x0, y0, 0]), np.array([sx, 0, 0]), np.array([0, 0, h]), np.array([0, -1.0, 0])),
            (np.array([x0, y1, 0]), np.array([sx, 0, 0]), np.array([0, 0, h]), np.array([0, 1.0, 0])),
            (np.array([x0, y0, 0]), np.array([0, sy, 0]), np.array([0, 0, h]), np.array([-1.0, 0, 0])),
            (np.array([x1, y0, 0]), np.array([0, sy, 0]), np.array([0, 0, h]), np.array([1.0, 0, 0])),
        ]
    return rects


def box_room_scene(n=200_000, seed=0, sh_degree=1, scale=1.0, slice_log_scale=math.log(1e-3)):
    """LiDAR-map-like window: a floor plus three boxes (6x6x3 m at scale 1),
    points uniform by area, offset along the normal by N(0, 2 cm), rotation
    from the surface normal, tangential log-scales ~ N(-3, 0.5), normal-axis
    scale 1 mm (the slice axis), degree-0 colour from a procedural texture,
    coefficients of degree 1 to sh_degree (<= 3) ~ N(0, 0.1), opacity logit
    ~ N(0, 1)."""
    rng = _rng(seed)
    rects = _box_room_surfaces(scale)
    areas = np.array([np.linalg.norm(np.cross(u, v)) for _, u, v, _ in rects])
    which = rng.choice(len(rects), size=n, p=areas / areas.sum())
    a = rng.uniform(0, 1, n)
    b = rng.uniform(0, 1, n)
    origin = np.stack([rects[k][0] for k in range(len(rects))])[which]
    eu = np.stack([rects[k][1] for k in range(len(rects))])[which]
    ev = np.stack([rects[k][2] for k in range(len(rects))])[which]
    nrm = np.stack([rects[k][3] for k in range(len(rects))])[which]
    pts = origin + a[:, None] * eu + b[:, None] * ev + rng.normal(0, 0.02, n)[:, None] * nrm
    Rg = _normal_frame(nrm)
    quats = _rot_to_quat(Rg)
    log_scales = np.stack([rng.normal(-3.0, 0.5, n), rng.normal(-3.0, 0.5, n),
                           np.full(n, slice_log_scale)], 1)
    # Procedural texture: smooth stripes and a checker in world coordinates.
    tex = np.stack([0.5 + 0.35 * np.sin(3.1 * pts[:, 0] + 1.3 * pts[:, 2]),
                    0.5 + 0.35 * np.sin(2.3 * pts[:, 1] - 0.7 * pts[:, 0] + 1.0),
                    0.5 + 0.3 * np.sign(np.sin(4.0 * pts[:, 0]) * np.sin(4.0 * pts[:, 1]))], 1)
    K = (sh_degree + 1) ** 2
    sh = np.zeros((n, K, 3))
    sh[:, 0, :] = (tex - 0.5) * 2.0 * SQRT_PI
    if K > 1:
        sh[:, 1:, :] = rng.normal(0, 0.1, (n, K - 1, 3))
    opacity = rng.normal(0.0, 1.0, n)
    return dict(means=pts.astype(np.float32), log_scales=log_scales.astype(np.float32),
                quats=quats.astype(np.float32), opacity=opacity.astype(np.float32),
                sh=sh.astype(np.float32), sh_degree=sh_degree)


def arc_views(n_views=8, W=640, H=512, f=600.0, radius=4.0, arc_len=2.0, height=2.2,
              centre=(0.0, 0.0, 0.6), start_angle=-2.2, n_gaussians=0):
    """Keyframes on a horizontal arc of length `arc_len` at `radius` from the
    room centre, all looking at the centre."""
    views = []
    span = arc_len / radius
    for k in range(n_views):
        ang = start_angle + (span * k / max(n_views - 1, 1))
        eye = (centre[0] + radius * math.cos(ang), centre[1] + radius * math.sin(ang), height)
        views.append(lookat_view(eye, centre, W, H, f, 0, n_gaussians))
    return views


def perturbed_copy(params, seed=1, mean_std=0.01, log_scale_std=0.05, colour_std=0.05):
    """Copy with means += N(0, 1 cm), log-scales += N(0, 0.05) and the
    degree-0 colour += N(0, 0.05) (coefficient noise scaled accordingly)."""
    rng = _rng(seed)
    out = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in params.items()}
    n = params["means"].shape[0]
    out["means"] = (params["means"] + rng.normal(0, mean_std, (n, 3))).astype(np.float32)
    out["log_scales"] = (params["log_scales"] + rng.normal(0, log_scale_std, (n, 3))).astype(np.float32)
    sh = params["sh"].copy()
    sh[:, 0, :] += rng.normal(0, colour_std, (n, 3)) * 2.0 * SQRT_PI
    out["sh"] = sh.astype(np.float32)
    return out


def uneven_batch(n_views=16, n_total=2_000_000, seed=0, min_count=20_000, max_count=500_000,
                 widths=None):
    """Batched uneven window: `n_views` views with widths log-uniform over
    multiples of 64 in [320, 1280], H = 0.8 W, focal 600 * W / 640, each
    seeing a contiguous range of a box-room scene sorted by azimuth (like the
    paper's contiguous GPU window), with range lengths log-uniform in
    [min_count, max_count]."""
    rng = _rng(seed)
    params = box_room_scene(n_total, seed=seed, sh_degree=1, scale=2.0)
    az = np.arctan2(params["means"][:, 1], params["means"][:, 0])
    order = np.argsort(az, kind="stable")
    for k in ("means", "log_scales", "quats", "opacity", "sh"):
        params[k] = np.ascontiguousarray(params[k][order])
    az = az[order]
    if widths is None:
        cand = np.arange(320, 1281, 64)
        lw = rng.uniform(math.log(320), math.log(1280), n_views)
        widths = [int(cand[np.argmin(np.abs(cand - math.exp(x)))]) for x in lw]
    views = []
    for k in range(n_views):
        W = widths[k]
        H = int(round(0.8 * W / 16.0)) * 16 if (0.8 * W) % 16 else int(0.8 * W)
        cnt = int(math.exp(rng.uniform(math.log(min_count), math.log(max_count))))
        cnt = min(cnt, n_total)
        b = int(rng.integers(0, n_total - cnt + 1))
        mid_az = float(az[b + cnt // 2])
        look = (2.0 * math.cos(mid_az), 2.0 * math.sin(mid_az), 0.6)
        eye = (-4.0 * math.cos(mid_az) * 0.5, -4.0 * math.sin(mid_az) * 0.5, 3.0)
        views.append(lookat_view(eye, look, W, H, 600.0 * W / 640.0, b, b + cnt))
    return params, views


def axis_angle_to_R(w):
    th = float(np.linalg.norm(w))
    if th < 1e-15:
        return np.eye(3)
    k = np.asarray(w, np.float64) / th
    Kx = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    return np.eye(3) + math.sin(th) * Kx + (1 - math.cos(th)) * (Kx @ Kx)


def odometry_frames(n_frames=200, W=1280, H=1024, f=1200.0, seed=0, rot_deg=2.0, trans_m=0.05):
    """Smooth arc of true camera poses plus, per frame, a perturbed start
    pose: a random-axis rotation of `rot_deg` degrees and a random-direction
    translation of `trans_m` metres applied on the left of T_CW."""
    rng = _rng(seed)
    true_views, start_views = [], []
    for k in range(n_frames):
        ang = -2.2 + 1.0 * k / max(n_frames - 1, 1)
        eye = (4.0 * math.cos(ang), 4.0 * math.sin(ang), 2.2)
        v = lookat_view(eye, (0.0, 0.0, 0.6), W, H, f)
        true_views.append(v)
        axis = rng.standard_normal(3)
        axis /= np.linalg.norm(axis)
        dR = axis_angle_to_R(axis * math.radians(rot_deg))
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        p = dict(v)
        p["R"] = (dR @ v["R"].astype(np.float64)).astype(np.float32)
        p["t"] = (dR @ v["t"].astype(np.float64) + trans_m * d).astype(np.float32)
        start_views.append(p)
    return true_views, start_views


def mixed_precision_scene(n=2_000_000, seed=0):
    """Large window for the mixed-precision form: the box-room generator at
    twice the room size with 10 keyframes at 1280x1024."""
    params = box_room_scene(n, seed=seed, sh_degree=1, scale=2.0)
    views = arc_views(10, 1280, 1024, 1200.0, radius=8.0, arc_len=4.0, height=4.0,
                      centre=(0.0, 0.0, 1.0), n_gaussians=n)
    return params, views
