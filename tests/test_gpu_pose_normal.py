"""Pose normal equations of the photometric residual (Sec. II-D) through the
C ABI against the FP64 oracle's forward-mode pose Jacobian.

Per-pixel Jacobians H must match within 1e-3 relative L2 over pixels whose
threshold decisions are not borderline; the per-view sums A = sum H H^T,
b = sum H r, r.r must equal the FP64 sums of the kernel's own per-pixel terms
(reduction check) and the oracle's sums over the same pixels.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_2501_08672_b300 import binding as B  # noqa: E402
from paper_2501_08672_b300 import scenes  # noqa: E402
from paper_2501_08672_b300.render import GaussianWindow, PoseTracker, Renderer, apply_left  # noqa: E402

import parity_log  # noqa: E402

TOL = 1e-3


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    torch.cuda.init()


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def sums_from_H(H, r):
    """A (upper triangle as 21), b, r.r in FP64 from per-pixel H [n,3,6] and r [n,3]."""
    A = np.einsum("pci,pcj->ij", H, H)
    b = np.einsum("pci,pc->i", H, r)
    return A, b, float((r * r).sum())


def gpu_pose_normal(p, views, target, tile_size, **cfg):
    win = GaussianWindow(p, 0)
    r = Renderer(views, 0, tile_size, **cfg)
    g = win.struct()
    r.forward(g)
    H = torch.zeros(r.npx * 18, device="cuda", dtype=torch.float32)
    normal = r.pose_normal(g, target, H)
    torch.cuda.synchronize()
    return r, normal, H.view(-1, 3, 6).double().cpu().numpy()


@pytest.mark.parametrize("ts,sh_degree", [(16, 0), (8, 1), (16, 1), (16, 2), (16, 3)])
def test_pose_normal_full_images_match_oracle(orc, ts, sh_degree):
    """Two ragged views of a 20k-Gaussian room, every pixel: per-pixel H
    against the oracle, and the per-view normal equations."""
    n = 20_000
    p = scenes.box_room_scene(n, seed=7, sh_degree=sh_degree)
    views = scenes.arc_views(2, 168, 120, 140.0, n_gaussians=n)
    q = scenes.perturbed_copy(p, seed=8)
    rt = Renderer(views, 0, ts)
    wq = GaussianWindow(q, 0)   # keeps the parameters alive while the struct is used
    rt.forward(wq.struct())
    target = rt.rgb.clone()
    r, normal, Hg = gpu_pose_normal(p, views, target, ts)
    tgt = B.unpack_images(target, views, 3)
    rows = B.unpack_normal(normal)
    off = 0
    for v, view in enumerate(views):
        W, Hh = int(view["W"]), int(view["H"])
        vv, uu = np.mgrid[0:Hh, 0:W]
        Ho, rgbo, bd = orc.pose_jacobian(p, view, uu.reshape(-1), vv.reshape(-1))
        Hv = Hg[off:off + W * Hh]
        tv = tgt[v].detach().double().cpu().numpy().reshape(3, -1).T
        ok = ~bd
        parity_log.record("pixels", bd.mean(), 1e-3, int(bd.sum()), bd.size)
        assert bd.mean() < 1e-3, bd.mean()
        e = rel(Hv[ok], Ho[ok])
        print("view %d: H rel err %.2e, border %.1e" % (v, e, bd.mean()))
        assert e < TOL
        # the kernel's sums equal the FP64 sums of its own per-pixel terms
        img = B.unpack_images(r.rgb, views, 3)[v].detach().double().cpu().numpy().reshape(3, -1).T
        A_own, b_own, rr_own = sums_from_H(Hv, tv - img)
        A, b, rr = rows[v]
        assert rel(A, A_own) < 1e-5 and rel(b, b_own) < 1e-4 and abs(rr - rr_own) <= 1e-5 * rr_own
        # and the oracle's over the non-borderline pixels
        A_o, b_o, _ = sums_from_H(Ho[ok], tv[ok] - rgbo[ok])
        A_g, b_g, _ = sums_from_H(Hv[ok], tv[ok] - img[ok])
        assert rel(A_g, A_o) < TOL and rel(b_g, b_o) < 5 * TOL, (rel(A_g, A_o), rel(b_g, b_o))
        off += W * Hh


def test_pose_normal_odometry_sampled(orc):
    """Odometry size: 500k Gaussians, one 1280x1024 view at a perturbed pose:
    per-pixel H at sampled pixels against the oracle and the reduction
    against the FP64 sum of all per-pixel terms."""
    n = 500_000
    p = scenes.box_room_scene(n, seed=2, sh_degree=1)
    v_true = scenes.lookat_view((4.0 * math.cos(-1.7), 4.0 * math.sin(-1.7), 2.2), (0.0, 0.0, 0.6), 1280, 1024,
                                1200.0, 0, n)
    rt = Renderer([v_true], 0, 16)
    wp = GaussianWindow(p, 0)
    rt.forward(wp.struct())
    target = rt.rgb.clone()
    v = apply_left(v_true, np.array([0.02, -0.015, 0.01, 0.03, -0.02, 0.01]))
    r, normal, Hg = gpu_pose_normal(p, [v], target, 16)
    rng = np.random.default_rng(12)
    # pixels where something is rendered
    T = r.T.detach().cpu().numpy()
    cand = np.nonzero(T < 0.999)[0]
    pick = rng.choice(cand, 64, replace=False)
    px, py = pick % 1280, pick // 1280
    Ho, _, bd = orc.pose_jacobian(p, v, px, py)
    ok = ~bd
    parity_log.record("pixels", bd.mean(), 4.0 / 64, int(bd.sum()), bd.size)
    e = rel(Hg[pick][ok], Ho[ok])
    print("sampled H rel err %.2e over %d pixels" % (e, ok.sum()))
    assert ok.sum() >= 60 and e < TOL
    tv = target.view(3, -1).T.double().cpu().numpy()
    img = r.rgb.view(3, -1).T.double().cpu().numpy()
    A_own, b_own, rr_own = sums_from_H(Hg, tv - img)
    A, b, rr = B.unpack_normal(normal)[0]
    assert rel(A, A_own) < 1e-5 and rel(b, b_own) < 1e-4 and abs(rr - rr_own) <= 1e-5 * rr_own


def test_gauss_newton_pose_converges():
    """Gauss-Newton steps from the normal equations pull a pose perturbed by
    about 0.35 degree and 1.6 cm (a few pixels of image motion) back to the
    rendering pose."""
    n = 200_000
    p = scenes.box_room_scene(n, seed=3, sh_degree=1)
    v_true = scenes.lookat_view((4.0 * math.cos(-1.2), 4.0 * math.sin(-1.2), 2.2), (0.0, 0.0, 0.6), 640, 512,
                                600.0, 0, n)
    rt = Renderer([v_true], 0, 16)
    wp = GaussianWindow(p, 0)
    rt.forward(wp.struct())
    target = rt.rgb.clone()
    xi0 = np.array([0.004, -0.003, 0.003, 0.012, -0.008, 0.006])
    v = apply_left(v_true, xi0)
    tr = PoseTracker(p, v, 0, 16)

    def pose_err(a):
        Ta = np.eye(4); Ta[:3, :3] = a["R"]; Ta[:3, 3] = a["t"]
        Tb = np.eye(4); Tb[:3, :3] = v_true["R"]; Tb[:3, 3] = v_true["t"]
        D = Ta @ np.linalg.inv(Tb)
        ang = math.acos(max(-1.0, min(1.0, (np.trace(D[:3, :3]) - 1) / 2)))
        return ang, float(np.linalg.norm(D[:3, 3]))

    a0, t0 = pose_err(v)
    rrs = []
    for _ in range(6):
        v, (A, b, rr) = tr.gauss_newton(v, target)
        rrs.append(rr)
    a1, t1 = pose_err(v)
    print("rotation %.4f -> %.5f rad, translation %.4f -> %.5f m, r.r %s" % (a0, a1, t0, t1, rrs))
    assert a1 < 0.1 * a0 and t1 < 0.1 * t0
    assert rrs[-1] < 0.2 * rrs[0]


def test_pose_normal_rejects_unsupported_tile_size():
    n = 1000
    p = scenes.frustum_scene(n, seed=1)
    v = scenes.identity_view(64, 48, 60.0, 0, n)
    r = Renderer([v], 0, 32)
    win = GaussianWindow(p, 0)
    r.forward(win.struct())
    with pytest.raises(B.GsError) as ei:
        r.pose_normal(win.struct(), r.rgb.clone())
    assert ei.value.code == B.GS_ERR_UNSUPPORTED


def test_ieskf_visual_update_converges():
    """The IESKF pose update with the GPU's normal equations: the IMU pose
    perturbed by about 0.3 degree and 1.5 cm returns to the rendering pose,
    and the posterior covariance shrinks below the prior."""
    from paper_2501_08672_b300 import ieskf
    from paper_2501_08672_b300.render import IESKFPoseTracker
    from scipy.spatial.transform import Rotation
    n = 200_000
    p = scenes.box_room_scene(n, seed=4, sh_degree=1)
    v0 = scenes.lookat_view((4.0 * math.cos(-1.0), 4.0 * math.sin(-1.0), 2.2), (0.0, 0.0, 0.6), 640, 512,
                            600.0, 0, n)
    R_CI = Rotation.from_rotvec([0.01, -0.02, 0.015]).as_matrix()
    t_CI = np.array([0.04, 0.02, -0.03])
    # the IMU pose that puts the camera at v0: T_WI = T_CW^-1 T_CI
    T_CW = np.eye(4); T_CW[:3, :3] = v0["R"]; T_CW[:3, 3] = v0["t"]
    T_CI = np.eye(4); T_CI[:3, :3] = R_CI; T_CI[:3, 3] = t_CI
    T_WI = np.linalg.inv(T_CW) @ T_CI
    R_true, p_true = T_WI[:3, :3], T_WI[:3, 3]
    tr = IESKFPoseTracker(p, v0, R_CI, t_CI, 0, 16, sigma2=1e-3)
    tr.r.set_views([tr.camera_view(R_true, p_true)])
    tr.r.forward(tr.g)
    target = tr.r.rgb.clone()
    dx0 = np.array([0.004, -0.003, 0.003, 0.012, -0.008, 0.006])
    R0, p0 = ieskf.boxplus(R_true, p_true, dx0)
    P0 = np.diag([1e-4, 1e-4, 1e-4, 4e-4, 4e-4, 4e-4])
    R1, p1, P1, rrs = tr.update(R0, p0, P0, target, iters=5)
    e0 = np.linalg.norm(ieskf.boxminus(R0, p0, R_true, p_true))
    e1 = np.linalg.norm(ieskf.boxminus(R1, p1, R_true, p_true))
    print("pose error %.2e -> %.2e, r.r %s" % (e0, e1, ["%.3g" % x for x in rrs]))
    assert e1 < 0.05 * e0
    assert np.linalg.eigvalsh(P0 - P1).min() > -1e-12 and np.trace(P1) < 0.5 * np.trace(P0)
