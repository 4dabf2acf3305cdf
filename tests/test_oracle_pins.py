"""Pins of the FP64 oracle against things other than itself.

Closed forms of Eq. raster, textbook rotations and real spherical harmonics
from scipy, numerical Jacobians, central finite differences, torch.optim.Adam,
and the pose/Gaussian adjoint identity.  No GPU is used.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.linalg
import scipy.special
from scipy.spatial.transform import Rotation

from paper_2501_08672_b300 import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def one_gaussian(mu, log_scale, quat, logit, sh, sh_degree=0):
    K = (sh_degree + 1) ** 2
    sh = np.asarray(sh, np.float64).reshape(1, K, 3)
    return dict(means=np.asarray([mu], np.float64), log_scales=np.asarray([log_scale], np.float64),
                quats=np.asarray([quat], np.float64), opacity=np.asarray([logit], np.float64),
                sh=sh, sh_degree=sh_degree)


def stack(*gs):
    out = {k: np.concatenate([g[k] for g in gs]) for k in ("means", "log_scales", "quats", "opacity", "sh")}
    out["sh_degree"] = gs[0]["sh_degree"]
    return out


def k0_for(c):
    # degree-0 coefficient that gives colour c: c = k0 / (2 sqrt(pi)) + 0.5
    return (np.asarray(c, np.float64) - 0.5) * 2.0 * math.sqrt(math.pi)


def view(W, H, f, cx=None, cy=None, R=None, t=None):
    return dict(R=np.eye(3) if R is None else R, t=np.zeros(3) if t is None else t, fx=f, fy=f,
                cx=W / 2 if cx is None else cx, cy=H / 2 if cy is None else cy, W=W, H=H,
                g_begin=0, g_end=0)


# ---------------------------------------------------------------- projection

@pytest.mark.parametrize("axis", ["x", "y", "z"])
def test_quarter_turns_are_textbook(orc, axis):
    """90-degree turns about each axis permute the scales (Eq. 3dgs); on the
    optical axis J = diag(f/z, f/z) so Sigma2 = (f/z)^2 Sigma3[:2,:2] + b I."""
    s = np.array([0.1, 0.2, 0.3])
    z, f = 5.0, 100.0
    q = {"x": [math.cos(math.pi / 4), math.sin(math.pi / 4), 0, 0],
         "y": [math.cos(math.pi / 4), 0, math.sin(math.pi / 4), 0],
         "z": [math.cos(math.pi / 4), 0, 0, math.sin(math.pi / 4)]}[axis]
    # Rx(90): (x, y, z) scales -> diag(sx^2, sz^2, sy^2); Ry: (sz, sy, sx); Rz: (sy, sx, sz)
    perm = {"x": (0, 2), "y": (2, 1), "z": (1, 0)}[axis]
    p = one_gaussian([0, 0, z], np.log(s), q, 0.0, k0_for([0.5] * 3))
    pr = orc.project(p, view(64, 64, f), dict(blur=0.3))
    expect = np.array([(f / z) ** 2 * s[perm[0]] ** 2 + 0.3, 0.0, (f / z) ** 2 * s[perm[1]] ** 2 + 0.3])
    np.testing.assert_allclose(pr["sigma2"][0], expect, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(pr["q"][0], [32.0, 32.0], rtol=0, atol=1e-13)


def test_random_rotation_matches_scipy(orc):
    """Sigma3 = R S^2 R^T with R from scipy's quaternion convention (Eq. 3dgs)."""
    rng = np.random.default_rng(3)
    for _ in range(20):
        q = rng.standard_normal(4) * rng.uniform(0.5, 2.0)  # deliberately not unit
        s = rng.uniform(0.05, 0.4, 3)
        R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()  # scipy is scalar-last
        S3 = R @ np.diag(s ** 2) @ R.T
        z, f = 4.0, 150.0
        p = one_gaussian([0, 0, z], np.log(s), q, 0.0, k0_for([0.5] * 3))
        pr = orc.project(p, view(64, 64, f), dict(blur=0.0))
        e = (f / z) ** 2 * S3[:2, :2]
        np.testing.assert_allclose(pr["sigma2"][0], [e[0, 0], e[0, 1], e[1, 1]], rtol=1e-12, atol=1e-14)


def _pi(p, fx, fy, cx, cy):
    return np.array([fx * p[0] / p[2] + cx, fy * p[1] / p[2] + cy])


def test_offaxis_ewa_uses_exact_projection_jacobian(orc):
    """Eq. spat with J the Jacobian of pi, checked against a numerical
    Jacobian of the pinhole map and a posed camera."""
    rng = np.random.default_rng(4)
    R = Rotation.from_rotvec([0.3, -0.2, 0.5]).as_matrix()
    t = np.array([0.2, -0.1, 1.0])
    fx, fy, cx, cy = 300.0, 280.0, 161.0, 121.0
    for _ in range(10):
        mu = rng.uniform(-1, 1, 3) + np.array([0, 0, 4.0])
        mu = R.T @ (mu - t)  # world point that lands in front of the camera
        q = rng.standard_normal(4)
        s = rng.uniform(0.02, 0.3, 3)
        p = one_gaussian(mu, np.log(s), q, 0.0, k0_for([0.5] * 3))
        v = dict(R=R, t=t, fx=fx, fy=fy, cx=cx, cy=cy, W=320, H=240, g_begin=0, g_end=0)
        pr = orc.project(p, v, dict(blur=0.3))
        pc = R @ mu + t
        h = 1e-6
        Jn = np.zeros((2, 3))
        for k in range(3):
            e = np.zeros(3); e[k] = h
            Jn[:, k] = (_pi(pc + e, fx, fy, cx, cy) - _pi(pc - e, fx, fy, cx, cy)) / (2 * h)
        Rq = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        S3 = Rq @ np.diag(s ** 2) @ Rq.T
        S2 = Jn @ R @ S3 @ R.T @ Jn.T + 0.3 * np.eye(2)
        np.testing.assert_allclose(pr["sigma2"][0], [S2[0, 0], S2[0, 1], S2[1, 1]], rtol=1e-7)
        np.testing.assert_allclose(pr["q"][0], _pi(pc, fx, fy, cx, cy), rtol=1e-13)


def test_ewa_matches_monte_carlo_for_small_gaussians(orc):
    """Second moment of projected samples approaches Sigma2 - b I as the
    Gaussian shrinks relative to its depth (the local-affine approximation)."""
    rng = np.random.default_rng(5)
    R = Rotation.from_rotvec([0.1, 0.2, -0.1]).as_matrix()
    t = np.array([0.0, 0.0, 0.5])
    mu = np.array([0.4, -0.3, 5.0])
    q = np.array([0.8, 0.1, -0.3, 0.5])
    s = np.array([0.01, 0.02, 0.005])
    p = one_gaussian(mu, np.log(s), q, 0.0, k0_for([0.5] * 3))
    v = dict(R=R, t=t, fx=500.0, fy=500.0, cx=0.0, cy=0.0, W=8, H=8, g_begin=0, g_end=0)
    pr = orc.project(p, v, dict(blur=0.0))
    Rq = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
    x = mu + (rng.standard_normal((400_000, 3)) * s) @ Rq.T
    pc = x @ R.T + t
    uv = np.stack([500 * pc[:, 0] / pc[:, 2], 500 * pc[:, 1] / pc[:, 2]], 1)
    C = np.cov(uv.T)
    np.testing.assert_allclose(pr["sigma2"][0], [C[0, 0], C[0, 1], C[1, 1]], rtol=0.02, atol=0.02 * C[0, 0])


def test_degree_one_colour_is_real_sh(orc):
    """Colour = C0 k0 - k1 Y_{1,-1} + k2 Y_{1,0} - k3 Y_{1,1} + 0.5 with the
    real harmonics built from scipy's complex ones (the degree-1 reading)."""
    rng = np.random.default_rng(6)
    for _ in range(10):
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        if d[2] < 0.2:
            d[2] = 0.2 + abs(d[2])
            d /= np.linalg.norm(d)
        mu = 5.0 * d
        sh = rng.normal(0, 0.3, (4, 3))
        sh[0] = 1.0
        theta = math.acos(d[2])
        phi = math.atan2(d[1], d[0])
        Y = lambda l, m: scipy.special.sph_harm_y(l, m, theta, phi)  # noqa: E731
        y00 = Y(0, 0).real
        # real harmonics: Y_{1,-1} = -sqrt(2) Im Y_1^1, Y_{1,0} = Y_1^0, Y_{1,1} = -sqrt(2) Re Y_1^1
        y1m1 = -math.sqrt(2) * Y(1, 1).imag
        y10 = Y(1, 0).real
        y11 = -math.sqrt(2) * Y(1, 1).real
        np.testing.assert_allclose([y1m1, y10, y11], math.sqrt(3 / (4 * math.pi)) * d[[1, 2, 0]], rtol=1e-12)
        expect = y00 * sh[0] - y1m1 * sh[1] + y10 * sh[2] - y11 * sh[3] + 0.5
        p = one_gaussian(mu, np.log([0.1] * 3), [1, 0, 0, 0], 0.0, sh, sh_degree=1)
        pr = orc.project(p, view(64, 64, 50.0), dict(blur=0.3))
        np.testing.assert_allclose(pr["raw_colour"][0], expect, rtol=1e-12, atol=1e-13)


def _real_sh_from_scipy(d, lmax=3):
    """Real harmonics with the Condon-Shortley phase, k = l^2 + l + m, from
    scipy's complex Y_l^m (which carry the phase): sqrt(2) Im Y_l^|m| for
    m < 0, Y_l^0, sqrt(2) Re Y_l^m for m > 0."""
    theta = math.acos(max(-1.0, min(1.0, d[2])))
    phi = math.atan2(d[1], d[0])
    out = []
    for l in range(lmax + 1):
        for m in range(-l, l + 1):
            y = scipy.special.sph_harm_y(l, abs(m), theta, phi)
            out.append(math.sqrt(2) * y.imag if m < 0 else (y.real if m == 0 else math.sqrt(2) * y.real))
    return np.array(out)


def test_sh_basis_is_scipy_real_sh(orc):
    """Degrees 0-3: the oracle's basis equals the real harmonics built from
    scipy's complex ones (the degree-1 reading extended), and the basis of a
    lower degree is its prefix."""
    rng = np.random.default_rng(8)
    d = rng.standard_normal((40, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    Y, _ = orc.sh_basis(d, 3)
    for i in range(len(d)):
        np.testing.assert_allclose(Y[i], _real_sh_from_scipy(d[i]), rtol=1e-12, atol=1e-14)
    for deg in range(3):
        Yd, _ = orc.sh_basis(d, deg)
        K = (deg + 1) ** 2
        np.testing.assert_array_equal(Yd[:, :K], Y[:, :K])
        assert np.all(Yd[:, K:] == 0)


@pytest.mark.parametrize("l", [1, 2, 3])
def test_sh_addition_theorem(orc, l):
    """sum_m Y_lm(a) Y_lm(b) = (2l+1)/(4 pi) P_l(a.b) (textbook Legendre
    polynomials): any wrong constant, sign mix-up inside a product or missing
    term of degree l breaks it."""
    P = {1: lambda t: t, 2: lambda t: 1.5 * t * t - 0.5, 3: lambda t: 2.5 * t ** 3 - 1.5 * t}[l]
    rng = np.random.default_rng(9 + l)
    a = rng.standard_normal((50, 3))
    b = rng.standard_normal((50, 3))
    a /= np.linalg.norm(a, axis=1, keepdims=True)
    b /= np.linalg.norm(b, axis=1, keepdims=True)
    Ya, _ = orc.sh_basis(a, 3)
    Yb, _ = orc.sh_basis(b, 3)
    blk = slice(l * l, (l + 1) ** 2)
    lhs = (Ya[:, blk] * Yb[:, blk]).sum(1)
    rhs = (2 * l + 1) / (4 * math.pi) * P((a * b).sum(1))
    np.testing.assert_allclose(lhs, rhs, rtol=1e-12, atol=1e-14)


def test_sh_basis_derivatives_match_differences(orc):
    """dY: the partial derivatives of the homogeneous polynomials, against
    central differences off the sphere (the polynomials are evaluated as
    written, without renormalising the direction)."""
    rng = np.random.default_rng(10)
    d = rng.standard_normal((20, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    _, dY = orc.sh_basis(d, 3)
    h = 1e-6
    for c in range(3):
        e = np.zeros(3)
        e[c] = h
        Yp, _ = orc.sh_basis(d + e, 3)
        Ym, _ = orc.sh_basis(d - e, 3)
        np.testing.assert_allclose((Yp - Ym) / (2 * h), dY[:, :, c], rtol=1e-6, atol=1e-8)


# ---------------------------------------------------------------- compositing

def test_single_isotropic_gaussian_closed_form(orc):
    """Exact mode, one isotropic Gaussian on the axis:
    I(x) = c sigma exp(-r^2 / (2 (f^2 s^2 / z^2 + b)))."""
    f, z, s, b = 120.0, 3.0, 0.08, 0.3
    c = np.array([0.9, 0.4, 0.2])
    p = one_gaussian([0, 0, z], np.log([s] * 3), [0.3, 0.5, -0.2, 0.7], 0.4, k0_for(c))
    W, H = 40, 30
    v = view(W, H, f, cx=17.3, cy=14.1)
    out = orc.render_view(p, v, dict(orc.EXACT_CFG, blur=b))
    u, w = np.meshgrid(np.arange(W) + 0.5, np.arange(H) + 0.5)
    r2 = (u - 17.3) ** 2 + (w - 14.1) ** 2
    sig = 1 / (1 + math.exp(-0.4))
    prof = sig * np.exp(-r2 / (2 * (f * f * s * s / (z * z) + b)))
    for ch in range(3):
        np.testing.assert_allclose(out["rgb"][ch], c[ch] * prof, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(out["T"], 1 - prof, rtol=1e-12, atol=1e-14)


def test_cocentred_stack_golden(orc):
    g = json.load(open(os.path.join(GOLDEN, "cocentred_stack.json")))
    gs = []
    # inputs listed back to front so the oracle must sort by depth
    for sg, c, z in reversed(list(zip(g["sigma"], g["colour"], g["depth"]))):
        gs.append(one_gaussian([0, 0, z], np.log([0.05] * 3), [1, 0, 0, 0], math.log(sg / (1 - sg)),
                               k0_for([c] * 3)))
    p = stack(*gs)
    v = view(9, 9, 50.0, cx=4.5, cy=4.5)
    out = orc.render_view(p, v, dict(orc.EXACT_CFG))
    assert abs(out["T"][4, 4] - g["T_final"]) < 1e-13
    for ch in range(3):
        assert abs(out["rgb"][ch, 4, 4] - g["intensity"]) < 1e-13


def test_stack_product_and_termination(orc):
    """Random co-centred stacks: T_final = prod(1 - sigma_j) and
    I = sum c_j sigma_j prod_{k<j}(1 - sigma_k); with T_min the compositing
    stops before the Gaussian that would take T below T_min."""
    rng = np.random.default_rng(7)
    for trial in range(10):
        n = 12
        sig = rng.uniform(0.2, 0.6, n)
        col = rng.uniform(0.1, 0.9, n)
        zs = rng.permutation(np.linspace(2.0, 9.0, n))
        p = stack(*[one_gaussian([0, 0, zs[i]], np.log([0.05] * 3), [1, 0, 0, 0],
                                 math.log(sig[i] / (1 - sig[i])), k0_for([col[i]] * 3)) for i in range(n)])
        order = np.argsort(zs)
        Tmin = 10 ** rng.uniform(-4, -2)
        T, I = 1.0, 0.0
        for j in order:
            if T * (1 - sig[j]) < Tmin:
                break
            I += col[j] * sig[j] * T
            T *= 1 - sig[j]
        v = view(9, 9, 50.0, cx=4.5, cy=4.5)
        out = orc.render_view(p, v, dict(alpha_min=0.0, alpha_max=1.0, T_min=Tmin))
        assert abs(out["T"][4, 4] - T) < 1e-13
        assert abs(out["rgb"][0, 4, 4] - I) < 1e-13
        full = orc.render_view(p, v, dict(orc.EXACT_CFG))
        assert abs(full["T"][4, 4] - np.prod(1 - sig)) < 1e-13


def test_alpha_clamp_and_skip(orc):
    """alpha = min(alpha_max, sigma G); Gaussians below alpha_min are skipped."""
    v = view(9, 9, 50.0, cx=4.5, cy=4.5)
    strong = one_gaussian([0, 0, 3.0], np.log([0.05] * 3), [1, 0, 0, 0], 8.0, k0_for([1.0] * 3))
    out = orc.render_view(strong, v, dict(alpha_min=1 / 255, alpha_max=0.99, T_min=0.0))
    assert abs(out["T"][4, 4] - 0.01) < 1e-14
    faint = one_gaussian([0, 0, 2.0], np.log([0.05] * 3), [1, 0, 0, 0], math.log(0.003 / 0.997),
                         k0_for([0.3] * 3))
    both = orc.render_view(stack(strong, faint), v, dict(alpha_min=1 / 255, alpha_max=0.99, T_min=0.0))
    np.testing.assert_array_equal(both["rgb"], out["rgb"])


def test_permutation_invariance(orc):
    p = scenes.frustum_scene(600, seed=11)
    v = scenes.identity_view(64, 48, 60.0)
    a = orc.render_view(p, v)
    perm = np.random.default_rng(1).permutation(600)
    q = {k: (p[k][perm] if isinstance(p[k], np.ndarray) else p[k]) for k in p}
    b = orc.render_view(q, v)
    np.testing.assert_allclose(a["rgb"], b["rgb"], rtol=0, atol=1e-13)


def test_truncated_close_to_exact(orc):
    """Truncation (alpha_min, T_min) moves each pixel by at most the light
    it drops: skipped fragments (< alpha_min each) and the tail behind the
    stop (< T_min / (1 - alpha_max))."""
    p = scenes.frustum_scene(300, seed=12)
    p["opacity"][:] = np.clip(p["opacity"], -3, 3)
    v = scenes.identity_view(48, 40, 50.0)
    ex = orc.render_view(p, v, dict(orc.EXACT_CFG, alpha_max=0.99))
    tr = orc.render_view(p, v, dict(alpha_min=1 / 255, alpha_max=0.99, T_min=1e-4))
    bound = 300 * (1 / 255) * 1.0 + 1e-4 / 0.01
    assert np.abs(ex["rgb"] - tr["rgb"]).max() < bound
    assert np.abs(ex["rgb"] - tr["rgb"]).mean() < 0.05


# ---------------------------------------------------------------- gradients

def _tiny_scene(seed, n=5, sh_degree=1):
    rng = np.random.default_rng(seed)
    K = (sh_degree + 1) ** 2
    mu = np.stack([rng.uniform(-0.4, 0.4, n), rng.uniform(-0.3, 0.3, n), rng.uniform(2.0, 3.5, n)], 1)
    sh = rng.normal(0, 0.3, (n, K, 3))
    sh[:, 0, :] = k0_for(rng.uniform(0.4, 0.9, (n, 3)))
    return dict(means=mu, log_scales=rng.normal(-2.2, 0.3, (n, 3)), quats=rng.standard_normal((n, 4)),
                opacity=rng.normal(0, 0.8, n), sh=sh, sh_degree=sh_degree)


def _posed_view(W=24, H=20):
    R = Rotation.from_rotvec([0.05, -0.08, 0.03]).as_matrix()
    return dict(R=R, t=np.array([0.05, -0.02, 0.1]), fx=40.0, fy=42.0, cx=W / 2 + 0.3, cy=H / 2 - 0.2,
                W=W, H=H, g_begin=0, g_end=0)


def _loss(orc, p, views, w, cfg):
    outs = [orc.render_view(p, v, cfg) for v in views]
    return sum(float(np.sum(o["rgb"] * wi)) for o, wi in zip(outs, w))


@pytest.mark.parametrize("sh_degree", [0, 1, 2, 3])
def test_gaussian_gradients_match_central_differences(orc, sh_degree):
    """Exact mode, smooth loss L = sum w * I: analytic backward vs central
    differences for every parameter of every Gaussian, two views."""
    p = _tiny_scene(21 + sh_degree, sh_degree=sh_degree)
    views = [_posed_view(), view(24, 20, 38.0, cx=11.7, cy=10.2)]
    cfg = dict(orc.EXACT_CFG)
    rng = np.random.default_rng(2)
    w = [rng.standard_normal((3, v["H"], v["W"])) for v in views]
    g, pose, _ = orc.backward(p, views, w, cfg)
    h = 1e-6
    for key in ("means", "log_scales", "quats", "opacity", "sh"):
        flat = p[key].reshape(-1)
        num = np.zeros_like(flat)
        for k in range(flat.size):
            old = flat[k]
            flat[k] = old + h
            lp = _loss(orc, p, views, w, cfg)
            flat[k] = old - h
            lm = _loss(orc, p, views, w, cfg)
            flat[k] = old
            num[k] = (lp - lm) / (2 * h)
        ana = g[key].reshape(-1)
        err = np.linalg.norm(ana - num) / max(np.linalg.norm(num), 1e-30)
        assert err < 1e-6, (key, err)


def _se3_exp(xi):
    """Exp of xi = (dphi, dt) through the 4x4 matrix exponential (scipy)."""
    X = np.zeros((4, 4))
    wx, wy, wz = xi[:3]
    X[:3, :3] = [[0, -wz, wy], [wz, 0, -wx], [-wy, wx, 0]]
    X[:3, 3] = xi[3:]
    return scipy.linalg.expm(X)


def _perturb(v, xi):
    T = np.eye(4)
    T[:3, :3] = v["R"]
    T[:3, 3] = v["t"]
    Tp = _se3_exp(xi) @ T
    out = dict(v)
    out["R"] = Tp[:3, :3]
    out["t"] = Tp[:3, 3]
    return out


@pytest.mark.parametrize("loss", ["weighted", "l1"])
def test_pose_gradient_matches_central_differences(orc, loss):
    """dL/d(dphi, dt) for T_CW <- Exp(xi) T_CW (Appendix A perturbation model),
    against central differences through scipy's matrix exponential."""
    p = _tiny_scene(31, sh_degree=1)
    v = _posed_view(28, 22)
    cfg = dict(orc.EXACT_CFG)
    rng = np.random.default_rng(3)
    if loss == "weighted":
        w = rng.standard_normal((3, v["H"], v["W"]))
        lossf = lambda vv: float(np.sum(orc.render_view(p, vv, cfg)["rgb"] * w))  # noqa: E731
        dl = [w]
    else:
        base = orc.render_view(p, v, cfg)["rgb"]
        target = base + np.where(rng.uniform(size=base.shape) < 0.5, -1, 1) * rng.uniform(0.2, 0.4, base.shape)
        lossf = lambda vv: orc.l1_loss_grad([orc.render_view(p, vv, cfg)["rgb"]], [target])[0]  # noqa: E731
        dl = orc.l1_loss_grad([base], [target])[1]
    _, pose, _ = orc.backward(p, [v], dl, cfg)
    h = 1e-6
    num = np.zeros(6)
    for k in range(6):
        e = np.zeros(6); e[k] = h
        num[k] = (lossf(_perturb(v, e)) - lossf(_perturb(v, -e))) / (2 * h)
    np.testing.assert_allclose(pose[0], num, rtol=2e-6, atol=1e-9 * np.abs(num).max())


def test_pose_gradient_adjoint_identity(orc):
    """Degree-0 colour: moving the camera by Exp(xi) equals moving every
    Gaussian rigidly by T_CW^-1 Exp(xi) T_CW, so the pose gradient equals
    dt: W sum_i g_mu_i;  dphi: sum_i p_C,i x (W g_mu_i) + W g_omega_i with
    g_omega the gradient of a left rotation of the Gaussian's quaternion."""
    p = _tiny_scene(41, n=6, sh_degree=0)
    v = _posed_view(30, 26)
    cfg = dict(orc.EXACT_CFG)
    w = np.random.default_rng(4).standard_normal((3, v["H"], v["W"]))
    g, pose, _ = orc.backward(p, [v], [w], cfg)
    Wm = np.asarray(v["R"], np.float64)
    pc = p["means"] @ Wm.T + v["t"]
    gt = Wm @ g["means"].sum(0)
    gphi = np.zeros(3)
    for i in range(p["means"].shape[0]):
        gphi += np.cross(pc[i], Wm @ g["means"][i])
        qw, qv = p["quats"][i, 0], p["quats"][i, 1:]
        gw, gv = g["quats"][i, 0], g["quats"][i, 1:]
        gomega = 0.5 * (qw * gv - gw * qv + np.cross(qv, gv))
        gphi += Wm @ gomega
    np.testing.assert_allclose(pose[0], np.concatenate([gphi, gt]), rtol=1e-9, atol=1e-12)


def test_l1_gradient_matches_differences(orc):
    """Eq. gaussian_optimization with the L1 norm: the gradient of the
    per-Gaussian path under L1 (residuals bounded away from zero)."""
    p = _tiny_scene(51, sh_degree=1)
    v = _posed_view()
    cfg = dict(orc.EXACT_CFG)
    base = orc.render_view(p, v, cfg)["rgb"]
    rng = np.random.default_rng(5)
    target = base + np.where(rng.uniform(size=base.shape) < 0.5, -1, 1) * rng.uniform(0.2, 0.4, base.shape)
    L, dl = orc.l1_loss_grad([base], [target])
    assert abs(L - np.abs(base - target).mean()) < 1e-15
    g, _, _ = orc.backward(p, [v], dl, cfg)
    h = 1e-6
    flat = p["means"].reshape(-1)
    for k in range(flat.size):
        old = flat[k]
        flat[k] = old + h
        lp = orc.l1_loss_grad([orc.render_view(p, v, cfg)["rgb"]], [target])[0]
        flat[k] = old - h
        lm = orc.l1_loss_grad([orc.render_view(p, v, cfg)["rgb"]], [target])[0]
        flat[k] = old
        assert abs((lp - lm) / (2 * h) - g["means"].reshape(-1)[k]) < 1e-7 * max(1.0, abs(g["means"]).max())


# ---------------------------------------------------------------- Adam

def test_adam_matches_torch(orc):
    import torch
    rng = np.random.default_rng(9)
    n = 257
    p0 = rng.standard_normal(n)
    p = p0.copy(); m = np.zeros(n); v = np.zeros(n)
    tp = torch.tensor(p0.copy(), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([tp], lr=1e-3, betas=(0.9, 0.999), eps=1e-8, foreach=False)
    for step in range(1, 8):
        g = rng.standard_normal(n) * 10 ** rng.uniform(-3, 1)
        tp.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
        orc.adam(p, np.ascontiguousarray(g), m, v, 1e-3, 0.9, 0.999, 1e-8, step)
        np.testing.assert_allclose(p, tp.detach().numpy(), rtol=1e-14, atol=1e-15)


def test_borderline_pixels_are_rare(orc):
    p = scenes.frustum_scene(3000, seed=0)
    v = scenes.identity_view(160, 128, 150.0)
    out = orc.render_view(p, v)
    assert out["border"].mean() < 1e-3


def test_pixel_list_paths_agree_with_full_image(orc):
    """The pixel-list render/backward (used for sampled checks of full-size
    workloads) equals the full-image one on the same pixels."""
    p = _tiny_scene(61, n=40, sh_degree=1)
    v = _posed_view(30, 22)
    full = orc.render_view(p, v)
    yy, xx = np.mgrid[0:v["H"], 0:v["W"]]
    px, py = xx.reshape(-1), yy.reshape(-1)
    lst = orc.render_pixels(p, v, px, py)
    np.testing.assert_array_equal(lst["rgb"].T.reshape(3, v["H"], v["W"]), full["rgb"])
    np.testing.assert_array_equal(lst["T"].reshape(v["H"], v["W"]), full["T"])
    w = np.random.default_rng(7).standard_normal((3, v["H"], v["W"]))
    g1, pose1, _ = orc.backward(p, [v], [w])
    g2, pose2, _ = orc.backward(p, [v], [w.reshape(3, -1).T], pixels=[(px, py)])
    for k in g1:
        np.testing.assert_allclose(g2[k], g1[k], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(pose2, pose1, rtol=1e-12, atol=1e-15)


def test_backward_does_not_depend_on_thread_count(orc):
    """The pixel loop runs in parallel, but each pixel's contributions are
    added in pixel order and the projection backward's pose terms in
    Gaussian order, so the FP64 result is the same bit for bit on any number
    of host threads."""
    p = scenes.frustum_scene(800, seed=5)
    p["sh"] = np.concatenate([p["sh"], np.random.default_rng(1).normal(0, 0.2, (800, 3, 3)).astype(np.float32)], 1)
    p["sh_degree"] = 1
    v = scenes.lookat_view((0.3, -0.2, -0.5), (0.0, 0.0, 5.0), 64, 48, 60.0, 0, 800, up=(0, -1, 0))
    w = np.random.default_rng(2).standard_normal((3, 48, 64))
    outs = []
    for nt in (1, 3, 8):
        orc.set_threads(nt)
        try:
            outs.append(orc.backward(p, [v], [w], n_threads=nt))
        finally:
            orc.set_threads(0)
    for g, pose, border in outs[1:]:
        for k in g:
            np.testing.assert_array_equal(g[k], outs[0][0][k])
        np.testing.assert_array_equal(pose, outs[0][1])
        np.testing.assert_array_equal(border, outs[0][2])


def test_zero_gradient_pixels_contribute_and_flag_nothing(orc):
    """A pixel whose dL/dI is zero adds nothing to any gradient, so the
    backward over a pixel list with such pixels equals the backward over the
    list without them, borderline flags included."""
    p = scenes.frustum_scene(1500, seed=8)
    v = scenes.identity_view(96, 80, 90.0, 0, 1500)
    rng = np.random.default_rng(3)
    px, py = rng.integers(0, 96, 400), rng.integers(0, 80, 400)
    w = rng.standard_normal((400, 3))
    zero = rng.random(400) < 0.4
    w[zero] = 0.0
    ga, pa, ba = orc.backward(p, [v], [w], pixels=[(px, py)])
    keep = ~zero
    gb, pb, bb = orc.backward(p, [v], [w[keep]], pixels=[(px[keep], py[keep])])
    for k in ga:
        np.testing.assert_array_equal(ga[k], gb[k])
    np.testing.assert_array_equal(pa, pb)
    np.testing.assert_array_equal(ba, bb)
    # all zero: nothing at all
    g0, p0, b0 = orc.backward(p, [v], [np.zeros((400, 3))], pixels=[(px, py)])
    assert not b0.any() and not p0.any() and all(not g0[k].any() for k in g0)


def test_borderline_share_follows_contributor_count(orc):
    """The share of borderline pixels stays within twice the expectation
    2 REL (n (m + 1 / |ln T_min|) + 1) that the parity tests bound it by:
    over a footprint ln(alpha) is uniform between ln(alpha_min) and
    ln(sigma), so a covering Gaussian lands within REL of alpha_min with
    probability 2 REL / ln(sigma / alpha_min) (m is the mean of that
    reciprocal), and the step of ln T that crosses ln T_min lands within REL
    of it with probability 2 REL n / |ln T_min|; on a dense box-room view
    where pixels hold tens of contributors."""
    n = 20_000
    p = scenes.box_room_scene(n, seed=7)
    v = scenes.arc_views(1, 192, 160, 180.0, n_gaussians=n)[0]
    out = orc.render_view(p, v)
    nbar = float(out["n_contrib"].mean())
    assert nbar > 10
    share = float(out["border"].mean())
    s = out["sigma"][out["sigma"] > 1.0 / 255.0]
    m = float(np.mean(1.0 / np.maximum(np.log(s * 255.0), 1.0)))
    assert share <= 2.0 * 2.0 * 1e-5 * (nbar * (m + 1.0 / math.log(1e4)) + 1.0)


# ---- pose Jacobian and normal equations (Sec. II-D, Eq. minimization) ----

@pytest.mark.parametrize("sh_degree", [0, 1, 2, 3])
def test_pose_jacobian_matches_central_differences(orc, sh_degree):
    """Per-pixel dI/dxi by forward mode against central differences of the
    rendered image through scipy's matrix exponential, T_CW <- Exp(xi) T_CW,
    exact mode and a coloured background (so dT_final enters)."""
    p = _tiny_scene(41 + sh_degree, n=6, sh_degree=sh_degree)
    v = _posed_view(20, 16)
    cfg = dict(orc.EXACT_CFG)
    cfg["bg"] = (0.2, 0.5, 0.7)
    vv, uu = np.mgrid[0:v["H"], 0:v["W"]]
    Hj, rgb, _ = orc.pose_jacobian(p, v, uu.reshape(-1), vv.reshape(-1), cfg)
    base = orc.render_view(p, v, cfg)["rgb"]
    np.testing.assert_allclose(rgb.T.reshape(base.shape), base, atol=1e-13)
    h = 1e-6
    for k in range(6):
        e = np.zeros(6); e[k] = h
        num = (orc.render_view(p, _perturb(v, e), cfg)["rgb"] - orc.render_view(p, _perturb(v, -e), cfg)["rgb"]) / (2 * h)
        ana = Hj[:, :, k].T.reshape(num.shape)
        err = np.linalg.norm(ana - num) / max(np.linalg.norm(num), 1e-30)
        assert err < 1e-6, (k, err)


def test_pose_jacobian_agrees_with_reverse_mode(orc):
    """Truncated mode (alpha_min, alpha_max clamp, T_min early stop active):
    for any dL/dI, sum_p sum_ch dL/dI_ch(p) H_ch(p) equals the pose gradient of
    the reverse-mode backward, an independent derivation."""
    p = _tiny_scene(47, n=40, sh_degree=1)
    p["opacity"][:20] += 6.0   # sigma > 0.99: the alpha_max clamp and the T_min stop act
    v = _posed_view(24, 20)
    cfg = dict(orc.DEFAULT_CFG)
    cfg["bg"] = (0.1, 0.3, 0.2)
    vv, uu = np.mgrid[0:v["H"], 0:v["W"]]
    Hj, _, _ = orc.pose_jacobian(p, v, uu.reshape(-1), vv.reshape(-1), cfg)
    rng = np.random.default_rng(5)
    w = rng.standard_normal((3, v["H"], v["W"]))
    _, pose, _ = orc.backward(p, [v], [w], cfg)
    fwd = np.einsum("pck,pc->k", Hj, w.reshape(3, -1).T)
    np.testing.assert_allclose(fwd, pose[0], rtol=1e-10, atol=1e-12 * np.abs(pose[0]).max())
    out = orc.render_view(p, v, cfg)
    assert out["n_contrib"].max() >= 3
    assert (out["T"] < 1e-3).any()   # pixels that stopped at T_min


def test_pose_normal_equations_brute_force(orc):
    """A = sum H^T H and b = sum H^T (target - I) against an explicit loop over
    pixels and channels; A is symmetric positive semi-definite and the
    Gauss-Newton step A^-1 b reduces the residual of a pose perturbed by a
    small known xi (first-order model)."""
    p = _tiny_scene(53, n=12, sh_degree=1)
    v = _posed_view(20, 16)
    cfg = dict(orc.EXACT_CFG)
    xi_true = np.array([0.002, -0.003, 0.001, 0.004, -0.002, 0.003])
    target = orc.render_view(p, _perturb(v, xi_true), cfg)["rgb"]
    A, b, rr, _ = orc.pose_normal(p, v, target, cfg)
    vv, uu = np.mgrid[0:v["H"], 0:v["W"]]
    Hj, rgb, _ = orc.pose_jacobian(p, v, uu.reshape(-1), vv.reshape(-1), cfg)
    A2 = np.zeros((6, 6)); b2 = np.zeros(6); rr2 = 0.0
    for q in range(Hj.shape[0]):
        for ch in range(3):
            r = target[ch].reshape(-1)[q] - rgb[q, ch]
            A2 += np.outer(Hj[q, ch], Hj[q, ch]); b2 += Hj[q, ch] * r; rr2 += r * r
    np.testing.assert_allclose(A, A2, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(b, b2, rtol=1e-12, atol=1e-14)
    assert abs(rr - rr2) <= 1e-12 * rr2
    assert np.allclose(A, A.T) and np.linalg.eigvalsh(A).min() > -1e-9 * np.abs(A).max()
    step = np.linalg.solve(A, b)
    # the linearisation recovers the perturbation to first order
    np.testing.assert_allclose(step, xi_true, rtol=0.05, atol=2e-4)


# ---- sliding-window maintenance (Sec. II-C) and SH0 initialisation (Sec. II-B.2) ----

def test_window_compact_worked_example(orc):
    """Rows 0..7, rows 1, 4 and 6 leave: n_keep = 5; the holes 1 and 4 take the
    rear survivors 7 and 5; survivors 0, 2, 3 stay."""
    keep = np.array([1, 0, 1, 1, 0, 1, 0, 1], bool)
    np.testing.assert_array_equal(orc.window_compact(keep), [0, 7, 2, 3, 5])


def test_window_compact_invariants(orc):
    """Random masks: the window keeps exactly the survivors, survivors below
    n_keep never move, every mover comes from at or behind n_keep, and the
    k-th hole takes the k-th survivor from the rear (the closed form)."""
    rng = np.random.default_rng(9)
    for n in (1, 2, 7, 64, 1000):
        for p in (0.0, 0.1, 0.5, 0.9, 1.0):
            keep = rng.uniform(size=n) >= p
            mf = orc.window_compact(keep)
            nk = int(keep.sum())
            assert mf.size == nk
            assert sorted(mf.tolist()) == np.nonzero(keep)[0].tolist()
            for r in range(nk):
                if keep[r]:
                    assert mf[r] == r
                else:
                    assert mf[r] >= nk
            holes = [r for r in range(nk) if not keep[r]]
            movers = [r for r in range(nk, n) if keep[r]][::-1]
            assert [int(mf[h]) for h in holes] == movers


def test_sh0_bilinear_pins(orc):
    """At a pixel centre the colour is that pixel's; a linear image is
    reproduced exactly (bilinear interpolation is exact on it); inside the
    image it matches scipy's order-1 map_coordinates; outside, grey."""
    from scipy import ndimage
    rng = np.random.default_rng(10)
    W, H = 9, 7
    view = dict(R=np.eye(3), t=np.zeros(3), fx=10.0, fy=10.0, cx=4.5, cy=3.5, W=W, H=H)
    img = rng.uniform(0.1, 0.9, (3, H, W))
    z = 2.0
    c0 = 0.5 / np.sqrt(np.pi)
    # pixel centre (u, v) = (3, 2): q = (3.5, 2.5)
    mu = np.array([[(3.5 - 4.5) * z / 10.0, (2.5 - 3.5) * z / 10.0, z]])
    sh = orc.sh0_bilinear(mu, view, img, 1)
    np.testing.assert_allclose(sh[0, 0] * c0 + 0.5, img[:, 2, 3], atol=1e-12)
    assert np.all(sh[0, 1:] == 0)
    uu, vv = np.meshgrid(np.arange(W), np.arange(H))
    lin = np.stack([0.2 + 0.03 * uu - 0.02 * vv, 0.5 + 0.01 * vv, 0.3 - 0.01 * uu])
    pts = rng.uniform([0.3, 0.3], [W - 1.3, H - 1.3], (50, 2))   # continuous pixel coordinates
    mus = np.stack([(pts[:, 0] + 0.5 - 4.5) * z / 10.0, (pts[:, 1] + 0.5 - 3.5) * z / 10.0, np.full(50, z)], 1)
    got = orc.sh0_bilinear(mus, view, lin, 0)[:, 0] * c0 + 0.5
    exact = np.stack([0.2 + 0.03 * pts[:, 0] - 0.02 * pts[:, 1], 0.5 + 0.01 * pts[:, 1], 0.3 - 0.01 * pts[:, 0]], 1)
    np.testing.assert_allclose(got, exact, atol=1e-12)
    got = orc.sh0_bilinear(mus, view, img, 0)[:, 0] * c0 + 0.5
    ref = np.stack([ndimage.map_coordinates(img[ch], [pts[:, 1], pts[:, 0]], order=1) for ch in range(3)], 1)
    np.testing.assert_allclose(got, ref, atol=1e-12)
    far = np.array([[10.0, 0.0, z], [0.0, 0.0, -1.0]])
    np.testing.assert_array_equal(orc.sh0_bilinear(far, view, img, 0)[:, 0], 0.0)


# ---------------------------------------------------------------- D-SSIM term

def _ssim_brute(x, y, size=11, sigma=1.5, C1=1e-4, C2=9e-4):
    """SSIM map by explicit loops: at each pixel the Gaussian-weighted means,
    variances and covariance over the window's pixels inside the image (the
    outside counts as zeros, its weight still in the normalisation)."""
    r = size // 2
    k = np.arange(size) - r
    g = np.exp(-k * k / (2 * sigma * sigma))
    w = np.outer(g, g) / np.outer(g, g).sum()
    C, H, W = x.shape
    out = np.zeros((C, H, W))
    for c in range(C):
        for i in range(H):
            for j in range(W):
                m = {"x": 0.0, "y": 0.0, "xx": 0.0, "yy": 0.0, "xy": 0.0}
                for a in range(size):
                    for b in range(size):
                        ii, jj = i + a - r, j + b - r
                        if 0 <= ii < H and 0 <= jj < W:
                            u, v = x[c, ii, jj], y[c, ii, jj]
                            m["x"] += w[a, b] * u
                            m["y"] += w[a, b] * v
                            m["xx"] += w[a, b] * u * u
                            m["yy"] += w[a, b] * v * v
                            m["xy"] += w[a, b] * u * v
                sx = m["xx"] - m["x"] ** 2
                sy = m["yy"] - m["y"] ** 2
                sxy = m["xy"] - m["x"] * m["y"]
                out[c, i, j] = ((2 * m["x"] * m["y"] + C1) * (2 * sxy + C2)) / \
                               ((m["x"] ** 2 + m["y"] ** 2 + C1) * (sx + sy + C2))
    return out


def test_ssim_map_brute_force(orc):
    rng = np.random.default_rng(12)
    x = rng.uniform(0, 1, (2, 9, 13))
    y = np.clip(x + rng.normal(0, 0.2, x.shape), 0, 1)
    np.testing.assert_allclose(orc.ssim_map(x, y), _ssim_brute(x, y), rtol=1e-12, atol=1e-13)


def test_ssim_window_taps(orc):
    g = orc.ssim_window()
    assert g.size == 11 and abs(g.sum() - 1.0) < 1e-15
    np.testing.assert_allclose(g, g[::-1], rtol=0, atol=0)
    k = np.arange(10) - 5
    np.testing.assert_allclose(g[1:] / g[:-1], np.exp(-(2 * k + 1) / (2 * 1.5 ** 2)), rtol=1e-13)


def test_ssim_constant_images_interior_closed_form(orc):
    """Constant planes a and b: away from the border (window inside the
    image) the variances vanish and s = (2ab + C1) / (a^2 + b^2 + C1)."""
    a, b = 0.7, 0.25
    x = np.full((1, 24, 24), a)
    y = np.full((1, 24, 24), b)
    s = orc.ssim_map(x, y)
    np.testing.assert_allclose(s[0, 5:19, 5:19], (2 * a * b + 1e-4) / (a * a + b * b + 1e-4), rtol=1e-12)


def test_dssim_identical_images_is_stationary(orc):
    """x = y: every s(q) is at its maximum 1, so the SSIM term and its gradient
    vanish (and sign(0) = 0 for the L1 part)."""
    rng = np.random.default_rng(13)
    x = rng.uniform(0, 1, (3, 16, 12))
    L, g = orc.dssim_loss_grad([x], [x], lam=1.0)
    assert abs(L) < 1e-14
    assert np.abs(g[0]).max() < 1e-12


def test_dssim_lambda_zero_is_l1(orc):
    rng = np.random.default_rng(14)
    xs = [rng.uniform(0, 1, (3, 10, 14)), rng.uniform(0, 1, (3, 7, 9))]
    ys = [rng.uniform(0, 1, x.shape) for x in xs]
    L, g = orc.dssim_loss_grad(xs, ys, lam=0.0)
    L1, g1 = orc.l1_loss_grad(xs, ys)
    assert abs(L - L1) < 1e-15
    for a, b in zip(g, g1):
        np.testing.assert_array_equal(a, b)


def test_dssim_gradient_matches_differences(orc):
    """Central differences of the loss at interior, edge and corner pixels of
    two views of different sizes."""
    rng = np.random.default_rng(15)
    xs = [rng.uniform(0.05, 0.95, (3, 14, 19)), rng.uniform(0.05, 0.95, (3, 11, 8))]
    ys = [np.clip(x + rng.normal(0, 0.15, x.shape), 0, 1) for x in xs]
    lam = 0.2
    _, g = orc.dssim_loss_grad(xs, ys, lam)
    h = 1e-6
    for v, idx in [(0, (0, 0, 0)), (0, (1, 7, 9)), (0, (2, 13, 18)), (1, (0, 0, 4)), (1, (2, 10, 7)), (1, (1, 5, 5))]:
        xp = [x.copy() for x in xs]
        xm = [x.copy() for x in xs]
        xp[v][idx] += h
        xm[v][idx] -= h
        fd = (orc.dssim_loss_grad(xp, ys, lam)[0] - orc.dssim_loss_grad(xm, ys, lam)[0]) / (2 * h)
        assert abs(fd - g[v][idx]) <= 1e-6 * abs(g[v][idx]) + 1e-11, (v, idx, fd, g[v][idx])
