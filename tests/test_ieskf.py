"""Camera-IMU chain and IESKF pose update (Appendix A) on the host, pinned by
finite differences through the matrix exponential, closed-form identities
and the FP64 oracle's photometric normal equations."""
import numpy as np
import pytest
import scipy.linalg
from scipy.spatial.transform import Rotation

from paper_2501_08672_b300 import ieskf


def _rand_pose(rng, scale=1.0):
    return Rotation.from_rotvec(rng.normal(0, 0.6, 3)).as_matrix(), rng.normal(0, scale, 3)


def _T(R, t):
    T = np.eye(4)
    T[:3, :3] = R
    T[:3, 3] = t
    return T


def test_so3_exp_log_against_scipy():
    rng = np.random.default_rng(1)
    for _ in range(20):
        w = rng.normal(0, 1.0, 3)
        R = ieskf.so3_exp(w)
        np.testing.assert_allclose(R, Rotation.from_rotvec(w).as_matrix(), atol=1e-12)
        np.testing.assert_allclose(ieskf.so3_log(R), Rotation.from_matrix(R).as_rotvec(), atol=1e-10)
    np.testing.assert_allclose(ieskf.so3_exp(np.zeros(3)), np.eye(3))


def test_camera_from_imu_jacobian_matches_central_differences():
    """xi = Log(T_CW' T_CW^-1) for T_CW' = T_CI (T_WI [+] dx)^-1, by central
    differences of scipy's logm, against J."""
    rng = np.random.default_rng(2)
    for _ in range(5):
        R_WI, p_WI = _rand_pose(rng, 3.0)
        R_CI, t_CI = _rand_pose(rng, 0.2)
        R_CW, t_CW = ieskf.camera_pose(R_WI, p_WI, R_CI, t_CI)
        np.testing.assert_allclose(_T(R_CW, t_CW), _T(R_CI, t_CI) @ np.linalg.inv(_T(R_WI, p_WI)), atol=1e-12)
        J = ieskf.camera_from_imu_jacobian(R_CI, t_CI, R_CW)
        h = 1e-6
        num = np.zeros((6, 6))
        for k in range(6):
            xs = []
            for sgn in (1.0, -1.0):
                dx = np.zeros(6)
                dx[k] = sgn * h
                R2, p2 = ieskf.boxplus(R_WI, p_WI, dx)
                Rc, tc = ieskf.camera_pose(R2, p2, R_CI, t_CI)
                X = np.real(scipy.linalg.logm(_T(Rc, tc) @ np.linalg.inv(_T(R_CW, t_CW))))
                xs.append(np.array([X[2, 1], X[0, 2], X[1, 0], X[0, 3], X[1, 3], X[2, 3]]))
            num[:, k] = (xs[0] - xs[1]) / (2 * h)
        np.testing.assert_allclose(J, num, atol=1e-6)
        # the rotation block is the paper's -R_CI
        np.testing.assert_allclose(J[:3, :3], -R_CI)


def test_update_without_prior_is_the_camera_gauss_newton_step():
    """P -> infinity: J dx = A_cam^-1 b_cam (J is invertible), and the
    posterior covariance vanishes with the prior's information."""
    rng = np.random.default_rng(3)
    M = rng.normal(size=(40, 6))
    A = M.T @ M
    b = rng.normal(size=6)
    R_CI, t_CI = _rand_pose(rng, 0.2)
    R_CW, _ = _rand_pose(rng)
    J = ieskf.camera_from_imu_jacobian(R_CI, t_CI, R_CW)
    dx, P = ieskf.ieskf_pose_update(A, b, J, 0.5, np.eye(6) * 1e12)
    np.testing.assert_allclose(J @ dx, np.linalg.solve(A, b), rtol=1e-6, atol=1e-9)
    np.testing.assert_allclose(P, 0.5 * np.linalg.inv(J.T @ A @ J), rtol=1e-5, atol=1e-12)


def test_update_properties_with_a_prior():
    """Posterior covariance symmetric, positive definite, below the prior;
    a zero measurement leaves the state at the prior mean."""
    rng = np.random.default_rng(4)
    M = rng.normal(size=(30, 6))
    A = M.T @ M
    b = rng.normal(size=6)
    R_CI, t_CI = _rand_pose(rng, 0.2)
    R_CW, _ = _rand_pose(rng)
    J = ieskf.camera_from_imu_jacobian(R_CI, t_CI, R_CW)
    L = rng.normal(size=(6, 6))
    P = L @ L.T + 0.1 * np.eye(6)
    dx, Pp = ieskf.ieskf_pose_update(A, b, J, 2.0, P)
    assert np.allclose(Pp, Pp.T)
    assert np.linalg.eigvalsh(Pp).min() > 0
    assert np.linalg.eigvalsh(P - Pp).min() > -1e-9
    off = rng.normal(0, 0.01, 6)
    dx0, _ = ieskf.ieskf_pose_update(np.zeros((6, 6)), np.zeros(6), J, 2.0, P, offset=off)
    np.testing.assert_allclose(dx0, -off, atol=1e-12)


def test_ieskf_recovers_imu_pose_from_oracle_normal_equations(orc):
    """Tiny scene, exact mode: the camera renders from T_CI T_WI^-1; starting
    from the true IMU pose perturbed by a small known dx, iterated updates
    with the oracle's photometric normal equations and a weak prior return to
    the true pose."""
    rng = np.random.default_rng(5)
    n = 30
    K = 4
    mu = np.stack([rng.uniform(-0.5, 0.5, n), rng.uniform(-0.4, 0.4, n), rng.uniform(2.0, 3.0, n)], 1)
    sh = rng.normal(0, 0.3, (n, K, 3))
    sh[:, 0, :] = rng.uniform(0.5, 1.5, (n, 3))
    p = dict(means=mu, log_scales=rng.normal(-2.0, 0.2, (n, 3)), quats=rng.standard_normal((n, 4)),
             opacity=rng.normal(0.5, 0.5, n), sh=sh, sh_degree=1)
    R_CI = Rotation.from_rotvec([0.02, -0.01, 0.03]).as_matrix()
    t_CI = np.array([0.05, -0.02, 0.01])
    R_WI_true = Rotation.from_rotvec([0.01, 0.02, -0.015]).as_matrix()
    p_WI_true = np.array([0.02, -0.01, 0.03])
    W, H = 48, 36

    def view(R_WI, p_WI):
        R_CW, t_CW = ieskf.camera_pose(R_WI, p_WI, R_CI, t_CI)
        return dict(R=R_CW, t=t_CW, fx=50.0, fy=50.0, cx=W / 2, cy=H / 2, W=W, H=H, g_begin=0, g_end=0)

    cfg = dict(orc.EXACT_CFG)
    target = orc.render_view(p, view(R_WI_true, p_WI_true), cfg)["rgb"]
    R, t = ieskf.boxplus(R_WI_true, p_WI_true, np.array([0.004, -0.003, 0.002, 0.006, -0.004, 0.005]))
    R_bar, t_bar = R.copy(), t.copy()
    P = np.eye(6) * 1.0
    e0 = np.linalg.norm(ieskf.boxminus(R, t, R_WI_true, p_WI_true))
    for _ in range(4):
        v = view(R, t)
        A, b, _, _ = orc.pose_normal(p, v, target, cfg)
        J = ieskf.camera_from_imu_jacobian(R_CI, t_CI, np.asarray(v["R"]))
        dx, P_post = ieskf.ieskf_pose_update(A, b, J, 1e-4, P, offset=ieskf.boxminus(R, t, R_bar, t_bar))
        R, t = ieskf.boxplus(R, t, dx)
    e1 = np.linalg.norm(ieskf.boxminus(R, t, R_WI_true, p_WI_true))
    assert e1 < 1e-3 * e0, (e0, e1)
