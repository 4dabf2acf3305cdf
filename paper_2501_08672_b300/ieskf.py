"""Camera-to-IMU pose chain and the pose block of the IESKF update (Sec. II-D,
Appendix A), on the host.

The state is the IMU pose T_WI = (R_WI, p_WI) with the error-state
perturbation dx = [dtheta; dp] of the paper's perturbation model (Appendix A):
R_WI <- R_WI Exp(dtheta), p_WI <- p_WI + dp.  The camera pose follows as
T_CW = T_CI T_WI^-1 with T_CI the fixed camera-IMU extrinsic.  The renderer's
pose derivatives are taken with respect to the left perturbation of the
camera, T_CW <- Exp(xi) T_CW, xi = [dphi; dt]; `camera_from_imu_jacobian`
gives the exact 6 x 6 map J = d xi / d dx at dx = 0:
    dphi = -R_CI dtheta,
    dt   = -[t_CI]x R_CI dtheta - R_CW dp.
The rotation block matches the paper's Eq. rot_jacobian; the translation
rows are derived here directly (the paper's decomposition of the
translation equation is garbled) and pinned by finite differences through
the matrix exponential in the tests.

`ieskf_pose_update` is one iteration of the iterated error-state Kalman
filter update (Appendix A, "IESKF Update Framework") for the pose block,
given the photometric normal equations from the GPU (gs_pose_normal):
A_cam = sum H_cam^T H_cam, b_cam = sum H_cam^T (target - render).  With
H = H_cam J, R = sigma^2 I and the prior covariance P of dx:
    K H = (J^T A_cam J / sigma^2 + P^-1)^-1 J^T A_cam J / sigma^2,
    dx  = (J^T A_cam J / sigma^2 + P^-1)^-1 (J^T b_cam / sigma^2)
          - (I - K H) (x_hat [-] x_bar),
    P+  = (I - K H) P = (J^T A_cam J / sigma^2 + P^-1)^-1,
where x_hat [-] x_bar is the current estimate's offset from the prior mean
(zero at the first iteration).  The Jacobian of [-] is taken as identity
(first order), as the paper's update does for small offsets.
"""
from __future__ import annotations

import math

import numpy as np


def skew(v):
    x, y, z = (float(c) for c in v)
    return np.array([[0.0, -z, y], [z, 0.0, -x], [-y, x, 0.0]])


def so3_exp(w):
    """Rodrigues' formula for Exp of a rotation vector."""
    w = np.asarray(w, np.float64)
    th = float(np.linalg.norm(w))
    K = skew(w)
    if th < 1e-12:
        return np.eye(3) + K + 0.5 * K @ K
    return np.eye(3) + math.sin(th) / th * K + (1.0 - math.cos(th)) / (th * th) * K @ K


def so3_log(R):
    """Rotation vector of a rotation matrix."""
    R = np.asarray(R, np.float64)
    c = max(-1.0, min(1.0, (np.trace(R) - 1.0) / 2.0))
    th = math.acos(c)
    v = np.array([R[2, 1] - R[1, 2], R[0, 2] - R[2, 0], R[1, 0] - R[0, 1]])
    if th < 1e-8:
        return 0.5 * v
    return th / (2.0 * math.sin(th)) * v


def camera_pose(R_WI, p_WI, R_CI, t_CI):
    """T_CW = T_CI T_WI^-1 as (R_CW, t_CW)."""
    R_WI = np.asarray(R_WI, np.float64)
    R_CW = np.asarray(R_CI, np.float64) @ R_WI.T
    t_CW = np.asarray(t_CI, np.float64) - R_CW @ np.asarray(p_WI, np.float64)
    return R_CW, t_CW


def camera_from_imu_jacobian(R_CI, t_CI, R_CW):
    """J = d xi / d dx (6 x 6), rows [dphi; dt], columns [dtheta; dp]."""
    R_CI = np.asarray(R_CI, np.float64)
    J = np.zeros((6, 6))
    J[:3, :3] = -R_CI
    J[3:, :3] = -skew(t_CI) @ R_CI
    J[3:, 3:] = -np.asarray(R_CW, np.float64)
    return J


def boxplus(R_WI, p_WI, dx):
    """T_WI [+] dx = (R_WI Exp(dtheta), p_WI + dp)."""
    dx = np.asarray(dx, np.float64)
    return np.asarray(R_WI, np.float64) @ so3_exp(dx[:3]), np.asarray(p_WI, np.float64) + dx[3:]


def boxminus(R_a, p_a, R_b, p_b):
    """(R_a, p_a) [-] (R_b, p_b) = [Log(R_b^T R_a); p_a - p_b]."""
    return np.concatenate([so3_log(np.asarray(R_b, np.float64).T @ np.asarray(R_a, np.float64)),
                           np.asarray(p_a, np.float64) - np.asarray(p_b, np.float64)])


def ieskf_pose_update(A_cam, b_cam, J, sigma2, P, offset=None):
    """One iterated update of the pose block: returns (dx, P_post)."""
    A = J.T @ np.asarray(A_cam, np.float64) @ J / sigma2
    b = J.T @ np.asarray(b_cam, np.float64) / sigma2
    Pinv = np.linalg.inv(np.asarray(P, np.float64))
    S = np.linalg.inv(A + Pinv)
    KH = S @ A
    dx = S @ b
    if offset is not None:
        dx = dx - (np.eye(6) - KH) @ np.asarray(offset, np.float64)
    # (I - K H) P = S P^-1 P = S, formed directly (no cancellation)
    return dx, 0.5 * (S + S.T)
