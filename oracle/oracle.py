"""FP64 CPU oracle for the Gaussian-splatting path (test infrastructure only).

Only the tests, the smoke check and the benchmark's CPU-baseline leg may use
this module.  It wraps the plain C implementation in `gs_oracle.c` (compiled
with gcc, loaded with ctypes) and adds the loss in numpy.  It imports nothing
from the CUDA package.

Functions, with the passage each restates:
  project        Sec. II-B.1, Eqs. 3dgs, q, spat
  render         Sec. II-B.2, Eq. raster (per pixel, front to back)
  l1_loss_grad   Sec. II-B.2, Eq. gaussian_optimization with the L1 norm
  backward       chain rule through all of the above, to the Gaussian
                 parameters and to the left-perturbed camera pose
                 (Appendix A, perturbation model)
  adam           Sec. II-B.2 ("Adam optimizer"), Kingma & Ba with bias
                 correction
  pose_jacobian  Sec. II-D, Eq. minimization: per-pixel d(rendered colour) /
                 d(left pose perturbation), forward mode
  pose_normal    the Gauss-Newton normal equations of the photometric
                 residual in the pose: sum H^T H, sum H^T (target - I)
  window_compact Sec. II-C Step 2: deletion and compaction of the window by
                 swapping survivors from the rear into the holes
  sh0_bilinear   Sec. II-B.2: SH0 initialisation from the bilinear colour of
                 the image at the projected mean
  sh_basis       the real spherical harmonics of degree <= 3 the colour uses
  ssim_map,      the photometric loss with a structural term, (1 - lambda) L1
  dssim_loss_grad  + lambda (1 - SSIM), SSIM of Wang et al. (2004) with an
                 11 x 11 Gaussian window (sigma 1.5), zero padding,
                 C1 = 0.01^2, C2 = 0.03^2 (the paper names only the L1 norm
                 of Eq. gaussian_optimization; this is the common 3D-GS
                 variant)
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gs_oracle.c")
_LIB = os.path.join(_HERE, "libgs_oracle.so")
_lib = None

# Truncated-mode defaults (the reading of the 3D-GS rasteriser constants).
DEFAULT_CFG = dict(alpha_min=1.0 / 255.0, alpha_max=0.99, T_min=1e-4, blur=0.3, z_near=0.2,
                   bg=(0.0, 0.0, 0.0))
# Exact mode: Eq. raster literally, every Gaussian at every pixel.
EXACT_CFG = dict(alpha_min=0.0, alpha_max=1.0, T_min=0.0, blur=0.3, z_near=0.2, bg=(0.0, 0.0, 0.0))


def build(force=False):
    """Compile gs_oracle.c into libgs_oracle.so next to it."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-shared", "-fPIC", _SRC, "-o", _LIB, "-lm"]
        subprocess.run(cmd, check=True)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        L.orc_project.argtypes = [ctypes.c_long] + [P] * 5 + [ctypes.c_int] + [P] * 11
        L.orc_render.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_long] + [P] * 12 + [ctypes.c_int]
        L.orc_render_pixels.argtypes = ([ctypes.c_long, P, P, ctypes.c_long] + [P] * 12 + [ctypes.c_int])
        L.orc_render_backward.argtypes = ([ctypes.c_int, ctypes.c_int, ctypes.c_long] + [P] * 14 +
                                          [ctypes.c_int])
        L.orc_render_backward_pixels.argtypes = ([ctypes.c_long, P, P, ctypes.c_long] + [P] * 14 +
                                                 [ctypes.c_int])
        L.orc_project_backward.argtypes = ([ctypes.c_long] + [P] * 5 + [ctypes.c_int] + [P] * 2 +
                                           [P] * 4 + [P] * 7)
        L.orc_adam.argtypes = [ctypes.c_long, P, P, P, P, ctypes.c_double, ctypes.c_double,
                               ctypes.c_double, ctypes.c_double, ctypes.c_long]
        L.orc_adam.restype = None
        L.orc_num_threads.restype = ctypes.c_int
        L.orc_set_num_threads.argtypes = [ctypes.c_int]
        L.orc_set_num_threads.restype = None
        L.orc_pose_jacobian_pixels.argtypes = ([ctypes.c_long, P, P, ctypes.c_long] + [P] * 5 + [ctypes.c_int] +
                                               [P] * 5 + [ctypes.c_int])
        L.orc_sh_basis.argtypes = [ctypes.c_long, P, ctypes.c_int, P, P]
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def cfg_array(cfg):
    c = dict(DEFAULT_CFG)
    c.update(cfg or {})
    return np.array([c["alpha_min"], c["alpha_max"], c["T_min"], c["blur"], c["z_near"],
                     *c["bg"]], dtype=np.float64)


def cam_array(view):
    R = np.asarray(view["R"], np.float64).reshape(9)
    t = np.asarray(view["t"], np.float64).reshape(3)
    return np.concatenate([R, t, [view["fx"], view["fy"], view["cx"], view["cy"]]]).astype(np.float64)


def _slice(params, view):
    b = int(view.get("g_begin", 0))
    e = int(view.get("g_end", 0)) or params["means"].shape[0]
    return b, e


def _params64(params, b, e):
    return (_f64(params["means"][b:e]), _f64(params["log_scales"][b:e]), _f64(params["quats"][b:e]),
            _f64(params["opacity"][b:e]), _f64(params["sh"][b:e]))


def project(params, view, cfg=None):
    """Per-Gaussian projection of one view (Eqs. 3dgs, q, spat)."""
    b, e = _slice(params, view)
    n = e - b
    mu, ls, qt, op, sh = _params64(params, b, e)
    out = dict(valid=np.zeros(n, np.int32), pc=np.zeros((n, 3)), q=np.zeros((n, 2)),
               sigma2=np.zeros((n, 3)), conic=np.zeros((n, 3)), opac=np.zeros(n),
               colour=np.zeros((n, 3)), raw_colour=np.zeros((n, 3)), depth_err=np.zeros(n))
    lib().orc_project(n, _p(mu), _p(ls), _p(qt), _p(op), _p(sh), int(params["sh_degree"]),
                      _p(cam_array(view)), _p(cfg_array(cfg)), _p(out["valid"]), _p(out["pc"]),
                      _p(out["q"]), _p(out["sigma2"]), _p(out["conic"]), _p(out["opac"]),
                      _p(out["colour"]), _p(out["raw_colour"]), _p(out["depth_err"]))
    out["depth"] = out["pc"][:, 2].copy()
    return out


def render_view(params, view, cfg=None, n_threads=0, proj=None):
    """Eq. raster for one view: returns rgb [3,H,W], T_final [H,W], contributor
    count [H,W], the borderline-pixel mask [H,W] and the opacities sigma of
    the Gaussians in front of the camera."""
    W, H = int(view["W"]), int(view["H"])
    pr = proj if proj is not None else project(params, view, cfg)
    n = pr["valid"].shape[0]
    rgb = np.zeros((3, H, W))
    T = np.zeros((H, W))
    nc = np.zeros((H, W), np.int32)
    bd = np.zeros((H, W), np.uint8)
    lib().orc_render(W, H, n, _p(pr["valid"]), _p(pr["q"]), _p(pr["conic"]), _p(pr["opac"]),
                     _p(pr["colour"]), _p(pr["depth"]), _p(pr["depth_err"]), _p(cfg_array(cfg)), _p(rgb), _p(T), _p(nc),
                     _p(bd), int(n_threads))
    return dict(rgb=rgb, T=T, n_contrib=nc, border=bd.astype(bool), sigma=pr["opac"][pr["valid"] == 1])


def render_pixels(params, view, px, py, cfg=None, n_threads=0, proj=None):
    """Eq. raster at the listed pixels of one view (same per-pixel compositing
    as render_view): rgb [n,3], T_final [n], contributor count [n], border [n]."""
    pr = proj if proj is not None else project(params, view, cfg)
    n = pr["valid"].shape[0]
    px = np.ascontiguousarray(px, np.int32)
    py = np.ascontiguousarray(py, np.int32)
    k = px.size
    rgb = np.zeros((k, 3))
    T = np.zeros(k)
    nc = np.zeros(k, np.int32)
    bd = np.zeros(k, np.uint8)
    lib().orc_render_pixels(k, _p(px), _p(py), n, _p(pr["valid"]), _p(pr["q"]), _p(pr["conic"]),
                            _p(pr["opac"]), _p(pr["colour"]), _p(pr["depth"]), _p(pr["depth_err"]), _p(cfg_array(cfg)), _p(rgb),
                            _p(T), _p(nc), _p(bd), int(n_threads))
    return dict(rgb=rgb, T=T, n_contrib=nc, border=bd.astype(bool), sigma=pr["opac"][pr["valid"] == 1])


def render(params, views, cfg=None, n_threads=0):
    return [render_view(params, v, cfg, n_threads) for v in views]


def l1_loss_grad(rgbs, targets):
    """L = (1/V) sum_v mean |I_hat - I| and dL/dI_hat = sign(I_hat - I)/(3HW V),
    sign(0) = 0 (Eq. gaussian_optimization with the L1 norm)."""
    V = len(rgbs)
    L = 0.0
    grads = []
    for r, t in zip(rgbs, targets):
        d = np.asarray(r, np.float64) - np.asarray(t, np.float64)
        L += np.abs(d).mean() / V
        grads.append(np.sign(d) / (d.size * V))
    return L, grads


SSIM_C1 = 0.01 ** 2
SSIM_C2 = 0.03 ** 2


def ssim_window(size=11, sigma=1.5):
    """Normalised 1D Gaussian taps g[k] ~ exp(-(k - size//2)^2 / (2 sigma^2));
    the 2D window is the outer product g g^T."""
    k = np.arange(size) - size // 2
    g = np.exp(-(k * k) / (2.0 * sigma * sigma))
    return g / g.sum()


def _window_mean(img, g):
    """Windowed mean of a [H, W] plane: sum_{a,b} g[a] g[b] img[y + a - r,
    x + b - r] over the pixels inside the image (zero padding), the window
    centred on each pixel.  scipy's correlate serves as the step."""
    import scipy.ndimage
    return scipy.ndimage.correlate(img, np.outer(g, g), mode="constant", cval=0.0)


def ssim_map(x, y, size=11, sigma=1.5):
    """Per-pixel SSIM of [C, H, W] images x (rendered) and y (target):
    ((2 mu_x mu_y + C1)(2 s_xy + C2)) / ((mu_x^2 + mu_y^2 + C1)(s_x^2 + s_y^2 + C2))
    with mu, s^2, s_xy the windowed means, variances E[x^2] - mu^2 and
    covariance E[xy] - mu_x mu_y, per channel."""
    g = ssim_window(size, sigma)
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    out = np.empty_like(x)
    for c in range(x.shape[0]):
        mx, my = _window_mean(x[c], g), _window_mean(y[c], g)
        sxx = _window_mean(x[c] * x[c], g) - mx * mx
        syy = _window_mean(y[c] * y[c], g) - my * my
        sxy = _window_mean(x[c] * y[c], g) - mx * my
        out[c] = ((2 * mx * my + SSIM_C1) * (2 * sxy + SSIM_C2)) / \
                 ((mx * mx + my * my + SSIM_C1) * (sxx + syy + SSIM_C2))
    return out


def dssim_loss_grad(rgbs, targets, lam=0.2, size=11, sigma=1.5):
    """L = (1/V) sum_v [(1 - lam) mean |x - y| + lam (1 - mean SSIM(x, y))] over
    views v with x the rendered image [3, H, W] and y the target; returns L
    and dL/dx per view.  The SSIM term's gradient: with s the SSIM map and
    the window means mu_x = G * x, E_xx = G * x^2, E_xy = G * (x y),
    ds(q)/dx(p) = G(q - p) [ds/dmu_x + 2 x(p) ds/dE_xx + y(p) ds/dE_xy](q),
    and the window G is symmetric, so the sum over q is again a windowed mean
    of the three partial-derivative maps."""
    g = ssim_window(size, sigma)
    V = len(rgbs)
    L = 0.0
    grads = []
    for xr, yr in zip(rgbs, targets):
        x = np.asarray(xr, np.float64)
        y = np.asarray(yr, np.float64)
        n = x.size
        d = x - y
        grad = (1.0 - lam) * np.sign(d) / (n * V)
        smean = 0.0
        for c in range(x.shape[0]):
            mx, my = _window_mean(x[c], g), _window_mean(y[c], g)
            exx, eyy, exy = _window_mean(x[c] * x[c], g), _window_mean(y[c] * y[c], g), _window_mean(x[c] * y[c], g)
            a1 = 2 * mx * my + SSIM_C1
            a2 = 2 * (exy - mx * my) + SSIM_C2
            b1 = mx * mx + my * my + SSIM_C1
            b2 = (exx - mx * mx) + (eyy - my * my) + SSIM_C2
            s = a1 * a2 / (b1 * b2)
            smean += s.sum()
            # partial derivatives of s with respect to mu_x, E_xx, E_xy
            d_mx = (2 * my * a2 - 2 * my * a1) / (b1 * b2) - s * (2 * mx / b1 - 2 * mx / b2)
            d_exx = -s / b2
            d_exy = 2 * a1 / (b1 * b2)
            ds_dx = _window_mean(d_mx, g) + 2 * x[c] * _window_mean(d_exx, g) + y[c] * _window_mean(d_exy, g)
            grad[c] -= lam * ds_dx / (n * V)
        L += ((1.0 - lam) * np.abs(d).mean() + lam * (1.0 - smean / n)) / V
        grads.append(grad)
    return L, grads


def backward(params, views, dL_drgbs, cfg=None, n_threads=0, pixels=None):
    """Gradients of a loss with dL/d(rgb) given per view, with respect to every
    Gaussian parameter (summed over views) and to each view's pose
    (dL/d(dphi, dt) for T_CW <- Exp(dphi, dt) T_CW).  Also returns a per-Gaussian
    mask of gradients that FP32 may legitimately decide differently.

    pixels: None (dL_drgbs[v] is [3,H,W]) or a list of (px, py) index arrays
    per view, with dL_drgbs[v] of shape [len(px), 3]: the loss then depends
    only on those pixels."""
    N = params["means"].shape[0]
    K = params["sh"].shape[1]
    g = dict(means=np.zeros((N, 3)), log_scales=np.zeros((N, 3)), quats=np.zeros((N, 4)),
             opacity=np.zeros(N), sh=np.zeros((N, K, 3)))
    pose = np.zeros((len(views), 6))
    border = np.zeros(N, bool)
    ca = cfg_array(cfg)
    for vi, view in enumerate(views):
        b, e = _slice(params, view)
        n = e - b
        pr = project(params, view, cfg)
        gq = np.zeros((n, 2)); gc = np.zeros((n, 3)); go = np.zeros(n); gcol = np.zeros((n, 3))
        gb = np.zeros(n, np.uint8)
        dl = _f64(dL_drgbs[vi])
        if pixels is None:
            W, H = int(view["W"]), int(view["H"])
            lib().orc_render_backward(W, H, n, _p(pr["valid"]), _p(pr["q"]), _p(pr["conic"]),
                                      _p(pr["opac"]), _p(pr["colour"]), _p(pr["depth"]), _p(pr["depth_err"]), _p(ca), _p(dl),
                                      _p(gq), _p(gc), _p(go), _p(gcol), _p(gb), int(n_threads))
        else:
            px = np.ascontiguousarray(pixels[vi][0], np.int32)
            py = np.ascontiguousarray(pixels[vi][1], np.int32)
            lib().orc_render_backward_pixels(px.size, _p(px), _p(py), n, _p(pr["valid"]), _p(pr["q"]),
                                             _p(pr["conic"]), _p(pr["opac"]), _p(pr["colour"]),
                                             _p(pr["depth"]), _p(pr["depth_err"]), _p(ca), _p(dl), _p(gq),
                                             _p(gc), _p(go),
                                             _p(gcol), _p(gb), int(n_threads))
        mu, ls, qt, op, sh = _params64(params, b, e)
        gm = np.zeros((n, 3)); gl = np.zeros((n, 3)); gqt = np.zeros((n, 4)); gop = np.zeros(n)
        gsh = np.zeros((n, K, 3)); gpose = np.zeros(6); gbc = np.zeros(n, np.uint8)
        lib().orc_project_backward(n, _p(mu), _p(ls), _p(qt), _p(op), _p(sh), int(params["sh_degree"]),
                                   _p(cam_array(view)), _p(ca), _p(gq), _p(gc), _p(go), _p(gcol),
                                   _p(gm), _p(gl), _p(gqt), _p(gop), _p(gsh), _p(gpose), _p(gbc))
        g["means"][b:e] += gm
        g["log_scales"][b:e] += gl
        g["quats"][b:e] += gqt
        g["opacity"][b:e] += gop
        g["sh"][b:e] += gsh
        pose[vi] = gpose
        border[b:e] |= (gb != 0) | (gbc != 0)
    return g, pose, border


def adam(p, g, m, v, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8, step=1):
    """One Adam step in place on float64 arrays."""
    for a in (p, g, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    lib().orc_adam(p.size, _p(p), _p(g), _p(m), _p(v), lr, b1, b2, eps, int(step))


def num_threads():
    """Host threads the parallel loops use when a call passes n_threads=0."""
    return int(lib().orc_num_threads())


def set_threads(n):
    """Sets the host thread count of calls that pass n_threads=0 (n <= 0:
    every processor).  Results do not depend on it."""
    lib().orc_set_num_threads(int(n))


def pose_jacobian(params, view, px, py, cfg=None, n_threads=0):
    """Per-pixel pose Jacobian H [n, 3, 6] of the rendered colour at pixels
    (px, py) of one view, with respect to xi = [dphi; dt], T_CW <- Exp(xi) T_CW
    (forward mode through Eq. raster); also rgb [n, 3] and the borderline
    mask [n]."""
    b, e = _slice(params, view)
    n = e - b
    mu, ls, qt, op, sh = _params64(params, b, e)
    px = np.ascontiguousarray(px, np.int32)
    py = np.ascontiguousarray(py, np.int32)
    k = px.size
    H = np.zeros((k, 3, 6))
    rgb = np.zeros((k, 3))
    bd = np.zeros(k, np.uint8)
    lib().orc_pose_jacobian_pixels(k, _p(px), _p(py), n, _p(mu), _p(ls), _p(qt), _p(op), _p(sh),
                                   int(params["sh_degree"]), _p(cam_array(view)), _p(cfg_array(cfg)), _p(H),
                                   _p(rgb), _p(bd), int(n_threads))
    return H, rgb, bd.astype(bool)


def pose_normal(params, view, target, cfg=None, n_threads=0):
    """Normal equations of the photometric residual r = target - I over every
    pixel of one view: A = sum_p sum_ch H H^T (6 x 6), b = sum H r (6),
    rr = sum r^2, with H from pose_jacobian (target is [3, H, W]).  Also
    returns the borderline mask [H, W]."""
    W, Hh = int(view["W"]), int(view["H"])
    vv, uu = np.mgrid[0:Hh, 0:W]
    Hj, rgb, bd = pose_jacobian(params, view, uu.reshape(-1), vv.reshape(-1), cfg, n_threads)
    r = np.asarray(target, np.float64).reshape(3, -1).T - rgb          # [n, 3]
    A = np.einsum("pci,pcj->ij", Hj, Hj)
    b = np.einsum("pci,pc->i", Hj, r)
    return A, b, float((r * r).sum()), bd.reshape(Hh, W)


def sh_basis(dirs, degree):
    """Real spherical harmonics (Condon-Shortley phase, k = l^2 + l + m) of
    degree <= 3 at unit directions dirs [n, 3], and their partial derivatives
    as homogeneous polynomials: (Y [n, 16], dY [n, 16, 3]); entries above the
    degree are 0."""
    d = _f64(dirs).reshape(-1, 3)
    n = d.shape[0]
    Y = np.zeros((n, 16))
    dY = np.zeros((n, 16, 3))
    if lib().orc_sh_basis(n, _p(d), int(degree), _p(Y), _p(dY)) != 0:
        raise ValueError("degree %d outside [0, 3]" % degree)
    return Y, dY


def window_compact(keep):
    """Sec. II-C Step 2 (deletion and compaction).  Rows whose keep flag is
    false are removed by swapping rows from the rear of the window into them:
    walking the holes front to back, each takes the last surviving row that
    has not moved yet, as long as that row lies behind the hole.  Returns
    moved_from: for every row r < n_keep, the row whose data r holds."""
    keep = np.asarray(keep).astype(bool)
    n = keep.size
    rows = list(range(n))
    alive = keep.copy()
    tail = n - 1
    for h in range(n):
        if alive[h]:
            continue
        while tail > h and not alive[tail]:
            tail -= 1
        if tail <= h:
            break
        rows[h], alive[h] = rows[tail], True
        alive[tail] = False
        tail -= 1
    n_keep = int(keep.sum())
    return np.array(rows[:n_keep], dtype=np.int64)


def sh0_bilinear(means, view, image, sh_degree, z_near=0.2):
    """Sec. II-B.2: SH coefficients of new Gaussians whose degree-0 colour is
    the bilinear interpolation of image [3, H, W] at the projected mean (pixel
    (u, v) at (u + 0.5, v + 0.5), weights the areas of the opposite
    sub-rectangles, clamped at the border); c = 0.5 where the mean is behind
    z_near or projects outside the image.  Returns [n, (D+1)^2, 3]."""
    means = np.asarray(means, np.float64)
    R = np.asarray(view["R"], np.float64)
    t = np.asarray(view["t"], np.float64)
    W, H = int(view["W"]), int(view["H"])
    img = np.asarray(image, np.float64)
    K = (sh_degree + 1) ** 2
    out = np.zeros((means.shape[0], K, 3))
    c0 = 0.5 / np.sqrt(np.pi)
    for i, mu in enumerate(means):
        pc = R @ mu + t
        c = np.full(3, 0.5)
        if pc[2] > z_near:
            u = view["fx"] * pc[0] / pc[2] + view["cx"] - 0.5
            v = view["fy"] * pc[1] / pc[2] + view["cy"] - 0.5
            if -0.5 < u < W - 0.5 and -0.5 < v < H - 0.5:
                u = min(max(u, 0.0), W - 1.0)
                v = min(max(v, 0.0), H - 1.0)
                u0, v0 = int(np.floor(u)), int(np.floor(v))
                u1, v1 = min(u0 + 1, W - 1), min(v0 + 1, H - 1)
                a, b = u - u0, v - v0
                c = ((1 - a) * (1 - b) * img[:, v0, u0] + a * (1 - b) * img[:, v0, u1] +
                     (1 - a) * b * img[:, v1, u0] + a * b * img[:, v1, u1])
        out[i, 0, :] = (c - 0.5) / c0
    return out

