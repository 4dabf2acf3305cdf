"""ctypes binding of libgs_b300.so (include/gs.h): argument marshalling only.

Every step of the path runs in the library's CUDA kernels; this module builds
the C structs from torch tensors and view dicts and checks return codes.  It
raises if the library is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np
import torch  # noqa: F401  (loads the CUDA runtime the library links against)

HERE = os.path.dirname(os.path.abspath(__file__))
# GS_B300_LIB=checked loads the checked build (bounds-checked compositing
# kernels, `python -m paper_2501_08672_b300.build --checked`).
LIB_NAME = "libgs_b300_checked.so" if os.environ.get("GS_B300_LIB", "") == "checked" else "libgs_b300.so"
LIB_PATH = os.path.join(HERE, LIB_NAME)

GS_OK = 0
GS_ERR_INVALID_ARG = -1
GS_ERR_CUDA = -2
GS_ERR_OOM = -3
GS_ERR_CAPACITY = -4
GS_ERR_TIMEOUT = -5
GS_ERR_NONFINITE = -6
GS_ERR_UNSUPPORTED = -7
GS_ERR_BOUNDS = -8
GS_F32, GS_F16, GS_BF16 = 0, 1, 2
GS_MAX_VIEWS = 64

_DTYPE = {torch.float32: GS_F32, torch.float16: GS_F16, torch.bfloat16: GS_BF16}

EXPORTED = ["gs_config_default", "gs_version", "gs_context_create", "gs_context_destroy", "gs_last_error",
            "gs_get_config", "gs_workspace_query", "gs_workspace_layout", "gs_project", "gs_bin",
            "gs_render_fwd", "gs_l1_loss", "gs_render_bwd", "gs_pose_grad", "gs_adam_step", "gs_sync_status",
            "gs_profile_enable", "gs_profile_collect", "gs_launch_count", "gs_adam_step_dev",
            "gs_l1_loss_noalloc", "gs_calibrate_alu", "gs_pose_normal_scratch", "gs_pose_normal",
            "gs_window_scratch_bytes", "gs_window_compact", "gs_window_remove", "gs_window_gather", "gs_window_clear",
            "gs_sh_init_bilinear", "gs_dssim_scratch_floats", "gs_dssim_loss", "gs_adam_step_ranges",
            "gs_selftest_wait_scratch_bytes", "gs_selftest_bounded_wait", "gs_render_fwd_l1",
            "gs_render_bwd_accumulate", "gs_checked_build"]

KERNEL_FAMILIES = ["project", "depth_sort", "tile_scan", "emit", "tile_sort", "ranges", "raster_fwd", "l1",
                   "raster_bwd", "project_bwd", "adam", "pose_normal", "window", "ssim", "refine"]


class WindowColumn(ctypes.Structure):
    _fields_ = [("ptr", ctypes.c_void_p), ("bytes_per_gaussian", ctypes.c_int32)]


class GsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("gs status %d: %s" % (code, msg))
        self.code = code


class Config(ctypes.Structure):
    _fields_ = [("tile_size", ctypes.c_int32), ("alpha_min", ctypes.c_float), ("alpha_max", ctypes.c_float),
                ("T_min", ctypes.c_float), ("blur", ctypes.c_float), ("z_near", ctypes.c_float),
                ("bg", ctypes.c_float * 3), ("pixels_per_thread", ctypes.c_int32), ("batch", ctypes.c_int32),
                ("deterministic", ctypes.c_int32), ("bin_tile_size", ctypes.c_int32)]


class View(ctypes.Structure):
    _fields_ = [("R_cw", ctypes.c_float * 9), ("t_cw", ctypes.c_float * 3), ("fx", ctypes.c_float),
                ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32), ("g_begin", ctypes.c_int64),
                ("g_end", ctypes.c_int64)]


class Gaussians(ctypes.Structure):
    _fields_ = [("means", ctypes.c_void_p), ("log_scales", ctypes.c_void_p), ("quats", ctypes.c_void_p),
                ("opacity", ctypes.c_void_p), ("sh", ctypes.c_void_p), ("scale_dtype", ctypes.c_int32),
                ("rot_dtype", ctypes.c_int32), ("opacity_dtype", ctypes.c_int32), ("sh_dtype", ctypes.c_int32),
                ("n", ctypes.c_int64), ("sh_degree", ctypes.c_int32)]


class Grads(ctypes.Structure):
    _fields_ = [("means", ctypes.c_void_p), ("log_scales", ctypes.c_void_p), ("quats", ctypes.c_void_p),
                ("opacity", ctypes.c_void_p), ("sh", ctypes.c_void_p)]


class Workspace(ctypes.Structure):
    _fields_ = [("ptr", ctypes.c_void_p), ("bytes", ctypes.c_size_t), ("max_pairs", ctypes.c_int64)]


class WsLayout(ctypes.Structure):
    _fields_ = [(n, ctypes.c_size_t) for n in ("records", "rects", "tiles_touched", "depth_keys", "depth_hi",
                                               "depth_vals",
                                               "pair_offsets", "pair_keys", "pair_vals", "sorted_vals",
                                               "tile_ranges", "grad2d", "counters", "total")] + [
        ("n_records", ctypes.c_int64), ("n_tiles", ctypes.c_int32), ("n_pixels", ctypes.c_int64),
        ("bin_keys", ctypes.c_size_t), ("bin_vals", ctypes.c_size_t), ("bin_ranges", ctypes.c_size_t),
        ("n_bins", ctypes.c_int32),
        ("bin_size", ctypes.c_int32)]


class ProfileEntry(ctypes.Structure):
    _fields_ = [("family", ctypes.c_int32), ("launches", ctypes.c_int32), ("total_ms", ctypes.c_double)]


class Range(ctypes.Structure):
    _fields_ = [("begin", ctypes.c_int64), ("end", ctypes.c_int64)]


class LowpSegment(ctypes.Structure):
    _fields_ = [("begin", ctypes.c_int64), ("end", ctypes.c_int64), ("dtype", ctypes.c_int32),
                ("dst", ctypes.c_void_p)]


_lib = None


def lib():
    """Loads libgs_b300.so; raises if it is missing (build it with
    `python -m paper_2501_08672_b300.build`)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("%s not found at %s: build it with `python -m paper_2501_08672_b300.build%s`"
                               % (LIB_NAME, LIB_PATH, " --checked" if "checked" in LIB_NAME else ""))
        L = ctypes.CDLL(LIB_PATH)
        P, I, I64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
        L.gs_config_default.argtypes = [ctypes.POINTER(Config)]
        L.gs_config_default.restype = None
        L.gs_checked_build.restype = ctypes.c_int32
        L.gs_version.restype = ctypes.c_char_p
        L.gs_context_create.argtypes = [ctypes.POINTER(P), I, ctypes.POINTER(Config)]
        L.gs_context_destroy.argtypes = [P]
        L.gs_last_error.argtypes = [P]
        L.gs_last_error.restype = ctypes.c_char_p
        L.gs_get_config.argtypes = [P, ctypes.POINTER(Config)]
        L.gs_workspace_query.argtypes = [P, ctypes.POINTER(View), I, I64, ctypes.POINTER(ctypes.c_size_t)]
        L.gs_workspace_layout.argtypes = [P, ctypes.POINTER(View), I, I64, ctypes.POINTER(WsLayout)]
        L.gs_project.argtypes = [P, ctypes.POINTER(Gaussians), ctypes.POINTER(View), I, ctypes.POINTER(Workspace), P]
        L.gs_bin.argtypes = [P, ctypes.POINTER(View), I, ctypes.POINTER(Workspace), ctypes.POINTER(ctypes.c_uint64), P]
        L.gs_render_fwd.argtypes = [P, ctypes.POINTER(View), I, ctypes.POINTER(Workspace), P, P, P, P, P]
        L.gs_l1_loss.argtypes = [P, ctypes.POINTER(View), I, ctypes.POINTER(Workspace), P, P, P, P, P]
        L.gs_render_fwd_l1.argtypes = [P, ctypes.POINTER(View), I, ctypes.POINTER(Workspace), P, P, P, P, P, P, P,
                                       P]
        L.gs_render_bwd.argtypes = [P, ctypes.POINTER(Gaussians), ctypes.POINTER(View), I, ctypes.POINTER(Workspace),
                                    P, P, P, ctypes.POINTER(Grads), P, P]
        L.gs_render_bwd_accumulate.argtypes = L.gs_render_bwd.argtypes
        L.gs_pose_grad.argtypes = [P, ctypes.POINTER(Gaussians), ctypes.POINTER(View), I, ctypes.POINTER(Workspace),
                                   P, P, P, P, P]
        L.gs_adam_step.argtypes = [P, P, P, P, P, I64, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                   ctypes.c_float, I64, ctypes.POINTER(LowpSegment), I, P]
        L.gs_adam_step_dev.argtypes = [P, P, P, P, P, I64, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                       ctypes.c_float, P, ctypes.POINTER(LowpSegment), I, P]
        L.gs_adam_step_ranges.argtypes = [P, P, P, P, P, I64, ctypes.POINTER(Range), I, ctypes.c_float,
                                          ctypes.c_float, ctypes.c_float, ctypes.c_float, I64, P,
                                          ctypes.POINTER(LowpSegment), I, P]
        L.gs_sync_status.argtypes = [P, P, ctypes.POINTER(ctypes.c_uint64)]
        L.gs_selftest_wait_scratch_bytes.argtypes = []
        L.gs_selftest_wait_scratch_bytes.restype = ctypes.c_size_t
        L.gs_selftest_bounded_wait.argtypes = [P, P, P]
        L.gs_dssim_scratch_floats.argtypes = [ctypes.POINTER(View), I]
        L.gs_dssim_scratch_floats.restype = ctypes.c_size_t
        L.gs_dssim_loss.argtypes = [P, ctypes.POINTER(View), I, P, P, ctypes.c_float, P, P, P, P]
        L.gs_l1_loss_noalloc.argtypes = [ctypes.POINTER(View), I, P, P, P, P, P, ctypes.c_char_p, ctypes.c_size_t]
        L.gs_profile_enable.argtypes = [P, ctypes.c_uint32]
        L.gs_profile_collect.argtypes = [P, P, ctypes.POINTER(ProfileEntry), I, ctypes.POINTER(ctypes.c_int)]
        L.gs_launch_count.argtypes = [P]
        L.gs_launch_count.restype = ctypes.c_int64
        L.gs_calibrate_alu.argtypes = [P, P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
        L.gs_pose_normal_scratch.argtypes = [P, ctypes.POINTER(View), I, ctypes.POINTER(ctypes.c_size_t)]
        L.gs_window_scratch_bytes.argtypes = [I64]
        L.gs_window_scratch_bytes.restype = ctypes.c_size_t
        L.gs_window_compact.argtypes = [P, ctypes.POINTER(WindowColumn), I, I64, P, P, P, P, P]
        L.gs_window_remove.argtypes = [P, ctypes.POINTER(WindowColumn), ctypes.POINTER(WindowColumn), I, I64, P, P, P,
                                       P, P, P]
        L.gs_window_gather.argtypes = [P, ctypes.POINTER(WindowColumn), ctypes.POINTER(WindowColumn), I, I64, P,
                                       I64, P]
        L.gs_window_clear.argtypes = [P, ctypes.POINTER(WindowColumn), I, I64, I64, P]
        L.gs_sh_init_bilinear.argtypes = [P, ctypes.POINTER(Gaussians), ctypes.POINTER(View), P, I64, I64, P, P]
        L.gs_pose_normal.argtypes = [P, ctypes.POINTER(Gaussians), ctypes.POINTER(View), I,
                                     ctypes.POINTER(Workspace), P, P, P, P, P]
        _lib = L
    return _lib


def default_config(**kw):
    c = Config()
    lib().gs_config_default(ctypes.byref(c))
    for k, v in kw.items():
        if k == "bg":
            for i in range(3):
                c.bg[i] = float(v[i])
        else:
            setattr(c, k, v)
    return c


def make_views(views):
    """Host array of gs_view from view dicts (R, t, fx, fy, cx, cy, W, H,
    g_begin, g_end)."""
    arr = (View * len(views))()
    for i, v in enumerate(views):
        R = np.asarray(v["R"], np.float32).reshape(9)
        t = np.asarray(v["t"], np.float32).reshape(3)
        for k in range(9):
            arr[i].R_cw[k] = float(R[k])
        for k in range(3):
            arr[i].t_cw[k] = float(t[k])
        arr[i].fx, arr[i].fy, arr[i].cx, arr[i].cy = float(v["fx"]), float(v["fy"]), float(v["cx"]), float(v["cy"])
        arr[i].width, arr[i].height = int(v["W"]), int(v["H"])
        arr[i].g_begin, arr[i].g_end = int(v["g_begin"]), int(v["g_end"])
    return arr


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _check_dev(t, name, dtype=None, numel=None):
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous()):
        raise ValueError("%s must be a contiguous CUDA tensor" % name)
    if dtype is not None and t.dtype != dtype:
        raise ValueError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if numel is not None and t.numel() != numel:
        raise ValueError("%s must have %d elements, got %d" % (name, numel, t.numel()))


def gaussians_struct(means, log_scales, quats, opacity, sh, sh_degree):
    n = means.shape[0]
    K = (sh_degree + 1) ** 2
    _check_dev(means, "means", torch.float32, 3 * n)
    _check_dev(log_scales, "log_scales", None, 3 * n)
    _check_dev(quats, "quats", None, 4 * n)
    _check_dev(opacity, "opacity", None, n)
    _check_dev(sh, "sh", None, 3 * K * n)
    g = Gaussians()
    g.means, g.log_scales, g.quats = means.data_ptr(), log_scales.data_ptr(), quats.data_ptr()
    g.opacity, g.sh = opacity.data_ptr(), sh.data_ptr()
    g.scale_dtype, g.rot_dtype = _DTYPE[log_scales.dtype], _DTYPE[quats.dtype]
    g.opacity_dtype, g.sh_dtype = _DTYPE[opacity.dtype], _DTYPE[sh.dtype]
    g.n = n
    g.sh_degree = sh_degree
    return g


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Context:
    """One gs_ctx: configuration, status block, and the C-ABI calls."""

    def __init__(self, device=0, **cfg):
        self.cfg = default_config(**cfg)
        self.device = device
        h = ctypes.c_void_p()
        rc = lib().gs_context_create(ctypes.byref(h), int(device), ctypes.byref(self.cfg))
        if rc != GS_OK:
            raise GsError(rc, "gs_context_create failed")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().gs_context_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _ck(self, rc):
        if rc != GS_OK:
            raise GsError(rc, lib().gs_last_error(self.h).decode())
        return rc

    def workspace_bytes(self, views, max_pairs):
        n = ctypes.c_size_t()
        self._ck(lib().gs_workspace_query(self.h, views, len(views), int(max_pairs), ctypes.byref(n)))
        return n.value

    def layout(self, views, max_pairs):
        L = WsLayout()
        self._ck(lib().gs_workspace_layout(self.h, views, len(views), int(max_pairs), ctypes.byref(L)))
        return L

    @staticmethod
    def ws_struct(ws_tensor, max_pairs):
        w = Workspace()
        w.ptr, w.bytes, w.max_pairs = ws_tensor.data_ptr(), ws_tensor.numel(), int(max_pairs)
        return w

    def project(self, g, views, ws, stream=None):
        self._ck(lib().gs_project(self.h, ctypes.byref(g), views, len(views), ctypes.byref(ws), _stream(stream)))

    def bin(self, views, ws, want_count=False, stream=None):
        """Returns the pair count (synchronising) when want_count, else None.
        Raises GsError(GS_ERR_CAPACITY) when want_count and the workspace is
        too small."""
        if want_count:
            n = ctypes.c_uint64()
            rc = lib().gs_bin(self.h, views, len(views), ctypes.byref(ws), ctypes.byref(n), _stream(stream))
            if rc == GS_ERR_CAPACITY:
                err = GsError(rc, lib().gs_last_error(self.h).decode())
                err.pairs_needed = n.value
                # clear the latched device status as well
                lib().gs_sync_status(self.h, _stream(stream), None)
                raise err
            self._ck(rc)
            return n.value
        self._ck(lib().gs_bin(self.h, views, len(views), ctypes.byref(ws), None, _stream(stream)))
        return None

    def render_fwd(self, views, ws, rgb, T_final, n_contrib, n_used=None, stream=None):
        self._ck(lib().gs_render_fwd(self.h, views, len(views), ctypes.byref(ws), _ptr(rgb), _ptr(T_final),
                                     _ptr(n_contrib), _ptr(n_used), _stream(stream)))

    def render_fwd_l1(self, views, ws, target, rgb, T_final, n_contrib, dL_drgb, loss=None, n_used=None,
                      stream=None):
        """Compositing with the L1 loss folded in (rgb may be None: image not written)."""
        self._ck(lib().gs_render_fwd_l1(self.h, views, len(views), ctypes.byref(ws), _ptr(target), _ptr(rgb),
                                        _ptr(T_final), _ptr(n_contrib), _ptr(n_used), _ptr(dL_drgb), _ptr(loss),
                                        _stream(stream)))

    def l1_loss(self, views, ws, rgb, target, dL_drgb, loss=None, stream=None):
        self._ck(lib().gs_l1_loss(self.h, views, len(views), ctypes.byref(ws), _ptr(rgb), _ptr(target),
                                  _ptr(dL_drgb), _ptr(loss), _stream(stream)))

    def dssim_loss(self, views, rgb, target, lam, scratch, dL_drgb, loss=None, stream=None):
        """(1 - lam) L1 + lam (1 - SSIM) and its gradient; scratch: FP32 device
        tensor of dssim_scratch_floats(views) elements."""
        _check_dev(scratch, "scratch", torch.float32, int(lib().gs_dssim_scratch_floats(views, len(views))))
        self._ck(lib().gs_dssim_loss(self.h, views, len(views), _ptr(rgb), _ptr(target), float(lam), _ptr(scratch),
                                     _ptr(dL_drgb), _ptr(loss), _stream(stream)))

    def render_bwd(self, g, views, ws, T_final, n_contrib, dL_drgb, grads=None, dL_dpose=None, stream=None,
                   accumulate=False):
        gr = None
        if grads is not None:
            gr = Grads()
            gr.means, gr.log_scales, gr.quats, gr.opacity, gr.sh = [t.data_ptr() for t in grads]
        fn = lib().gs_render_bwd_accumulate if accumulate else lib().gs_render_bwd
        self._ck(fn(self.h, ctypes.byref(g), views, len(views), ctypes.byref(ws), _ptr(T_final),
                    _ptr(n_contrib), _ptr(dL_drgb), ctypes.byref(gr) if gr is not None else None,
                    _ptr(dL_dpose), _stream(stream)))

    def pose_grad(self, g, views, ws, T_final, n_contrib, dL_drgb, dL_dpose, stream=None):
        self._ck(lib().gs_pose_grad(self.h, ctypes.byref(g), views, len(views), ctypes.byref(ws), _ptr(T_final),
                                    _ptr(n_contrib), _ptr(dL_drgb), _ptr(dL_dpose), _stream(stream)))

    def pose_normal_scratch(self, views):
        """FP32 scratch floats gs_pose_normal needs for this batch of views."""
        n = ctypes.c_size_t()
        self._ck(lib().gs_pose_normal_scratch(self.h, views, len(views), ctypes.byref(n)))
        return int(n.value)

    def pose_normal(self, g, views, ws, target, scratch, normal, H_pix=None, stream=None):
        """Per-view Gauss-Newton normal equations of the photometric residual in
        the pose: normal [n_views, 28] float64 (A upper triangle, b, r.r)."""
        _check_dev(normal, "normal", torch.float64, 28 * len(views))
        self._ck(lib().gs_pose_normal(self.h, ctypes.byref(g), views, len(views), ctypes.byref(ws), _ptr(target),
                                      _ptr(scratch), _ptr(normal), _ptr(H_pix), _stream(stream)))

    @staticmethod
    def _columns(tensors):
        """WindowColumn array for [n, ...] tensors (row i = Gaussian i)."""
        cols = (WindowColumn * len(tensors))()
        for k, t in enumerate(tensors):
            _check_dev(t, "window column")
            rows = t.shape[0]
            cols[k].ptr = t.data_ptr()
            cols[k].bytes_per_gaussian = t.numel() * t.element_size() // max(rows, 1)
        return cols

    def window_compact(self, tensors, keep, n_keep, moved_from=None, scratch=None, stream=None):
        """Deletion and compaction of the window rows (keep: uint8 [n]); n_keep:
        int64 tensor [1] receiving the survivors; moved_from: None or int32 [n]."""
        n = int(keep.numel())
        if scratch is None:
            scratch = torch.empty(int(lib().gs_window_scratch_bytes(n)), dtype=torch.uint8, device=keep.device)
        _check_dev(keep, "keep", torch.uint8, n)
        _check_dev(n_keep, "n_keep", torch.int64, 1)
        if moved_from is not None:
            _check_dev(moved_from, "moved_from", torch.int32, n)
        cols = self._columns(tensors)
        self._ck(lib().gs_window_compact(self.h, cols, len(tensors), n, _ptr(keep), _ptr(n_keep), _ptr(moved_from),
                                         _ptr(scratch), _stream(stream)))

    def window_remove(self, tensors, leave_dst, keep, n_keep, moved_from=None, leaving_rows=None, scratch=None,
                      stream=None):
        """Gather of the rows with keep == 0 into leave_dst (a list matching
        tensors, None entries skipped; each with room for n rows) and the
        compaction, in one stream-ordered call."""
        n = int(keep.numel())
        if scratch is None:
            scratch = torch.empty(int(lib().gs_window_scratch_bytes(n)), dtype=torch.uint8, device=keep.device)
        _check_dev(keep, "keep", torch.uint8, n)
        _check_dev(n_keep, "n_keep", torch.int64, 1)
        for name, t in (("moved_from", moved_from), ("leaving_rows", leaving_rows)):
            if t is not None:
                _check_dev(t, name, torch.int32, n)
        cols = self._columns(tensors)
        dst = None
        if leave_dst is not None:
            if len(leave_dst) != len(tensors):
                raise ValueError("leave_dst has %d entries for %d columns" % (len(leave_dst), len(tensors)))
            dst = (WindowColumn * len(tensors))()
            for k, (t, d) in enumerate(zip(tensors, leave_dst)):
                dst[k].bytes_per_gaussian = cols[k].bytes_per_gaussian
                if d is not None:
                    _check_dev(d, "leave_dst column")
                    if d.shape[0] < n or d.numel() * d.element_size() // max(d.shape[0], 1) != cols[k].bytes_per_gaussian:
                        raise ValueError("leave_dst column %d must hold %d rows of the column's width" % (k, n))
                    dst[k].ptr = d.data_ptr()
        self._ck(lib().gs_window_remove(self.h, cols, dst, len(tensors), n, _ptr(keep), _ptr(n_keep),
                                        _ptr(moved_from), _ptr(leaving_rows), _ptr(scratch), _stream(stream)))

    def window_gather(self, src, dst, idx, stream=None):
        """Rows idx (int32 device) of every src tensor into rows 0.. of dst."""
        _check_dev(idx, "idx", torch.int32)
        n = int(src[0].shape[0])
        self._ck(lib().gs_window_gather(self.h, self._columns(src), self._columns(dst), len(src), n, _ptr(idx),
                                        int(idx.numel()), _stream(stream)))

    def window_clear(self, tensors, begin, end, stream=None):
        """Rows [begin, end) of every tensor set to zero."""
        self._ck(lib().gs_window_clear(self.h, self._columns(tensors), len(tensors), int(begin), int(end),
                                       _stream(stream)))

    def sh_init_bilinear(self, g, view, image, begin, end, sh_out, stream=None):
        """k0 of Gaussians [begin, end) from the bilinear colour of image [3, H, W] (FP32 device)."""
        _check_dev(image, "image", torch.float32)
        _check_dev(sh_out, "sh_out", torch.float32)
        v = make_views([view])
        self._ck(lib().gs_sh_init_bilinear(self.h, ctypes.byref(g), v, _ptr(image), int(begin), int(end),
                                           _ptr(sh_out), _stream(stream)))

    def adam_step(self, param, grad, m, v, lr, b1, b2, eps, step, segments=(), stream=None):
        segs = None
        ns = len(segments)
        if ns:
            segs = (LowpSegment * ns)()
            for k, (b, e, dst) in enumerate(segments):
                segs[k].begin, segs[k].end, segs[k].dtype, segs[k].dst = int(b), int(e), _DTYPE[dst.dtype], dst.data_ptr()
        self._ck(lib().gs_adam_step(self.h, _ptr(param), _ptr(grad), _ptr(m), _ptr(v), param.numel(), float(lr),
                                    float(b1), float(b2), float(eps), int(step), segs, ns, _stream(stream)))

    def profile(self, families):
        """Times every launch of the named kernel families with CUDA events."""
        mask = 0
        for f in families:
            mask |= 1 << KERNEL_FAMILIES.index(f)
        self._ck(lib().gs_profile_enable(self.h, mask))

    def profile_collect(self, stream=None):
        """{family: (launches, total_ms)} since the last collect (synchronises)."""
        out = (ProfileEntry * len(KERNEL_FAMILIES))()
        n = ctypes.c_int()
        self._ck(lib().gs_profile_collect(self.h, _stream(stream), out, len(KERNEL_FAMILIES), ctypes.byref(n)))
        return {KERNEL_FAMILIES[out[k].family]: (out[k].launches, out[k].total_ms) for k in range(n.value)}

    def launch_count(self):
        return int(lib().gs_launch_count(self.h))

    def adam_step_dev(self, param, grad, m, v, lr, b1, b2, eps, step_dev, segments=(), stream=None):
        """Adam with the step counter in device memory (int64 tensor, incremented by the call)."""
        segs = None
        ns = len(segments)
        if ns:
            segs = (LowpSegment * ns)()
            for k, (b, e, dst) in enumerate(segments):
                segs[k].begin, segs[k].end, segs[k].dtype, segs[k].dst = int(b), int(e), _DTYPE[dst.dtype], dst.data_ptr()
        _check_dev(step_dev, "step_dev", torch.int64, 1)
        self._ck(lib().gs_adam_step_dev(self.h, _ptr(param), _ptr(grad), _ptr(m), _ptr(v), param.numel(), float(lr),
                                        float(b1), float(b2), float(eps), _ptr(step_dev), segs, ns, _stream(stream)))

    def adam_step_ranges(self, param, grad, m, v, ranges, lr, b1, b2, eps, step=0, step_dev=None, segments=(),
                         stream=None):
        """Adam over the element ranges [(begin, end), ...] of the flat buffers
        only; the step count from step_dev (device int64, incremented) when
        given, else the host step."""
        rg = (Range * len(ranges))()
        for k, (b, e) in enumerate(ranges):
            rg[k].begin, rg[k].end = int(b), int(e)
        segs = None
        ns = len(segments)
        if ns:
            segs = (LowpSegment * ns)()
            for k, (b, e, dst) in enumerate(segments):
                segs[k].begin, segs[k].end, segs[k].dtype, segs[k].dst = int(b), int(e), _DTYPE[dst.dtype], dst.data_ptr()
        if step_dev is not None:
            _check_dev(step_dev, "step_dev", torch.int64, 1)
        self._ck(lib().gs_adam_step_ranges(self.h, _ptr(param), _ptr(grad), _ptr(m), _ptr(v), param.numel(), rg,
                                           len(ranges), float(lr), float(b1), float(b2), float(eps), int(step),
                                           _ptr(step_dev), segs, ns, _stream(stream)))

    def selftest_bounded_wait(self, stream=None):
        """Makes the binning scan's bounded wait expire (see gs.h); the next
        sync_status returns GS_ERR_TIMEOUT."""
        scratch = torch.empty(int(lib().gs_selftest_wait_scratch_bytes()), dtype=torch.uint8, device="cuda")
        self._ck(lib().gs_selftest_bounded_wait(self.h, _ptr(scratch), _stream(stream)))
        return scratch  # kept alive by the caller until the stream has run

    def calibrate_alu(self, stream=None):
        """Measured FP32 FMA throughput (TFLOP/s) and ex2 throughput (G/s) of this device."""
        f, x = ctypes.c_double(), ctypes.c_double()
        self._ck(lib().gs_calibrate_alu(self.h, _stream(stream), ctypes.byref(f), ctypes.byref(x)))
        return f.value, x.value

    def sync_status(self, stream=None):
        n = ctypes.c_uint64()
        rc = lib().gs_sync_status(self.h, _stream(stream), ctypes.byref(n))
        return rc, n.value


def pixel_counts(views):
    return [int(v["W"]) * int(v["H"]) for v in views]


def unpack_images(flat, views, channels=3):
    """Splits a packed per-view buffer into a list of [C,H,W] (or [H,W]) views."""
    out, off = [], 0
    for v in views:
        n = int(v["W"]) * int(v["H"]) * channels
        t = flat[off:off + n]
        out.append(t.view(channels, int(v["H"]), int(v["W"])) if channels > 1 else t.view(int(v["H"]), int(v["W"])))
        off += n
    return out


def suggest_capacity(n_pairs, headroom=1.25):
    return int(math.ceil(max(n_pairs, 1024) * headroom))


def unpack_normal(normal):
    """[n_views, 28] normal-equation rows -> list of (A 6x6, b 6, r.r) in float64 numpy."""
    out = []
    rows = normal.detach().double().cpu().numpy().reshape(-1, 28)
    iu = np.triu_indices(6)
    for r in rows:
        A = np.zeros((6, 6))
        A[iu] = r[:21]
        A = A + np.triu(A, 1).T
        out.append((A, r[21:27].copy(), float(r[27])))
    return out

