"""High-level API over the C ABI: a renderer for a batch of keyframe views, a
torch.autograd.Function, the sliding-window optimisation step (Sec. II-B.2)
and the photometric pose-gradient step (Sec. II-D).

Torch provides device memory and streams only; every computation is a call
into libgs_b300.so.
"""
from __future__ import annotations

import warnings

import numpy as np
import torch

from . import binding as B


class Renderer:
    """Renders a fixed batch of views (layout fixed, poses may change via
    `set_views`) and owns the image buffers and the workspace."""

    def __init__(self, views, device=0, tile_size=16, capacity=None, **cfg):
        self.device = torch.device("cuda", device)
        self.ctx = B.Context(device, tile_size=tile_size, **cfg)
        self.view_dicts = [dict(v) for v in views]
        self.views = B.make_views(self.view_dicts)
        self.n_views = len(views)
        self.npx = sum(B.pixel_counts(self.view_dicts))
        dev = self.device
        self.rgb = torch.empty(3 * self.npx, device=dev, dtype=torch.float32)
        self.T = torch.empty(self.npx, device=dev, dtype=torch.float32)
        self.n_contrib = torch.empty(self.npx, device=dev, dtype=torch.int32)
        self.dL_drgb = torch.empty(3 * self.npx, device=dev, dtype=torch.float32)
        self.loss = torch.zeros(1, device=dev, dtype=torch.float32)
        # forwards run so far: the autograd wrapper checks that the bins its
        # backward recomputes alpha from still belong to its own forward
        self.forward_count = 0
        self.dL_dpose = torch.zeros(self.n_views * 6, device=dev, dtype=torch.float32)
        self.cap = 0
        self.ws = None
        self.ws_struct = None
        self._counted = False
        self.ensure_capacity(capacity or 1 << 16)

    def set_views(self, views):
        """Replaces camera poses / intrinsics; the layout (sizes, ranges) must
        not change."""
        for old, new in zip(self.view_dicts, views):
            for k in ("W", "H", "g_begin", "g_end"):
                if int(old[k]) != int(new[k]):
                    raise ValueError("set_views may not change the view layout")
        self.view_dicts = [dict(v) for v in views]
        self.views = B.make_views(self.view_dicts)

    def ensure_capacity(self, pairs):
        if pairs <= self.cap and self.ws is not None:
            return False
        self.cap = B.suggest_capacity(pairs)
        nbytes = self.ctx.workspace_bytes(self.views, self.cap)
        self.ws = torch.empty(nbytes, device=self.device, dtype=torch.uint8)
        self.ws_struct = B.Context.ws_struct(self.ws, self.cap)
        return True

    def layout(self):
        return self.ctx.layout(self.views, self.cap)

    def list_entries(self):
        """Entries of all tiles' lists after the last binning (the pair count,
        or with bins larger than the tiles the entries split from them);
        synchronises."""
        L = self.layout()
        rg = self.ws[L.tile_ranges:L.tile_ranges + 8 * L.n_tiles].view(torch.int32).view(-1, 2).long() & 0xFFFFFFFF
        return int((rg[:, 1] - rg[:, 0]).sum().item())

    def forward(self, g, count=None, n_used=None, target=None):
        """project + bin + composite into self.rgb / self.T / self.n_contrib.
        count: True synchronises to read the pair count and grows the workspace
        if needed (default: only on the first call).  target: also the L1 loss
        against it, folded into the compositing (self.loss, self.dL_drgb)."""
        if count is None:
            count = not self._counted
        self.forward_count += 1
        self.ctx.project(g, self.views, self.ws_struct)
        if count:
            while True:
                try:
                    n = self.ctx.bin(self.views, self.ws_struct, want_count=True)
                    break
                except B.GsError as e:
                    if e.code != B.GS_ERR_CAPACITY:
                        raise
                    self.ensure_capacity(e.pairs_needed)
                    self.ctx.project(g, self.views, self.ws_struct)
            self._counted = True
            self.last_pairs = n
        else:
            self.ctx.bin(self.views, self.ws_struct)
        if target is None:
            self.ctx.render_fwd(self.views, self.ws_struct, self.rgb, self.T, self.n_contrib, n_used)
        else:
            self.ctx.render_fwd_l1(self.views, self.ws_struct, target, self.rgb, self.T, self.n_contrib,
                                   self.dL_drgb, self.loss, n_used)

    def forward_loss(self, g, target, ssim_lambda=0.0, count=None):
        """forward + photometric loss and its gradient into self.loss and
        self.dL_drgb: L1 in the same pass as the compositing, or the D-SSIM
        variant after it when ssim_lambda > 0."""
        if ssim_lambda > 0.0:
            self.forward(g, count=count)
            self.dssim(target, ssim_lambda)
        else:
            self.forward(g, count=count, target=target)

    def l1(self, target):
        self.ctx.l1_loss(self.views, self.ws_struct, self.rgb, target, self.dL_drgb, self.loss)

    def dssim(self, target, lam=0.2):
        """(1 - lam) L1 + lam (1 - SSIM) of the last forward against target,
        into self.loss and self.dL_drgb."""
        n = int(B.lib().gs_dssim_scratch_floats(self.views, len(self.views)))
        if getattr(self, "_ssim_scratch", None) is None or self._ssim_scratch.numel() != n:
            self._ssim_scratch = torch.empty(n, dtype=torch.float32, device=self.rgb.device)
        self.ctx.dssim_loss(self.views, self.rgb, target, lam, self._ssim_scratch, self.dL_drgb, self.loss)

    def loss_and_grad(self, target, ssim_lambda=0.0):
        if ssim_lambda > 0.0:
            self.dssim(target, ssim_lambda)
        else:
            self.l1(target)

    def backward(self, g, dL_drgb, grads=None, want_pose=False, accumulate=False):
        """Gradients of the last forward's views.  accumulate: add to `grads`
        instead of overwriting them (views back-propagated in several calls)."""
        self.ctx.render_bwd(g, self.views, self.ws_struct, self.T, self.n_contrib, dL_drgb, grads,
                            self.dL_dpose if want_pose else None, accumulate=accumulate)

    def pose_grad(self, g, dL_drgb):
        self.ctx.pose_grad(g, self.views, self.ws_struct, self.T, self.n_contrib, dL_drgb, self.dL_dpose)

    def pose_normal(self, g, target, H_pix=None):
        """Per-view Gauss-Newton normal equations of target - render in the pose
        (Sec. II-D) over the bins of the last forward: returns [n_views, 28]
        float64 (see gs_pose_normal)."""
        need = self.ctx.pose_normal_scratch(self.views)
        if getattr(self, "_pn_scratch", None) is None or self._pn_scratch.numel() < need:
            self._pn_scratch = torch.empty(need, device=self.device, dtype=torch.float32)
            self.normal = torch.zeros(self.n_views, 28, device=self.device, dtype=torch.float64)
        self.ctx.pose_normal(g, self.views, self.ws_struct, target, self._pn_scratch, self.normal, H_pix)
        return self.normal

    def images(self, flat=None):
        return B.unpack_images(self.rgb if flat is None else flat, self.view_dicts, 3)

    def check_status(self):
        rc, n = self.ctx.sync_status()
        if rc == B.GS_ERR_CAPACITY:
            self.ensure_capacity(n)
        return rc, n


class GaussianWindow:
    """The window's parameters as one flat FP32 master vector (Adam runs over
    it in one launch) with per-group views, gradients, Adam moments and
    optional FP16/BF16 render copies of the non-mean groups.

    Rows [0, n) are the active window; `capacity` rows are allocated so that
    new Gaussians can be appended in place (Sec. II-C, Step 4).  `maintain`
    removes leaving Gaussians by the swap-with-tail compaction of Step 2 on
    the device and returns their parameters for the global map (Step 1)."""

    GROUPS = ("means", "log_scales", "quats", "opacity", "sh")

    def __init__(self, params, device=0, storage=None, capacity=None):
        self.device = torch.device("cuda", device)
        self.sh_degree = int(params["sh_degree"])
        self.K = (self.sh_degree + 1) ** 2
        self.n = int(params["means"].shape[0])
        self.capacity = max(int(capacity or 0), self.n)
        cap, K = self.capacity, self.K
        self.widths = dict(means=(3,), log_scales=(3,), quats=(4,), opacity=(), sh=(K, 3))
        self.sizes = {k: cap * int(np.prod(w)) for k, w in self.widths.items()}
        self.offsets = {}
        off = 0
        for k in self.GROUPS:
            self.offsets[k] = off
            off += self.sizes[k]
            off = (off + 3) // 4 * 4  # keep each group 16-byte aligned
        self.total = off
        dev = self.device
        self.flat = torch.zeros(self.total, device=dev, dtype=torch.float32)
        self.gflat = torch.zeros(self.total, device=dev, dtype=torch.float32)
        self.m = torch.zeros(self.total, device=dev, dtype=torch.float32)
        self.v = torch.zeros(self.total, device=dev, dtype=torch.float32)
        self.step_count = 0
        for k in self.GROUPS:
            self.group(k).copy_(torch.as_tensor(np.ascontiguousarray(params[k], np.float32)).view(self.shape(k)))
        self.storage = dict(storage or {})
        self.lowp = {}
        for k, dt in self.storage.items():
            if k == "means":
                raise ValueError("means are always FP32")
            self.lowp[k] = self.column(k).to(dt).contiguous()
        self._ctx = None

    def shape(self, k, rows=None):
        return (self.n if rows is None else rows,) + self.widths[k]

    def column(self, k, flat=None):
        """All `capacity` rows of group k in `flat` (default: the parameters)."""
        f = self.flat if flat is None else flat
        o = self.offsets[k]
        return f[o:o + self.sizes[k]].view(self.shape(k, self.capacity))

    def group(self, k, flat=None):
        """The active rows [0, n) of group k."""
        return self.column(k, flat)[:self.n]

    def grad(self, k):
        return self.group(k, self.gflat)

    def render_tensors(self):
        return [self.lowp[k][:self.n] if k in self.lowp else self.group(k) for k in self.GROUPS]

    def struct(self):
        """The C-ABI view of the render tensors.  It keeps this window alive as
        long as it is referenced, so its device pointers stay valid."""
        t = self.render_tensors()
        g = B.gaussians_struct(*t, self.sh_degree)
        g._owner = self
        return g

    def grad_tensors(self):
        return [self.grad(k) for k in self.GROUPS]

    def segments(self):
        return [(self.offsets[k], self.offsets[k] + self.sizes[k], self.lowp[k]) for k in self.lowp]

    def active_ranges(self):
        """Element ranges of the flat buffers that hold rows [0, n) of each group."""
        return [(self.offsets[k], self.offsets[k] + self.n * int(np.prod(self.widths[k]))) for k in self.GROUPS]

    def numpy(self, use_render_copy=False):
        out = {}
        for k in self.GROUPS:
            t = self.lowp[k][:self.n] if (use_render_copy and k in self.lowp) else self.group(k)
            out[k] = t.float().cpu().numpy()
        out["sh_degree"] = self.sh_degree
        return out

    # ---- sliding-window maintenance (Sec. II-C) ----

    def ctx(self):
        if self._ctx is None:
            self._ctx = B.Context(self.device.index or 0)
        return self._ctx

    def _columns(self, rows):
        """The per-Gaussian state that maintenance carries: parameters, Adam
        moments and render copies.  The gradients are not carried: every
        backward overwrites all of them."""
        cols = []
        for k in self.GROUPS:
            for f in (self.flat, self.m, self.v):
                cols.append(self.column(k, f)[:rows].reshape(rows, -1))
            if k in self.lowp:
                cols.append(self.lowp[k][:rows].reshape(rows, -1))
        return cols

    def maintain(self, keep):
        """Steps 1 and 2: `keep` (bool or uint8 [n], device or host) marks the
        Gaussians that stay.  One stream-ordered library call gathers the
        leaving Gaussians' parameters (ascending row order) into a device
        staging area and compacts the window by swapping rear survivors into
        the holes; the host then reads the survivor count and copies the
        leaving parameters and the row map back.  Returns (leaving params as
        a host dict, moved_from [n_keep] int64 host: the old row of every new
        row)."""
        n = self.n
        keep = torch.as_tensor(keep, device=self.device).to(torch.uint8).contiguous()
        if keep.numel() != n:
            raise ValueError("keep has %d entries for %d Gaussians" % (keep.numel(), n))
        if getattr(self, "_leave", None) is None:
            self._leave = {k: torch.empty((self.capacity,) + self.widths[k], dtype=torch.float32, device=self.device)
                           for k in self.GROUPS}
        cols = self._columns(n)
        leave = [None] * len(cols)
        c = 0
        for k in self.GROUPS:
            leave[c] = self._leave[k][:n].reshape(n, -1)  # the parameter column of group k
            c += 3 + (1 if k in self.lowp else 0)
        n_keep = torch.zeros(1, dtype=torch.int64, device=self.device)
        moved = torch.empty(max(n, 1), dtype=torch.int32, device=self.device)
        self.ctx().window_remove(cols, leave, keep, n_keep, moved[:n] if n else None)
        nk = int(n_keep.item())
        m = n - nk
        leaving = {k: self._leave[k][:m].cpu().numpy() for k in self.GROUPS}
        leaving["sh_degree"] = self.sh_degree
        self.n = nk
        return leaving, moved[:nk].to(torch.int64).cpu().numpy()

    def append(self, params, image=None, view=None, stream=None):
        """Step 4: appends the Gaussians of `params` (host arrays, or pinned
        FP32 host tensors, which are copied without staging) at rows [n, n + m)
        (parameters copied host to device, Adam moments zeroed); with `image` ([3, H, W] device FP32) and `view`
        their SH start from the bilinear image colour (Sec. II-B.2).  The
        copies are issued on `stream` (default: the current stream)."""
        m = int(params["means"].shape[0])
        if self.n + m > self.capacity:
            raise ValueError("window capacity %d exceeded (%d + %d)" % (self.capacity, self.n, m))
        a, b = self.n, self.n + m
        s = stream or torch.cuda.current_stream(self.device)
        with torch.cuda.stream(s):
            for k in self.GROUPS:
                src = params[k]
                if isinstance(src, torch.Tensor) and src.is_pinned() and src.dtype == torch.float32:
                    host = src.reshape(self.shape(k, m))  # already pinned (e.g. a pinned host map): no staging copy
                else:
                    host = torch.as_tensor(np.ascontiguousarray(src, np.float32)).view(self.shape(k, m)).pin_memory()
                self.column(k)[a:b].copy_(host, non_blocking=True)
            self.ctx().window_clear([self.column(k, f) for k in self.GROUPS for f in (self.m, self.v)], a, b, stream=s)
            self.n = b
            if image is not None:
                g = self.struct()
                self.ctx().sh_init_bilinear(g, view, image, a, b, self.column("sh"), stream=s)
            for k in self.lowp:
                self.lowp[k][a:b].copy_(self.column(k)[a:b])
        return a, b


class WindowOptimizer:
    """One sliding-window optimisation iteration (Sec. II-B.2): render every
    keyframe, photometric loss (L1; with ssim_lambda > 0 the D-SSIM variant
    (1 - lambda) L1 + lambda (1 - SSIM)), backward to the Gaussians, Adam."""

    def __init__(self, params, views, targets, lr=1e-3, betas=(0.9, 0.999), eps=1e-8, device=0,
                 tile_size=16, storage=None, ssim_lambda=0.0, capacity=None, **cfg):
        self.win = GaussianWindow(params, device, storage, capacity)
        self.r = Renderer(views, device, tile_size, **cfg)
        self.targets = targets
        self.ssim_lambda = float(ssim_lambda)
        self.lr, self.betas, self.eps = lr, betas, eps
        self._g = self.win.struct()
        self._grads = self.win.grad_tensors()
        self._segs = self.win.segments()

        self.graph = None
        self.step_dev = None

    def step(self, count=None, slot=0):
        """One iteration through the C ABI (host-issued launches), or, once
        captured, a replay of the graph of target buffer `slot`."""
        if self.graph is not None:
            return self.replay(slot)
        w, r = self.win, self.r
        r.forward_loss(self._g, self.targets, self.ssim_lambda, count=count)
        r.backward(self._g, r.dL_drgb, grads=self._grads)
        w.step_count += 1
        if w.capacity > w.n:  # spare rows (appends may be in flight there): Adam on the active rows only
            r.ctx.adam_step_ranges(w.flat, w.gflat, w.m, w.v, w.active_ranges(), self.lr, self.betas[0],
                                   self.betas[1], self.eps, step=w.step_count, segments=self._segs)
        else:
            r.ctx.adam_step(w.flat, w.gflat, w.m, w.v, self.lr, self.betas[0], self.betas[1], self.eps,
                            w.step_count, self._segs)
        return r.loss

    def _capture_one(self, targets):
        w, r = self.win, self.r
        for attempt in range(3):
            torch.cuda.synchronize()
            g = torch.cuda.CUDAGraph()
            try:
                # relaxed capture: a host-side CUDA call that is not part of
                # the iteration (a tensor or context another part of the
                # program frees meanwhile) does not invalidate it
                with torch.cuda.graph(g, capture_error_mode="relaxed"):
                    r.forward_loss(self._g, targets, self.ssim_lambda, count=False)
                    r.backward(self._g, r.dL_drgb, grads=self._grads)
                    if w.capacity > w.n:
                        r.ctx.adam_step_ranges(w.flat, w.gflat, w.m, w.v, w.active_ranges(), self.lr,
                                               self.betas[0], self.betas[1], self.eps, step_dev=self.step_dev,
                                               segments=self._segs)
                    else:
                        r.ctx.adam_step_dev(w.flat, w.gflat, w.m, w.v, self.lr, self.betas[0], self.betas[1],
                                            self.eps, self.step_dev, self._segs)
            except (RuntimeError, B.GsError) as e:
                if attempt == 2:
                    raise
                warnings.warn("graph capture failed (%s); capturing again" % e)
                torch.cuda.synchronize()
                continue
            return g

    def capture(self, targets=None):
        """Captures one iteration in a CUDA graph (the workspace must already
        be sized, i.e. after one step).  Later `step()` calls replay it; the
        Adam step count lives on the device, and a pair-capacity overflow is
        latched and reported by `r.check_status()`.

        targets: a list of target buffers (each shaped like the optimiser's
        targets) to capture one graph per buffer; `step(slot)` then replays
        the graph that reads targets[slot].  With two buffers the next
        iteration's keyframe images can be copied into one while the other is
        in use, and no copy into a fixed buffer is needed."""
        w, r = self.win, self.r
        if not r._counted:
            raise RuntimeError("run one step before capturing (sizes the pair workspace)")
        bufs = list(targets) if targets is not None else [self.targets]
        for t in bufs:
            if t.shape != self.targets.shape or t.dtype != self.targets.dtype or t.device != self.targets.device:
                raise ValueError("a target buffer differs from the optimiser's targets in shape, dtype or device")
            if not t.is_contiguous():
                raise ValueError("a target buffer is not contiguous (the kernels read it as one packed array)")
        self.step_dev = torch.tensor([w.step_count], dtype=torch.int64, device=w.device)
        self.graphs = [self._capture_one(t) for t in bufs]
        self.graph = self.graphs[0]
        self.target_buffers = bufs
        return self.graph

    def replay(self, slot=0):
        self.graphs[slot].replay()
        self.win.step_count += 1
        return self.r.loss


class PerViewOptimizer:
    """The window iteration of WindowOptimizer in the plain per-view form, the
    baseline the batched form is measured against: every view is projected,
    binned, composited and back-propagated by its own sequence of launches
    (one Renderer per view, writing into its view's slice of the packed
    images), the L1 loss is taken over all views in one call (the batched
    form's normalisation), the per-view backward passes add their parameter
    gradients up (gs_render_bwd_accumulate) and one Adam step follows.  Its
    result equals the batched form's up to the order of float atomics."""

    def __init__(self, params, views, targets, lr=1e-3, betas=(0.9, 0.999), eps=1e-8, device=0,
                 tile_size=16, storage=None, **cfg):
        self.win = GaussianWindow(params, device, storage)
        self.targets = targets
        self.lr, self.betas, self.eps = lr, betas, eps
        # packed images of all views and the loss over them
        self.all = Renderer(views, device, tile_size, capacity=1024, **cfg)
        self.rs = []
        off = 0
        for v in views:
            r = Renderer([v], device, tile_size, **cfg)
            n = int(v["W"]) * int(v["H"])
            r.rgb = self.all.rgb[3 * off:3 * (off + n)]
            r.T = self.all.T[off:off + n]
            r.n_contrib = self.all.n_contrib[off:off + n]
            r.dL_drgb = self.all.dL_drgb[3 * off:3 * (off + n)]
            self.rs.append(r)
            off += n
        self._g = self.win.struct()
        self._grads = self.win.grad_tensors()
        self._segs = self.win.segments()
        self.graph = None
        self.step_dev = None

    @property
    def r(self):
        return self.all

    def _iteration(self, count, step_dev=None):
        w = self.win
        for r in self.rs:
            r.forward(self._g, count=count)
        self.all.l1(self.targets)
        for i, r in enumerate(self.rs):
            r.backward(self._g, r.dL_drgb, grads=self._grads, accumulate=i > 0)
        ctx = self.all.ctx
        if step_dev is None:
            ctx.adam_step(w.flat, w.gflat, w.m, w.v, self.lr, self.betas[0], self.betas[1], self.eps,
                          w.step_count, self._segs)
        else:
            ctx.adam_step_dev(w.flat, w.gflat, w.m, w.v, self.lr, self.betas[0], self.betas[1], self.eps,
                              step_dev, self._segs)

    def step(self, count=None):
        if self.graph is not None:
            self.graph.replay()
            self.win.step_count += 1
            return self.all.loss
        self.win.step_count += 1
        self._iteration(count)
        return self.all.loss

    def pairs(self):
        return sum(int(r.last_pairs) for r in self.rs)

    def check_status(self):
        out = [r.check_status() for r in self.rs]
        bad = [o for o in out if o[0] != B.GS_OK]
        return bad[0] if bad else (B.GS_OK, self.pairs())

    def capture(self):
        """Captures one iteration in a CUDA graph (after one step, which sizes
        every view's pair workspace)."""
        if not all(r._counted for r in self.rs):
            raise RuntimeError("run one step before capturing (sizes the pair workspaces)")
        self.step_dev = torch.tensor([self.win.step_count], dtype=torch.int64, device=self.win.device)
        for attempt in range(3):
            torch.cuda.synchronize()
            g = torch.cuda.CUDAGraph()
            try:
                with torch.cuda.graph(g, capture_error_mode="relaxed"):
                    self._iteration(False, self.step_dev)
            except (RuntimeError, B.GsError) as e:
                if attempt == 2:
                    raise
                warnings.warn("graph capture failed (%s); capturing again" % e)
                torch.cuda.synchronize()
                continue
            self.graph = g
            return g


class _Rasterize(torch.autograd.Function):
    @staticmethod
    def forward(ctx, renderer, sh_degree, means, log_scales, quats, opacity, sh):
        g = B.gaussians_struct(means, log_scales, quats, opacity, sh, sh_degree)
        renderer.forward(g)
        ctx.renderer = renderer
        ctx.forward_count = renderer.forward_count
        ctx.sh_degree = sh_degree
        ctx.save_for_backward(means, log_scales, quats, opacity, sh)
        rgb = renderer.rgb.clone()
        T = renderer.T.clone()
        ctx.mark_non_differentiable(T)
        return rgb, T

    @staticmethod
    def backward(ctx, dL_drgb, _dT):
        means, log_scales, quats, opacity, sh = ctx.saved_tensors
        r = ctx.renderer
        if r.forward_count != ctx.forward_count:
            raise RuntimeError("rasterize: the renderer ran another forward after this one; its bins, T and "
                               "n_contrib (from which backward recomputes alpha) belong to that forward now. "
                               "Use one Renderer per rasterize call that is differentiated.")
        g = B.gaussians_struct(means, log_scales, quats, opacity, sh, ctx.sh_degree)
        grads = [torch.empty(t.shape, device=t.device, dtype=torch.float32) for t in
                 (means, log_scales, quats, opacity, sh)]
        r.backward(g, dL_drgb.contiguous().float(), grads=grads)
        out = [gr.to(t.dtype) for gr, t in zip(grads, (means, log_scales, quats, opacity, sh))]
        return (None, None, *out)


def rasterize(renderer, means, log_scales, quats, opacity, sh, sh_degree):
    """Differentiable render of the renderer's views.  Returns the packed rgb
    ([sum 3 H W]) and the final transmittance ([sum H W], not differentiable).
    Alpha is recomputed in the backward pass from the saved bins: call
    backward before the next forward on the same renderer."""
    return _Rasterize.apply(renderer, int(sh_degree), means.contiguous(), log_scales.contiguous(),
                            quats.contiguous(), opacity.contiguous(), sh.contiguous())


def se3_exp(xi):
    """4x4 Exp of xi = (dphi, dt) (closed form, float64)."""
    phi = np.asarray(xi[:3], np.float64)
    rho = np.asarray(xi[3:], np.float64)
    th = float(np.linalg.norm(phi))
    K = np.array([[0, -phi[2], phi[1]], [phi[2], 0, -phi[0]], [-phi[1], phi[0], 0]])
    if th < 1e-12:
        R = np.eye(3) + K
        V = np.eye(3) + 0.5 * K
    else:
        R = np.eye(3) + np.sin(th) / th * K + (1 - np.cos(th)) / th ** 2 * (K @ K)
        V = np.eye(3) + (1 - np.cos(th)) / th ** 2 * K + (th - np.sin(th)) / th ** 3 * (K @ K)
    T = np.eye(4)
    T[:3, :3] = R
    T[:3, 3] = V @ rho
    return T


def apply_left(view, xi):
    """View with T_CW <- Exp(xi) T_CW."""
    T = np.eye(4)
    T[:3, :3] = np.asarray(view["R"], np.float64)
    T[:3, 3] = np.asarray(view["t"], np.float64)
    Tn = se3_exp(xi) @ T
    out = dict(view)
    out["R"] = Tn[:3, :3].astype(np.float32)
    out["t"] = Tn[:3, 3].astype(np.float32)
    return out


class PoseTracker:
    """Photometric pose update (Sec. II-D, Eq. minimization) for fixed
    Gaussians: render at the current pose, L1 against the frame, pose-only
    backward, then a host step T <- Exp(-eta g) T (the paper feeds the
    gradient to its IESKF instead; the step rule does not change the GPU
    work)."""

    def __init__(self, params, view, device=0, tile_size=16, step_sizes=(2e-2, 2e-2), **cfg):
        self.win = GaussianWindow(params, device)
        self.r = Renderer([view], device, tile_size, **cfg)
        self.g = self.win.struct()
        self.eta_rot, self.eta_trans = step_sizes

    def iterate(self, view, target):
        self.r.set_views([view])
        self.r.forward(self.g, target=target)
        self.r.pose_grad(self.g, self.r.dL_drgb)
        return self.r.dL_dpose

    def step(self, view, target):
        gpose = self.iterate(view, target).double().cpu().numpy()
        xi = np.concatenate([-self.eta_rot * gpose[:3], -self.eta_trans * gpose[3:]])
        return apply_left(view, xi), gpose

    def gauss_newton(self, view, target, damping=1e-6):
        """One Gauss-Newton pose update from the normal equations of the
        photometric residual (the linearisation the IESKF's visual update
        uses, Sec. II-D): xi = (A + damping tr(A)/6 I)^-1 b, T <- Exp(xi) T.
        Returns the new view and (A, b, r.r)."""
        self.r.set_views([view])
        self.r.forward(self.g)
        A, b, rr = B.unpack_normal(self.r.pose_normal(self.g, target))[0]
        xi = np.linalg.solve(A + damping * np.trace(A) / 6.0 * np.eye(6), b)
        return apply_left(view, xi), (A, b, rr)


class IESKFPoseTracker:
    """The visual update of the paper's IESKF for the IMU pose (Sec. II-D,
    Appendix A): iterated updates of T_WI from the photometric normal
    equations computed on the GPU (gs_pose_normal), mapped through the
    camera-IMU Jacobian, against a prior (mean, covariance) on the host.
    `view` gives the camera intrinsics and image size; T_CI is the fixed
    camera-IMU extrinsic; sigma2 the photometric noise variance per channel."""

    def __init__(self, params, view, R_CI, t_CI, device=0, tile_size=16, sigma2=1e-3, **cfg):
        from . import ieskf
        self.ieskf = ieskf
        self.win = GaussianWindow(params, device)
        self.r = Renderer([view], device, tile_size, **cfg)
        self.g = self.win.struct()
        self.view = dict(view)
        self.R_CI, self.t_CI = np.asarray(R_CI, np.float64), np.asarray(t_CI, np.float64)
        self.sigma2 = float(sigma2)

    def camera_view(self, R_WI, p_WI):
        R_CW, t_CW = self.ieskf.camera_pose(R_WI, p_WI, self.R_CI, self.t_CI)
        v = dict(self.view)
        v["R"], v["t"] = R_CW.astype(np.float32), t_CW.astype(np.float32)
        return v

    def update(self, R_prior, p_prior, P_prior, target, iters=5):
        """Iterated update from the prior; returns (R_WI, p_WI, P_post, residuals r.r)."""
        R, p = np.asarray(R_prior, np.float64), np.asarray(p_prior, np.float64)
        P_post = np.asarray(P_prior, np.float64)
        rrs = []
        for _ in range(iters):
            v = self.camera_view(R, p)
            self.r.set_views([v])
            self.r.forward(self.g)
            A, b, rr = B.unpack_normal(self.r.pose_normal(self.g, target))[0]
            rrs.append(rr)
            J = self.ieskf.camera_from_imu_jacobian(self.R_CI, self.t_CI, np.asarray(v["R"], np.float64))
            off = self.ieskf.boxminus(R, p, R_prior, p_prior)
            dx, P_post = self.ieskf.ieskf_pose_update(A, b, J, self.sigma2, P_prior, offset=off)
            R, p = self.ieskf.boxplus(R, p, dx)
        return R, p, P_post, rrs


# Compiled launch shapes of the compositing kernels: (tile size, pixels per
# thread, records per staged batch).  Every one renders the same image.
RASTER_VARIANTS = [(8, 1, 128), (8, 1, 256), (8, 2, 128), (8, 2, 256),
                   (16, 1, 256), (16, 2, 128), (16, 2, 256), (16, 4, 128), (16, 4, 256), (16, 8, 128),
                   (16, 8, 256), (32, 4, 256), (32, 8, 128), (32, 8, 256)]


def launch_candidates(deterministic=False):
    """The launch shapes autotune times: every compiled (tile size, pixels
    per thread, batch) with binning at the tile size (bin 0), and, outside
    the deterministic mode, with bins of 2 and 4 times the tile size (at most
    32 pixels) split into per-tile lists."""
    out = [v + (0,) for v in RASTER_VARIANTS]
    if not deterministic:
        out += [v + (b,) for v in RASTER_VARIANTS for b in (2 * v[0], 4 * v[0]) if b <= 32]
    return out


def autotune(params, views, targets, candidates=None, steps=3, device=0, storage=None, verbose=False, **cfg):
    """Picks the fastest (tile size, pixels per thread, batch, bin tile size)
    for this window and batch of views by timing whole optimisation
    iterations (projection to Adam, lr = 0 so the parameters do not move)
    with CUDA events on the launching stream; cfg: further configuration
    (e.g. deterministic=1).  Returns (best, table) with table[(ts, ppt,
    batch, bin)] = ms per iteration (bin 0: binning at the tile size)."""
    cands = candidates or launch_candidates(bool(cfg.get("deterministic", 0)))
    table = {}
    for cand in cands:
        ts, ppt, batch = cand[:3]
        bin_ts = cand[3] if len(cand) > 3 else 0
        opt = WindowOptimizer(params, views, targets, lr=0.0, device=device, tile_size=ts, storage=storage,
                              pixels_per_thread=ppt, batch=batch, bin_tile_size=bin_ts, **cfg)
        opt.step(count=True)
        opt.step(count=False)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        for _ in range(steps):
            opt.step(count=False)
        b.record()
        torch.cuda.synchronize()
        rc, _ = opt.r.check_status()
        if rc != B.GS_OK:
            continue
        table[(ts, ppt, batch, bin_ts)] = a.elapsed_time(b) / steps
        if verbose:
            print("autotune tile %2d ppt %d batch %3d bin %2d: %.3f ms" % (ts, ppt, batch, bin_ts,
                                                                       table[(ts, ppt, batch, bin_ts)]))
        del opt
    best = min(table, key=table.get)
    return best, table
