"""The checked build against the normal one.

libgs_b300_checked.so is the library compiled with GS_CHECKED: its
compositing kernels (forward, backward, pose normal equations) test every
index they read from device memory, a tile's pair range against the
workspace capacity and a pair's record against the record count, and latch
GS_ERR_BOUNDS instead of reading out of bounds.  It stands in for a memory
checker: the same workloads run through both libraries (one process each,
as the binding loads one of them), no check may fail (gs_sync_status stays
GS_OK), and the outputs must be those of the normal build: bit for bit where
the arithmetic is ordered (images, T, contributor counts, deterministic
gradients), to rounding where float atomics add in arrival order.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

WORKER = r"""
import os, sys
import numpy as np
import torch
sys.path.insert(0, os.environ["GS_ROOT"])
from paper_2501_08672_b300 import binding as B
from paper_2501_08672_b300 import scenes
from paper_2501_08672_b300.render import GaussianWindow, Renderer

out = {"checked": np.array([int(B.lib().gs_checked_build())])}


def status_ok(r, name):
    rc, _ = r.ctx.sync_status()
    assert rc == B.GS_OK, (name, rc)


def cases():
    n = 3000
    p = scenes.frustum_scene(n, seed=61)
    v0 = scenes.identity_view(200, 136, 160.0, 0, n)
    v1 = scenes.lookat_view((0.6, -0.4, -1.0), (0.0, 0.0, 5.0), 150, 100, 120.0, 0, n, up=(0, -1, 0))
    yield "ragged", p, [v0, v1], {}
    yield "ragged_det", p, [v0, v1], {"deterministic": 1}
    yield "ragged_t8", p, [v0, v1], {"tile_size": 8}
    yield "ragged_bins", p, [v0, v1], {"tile_size": 8, "pixels_per_thread": 2, "batch": 128, "bin_tile_size": 32}
    big = scenes.frustum_scene(2000, seed=62)
    big["log_scales"][:6] = np.log(np.array([[1.5, 1.2, 0.4]] * 6, np.float32))
    big["means"][:6, 2] = np.linspace(3.0, 7.0, 6)
    yield "huge_splats", big, [scenes.identity_view(256, 192, 200.0, 0, 2000)], {}
    m = scenes.frustum_scene(1500, seed=63)
    views = [scenes.identity_view(40 + 3 * k, 24 + 2 * (k % 5), 30.0, 0, 1500) for k in range(64)]
    yield "64_views", m, views, {"tile_size": 8}
    yield "64_views_bins", m, views, {"tile_size": 8, "bin_tile_size": 16}


for name, p, views, cfg in cases():
    cfg = dict(cfg)
    ts = cfg.pop("tile_size", 16)
    win = GaussianWindow(p, 0)
    r = Renderer(views, 0, ts, **cfg)
    r.forward(win.struct())
    w = torch.randn(r.rgb.numel(), device="cuda", generator=torch.Generator(device="cuda").manual_seed(1))
    r.backward(win.struct(), w, grads=win.grad_tensors(), want_pose=True)
    torch.cuda.synchronize()
    status_ok(r, name)
    out[name + "/rgb"] = r.rgb.cpu().numpy()
    out[name + "/T"] = r.T.cpu().numpy()
    out[name + "/n_contrib"] = r.n_contrib.cpu().numpy()
    out[name + "/grad"] = win.gflat.cpu().numpy()
    out[name + "/pose"] = r.dL_dpose.cpu().numpy()
    if name in ("ragged", "ragged_bins"):
        target = (r.rgb + 0.05 * w).contiguous()
        H = r.pose_normal(win.struct(), target)
        torch.cuda.synchronize()
        status_ok(r, name + " pose normal")
        out[name + "/pose_normal"] = H.cpu().numpy()

# a workspace too small for the pairs: the capacity overflow is what the
# status reports, and the truncated lists are read within bounds
p = scenes.frustum_scene(3000, seed=61)
views = [scenes.identity_view(200, 136, 160.0, 0, 3000)]
win = GaussianWindow(p, 0)
r = Renderer(views, 0, 16, capacity=100)
r._counted = True
r.forward(win.struct())
torch.cuda.synchronize()
rc, need = r.ctx.sync_status()
out["overflow_rc"] = np.array([rc])
rc2, _ = r.ctx.sync_status()
out["overflow_rc_after"] = np.array([rc2])
# the same with bins split into tile lists
r = Renderer(views, 0, 8, capacity=100, pixels_per_thread=2, batch=128, bin_tile_size=32)
r._counted = True
r.forward(win.struct())
torch.cuda.synchronize()
rc, need = r.ctx.sync_status()
out["overflow_bins_rc"] = np.array([rc])
np.savez(os.environ["GS_OUT"], **out)
"""


def _run(tmp_path, which):
    dst = str(tmp_path / ("%s.npz" % which))
    env = dict(os.environ, GS_ROOT=ROOT, GS_OUT=dst, GS_B300_LIB=which)
    p = subprocess.run([sys.executable, "-c", WORKER], env=env, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-3000:]
    return dict(np.load(dst))


def test_checked_build_matches_the_normal_build(tmp_path):
    pytest.importorskip("torch")
    lib = os.path.join(ROOT, "paper_2501_08672_b300", "libgs_b300_checked.so")
    assert os.path.exists(lib), "build it: python -m paper_2501_08672_b300.build --checked"
    a = _run(tmp_path, "normal")
    b = _run(tmp_path, "checked")
    assert int(a["checked"][0]) == 0 and int(b["checked"][0]) == 1
    for k in a:
        if k in ("checked",):
            continue
        if k.startswith("overflow"):
            continue
        x, y = a[k], b[k]
        exact = k.endswith(("/rgb", "/T", "/n_contrib")) or k.startswith("ragged_det/")
        if exact:
            np.testing.assert_array_equal(x, y, err_msg=k)
        else:
            rel = np.linalg.norm(x.astype(np.float64) - y) / max(np.linalg.norm(x.astype(np.float64)), 1e-30)
            assert rel < 1e-5, (k, rel)
    assert int(b["overflow_rc"][0]) == -4  # GS_ERR_CAPACITY, reported once
    assert int(b["overflow_rc_after"][0]) == 0
    assert int(b["overflow_bins_rc"][0]) == -4
