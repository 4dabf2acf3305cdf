"""Binning at a larger bin size split into per-tile lists (gs_config
bin_tile_size): the per-tile lists against binning at the tile size
directly, the images bit for bit, and the whole path against the FP64
oracle."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_2501_08672_b300 import scenes  # noqa: E402
from paper_2501_08672_b300.render import GaussianWindow, Renderer  # noqa: E402

from test_gpu_parity import (_footprint_min, compare_images, gpu_forward, l1_parity, l1_target,  # noqa: E402
                             ragged_views, ws_view)

# (tile size, pixels per thread, bin size): factors 2 and 4
SPLITS = [(8, 2, 16), (8, 2, 32), (8, 1, 32), (16, 2, 32)]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")


def tile_lists(r):
    torch.cuda.synchronize()
    L = r.layout()
    T = L.n_tiles
    rg = ws_view(r, L.tile_ranges, np.uint32, 2 * T).reshape(T, 2)
    sv = ws_view(r, L.sorted_vals, np.uint32, int(rg[:, 1].max()) if T else 0)
    return [sv[a:b].copy() for a, b in rg], L


def render(win, views, ts, ppt, bin_ts):
    r = Renderer(views, 0, ts, pixels_per_thread=ppt, batch=128, bin_tile_size=bin_ts)
    r.forward(win.struct())
    torch.cuda.synchronize()
    return r


def _is_subsequence(a, b):
    it = iter(b.tolist())
    return all(x in it for x in a.tolist())


def split_from_bins(r, ts, views):
    """Every tile's full list rebuilt on the host from the sorted (bin,
    record) pairs: the records of the tile's bin, in the bin's order, whose
    key carries the tile's bit."""
    torch.cuda.synchronize()
    L = r.layout()
    F = L.bin_size // ts
    rb = ws_view(r, L.bin_ranges, np.uint32, 2 * L.n_bins).reshape(-1, 2)
    n = int(rb[:, 1].max()) if L.n_bins else 0
    keys = ws_view(r, L.bin_keys, np.uint32, n)
    vals = ws_view(r, L.bin_vals, np.uint32, n)
    out = []
    bin_off = 0
    for v in views:
        tx_n, ty_n = (v["W"] + ts - 1) // ts, (v["H"] + ts - 1) // ts
        bx_n = (v["W"] + L.bin_size - 1) // L.bin_size
        by_n = (v["H"] + L.bin_size - 1) // L.bin_size
        for ty in range(ty_n):
            for tx in range(tx_n):
                b = bin_off + (ty // F) * bx_n + tx // F
                a, e = rb[b]
                bit = 32 - F * F + (ty % F) * F + tx % F
                k = keys[a:e]
                out.append(vals[a:e][((k >> np.uint32(bit)) & np.uint32(1)).astype(bool)].copy())
        bin_off += bx_n * by_n
    return out


@pytest.mark.parametrize("ts,ppt,bin_ts", SPLITS)
def test_split_lists_match_binning_at_the_tile_size(ts, ppt, bin_ts):
    """Ragged views (sizes not multiples of the bin, so edge bins hold tiles
    past the image): every tile's list split from the bins (rebuilt from the
    bin lists and the tile masks in their keys) holds the list that binning
    at the tile size gives, in the same order, plus at most records whose
    footprint only grazes the tile (within the binning test's margin); the
    lists gs_bin split out are those; the images and T agree bit for bit."""
    n = 6000
    p = scenes.frustum_scene(n, seed=31)
    views = ragged_views(n)
    win = GaussianWindow(p, 0)
    r0 = render(win, views, ts, ppt, 0)
    r1 = render(win, views, ts, ppt, bin_ts)
    l0, L0 = tile_lists(r0)
    written, L1 = tile_lists(r1)
    l1 = split_from_bins(r1, ts, views)
    assert L1.bin_size == bin_ts and L1.n_tiles == L0.n_tiles and L1.n_bins < L0.n_tiles
    assert len(l1) == len(l0) == len(written)
    for t, (w, full) in enumerate(zip(written, l1)):
        assert np.array_equal(w, full), "tile %d: the split list differs from its bin's entries with its bit" % t
    assert int(r1.last_pairs) < int(r0.last_pairs)
    M = L1.n_records
    rec = ws_view(r1, L1.records, np.float32, 12 * M).reshape(M, 12)
    log2_amin = math.log2(1.0 / 255.0)
    tile_xy = []
    for v in views:
        tx_n = (v["W"] + ts - 1) // ts
        ty_n = (v["H"] + ts - 1) // ts
        tile_xy += [(tx, ty) for ty in range(ty_n) for tx in range(tx_n)]
    extra = 0
    for t, (a, b) in enumerate(zip(l0, l1)):
        assert _is_subsequence(a, b), "tile %d: the direct list is not a subsequence of the split one" % t
        for i in set(b.tolist()) - set(a.tolist()):
            tx, ty = tile_xy[t]
            m = _footprint_min(rec[i], tx * ts + 0.5, tx * ts + ts - 0.5, ty * ts + 0.5, ty * ts + ts - 0.5)
            Lim = float(rec[i, 6]) - log2_amin
            assert m > Lim * (1 - 1e-4), "tile %d: record %d clearly reached yet missing from the direct list" % (t, i)
            assert m <= Lim * 1.01 + 0.01, "tile %d: record %d clearly missed yet listed" % (t, i)
            extra += 1
    total = sum(len(a) for a in l0)
    assert extra <= 1e-3 * total + 3
    # front to back along every split list
    depth = rec[:, 10].astype(np.float64)
    for t, b in enumerate(l1):
        d = depth[b]
        assert np.all(d[1:] >= d[:-1] - 1e-6 * np.abs(d[:-1])), "tile %d is not front to back" % t
    assert torch.equal(r0.rgb, r1.rgb) and torch.equal(r0.T, r1.T)


def test_split_applies_only_in_truncated_mode_without_determinism():
    """Exact mode and the deterministic backward bin at the tile size."""
    n = 2000
    p = scenes.frustum_scene(n, seed=32)
    views = ragged_views(n)
    for cfg in (dict(alpha_min=0.0, alpha_max=1.0, T_min=0.0), dict(deterministic=1)):
        _, r = gpu_forward(p, views, tile_size=8, bin_tile_size=32, **cfg)
        L = r.layout()
        assert L.bin_size == 8 and L.n_bins == L.n_tiles and L.sorted_vals == L.bin_vals


@pytest.mark.parametrize("ts,ppt,bin_ts", [(8, 2, 32), (16, 2, 32)])
def test_split_path_matches_oracle(orc, ts, ppt, bin_ts):
    """Forward images and the L1 loss's gradients (every parameter group and
    the pose) through the split lists against the FP64 oracle."""
    p = scenes.frustum_scene(1500, seed=33)
    views = ragged_views(1500)
    win, r = gpu_forward(p, views, tile_size=ts, pixels_per_thread=ppt, batch=128, bin_tile_size=bin_ts)
    for v, img, T in zip(views, r.images(), B_unpack_T(r, views)):
        out = orc.render_view(p, v)
        compare_images(out, img.cpu().numpy(), T)
    l1_parity(orc, win, r, p, views, l1_target(p, views))


def B_unpack_T(r, views):
    out, off = [], 0
    T = r.T.cpu().numpy()
    for v in views:
        n = v["W"] * v["H"]
        out.append(T[off:off + n].reshape(v["H"], v["W"]))
        off += n
    return out


def test_box_room_window_split_matches_oracle(orc):
    """The box-room window (SH degree 1) with 8 x 8 tiles from 32 x 32 bins,
    the headline's launch shape, against the oracle."""
    n = 20_000
    p = scenes.box_room_scene(n, seed=34)
    views = scenes.arc_views(3, 192, 160, 180.0, n_gaussians=n)
    views[1] = dict(views[1], W=176, H=144, cx=88.0, cy=72.0)
    win, r = gpu_forward(p, views, tile_size=8, pixels_per_thread=2, batch=128, bin_tile_size=32)
    assert r.layout().bin_size == 32
    l1_parity(orc, win, r, p, views, l1_target(p, views))


def test_pose_normal_with_bins_matches_binning_at_the_tile_size():
    """gs_pose_normal over the lists split from 32 x 32 bins: its per-view
    normal equations equal those of binning at the tile size (the extra
    grazing records add nothing)."""
    n = 4000
    p = scenes.box_room_scene(n, seed=35)
    views = scenes.arc_views(2, 176, 144, 160.0, n_gaussians=n)
    win = GaussianWindow(p, 0)
    res = []
    for bin_ts in (0, 32):
        r = Renderer(views, 0, 8, pixels_per_thread=2, batch=128, bin_tile_size=bin_ts)
        r.forward(win.struct())
        target = torch.zeros_like(r.rgb)
        normal = r.pose_normal(win.struct(), target)
        torch.cuda.synchronize()
        res.append(np.asarray(normal.cpu().numpy(), np.float64))
        assert r.layout().bin_size == (bin_ts or 8)
    np.testing.assert_allclose(res[1], res[0], rtol=1e-12, atol=0)


def test_bins_that_would_not_fit_below_the_mask_bin_at_the_tile_size():
    """4 x 4 tiles per bin leave 16 bits for the bin id: 64 views of
    1280 x 1024 (81920 bins of 32 x 32) bin at the tile size instead, while
    2 x 2 tiles per bin (28 bits) still split."""
    from paper_2501_08672_b300 import binding as B
    views = [scenes.identity_view(1280, 1024, 1000.0, 0, 10) for _ in range(64)]
    vc = B.make_views(views)
    for bin_ts, expect in ((32, 8), (16, 16)):
        ctx = B.Context(0, tile_size=8, pixels_per_thread=2, batch=128, bin_tile_size=bin_ts)
        L = ctx.layout(vc, 1024)
        assert L.bin_size == expect and (L.n_bins == L.n_tiles) == (expect == 8)


def test_dispatch_order_by_walk_depth_changes_no_result():
    """The first forward dispatches tiles by list length, the next ones by the
    walk depths the previous forward reached: images, T and n_contrib are
    identical, and the deterministic backward's gradients bit for bit."""
    n = 8000
    p = scenes.box_room_scene(n, seed=36)
    views = scenes.arc_views(3, 192, 160, 180.0, n_gaussians=n)
    win = GaussianWindow(p, 0)
    for cfg in (dict(tile_size=8, pixels_per_thread=2, batch=128, bin_tile_size=32),
                dict(tile_size=16, deterministic=1)):
        ts = cfg.pop("tile_size")
        r = Renderer(views, 0, ts, **cfg)
        outs = []
        for it in range(3):
            r.forward(win.struct(), count=(it == 0))
            torch.cuda.synchronize()
            order = r.ws[r.layout().counters:r.layout().counters + 64].view(torch.int64).cpu().numpy()
            g = win.grad_tensors()
            r.backward(win.struct(), torch.full_like(r.rgb, 1e-3), grads=g)
            torch.cuda.synchronize()
            outs.append((r.rgb.clone(), r.T.clone(), r.n_contrib.clone(), win.gflat.clone(), int(order[4])))
        assert outs[1][4] == outs[2][4] == r.layout().n_tiles  # walk-depth keys in use
        for o in outs[1:]:
            assert torch.equal(o[0], outs[0][0]) and torch.equal(o[1], outs[0][1]) and torch.equal(o[2], outs[0][2])
            if cfg.get("deterministic"):
                assert torch.equal(o[3], outs[0][3])
            else:
                assert float((o[3] - outs[0][3]).norm() / outs[0][3].norm()) < 1e-5
