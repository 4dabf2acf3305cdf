"""D-SSIM photometric loss through the C ABI against the FP64 oracle.

Tolerance: the kernels form the five windowed moments by two 11-tap FP32
passes (relative rounding of each moment below 22 u with u = 2^-24, i.e. an
absolute error below 1.4e-6 for images in [0, 1]); a variance is a
difference of two such moments, and the denominator s_x^2 + s_y^2 + C2 is at
least C2 = 9e-4, so the SSIM value of a pixel and its derivatives carry a
relative error up to about 6e-3 where the window is flat and far less where
it is textured.  Averaged over an image the loss agrees to 1e-5 absolute;
the gradient is compared by its relative L2 norm (1e-3) and element-wise
against 1 % of its largest magnitude.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_2501_08672_b300 import binding as B  # noqa: E402
from paper_2501_08672_b300 import scenes  # noqa: E402
from paper_2501_08672_b300.render import Renderer, WindowOptimizer  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    torch.cuda.init()


def _views(sizes):
    return [scenes.identity_view(w, h, 100.0, 0, 1) for w, h in sizes]


def _images(rng, sizes, smooth):
    """Rendered-like pairs: smooth shading plus texture (flat and textured
    windows both occur), target = a perturbed copy."""
    xs, ys = [], []
    for w, h in sizes:
        yy, xx = np.mgrid[0:h, 0:w]
        base = 0.5 + 0.3 * np.sin(xx / 9.0 + np.arange(3)[:, None, None]) * np.cos(yy / 13.0)
        if not smooth:
            base = base + rng.normal(0, 0.1, (3, h, w))
        x = np.clip(base, 0, 1)
        y = np.clip(x + rng.normal(0, 0.05, x.shape) + 0.02, 0, 1)
        xs.append(x.astype(np.float32))
        ys.append(y.astype(np.float32))
    return xs, ys


def _pack(imgs):
    return torch.as_tensor(np.concatenate([i.reshape(-1) for i in imgs])).cuda()


def _run(ctx, views_d, xs, ys, lam):
    views = B.make_views(views_d)
    rgb, tgt = _pack(xs), _pack(ys)
    scratch = torch.empty(int(B.lib().gs_dssim_scratch_floats(views, len(views))), device="cuda")
    dl = torch.full_like(rgb, 7.0)
    loss = torch.zeros(1, device="cuda")
    ctx.dssim_loss(views, rgb, tgt, lam, scratch, dl, loss)
    torch.cuda.synchronize()
    return float(loss.item()), dl.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("smooth", [True, False])
def test_dssim_matches_oracle_ragged_views(orc, smooth):
    sizes = [(200, 136), (150, 100), (33, 17), (7, 5), (640, 512)]
    rng = np.random.default_rng(20 + smooth)
    xs, ys = _images(rng, sizes, smooth)
    lam = 0.2
    L, g = _run(B.Context(0), _views(sizes), xs, ys, lam)
    Lo, go = orc.dssim_loss_grad(xs, ys, lam)
    assert abs(L - Lo) < 1e-5, (L, Lo)
    ref = np.concatenate([a.reshape(-1) for a in go])
    err = np.linalg.norm(g - ref) / np.linalg.norm(ref)
    assert err < 1e-3, err
    assert np.abs(g - ref).max() <= 1e-2 * np.abs(ref).max()


def test_dssim_lambda_zero_is_the_l1_gradient(orc):
    sizes = [(64, 48), (40, 33)]
    rng = np.random.default_rng(22)
    xs, ys = _images(rng, sizes, False)
    L, g = _run(B.Context(0), _views(sizes), xs, ys, 0.0)
    Lo, go = orc.l1_loss_grad(xs, ys)
    assert abs(L - Lo) < 1e-6
    # sign / (3 H W V) in FP32, as the L1 kernel writes it
    ref = np.concatenate([(np.sign(x.astype(np.float64) - y) *
                           np.float32(1.0 / (np.float32(x.size) * np.float32(len(xs))))).reshape(-1)
                          for x, y in zip(xs, ys)])
    np.testing.assert_array_equal(g.astype(np.float32), ref.astype(np.float32))


def test_dssim_identical_images_vanish():
    sizes = [(96, 80)]
    rng = np.random.default_rng(23)
    xs, _ = _images(rng, sizes, False)
    L, g = _run(B.Context(0), _views(sizes), xs, xs, 1.0)
    assert abs(L) < 1e-5
    assert np.abs(g).max() < 1e-7


def test_dssim_rejects_bad_arguments():
    ctx = B.Context(0)
    views = B.make_views(_views([(32, 16)]))
    rgb = torch.zeros(3 * 32 * 16, device="cuda")
    dl = torch.zeros_like(rgb)
    n = int(B.lib().gs_dssim_scratch_floats(views, 1))
    scratch = torch.empty(n, device="cuda")
    with pytest.raises(B.GsError):
        ctx.dssim_loss(views, rgb, rgb, 1.5, scratch, dl)
    with pytest.raises(ValueError):
        ctx.dssim_loss(views, rgb, rgb, 0.2, torch.empty(n - 1, device="cuda"), dl)
    assert int(B.lib().gs_dssim_scratch_floats(views, 0)) == 0


def test_window_optimizer_with_dssim_reduces_loss():
    n = 20_000
    p = scenes.box_room_scene(n, seed=31, sh_degree=1)
    views = scenes.arc_views(2, 160, 128, 150.0, n_gaussians=n)
    q = dict(p, sh=p["sh"] + np.random.default_rng(32).normal(0, 0.2, p["sh"].shape).astype(np.float32))
    r = Renderer(views, 0)
    from paper_2501_08672_b300.render import GaussianWindow
    wt = GaussianWindow(p, 0)
    r.forward(wt.struct())
    targets = r.rgb.clone()
    opt = WindowOptimizer(q, views, targets, lr=5e-3, ssim_lambda=0.2)
    first = float(opt.step().item())
    for _ in range(30):
        last = opt.step()
    torch.cuda.synchronize()
    assert float(last.item()) < 0.8 * first
