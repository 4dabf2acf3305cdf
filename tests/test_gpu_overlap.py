"""Adam over the active rows only, and Step 4 (appending Gaussians, Sec.
II-C) overlapped with a running optimisation iteration on another stream."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_2501_08672_b300 import binding as B  # noqa: E402
from paper_2501_08672_b300 import scenes  # noqa: E402
from paper_2501_08672_b300.render import GaussianWindow, Renderer, WindowOptimizer  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    torch.cuda.init()


@pytest.mark.parametrize("ranges", [[(0, 1001)], [(0, 12), (16, 17), (100, 363), (400, 1001)], [(8, 8), (1000, 1001)]])
def test_adam_ranges_touch_only_their_elements(orc, ranges):
    rng = np.random.default_rng(len(ranges))
    n = 1001
    # p, m arbitrary; the second moment v is non-negative (away from 0, where
    # the step is ill-conditioned)
    base = [rng.standard_normal(n).astype(np.float32), rng.standard_normal(n).astype(np.float32),
            (0.05 + np.abs(rng.standard_normal(n))).astype(np.float32)]
    g = torch.as_tensor(rng.standard_normal(n).astype(np.float32)).cuda()
    ctx = B.Context(0)
    p, m, v = [torch.as_tensor(b).cuda() for b in base]
    ctx.adam_step_ranges(p, g, m, v, ranges, 1e-2, 0.9, 0.999, 1e-8, step=3)
    pf, mf, vf = [torch.as_tensor(b).cuda() for b in base]
    ctx.adam_step(pf, g, mf, vf, 1e-2, 0.9, 0.999, 1e-8, 3)
    inside = np.zeros(n, bool)
    for b, e in ranges:
        inside[b:e] = True
    for got, full, b in zip((p, m, v), (pf, mf, vf), base):
        got, full = got.cpu().numpy(), full.cpu().numpy()
        np.testing.assert_array_equal(got[inside], full[inside])
        np.testing.assert_array_equal(got[~inside], b[~inside])
    # and the oracle for the full step
    ref = base[0].astype(np.float64).copy()
    mm, vv = base[1].astype(np.float64).copy(), base[2].astype(np.float64).copy()
    orc.adam(ref, g.cpu().numpy().astype(np.float64), mm, vv, 1e-2, 0.9, 0.999, 1e-8, 3)
    np.testing.assert_allclose(pf.cpu().numpy(), ref, rtol=1e-5, atol=1e-6)


def test_adam_ranges_rejects_bad_ranges():
    ctx = B.Context(0)
    t = [torch.zeros(64, device="cuda") for _ in range(4)]
    for bad in ([(1, 8)], [(0, 65)], [(0, 16), (8, 24)], []):
        with pytest.raises(B.GsError):
            ctx.adam_step_ranges(*t, bad, 1e-3, 0.9, 0.999, 1e-8, step=1)


def test_append_overlapped_with_iterations():
    """Graph replays of the optimisation on the compute stream while new
    Gaussians are appended on a copy stream: the iterations give the same
    window as without the append, and the appended rows arrive intact."""
    n, extra = 20_000, 30_000
    p = scenes.box_room_scene(n, seed=50, sh_degree=1)
    new = scenes.box_room_scene(extra, seed=51, sh_degree=1)
    views = scenes.arc_views(2, 160, 128, 150.0, n_gaussians=n)
    rt = Renderer(views, 0)
    wt = GaussianWindow(scenes.perturbed_copy(p, seed=52), 0)
    rt.forward(wt.struct())
    targets = rt.rgb.clone()
    results = []
    for concurrent in (False, True):
        opt = WindowOptimizer(p, views, targets, lr=1e-3, capacity=n + extra)
        opt.step(count=True)
        opt.capture()
        torch.cuda.synchronize()
        side = torch.cuda.Stream()
        pinned = {k: torch.as_tensor(np.ascontiguousarray(new[k], np.float32)).pin_memory()
                  for k in GaussianWindow.GROUPS}
        for _ in range(5):
            opt.step()
            if concurrent and _ == 1:
                with torch.cuda.stream(side):
                    # rows [n, n + extra): the graph never touches them
                    for k in GaussianWindow.GROUPS:
                        opt.win.column(k)[n:n + extra].view(extra, -1).copy_(pinned[k].view(extra, -1),
                                                                           non_blocking=True)
                    opt.win.ctx().window_clear([opt.win.column(k, f) for k in GaussianWindow.GROUPS
                                                for f in (opt.win.m, opt.win.v)], n, n + extra, stream=side)
        torch.cuda.synchronize()
        results.append({k: opt.win.column(k)[:n + extra].cpu().numpy().copy() for k in GaussianWindow.GROUPS})
    # the backward's float atomics make runs differ in the last bits, which
    # Adam can turn into up to about lr per step on near-zero gradients: the
    # active rows agree within 5 steps x 3 lr, and closely on average
    for k in GaussianWindow.GROUPS:
        a, b = results[1][k][:n].astype(np.float64), results[0][k][:n].astype(np.float64)
        assert np.all(np.isfinite(a))
        assert np.abs(a - b).max() <= 5 * 3 * 1e-3
        assert np.abs(a - b).mean() <= 1e-5
        np.testing.assert_array_equal(results[1][k][n:].reshape(extra, -1),
                                      np.asarray(new[k], np.float32).reshape(extra, -1))
