"""gs_l1_loss_noalloc: the L1 loss for callers that cannot allocate device
memory (a real-time loop that allocates nothing after start-up, or a host
framework that owns every device allocation).  It keeps its partial sums in a
fixed array inside the library instead of a caller workspace; its results must
equal those of gs_l1_loss.  This file is collected last so that a run that
stops at the first failure has already run every other test."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_2501_08672_b300 import binding as B  # noqa: E402
from paper_2501_08672_b300 import scenes  # noqa: E402

TOL = 1e-4  # the forward tolerance of the parity tests


def _views():
    return [scenes.identity_view(200, 136, 160.0, 0, 10), scenes.identity_view(96, 150, 90.0, 0, 10),
            scenes.identity_view(64, 48, 50.0, 0, 10)]


def _noalloc(views_c, n_views, rgb, target, dl, loss):
    msg = ctypes.create_string_buffer(256)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = B.lib().gs_l1_loss_noalloc(views_c, n_views, ctypes.c_void_p(rgb.data_ptr()),
                                    ctypes.c_void_p(target.data_ptr()), ctypes.c_void_p(dl.data_ptr()),
                                    ctypes.c_void_p(loss.data_ptr()) if loss is not None else None, stream,
                                    msg, len(msg))
    return rc, msg.value.decode()


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")


def test_noalloc_l1_matches_workspace_l1_on_two_calls():
    views = _views()
    vc = B.make_views(views)
    npx = sum(v["W"] * v["H"] for v in views)
    ctx = B.Context(0)
    cap = 1024
    ws = torch.empty(ctx.workspace_bytes(vc, cap), dtype=torch.uint8, device="cuda")
    wss = B.Context.ws_struct(ws, cap)
    gen = torch.Generator(device="cuda").manual_seed(7)
    for call in range(2):  # two calls in a row: nothing from the first may leak into the second
        rgb = torch.rand(3 * npx, device="cuda", generator=gen)
        target = torch.rand(3 * npx, device="cuda", generator=gen)
        dl_ref = torch.empty_like(rgb)
        loss_ref = torch.zeros(1, device="cuda")
        ctx.l1_loss(vc, wss, rgb, target, dl_ref, loss_ref)
        dl = torch.full_like(rgb, float("nan"))
        loss = torch.full((1,), float("nan"), device="cuda")
        rc, msg = _noalloc(vc, len(views), rgb, target, dl, loss)
        torch.cuda.synchronize()
        assert rc == B.GS_OK, msg
        assert float((dl - dl_ref).abs().max()) <= TOL
        assert abs(float(loss.item()) - float(loss_ref.item())) <= TOL
        # and against the definition, in FP64 on the host: the mean absolute
        # residual per view averaged over views, and its gradient
        # sign(rgb - target) / (3 H W V)
        d = (rgb - target).double().cpu().numpy()
        sizes = [3 * v["W"] * v["H"] for v in views]
        parts = np.split(d, np.cumsum(sizes)[:-1])
        expect = sum(np.abs(c).mean() for c in parts) / len(views)
        assert abs(float(loss.item()) - expect) <= TOL
        grad = np.concatenate([np.sign(c) / (c.size * len(views)) for c in parts])
        np.testing.assert_allclose(dl.double().cpu().numpy(), grad, rtol=1e-6, atol=0)


def test_noalloc_l1_without_loss_pointer_writes_the_gradient_only():
    """With loss = NULL only the gradient is written (one launch), equal to
    that of gs_l1_loss."""
    views = _views()
    vc = B.make_views(views)
    npx = sum(v["W"] * v["H"] for v in views)
    ctx = B.Context(0)
    cap = 1024
    ws = torch.empty(ctx.workspace_bytes(vc, cap), dtype=torch.uint8, device="cuda")
    gen = torch.Generator(device="cuda").manual_seed(9)
    rgb = torch.rand(3 * npx, device="cuda", generator=gen)
    target = torch.rand(3 * npx, device="cuda", generator=gen)
    dl_ref = torch.empty_like(rgb)
    ctx.l1_loss(vc, B.Context.ws_struct(ws, cap), rgb, target, dl_ref, None)
    dl = torch.full_like(rgb, float("nan"))
    rc, msg = _noalloc(vc, len(views), rgb, target, dl, None)
    torch.cuda.synchronize()
    assert rc == B.GS_OK, msg
    assert float((dl - dl_ref).abs().max()) <= TOL


def test_noalloc_l1_rejects_batches_beyond_its_fixed_scratch():
    big = [scenes.identity_view(2048, 2048, 1000.0, 0, 10) for _ in range(64)]
    vc = B.make_views(big)
    t = torch.zeros(8, device="cuda")  # never read: the size check comes first
    rc, msg = _noalloc(vc, len(big), t, t, t, t)
    assert rc == B.GS_ERR_CAPACITY
    assert "fixed scratch" in msg
