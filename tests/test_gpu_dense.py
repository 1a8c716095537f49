"""Exact per-pixel order in dense content (depth peeling), against the oracle.

The training views of the 500k-Gaussian cube (1280x832) and the serving views
from inside the 200k/1M cubes keep 20-80 contributors per pixel waiting at
once, beyond the 16-entry per-pixel queue: there the renderer defers its
farthest contributors to further passes over the tile.  These tests render
the full frames with the C-ABI calls and compare pixels sampled at random
with the oracle's exact (t*, index) order, element by element, and the
gradients of a loss on sampled pixels with the oracle's autograd."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2504_12811_gb300 import aaag, scenes
from _gpu_util import TOL_ABS, TOL_PSNR, check_gradient_elements, psnr

pytestmark = pytest.mark.gpu

# Largest fraction of ambiguous pixels that may be excused from the max-abs
# check.  Thousands of Gaussians touch every ray in these views (and with the
# camera inside the cloud, many straddle the near plane), so 0.5-1% of the
# pixels hold a decision within float32 reach of its threshold: alpha at
# 1/255, t* at z_near, or two nearly tied depths near the front.  The excused
# pixels still count in the PSNR.
AMBIG_MAX = 2e-2
GROUPS = ("means", "log_scales", "quats", "opacity_logits", "sh")


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_12811_gb300 import build
    build.build()


def _sampled_parity(scene, cam, m, seed, capacity):
    ds = aaag.DeviceScene(scene)
    ws = aaag.Workspace(scene.n, cam.width, cam.height, capacity)
    rgb, alpha = aaag.render(ds, cam, ws)
    st = aaag.stats(ws)
    torch.cuda.synchronize()
    rng = np.random.default_rng(seed)
    px = rng.integers(0, cam.width, m)
    py = rng.integers(0, cam.height, m)
    prep = O.prepare(scene, cam)
    ref, ref_a = O.render_pixels(scene, cam, px, py, prep=prep)
    amb = np.concatenate([O.ambiguous_pixels(prep, px[i:i + 256], py[i:i + 256]).numpy()
                          for i in range(0, m, 256)])
    g = rgb.cpu().numpy()[:, py, px].T.astype(np.float64)
    ga = alpha.cpu().numpy()[py, px].astype(np.float64)
    err = np.maximum(np.abs(g - ref.numpy()).max(1), np.abs(ga - ref_a.numpy()))
    print(f"stats={st} max|err| clean={err[~amb].max():.3e} all={err.max():.3e} "
          f"ambiguous={amb.mean():.4f} psnr={psnr(g, ref.numpy()):.1f}")
    assert st["status"] == "OK"
    assert st["misorders"] == 0
    if err.max() > TOL_ABS:
        # only pixels whose decisions sit within float32 reach of a threshold
        # may be excused
        assert amb.mean() < AMBIG_MAX
        assert err[~amb].max() <= TOL_ABS
    assert psnr(g, ref.numpy()) >= TOL_PSNR
    assert psnr(ga, ref_a.numpy()) >= TOL_PSNR
    return st


@pytest.mark.parametrize("view", [0, 2])
def test_training_view_exact_order(view):
    """500k Gaussians (SH 3), 1280x832: the per-pixel queue fills on most
    pixels, so most pixels take several passes."""
    scene, cams = scenes.workload("train500k")
    st = _sampled_parity(scene, cams[view], 2400, 40 + view, 64 << 20)
    assert st["extra_passes"] > 100_000      # the deferral path is what ran


def test_serving_stereo_eye_exact_order():
    """One 1832x1920, 110 deg eye of a stereo request from inside the 200k
    serving scene (uniform cube, SH 3)."""
    scene = scenes.serving_scenes({"s200k": 200_000})["s200k"]
    rng = np.random.default_rng(31)
    cam = scenes.request_cameras("stereo", rng)[0]
    st = _sampled_parity(scene, cam, 2000, 32, 96 << 20)
    assert st["extra_passes"] > 0


def test_serving_hd_view_exact_order():
    """A 1920x1080 view from inside the 1M serving scene."""
    scene = scenes.serving_scenes({"s1m": 1_000_000})["s1m"]
    rng = np.random.default_rng(33)
    cam = scenes.request_cameras("hd", rng)[0]
    st = _sampled_parity(scene, cam, 1024, 34, 96 << 20)
    assert st["extra_passes"] > 0


def test_training_view_gradients_sampled_pixels():
    """Gradients of a loss on 160 random pixels of a 500k-Gaussian training
    view through the autograd Function, against the oracle's autograd on the
    Gaussians that reach those pixels: per group relative L2 <= 1e-3, and the
    elementwise bound of `check_gradient_elements`."""
    from paper_2504_12811_gb300 import autograd as AG
    scene, cams = scenes.workload("train500k")
    cam = cams[1]
    rng = np.random.default_rng(12)
    m = 160
    px = rng.integers(0, cam.width, m)
    py = rng.integers(0, cam.height, m)
    prep = O.prepare(scene, cam)
    amb = O.ambiguous_pixels(prep, px, py).numpy()
    px, py = px[~amb], py[~amb]
    w_rgb = np.zeros((3, cam.height, cam.width), np.float32)
    w_alpha = np.zeros((cam.height, cam.width), np.float32)
    w_rgb[:, py, px] = rng.standard_normal((3, px.size))
    w_alpha[py, px] = rng.standard_normal(px.size)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda().requires_grad_(True)
    leaves = [t(getattr(scene, g)) for g in GROUPS]
    vt = torch.from_numpy(scene.vhat_train).cuda()
    ws = aaag.Workspace(scene.n, cam.width, cam.height, 64 << 20)
    rgb, alpha = AG.render(*leaves, vt, cam, ws)
    loss = (rgb * torch.from_numpy(w_rgb).cuda()).sum() + (alpha * torch.from_numpy(w_alpha).cuda()).sum()
    loss.backward()
    st = aaag.stats(ws, check=False)
    assert st["status"] == "OK" and st["replay_mismatch"] == 0 and st["misorders"] == 0
    assert st["extra_passes"] > 0
    g_gpu = {g: l.grad.detach().cpu().numpy().astype(np.float64) for g, l in zip(GROUPS, leaves)}
    # the Gaussians with alpha >= 1/255 at a sampled pixel (the only ones with a gradient)
    rho2, ts = O.ray_maximum(prep, px, py)
    _, contrib, _ = O.pixel_alphas(prep, rho2, ts)
    touched = np.nonzero(contrib.numpy().any(0))[0]
    sub = scene.subset(touched)
    stt = O.scene_tensors(sub, requires_grad=True)
    ref, ref_a = O.render_pixels(stt, cam, px, py)
    wr = torch.from_numpy(w_rgb[:, py, px].T.astype(np.float64))
    wa = torch.from_numpy(w_alpha[py, px].astype(np.float64))
    ((ref * wr).sum() + (ref_a * wa).sum()).backward()
    others = np.ones(scene.n, bool)
    others[touched] = False
    for g in GROUPS:
        assert np.all(g_gpu[g][others] == 0), g
    print(f"stats={st}")
    report = check_gradient_elements({g: g_gpu[g][touched] for g in GROUPS},
                                     {g: stt[g].grad.numpy() for g in GROUPS}, GROUPS)
    for g, (rel, _, _) in report.items():
        assert rel <= 1e-3, (g, report)
