"""Invariants and adversarial scenes of the forward path on the GPU: crop
invariance across tile boundaries (the synthetic analogue of the paper's
large-FOV cutout comparison, Sec. 5), rigid-transform invariance, extreme
anisotropy against the oracle, and the camera-inside discard (Sec. 3.3)."""
import dataclasses

import numpy as np
import pytest
import torch

import oracle as O
from paper_2504_12811_gb300 import scenes
from _gpu_util import (TOL_ABS, TOL_AMBIG, TOL_PSNR, compare_image, dev_array, oracle_image_and_mask, psnr,
                       run_frame, stats)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_12811_gb300 import build
    build.build()


def _ambiguous(scene, cam):
    prep = O.prepare(scene, cam)
    py, px = np.mgrid[0:cam.height, 0:cam.width]
    return O.ambiguous_pixels(prep, px.ravel(), py.ravel()).numpy().reshape(cam.height, cam.width)


def test_crop_invariance_across_tile_boundaries():
    """A larger image with the same focal length and the principal point moved
    by (37, 21) pixels sees the small image's rays at pixels shifted by that
    offset, but over tiles that cut them elsewhere: the crop must match."""
    scene, cams = scenes.workload("small")
    cam = cams[0]
    dx, dy = 37, 21
    big = dataclasses.replace(cam, width=cam.width + 61, height=cam.height + 45, cx=cam.cx + dx, cy=cam.cy + dy)
    ws, rgb, alpha, _ = run_frame(scene, cam)
    ws2, rgb2, alpha2, _ = run_frame(scene, big)
    assert stats(ws)["status"] == "OK" and stats(ws2)["status"] == "OK"
    crop = rgb2[:, dy:dy + cam.height, dx:dx + cam.width]
    crop_a = alpha2[dy:dy + cam.height, dx:dx + cam.width]
    amb = _ambiguous(scene, cam)
    r = compare_image(rgb, alpha, crop.cpu(), crop_a.cpu(), amb)
    assert r["ambiguous_fraction"] < TOL_AMBIG
    assert r["max_abs_clean"] <= TOL_ABS, r
    assert r["psnr_rgb"] >= TOL_PSNR and r["psnr_alpha"] >= TOL_PSNR


def _quat_mul(a, b):
    """Hamilton product of (w, x, y, z) quaternions, row-wise."""
    aw, ax, ay, az = np.moveaxis(a, -1, 0)
    bw, bx, by, bz = np.moveaxis(b, -1, 0)
    return np.stack([aw * bw - ax * bx - ay * by - az * bz, aw * bx + ax * bw + ay * bz - az * by,
                     aw * by - ax * bz + ay * bw + az * bx, aw * bz + ax * by - ay * bx + az * bw], -1)


def test_rigid_transform_invariance():
    """Moving the scene and the camera by the same rigid motion leaves the
    image unchanged (SH degree 0: view-independent colour)."""
    scene, cams = scenes.workload("small")
    assert scene.sh_degree == 0
    cam = cams[1]
    qr = np.array([0.9, 0.2, -0.3, 0.25])
    qr /= np.linalg.norm(qr)
    R = O.rotation_from_quaternion(torch.tensor(qr[None])).numpy()[0]
    t = np.array([0.3, -0.2, 0.5])
    moved = dataclasses.replace(
        scene, means=(scene.means.astype(np.float64) @ R.T + t).astype(np.float32),
        quats=_quat_mul(np.broadcast_to(qr, scene.quats.shape), scene.quats.astype(np.float64)).astype(np.float32))
    T = np.eye(4)
    T[:3, :3], T[:3, 3] = R, t
    cam2 = dataclasses.replace(cam, viewmat=(cam.viewmat.astype(np.float64) @ np.linalg.inv(T)).astype(np.float32))
    ws, rgb, alpha, _ = run_frame(scene, cam)
    ws2, rgb2, alpha2, _ = run_frame(moved, cam2)
    amb = _ambiguous(scene, cam)
    r = compare_image(rgb, alpha, rgb2.cpu(), alpha2.cpu(), amb)
    assert r["max_abs_clean"] <= TOL_ABS, r
    assert r["psnr_rgb"] >= TOL_PSNR


def test_needle_and_flat_gaussians_match_oracle():
    """Extreme anisotropy (log-scales of -12 on one or two axes): the adaptive
    3D filter keeps them renderable and the bounds conservative."""
    base = scenes.uniform_cube_scene(600, seed=8)
    ls = base.log_scales.copy()
    ls[:200] = [-2.5, -12.0, -12.0]     # needles
    ls[200:400] = [-2.5, -2.5, -12.0]   # flat discs
    scene = dataclasses.replace(base, log_scales=ls)
    cam = scenes.make_camera((0.4, -0.3, -2.6), target=(0, 0, 0), width=96, height=80)
    ws, rgb, alpha, _ = run_frame(scene, cam)
    st = stats(ws)
    assert st["status"] == "OK" and st["n_visible"] > 300
    prep, ref_rgb, ref_alpha, amb = oracle_image_and_mask(scene, cam)
    r = compare_image(rgb, alpha, ref_rgb, ref_alpha, amb)
    assert r["finite"]
    assert r["ambiguous_fraction"] < TOL_AMBIG
    assert r["max_abs_clean"] <= TOL_ABS, r
    assert r["psnr_rgb"] >= TOL_PSNR


def test_gaussian_enclosing_the_camera_is_discarded():
    """A Gaussian whose tau-ellipsoid contains the camera centre is dropped
    (Sec. 3.3): it is not visible and the image equals the render without it."""
    sc = scenes.uniform_cube_scene(300, seed=9)
    pos = np.array([0.1, -0.1, -0.5])
    sc.means[0] = pos + np.array([0.05, 0.0, 0.1])
    sc.log_scales[0] = [-0.5, -0.5, -0.5]
    sc.opacity_logits[0] = 4.0
    cam = scenes.make_camera(tuple(pos), target=(0, 0, 0), width=64, height=64)
    prep = O.prepare(sc, cam)
    assert not bool(prep["alive"][0])                         # the oracle discards it too
    ws, rgb, alpha, _ = run_frame(sc, cam)
    counts = dev_array(ws, ws.view().counts, sc.n, np.uint32)
    assert counts[0] == 0
    ws2, rgb2, alpha2, _ = run_frame(sc.subset(np.arange(1, sc.n)), cam)
    np.testing.assert_allclose(rgb.cpu().numpy(), rgb2.cpu().numpy(), atol=1e-6)
    np.testing.assert_allclose(alpha.cpu().numpy(), alpha2.cpu().numpy(), atol=1e-6)
