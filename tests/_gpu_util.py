"""Helpers shared by the GPU tests: run the CUDA path through the C-ABI binding
and compare with the oracle."""
import math

import numpy as np
import torch

import oracle as O
from paper_2504_12811_gb300 import aaag, scenes

TOL_ABS = 2e-3        # max abs error on non-ambiguous pixels
TOL_PSNR = 55.0       # dB over all pixels
TOL_AMBIG = 1e-3      # largest allowed fraction of ambiguous pixels (0.1%)


# Gradients, element by element: |g - g_ref| <= 1e-3 max(|g_ref|, 1e-3 max|g_ref|)
# must hold for all but GRAD_ELEM_FRAC of the elements of a group, and every
# element must stay within GRAD_ELEM_LOOSE times that bound.  An element whose
# value is a sum of per-pixel terms that cancel (a Gaussian seen over
# thousands of pixels from both sides: the sum of the terms' magnitudes can
# be 100 times the sum) amplifies float32 rounding of the terms by that ratio.
GRAD_ELEM_FRAC = 5e-3
GRAD_ELEM_LOOSE = 250.0


def check_gradient_elements(g_gpu, g_ref, groups):
    """Per group: (relative L2, fraction of elements beyond the elementwise
    bound, largest ratio to it) over the elements whose reference is not 0
    or whose GPU value is not 0; asserts the limits above."""
    report = {}
    for g in groups:
        a, b = np.asarray(g_gpu[g], np.float64).ravel(), np.asarray(g_ref[g], np.float64).ravel()
        live = (a != 0) | (b != 0)
        a, b = a[live], b[live]
        rel = float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))
        bound = 1e-3 * np.maximum(np.abs(b), 1e-3 * np.abs(b).max())
        ratio = np.abs(a - b) / bound
        report[g] = (rel, float(np.mean(ratio > 1.0)), float(ratio.max()))
    print("gradients (relative L2, fraction beyond the elementwise bound, largest ratio):", report)
    for g, (rel, frac, worst) in report.items():
        assert frac <= GRAD_ELEM_FRAC, (g, report)
        assert worst <= GRAD_ELEM_LOOSE, (g, report)
    return report


def run_frame(scene, cam, capacity=None, params=None, stages=("pre", "cull", "sort", "render")):
    """Run the requested stages on a fresh workspace; returns (ws, rgb, alpha, dscene)."""
    ds = aaag.DeviceScene(scene)
    cap = capacity if capacity is not None else max(1 << 16, 64 * scene.n)
    ws = aaag.Workspace(scene.n, cam.width, cam.height, cap)
    st = aaag.current_stream()
    prm = params if params is not None else aaag.make_params()
    rgb = torch.full((3, cam.height, cam.width), float("nan"), device="cuda")
    alpha = torch.full((cam.height, cam.width), float("nan"), device="cuda")
    if "pre" in stages:
        aaag.aaag_preprocess(ds.struct(), aaag.make_camera(cam), prm, ws.handle, st)
    if "cull" in stages:
        aaag.aaag_cull(ws.handle, st)
    if "sort" in stages:
        aaag.aaag_sort(ws.handle, st)
    if "render" in stages:
        aaag.aaag_render(ws.handle, rgb.data_ptr(), alpha.data_ptr(), st)
    torch.cuda.synchronize()
    return ws, rgb, alpha, ds


def dev_array(ws, ptr, count, dtype):
    """Copy `count` elements of a workspace array (device pointer into the
    workspace buffer) to numpy, by slicing the torch tensor that backs it."""
    itemsize = np.dtype(dtype).itemsize
    if count == 0:
        return np.empty(0, dtype=dtype)
    off = int(ptr) - ws.buffer.data_ptr()
    assert 0 <= off and off + count * itemsize <= ws.buffer.numel()
    torch.cuda.synchronize()
    raw = ws.buffer[off:off + count * itemsize].cpu().numpy()
    return raw.view(dtype).copy()


def stats(ws):
    return aaag.stats(ws, check=False)


def psnr(a, b):
    mse = float(np.mean((a - b) ** 2))
    return math.inf if mse == 0 else 10 * math.log10(1.0 / mse)


def compare_image(gpu_rgb, gpu_alpha, ref_rgb, ref_alpha, ambiguous):
    """Returns a dict of error figures; `ambiguous` [H,W] bool."""
    g = gpu_rgb.detach().cpu().numpy().astype(np.float64)
    ga = gpu_alpha.detach().cpu().numpy().astype(np.float64)
    r = ref_rgb.numpy() if torch.is_tensor(ref_rgb) else ref_rgb
    ra = ref_alpha.numpy() if torch.is_tensor(ref_alpha) else ref_alpha
    err = np.abs(g - r).max(0)
    err = np.maximum(err, np.abs(ga - ra))
    clean = ~ambiguous
    return {
        "max_abs_clean": float(err[clean].max()) if clean.any() else 0.0,
        "max_abs_all": float(err.max()),
        "psnr_rgb": psnr(g, r),
        "psnr_alpha": psnr(ga, ra),
        "ambiguous_fraction": float(ambiguous.mean()),
        "finite": bool(np.isfinite(g).all() and np.isfinite(ga).all()),
    }


def oracle_image_and_mask(scene, cam, k=O.K_FILTER, order="tstar", eval2d=False):
    prep = O.prepare(scene, cam, k)
    rgb, alpha = O.render(scene, cam, k, prep=prep, order=order, eval2d=eval2d)
    py, px = np.mgrid[0:cam.height, 0:cam.width]
    mask = []
    step = 2048
    fx, fy = px.ravel(), py.ravel()
    for i in range(0, fx.size, step):
        mask.append(O.ambiguous_pixels(prep, fx[i:i + step], fy[i:i + step], eval2d=eval2d).numpy())
    return prep, rgb, alpha, np.concatenate(mask).reshape(cam.height, cam.width)
