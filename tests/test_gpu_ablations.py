"""GPU parity of the ablation switches (Sec. 5 'Ablation'): no 3D filter, no
3D tile culling, no per-pixel re-sort, 2D splatting instead of 3D evaluation,
and the bounded-buffer approximate re-sort, each against the oracle's
definition of that variant or against the full method."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2504_12811_gb300 import aaag, scenes
from _gpu_util import (TOL_ABS, TOL_AMBIG, TOL_PSNR, compare_image, oracle_image_and_mask, psnr,
                       run_frame, stats)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_12811_gb300 import build
    build.build()


def _check(rgb, alpha, ref, st, tol_ambig=TOL_AMBIG):
    prep, ref_rgb, ref_alpha, amb = ref
    r = compare_image(rgb, alpha, ref_rgb, ref_alpha, amb)
    print(r, st)
    assert st["status"] == "OK", st
    assert r["finite"]
    assert r["ambiguous_fraction"] < tol_ambig
    assert r["max_abs_clean"] <= TOL_ABS
    assert r["psnr_rgb"] >= TOL_PSNR and r["psnr_alpha"] >= TOL_PSNR


@pytest.mark.parametrize("wl", ["small", "zoomout"])
def test_no_filter_matches_oracle_without_filter(wl):
    # AA off: s_hat = s^2 and amplitude factor 1, i.e. the oracle with k = 0
    scene, cams = scenes.workload(wl)
    cam = cams[0]
    ws, rgb, alpha, _ = run_frame(scene, cam, params=aaag.make_params(flags=aaag.AAAG_FLAG_NO_FILTER))
    _check(rgb, alpha, oracle_image_and_mask(scene, cam, k=0.0), stats(ws))
    # and it differs from the filtered image where the filter acts
    _, rgb_f, _, _ = run_frame(scene, cam)
    if wl == "zoomout":
        assert float((rgb - rgb_f).abs().max()) > 1e-2


@pytest.mark.parametrize("wl", ["small", "near"])
def test_no_resort_matches_mean_depth_order(wl):
    scene, cams = scenes.workload(wl)
    cam = cams[0]
    ws, rgb, alpha, _ = run_frame(scene, cam, params=aaag.make_params(flags=aaag.AAAG_FLAG_NO_RESORT))
    st = stats(ws)
    _check(rgb, alpha, oracle_image_and_mask(scene, cam, order="mean"), st)
    assert st["misorders"] == 0


@pytest.mark.parametrize("wl", ["small", "near"])
def test_no_cull_gives_the_same_image(wl):
    # culling only removes pairs that cannot contribute: same blends, same order
    scene, cams = scenes.workload(wl)
    cam = cams[0]
    ws0, rgb0, alpha0, _ = run_frame(scene, cam)
    ws1, rgb1, alpha1, _ = run_frame(scene, cam, params=aaag.make_params(flags=aaag.AAAG_FLAG_NO_CULL))
    s0, s1 = stats(ws0), stats(ws1)
    assert s1["status"] == "OK"
    assert s1["n_pairs"] > s0["n_pairs"]
    assert s1["blended"] == s0["blended"]
    assert float((rgb0 - rgb1).abs().max()) <= 1e-6
    assert float((alpha0 - alpha1).abs().max()) <= 1e-6


def test_kbuffer_is_exact_while_the_buffer_never_fills():
    # a sparse scene: fewer than 16 contributors per pixel, so the bounded
    # buffer holds every contributor and blends them in exact order at the end
    rng = np.random.default_rng(5)
    n = 200
    scene = scenes.Scene(rng.uniform(-1, 1, (n, 3)).astype(np.float32),
                         rng.normal(-3.0, 0.3, (n, 3)).astype(np.float32),
                         rng.standard_normal((n, 4)).astype(np.float32),
                         rng.normal(0.5, 1.0, n).astype(np.float32),
                         rng.normal(0, 0.3, (n, 1, 3)).astype(np.float32),
                         np.full(n, np.inf, np.float32), 0)
    cam = scenes.make_camera((0.0, 0.0, -3.0), target=(0.0, 0.0, 0.0), width=96, height=80)
    ws0, rgb0, alpha0, _ = run_frame(scene, cam)
    ws1, rgb1, alpha1, _ = run_frame(scene, cam, params=aaag.make_params(flags=aaag.AAAG_FLAG_KBUFFER))
    s0, s1 = stats(ws0), stats(ws1)
    assert s1["status"] == "OK" and s1["misorders"] == 0 and s0["misorders"] == 0
    assert s1["blended"] == s0["blended"]
    assert torch.equal(rgb0, rgb1) and torch.equal(alpha0, alpha1)


def _kbuffer_reference(scene, cam, px, py, rel_t=2e-6, rel_arrival=1e-6, budget=1e-3):
    """The oracle's bounded-buffer image at the given pixels and a mask of the
    pixels whose buffer decisions float32 may take differently: those of the
    exact-order mask (alpha, near-plane and per-Gaussian thresholds), and
    pairs of blended contributors whose t* or arrival keys (mean depths) tie
    within float32 reach.  Swapping two such contributors can at most swap two
    consecutive blends of the buffer's sequence, which moves the pixel by at
    most T a_i a_j |c_i - c_j| (T: transmittance before the earlier of them);
    a pixel is flagged when these bounds add up beyond `budget`."""
    prep = O.prepare(scene, cam)
    rgb, alpha, amb = [], [], []
    z = torch.clamp(prep["mu_view"][:, 2], min=prep["view"].znear).numpy()
    col = prep["rgb"].numpy()
    for i in range(0, px.size, 256):
        qx, qy = px[i:i + 256], py[i:i + 256]
        rho2, ts = O.ray_maximum(prep, qx, qy)
        a, contrib, _ = O.pixel_alphas(prep, rho2, ts)
        out, T, _, seqs = O.composite_kbuffer(a, ts, z, contrib, prep["rgb"], prep["view"].bg, sequences=True)
        rgb.append(out.numpy())
        alpha.append(1.0 - T.numpy())
        flag = O.ambiguous_pixels(prep, qx, qy, rel_t=0.0).numpy()
        an, tn = a.numpy(), ts.numpy()
        for p, seq in enumerate(seqs):
            if seq.size < 2:
                continue
            ap = an[p, seq]
            Tb = np.concatenate([[1.0], np.cumprod(1.0 - ap)[:-1]])
            eff = 0.0
            for key, rel in ((tn[p, seq], rel_t), (z[seq], rel_arrival)):
                o = np.argsort(key, kind="stable")
                k = key[o]
                close = np.nonzero(np.diff(k) <= rel * np.abs(k[:-1]))[0]
                for c in close:
                    i_, j_ = o[c], o[c + 1]
                    eff += Tb[min(i_, j_)] * ap[i_] * ap[j_] * np.abs(col[seq[i_]] - col[seq[j_]]).max()
            flag[p] |= eff > budget
        amb.append(flag)
    return np.concatenate(rgb), np.concatenate(alpha), np.concatenate(amb)


def _dense_cube(n=30_000):
    full, _ = scenes.workload("train500k")
    return full.subset(np.arange(n))


@pytest.mark.parametrize("wl,ci", [("small", 1), ("near", 0), ("dense", 0)])
def test_kbuffer_matches_oracle_bounded_buffer(wl, ci):
    """The bounded-buffer ablation against the oracle's restatement of it
    (`composite_kbuffer`: arrivals in mean-depth order, 16 entries, the
    nearest blended when full).  "dense": 30k Gaussians of the 500k cube at
    128x128, where about 150 contributors meet each pixel and the buffer
    overflows on most arrivals, so the image departs from the exact order;
    the sparse workloads barely fill it."""
    if wl == "dense":
        scene = _dense_cube()
        cam = scenes.make_camera((0.0, 0.0, -3.0), target=(0, 0, 0), width=128, height=128)
    else:
        scene, cams = scenes.workload(wl)
        cam = cams[ci]
    ws, rgb, alpha, _ = run_frame(scene, cam, capacity=1 << 22,
                                  params=aaag.make_params(flags=aaag.AAAG_FLAG_KBUFFER))
    st = stats(ws)
    assert st["status"] == "OK" and st["extra_passes"] == 0
    py, px = np.mgrid[0:cam.height, 0:cam.width]
    px, py = px.ravel(), py.ravel()
    if wl == "dense":
        sel = np.random.default_rng(6).choice(px.size, 4096, replace=False)
        px, py = px[sel], py[sel]
    ref, ref_a, amb = _kbuffer_reference(scene, cam, px, py)
    g = rgb.cpu().numpy()[:, py, px].T.astype(np.float64)
    ga = alpha.cpu().numpy()[py, px].astype(np.float64)
    err = np.maximum(np.abs(g - ref).max(1), np.abs(ga - ref_a))
    print(wl, st, f"max|err| clean={err[~amb].max():.3e} ambiguous={amb.mean():.4f} psnr={psnr(g, ref):.1f}")
    assert amb.mean() < TOL_AMBIG
    assert err[~amb].max() <= TOL_ABS
    assert psnr(g, ref) >= TOL_PSNR
    if wl == "dense":
        assert st["misorders"] > 100_000
        exact, _ = O.render_pixels(scene, cam, px[:512], py[:512])
        assert np.abs(exact.numpy() - ref[:512]).max() > 5e-3      # the buffer's order is not the exact one


@pytest.mark.parametrize("wl,ci", [("small", 0), ("small", 1), ("zoomout", 0)])
def test_eval_2d_matches_oracle_splats(wl, ci):
    scene, cams = scenes.workload(wl)
    cam = cams[ci]
    ws, rgb, alpha, ds = run_frame(scene, cam, params=aaag.make_params(flags=aaag.AAAG_FLAG_EVAL_2D))
    # every pixel of a splat has the same depth, so a near-tie of two means'
    # depths flags their whole overlap rather than a curve: a larger masked
    # fraction is expected than for the 3D evaluation
    _check(rgb, alpha, oracle_image_and_mask(scene, cam, eval2d=True), stats(ws), tol_ambig=1e-2)
    # it is a different image from the 3D evaluation
    _, rgb3, _, _ = run_frame(scene, cam)
    assert float((rgb - rgb3).abs().max()) > 1e-3
    # forward only
    grads = [torch.empty_like(t) for t in (ds.means, ds.log_scales, ds.quats, ds.opacity_logits, ds.sh)]
    gs = aaag.aaag_grads(*[t.data_ptr() for t in grads])
    d = torch.zeros_like(rgb)
    with pytest.raises(aaag.AaagError) as e:
        aaag.aaag_render_backward(ds.struct(), ws.handle, rgb.data_ptr(), d.data_ptr(), None, gs,
                                  aaag.current_stream())
    assert e.value.status == aaag.AAAG_ERR_UNSUPPORTED
