"""Parity at the full benchmark size: 1M Gaussians, 1920x1080, in the launch
configuration bench.py times (same workspace capacity), on pixels sampled at
random and computed one by one by the oracle."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2504_12811_gb300 import aaag, scenes
from _gpu_util import TOL_ABS, TOL_AMBIG, TOL_PSNR, psnr

pytestmark = pytest.mark.gpu

BENCH_CAPACITY = 48 << 20


@pytest.fixture(scope="module")
def scene1m():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_12811_gb300 import build
    build.build()
    return scenes.workload("scene1m")


@pytest.mark.parametrize("pose", [0, 5, 9, 13])
def test_scene1m_sampled_pixels(scene1m, pose):
    scene, poses = scene1m
    cam = poses[pose]
    ds = aaag.DeviceScene(scene)
    ws = aaag.Workspace(scene.n, cam.width, cam.height, BENCH_CAPACITY)
    rgb, alpha = aaag.render(ds, cam, ws)
    st = aaag.stats(ws)
    torch.cuda.synchronize()
    rng = np.random.default_rng(11 + pose)
    m = 512
    px = rng.integers(0, cam.width, m)
    py = rng.integers(0, cam.height, m)
    prep = O.prepare(scene, cam)
    ref, ref_a = O.render_pixels(scene, cam, px, py, prep=prep)
    amb = np.concatenate([O.ambiguous_pixels(prep, px[i:i + 128], py[i:i + 128]).numpy()
                          for i in range(0, m, 128)])
    g = rgb.cpu().numpy()[:, py, px].T.astype(np.float64)
    ga = alpha.cpu().numpy()[py, px].astype(np.float64)
    err = np.maximum(np.abs(g - ref.numpy()).max(1), np.abs(ga - ref_a.numpy()))
    print(f"pose {pose}: stats={st} max|err| clean={err[~amb].max():.3e} all={err.max():.3e} "
          f"ambiguous={amb.mean():.4f} psnr={psnr(g, ref.numpy()):.1f}")
    assert st["misorders"] == 0
    if err.max() > TOL_ABS:
        # only a rare pixel whose decisions sit within float32 reach of a
        # threshold may be excused
        assert amb.mean() < TOL_AMBIG
        assert err[~amb].max() <= TOL_ABS
    assert psnr(g, ref.numpy()) >= TOL_PSNR


def test_scene1m_graph_launch_matches_per_stage_calls(scene1m):
    # bench.py times each frame as one launch of the captured frame graph;
    # the graph replays the same kernels, so the images are bit-identical
    scene, poses = scene1m
    ds = aaag.DeviceScene(scene)
    cam0 = poses[0]
    ws = aaag.Workspace(scene.n, cam0.width, cam0.height, BENCH_CAPACITY)
    st = torch.cuda.Stream()
    rgb_g = torch.empty(3, cam0.height, cam0.width, device="cuda")
    alpha_g = torch.empty(cam0.height, cam0.width, device="cuda")
    stages = (aaag.AAAG_STAGE_PREPROCESS | aaag.AAAG_STAGE_CULL | aaag.AAAG_STAGE_SORT |
              aaag.AAAG_STAGE_RENDER)
    graph = aaag.aaag_graph_create(ds.struct(), aaag.make_camera(cam0), aaag.make_params(), ws.handle, stages,
                                   rgb_g.data_ptr(), alpha_g.data_ptr(), st.cuda_stream)
    try:
        for pose in (3, 7, 3):
            cam = poses[pose]
            aaag.aaag_graph_launch(graph, aaag.make_camera(cam), st.cuda_stream)
            st.synchronize()
            sg = aaag.stats(ws)
            ws2 = aaag.Workspace(scene.n, cam.width, cam.height, BENCH_CAPACITY)
            rgb_d, alpha_d = aaag.render(ds, cam, ws2)
            torch.cuda.synchronize()
            sd = aaag.stats(ws2)
            assert sg["status"] == "OK" and sg["n_pairs"] == sd["n_pairs"] and sg["blended"] == sd["blended"]
            assert torch.equal(rgb_g, rgb_d) and torch.equal(alpha_g, alpha_d)
    finally:
        aaag.aaag_graph_destroy(graph)
