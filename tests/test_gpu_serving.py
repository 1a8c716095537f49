"""Serving form: batched persistent render, frame graphs, memory admission,
and the same result for a request alone and in a mix."""
import numpy as np
import pytest
import torch

from paper_2504_12811_gb300 import aaag, scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_12811_gb300 import build
    build.build()


def single_frame(scene_struct, cam, ws, n_max=None):
    rgb = torch.empty(3, cam.height, cam.width, device="cuda")
    alpha = torch.empty(cam.height, cam.width, device="cuda")
    aaag.aaag_render_frame(scene_struct, aaag.make_camera(cam), aaag.make_params(), ws.handle, rgb.data_ptr(),
                           alpha.data_ptr(), aaag.current_stream())
    torch.cuda.synchronize()
    return rgb.cpu(), alpha.cpu()


def test_batch_render_equals_single_frames():
    sc, cams = scenes.workload("small")
    zs, zc = scenes.workload("zoomout")
    ns, nc = scenes.workload("near")
    frames = [(sc, cams[0]), (sc, cams[1]), (zs, zc[0]), (ns, nc[0])]
    ds = [aaag.DeviceScene(f[0]) for f in frames]
    # one workspace per frame, sized for the largest
    W = max(f[1].width for f in frames)
    H = max(f[1].height for f in frames)
    wss = [aaag.Workspace(f[0].n, W, H, 1 << 18) for f in frames]
    singles = [single_frame(d.struct(), f[1], w) for d, f, w in zip(ds, frames, wss)]
    st = aaag.current_stream()
    outs = []
    for d, f, w in zip(ds, frames, wss):
        aaag.aaag_preprocess(d.struct(), aaag.make_camera(f[1]), aaag.make_params(), w.handle, st)
        aaag.aaag_cull(w.handle, st)
        aaag.aaag_sort(w.handle, st)
        outs.append((torch.empty(3, f[1].height, f[1].width, device="cuda"),
                     torch.empty(f[1].height, f[1].width, device="cuda")))
    aaag.aaag_render_batch([w.handle for w in wss], [o[0].data_ptr() for o in outs],
                           [o[1].data_ptr() for o in outs], st)
    torch.cuda.synchronize()
    for (r1, a1), (r2, a2) in zip(singles, outs):
        assert torch.equal(r1, r2.cpu()) and torch.equal(a1, a2.cpu())


def test_graph_relaunch_with_new_camera():
    sc, cams = scenes.workload("small")
    ds = aaag.DeviceScene(sc)
    ws = aaag.Workspace(sc.n, 128, 128, 1 << 18)
    ws_ref = aaag.Workspace(sc.n, 128, 128, 1 << 18)
    rgb = torch.empty(3, 128, 128, device="cuda")
    alpha = torch.empty(128, 128, device="cuda")
    stream = torch.cuda.Stream()
    g = aaag.aaag_graph_create(ds.struct(), aaag.make_camera(cams[0]), aaag.make_params(), ws.handle, 15,
                               rgb.data_ptr(), alpha.data_ptr(), stream.cuda_stream)
    try:
        for cam in (cams[1], cams[0], cams[1]):
            aaag.aaag_graph_launch(g, aaag.make_camera(cam), stream.cuda_stream)
            stream.synchronize()
            ref = single_frame(ds.struct(), cam, ws_ref)
            assert torch.equal(rgb.cpu(), ref[0]) and torch.equal(alpha.cpu(), ref[1])
    finally:
        aaag.aaag_graph_destroy(g)


def small_serving_setup(budget_slots=None):
    from paper_2504_12811_gb300 import serve
    sc = {"a": scenes.uniform_cube_scene(20_000, seed=31, sh_degree=3),
          "b": scenes.uniform_cube_scene(60_000, seed=32, sh_degree=3)}
    rng = np.random.default_rng(3)
    reqs = []
    t = 0.0
    for i in range(40):
        t += rng.exponential(1 / 300.0)
        kind = ["vga", "stereo_small"][i % 2]
        pos = rng.uniform(-0.6, 0.6, 3)
        d = rng.standard_normal(3)
        if kind == "vga":
            cams = [scenes.make_camera(pos, forward=d, width=320, height=240)]
        else:
            cams = [scenes.make_camera(pos + o, forward=d, width=256, height=272, fov_x_deg=110.0)
                    for o in (np.array([-0.03, 0, 0]), np.array([0.03, 0, 0]))]
        reqs.append(scenes.Request(i, t, "ab"[i % 3 % 2], kind, cams))
    ws_bytes = aaag.aaag_workspace_bytes(60_000, 320, 272, 1 << 21) + 16 * 320 * 272
    budget = ws_bytes * (budget_slots or 6) + 1
    server = serve.Server(sc, budget, 320, 272, 1 << 21, max_batch_views=4)
    return serve, server, sc, reqs


def test_serving_results_same_alone_and_in_mix():
    serve, server, sc, reqs = small_serving_setup()
    try:
        server.warm(reqs)
        captured, captured_s, captured_p = {}, {}, {}
        lat = server.serve(reqs, capture=captured)
        assert len(lat) == len(reqs) and all(x > 0 for x in lat)
        lat = server.serve_streams(reqs, capture=captured_s)
        assert len(lat) == len(reqs) and all(x > 0 for x in lat)
        # stereo requests one at a time, the others on high-priority streams
        lat = server.serve_streams(reqs, capture=captured_p, urgent_pixels=320 * 240, heavy_pixels=320 * 240)
        assert len(lat) == len(reqs) and all(x > 0 for x in lat)
        ds = {k: aaag.DeviceScene(v) for k, v in sc.items()}
        ws = aaag.Workspace(60_000, 320, 272, 1 << 21)
        worst = 0.0
        for r in reqs:
            for cap in (captured, captured_s, captured_p):
                for (rgb_mix, a_mix), cam in zip(cap[r.rid], r.cams):
                    rgb_alone, a_alone = single_frame(ds[r.scene].struct(), cam, ws)
                    worst = max(worst, float((rgb_mix - rgb_alone).abs().max()),
                                float((a_mix - a_alone).abs().max()))
        # the same kernels on the same inputs: identical in practice, and
        # within the image tolerance in any case
        assert worst <= 2e-3
        print("max |alone - in mix| =", worst)
    finally:
        server.close()


def test_admission_respects_memory_budget():
    serve, server, sc, reqs = small_serving_setup(budget_slots=2)
    try:
        assert len(server.slots) == 2
        server.warm(reqs)
        policy = lambda r: server.serve_streams(r, urgent_pixels=320 * 240, heavy_pixels=320 * 240)
        for run in (server.serve, server.serve_streams, policy):
            lat = run(reqs)
            assert len(lat) == len(reqs)
            assert server.max_views_in_flight <= len(server.slots)
    finally:
        server.close()
