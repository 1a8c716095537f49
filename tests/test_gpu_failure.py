"""Failure detection on the GPU without a fault: a bounded device-side wait
whose predecessor never publishes gives up after about a second, raises the
workspace's timeout flag (reported as TIMEOUT by aaag_get_stats) and returns;
the context stays usable and the next frame renders normally."""
import time

import numpy as np
import pytest
import torch

from paper_2504_12811_gb300 import aaag, scenes
from _gpu_util import run_frame, stats

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_12811_gb300 import build
    build.build()


@pytest.mark.parametrize("which", [0, 1], ids=["cull_lookback", "sort_lookback"])
def test_bounded_wait_times_out_and_reports(which):
    scene, cams = scenes.workload("small")
    ws, rgb0, _, ds = run_frame(scene, cams[0])
    assert stats(ws)["status"] == "OK"
    rgb0 = rgb0.cpu().numpy()
    st = aaag.current_stream()
    torch.cuda.synchronize()
    t0 = time.time()
    aaag.aaag_selftest_wait_timeout(ws.handle, which, st)
    torch.cuda.synchronize()
    waited = time.time() - t0
    assert 0.3 < waited < 20.0, waited
    s = aaag.stats(ws, check=False)
    assert s["status"] == "TIMEOUT" and s["timeout"] == 1
    # the context is intact: the same workspace renders the same frame again
    cam = cams[0]
    rgb1 = torch.empty(3, cam.height, cam.width, device="cuda")
    alpha1 = torch.empty(cam.height, cam.width, device="cuda")
    aaag.aaag_preprocess(ds.struct(), aaag.make_camera(cam), aaag.make_params(), ws.handle, st)
    aaag.aaag_cull(ws.handle, st)
    aaag.aaag_sort(ws.handle, st)
    aaag.aaag_render(ws.handle, rgb1.data_ptr(), alpha1.data_ptr(), st)
    torch.cuda.synchronize()
    assert stats(ws)["status"] == "OK"
    np.testing.assert_array_equal(rgb0, rgb1.cpu().numpy())


def test_selftest_rejects_bad_arguments():
    scene, cams = scenes.workload("small")
    ws, _, _, _ = run_frame(scene, cams[0], stages=("pre",))
    with pytest.raises(aaag.AaagError) as e:
        aaag.aaag_selftest_wait_timeout(ws.handle, 3, aaag.current_stream())
    assert e.value.status == aaag.AAAG_ERR_INVALID_ARG
