"""GPU parity of aaag_vhat_train (Sec. 3.2, Eq. 5) against the oracle."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2504_12811_gb300 import aaag, scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_12811_gb300 import build
    build.build()


def _gpu(means, cams):
    m = torch.from_numpy(np.ascontiguousarray(means, np.float32)).cuda()
    out = torch.full((means.shape[0],), float("nan"), device="cuda")
    aaag.aaag_vhat_train(m.data_ptr(), means.shape[0], [aaag.make_camera(c) for c in cams], out.data_ptr(),
                         aaag.current_stream())
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _borderline(means, cams, eps_px=1e-3, eps_z=1e-5):
    """Gaussians whose visibility in some camera is within float32 reach of
    the image border or the near plane."""
    m = np.asarray(means, np.float64)
    amb = np.zeros(m.shape[0], bool)
    for c in cams:
        V = np.asarray(c.viewmat, np.float64)
        p = m @ V[:3, :3].T + V[:3, 3]
        z = p[:, 2]
        zs = np.where(np.abs(z) > 1e-9, z, 1e-9)
        u = c.fx * p[:, 0] / zs + c.cx
        v = c.fy * p[:, 1] / zs + c.cy
        near = np.abs(z - c.znear) < eps_z * max(1.0, c.znear)
        edge = (z > c.znear) & ((np.abs(u) < eps_px) | (np.abs(u - c.width) < eps_px) |
                                (np.abs(v) < eps_px) | (np.abs(v - c.height) < eps_px))
        amb |= near | edge
    return amb


@pytest.mark.parametrize("n_cams", [1, 7, 64, 65, 150])
def test_vhat_train_matches_oracle(n_cams):
    rng = np.random.default_rng(n_cams)
    means = rng.uniform(-2, 2, (20000, 3)).astype(np.float32)
    cams = scenes.orbit_cameras(rng, n_cams, 4.0, 320, 240, 60.0)
    got = _gpu(means, cams)
    ref = O.training_sampling_frequency(means, cams)
    ok = ~_borderline(means, cams)
    assert ok.mean() > 1.0 - 2e-4 * len(cams)
    assert np.array_equal(np.isinf(got[ok]), np.isinf(ref[ok]))
    fin = ok & np.isfinite(ref)
    assert fin.sum() > 1000
    np.testing.assert_allclose(got[fin], ref[fin], rtol=2e-6)
    assert np.all(got > 0)


def test_vhat_train_edge_cases():
    means = np.array([[0.0, 0.0, 4.0], [0.0, 0.0, -4.0]], np.float32)
    # no camera: every Gaussian unclamped
    assert np.all(np.isinf(_gpu(means, [])))
    # empty scene
    _gpu(np.zeros((0, 3), np.float32), scenes.orbit_cameras(np.random.default_rng(0), 3, 4.0, 64, 48, 60.0))
    # invalid camera is rejected on the host
    bad = scenes.Camera(np.eye(4, dtype=np.float32), float("nan"), 1.0, 1.0, 1.0, 8, 8)
    with pytest.raises(aaag.AaagError):
        _gpu(means, [bad])
