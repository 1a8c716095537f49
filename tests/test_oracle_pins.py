"""Pins of the FP64 oracle to things other than itself (CPU only).

Each test checks an oracle function against a closed form, a library routine
(scipy rotations / spherical harmonics / optimisation), brute-force sampling,
or an invariant of the paper, chosen so that a dropped term, a wrong sign or
index, or a transposed operand in the oracle fails at least one of them.
"""
import math

import numpy as np
import pytest
import torch
from scipy.optimize import minimize_scalar
from scipy.spatial.transform import Rotation
from scipy.special import sph_harm_y

import oracle as O
from paper_2504_12811_gb300 import scenes


# ---------------------------------------------------------------------------
# helpers written independently of the oracle
# ---------------------------------------------------------------------------

def scipy_rot(q):
    """Rotation matrices of (w,x,y,z) quaternions via scipy (scalar-last)."""
    q = np.asarray(q, dtype=np.float64)
    return Rotation.from_quat(q[:, [1, 2, 3, 0]]).as_matrix()


def one_gaussian_scene(mu, log_s, q=(1.0, 0.0, 0.0, 0.0), logit=2.0, sh_dc=(0.5, 0.2, -0.3),
                       vtrain=np.inf):
    n = len(mu)
    sh = np.zeros((n, 1, 3), np.float32)
    sh[:, 0, :] = sh_dc
    return scenes.Scene(np.asarray(mu, np.float32).reshape(n, 3),
                        np.asarray(log_s, np.float32).reshape(n, 3),
                        np.tile(np.asarray(q, np.float32), (n, 1)) if np.ndim(q) == 1 else np.asarray(q, np.float32),
                        np.full(n, logit, np.float32) if np.ndim(logit) == 0 else np.asarray(logit, np.float32),
                        sh, np.full(n, vtrain, np.float32), 0)


def random_scene(n, seed, spread=1.0, logs=(-2.5, 0.6), deg=0):
    rng = np.random.default_rng(seed)
    mu = rng.uniform(-spread, spread, (n, 3)).astype(np.float32)
    ls = rng.normal(logs[0], logs[1], (n, 3)).astype(np.float32)
    q = rng.standard_normal((n, 4)).astype(np.float32)
    lg = rng.normal(1.0, 1.0, n).astype(np.float32)
    sh = rng.normal(0, 0.3, (n, (deg + 1) ** 2, 3)).astype(np.float32)
    vt = rng.uniform(20, 200, n).astype(np.float32)
    return scenes.Scene(mu, ls, q, lg, sh, vt, deg)


def cam_at(pos, target=(0, 0, 0), W=64, H=48, fov=60.0, **kw):
    return scenes.make_camera(pos, target=target, width=W, height=H, fov_x_deg=fov, **kw)


# ---------------------------------------------------------------------------
# Sec. 3.1 Eq. 3: rotation
# ---------------------------------------------------------------------------

def test_rotation_matches_scipy():
    rng = np.random.default_rng(1)
    q = rng.standard_normal((64, 4)) * rng.uniform(0.1, 5, (64, 1))
    R = O.rotation_from_quaternion(torch.tensor(q)).numpy()
    np.testing.assert_allclose(R, scipy_rot(q), atol=1e-12)


# ---------------------------------------------------------------------------
# colour: real SH
# ---------------------------------------------------------------------------

def scipy_real_sh(dirs, degree):
    x, y, z = dirs.T
    theta = np.arccos(np.clip(z, -1, 1))
    phi = np.arctan2(y, x)
    cols = []
    for l in range(degree + 1):
        for m in range(-l, l + 1):
            Y = sph_harm_y(l, abs(m), theta, phi)
            if m == 0:
                cols.append(Y.real)
            elif m > 0:
                cols.append(math.sqrt(2) * Y.real)
            else:
                cols.append(math.sqrt(2) * Y.imag)
    return np.stack(cols, -1)


def test_sh_basis_matches_scipy():
    rng = np.random.default_rng(2)
    d = rng.standard_normal((200, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    ours = O.sh_basis(torch.tensor(d), 3).numpy()
    np.testing.assert_allclose(ours, scipy_real_sh(d, 3), atol=1e-12)


def test_sh_bands_0_1_closed_form_and_orthonormality():
    rng = np.random.default_rng(3)
    d = rng.standard_normal((50, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    Y = O.sh_basis(torch.tensor(d), 1).numpy()
    c0 = 0.5 / math.sqrt(math.pi)
    c1 = math.sqrt(3.0 / (4 * math.pi))
    np.testing.assert_allclose(Y[:, 0], c0, atol=1e-14)
    np.testing.assert_allclose(Y[:, 1:], c1 * np.stack([-d[:, 1], d[:, 2], -d[:, 0]], 1), atol=1e-14)
    # orthonormality by quadrature on a Fibonacci sphere
    n = 40000
    i = np.arange(n) + 0.5
    zz = 1 - 2 * i / n
    ph = math.pi * (1 + 5 ** 0.5) * i
    r = np.sqrt(1 - zz * zz)
    pts = np.stack([r * np.cos(ph), r * np.sin(ph), zz], 1)
    B = O.sh_basis(torch.tensor(pts), 3).numpy()
    gram = 4 * math.pi * B.T @ B / n
    np.testing.assert_allclose(gram, np.eye(16), atol=2e-3)


def test_sh_colour_offset_and_clamp():
    d = torch.tensor([[0.0, 0.0, 1.0]])
    sh = torch.zeros(1, 1, 3, dtype=torch.float64)
    sh[0, 0] = torch.tensor([1.0, 0.0, -5.0])
    c = O.sh_colour(sh, d, 0)[0].numpy()
    c0 = 0.5 / math.sqrt(math.pi)
    np.testing.assert_allclose(c, [c0 + 0.5, 0.5, 0.0], atol=1e-14)


# ---------------------------------------------------------------------------
# Sec. 3.2: adaptive filter
# ---------------------------------------------------------------------------

def test_isotropic_filter_factor_closed_form():
    # s_i = s for all i: Eq. 12 reduces to s^2 / s_hat for every direction
    rng = np.random.default_rng(4)
    s = torch.full((100, 3), 0.02, dtype=torch.float64)
    R = torch.tensor(scipy_rot(rng.standard_normal((100, 4))))
    d = torch.tensor(rng.standard_normal((100, 3)))
    d = d / d.norm(dim=1, keepdim=True)
    v = torch.tensor(rng.uniform(10, 300, 100))
    sh = O.filtered_variances(s, v, 0.3)
    phi = O.perpendicular_factor(s, sh, R, d)
    expect = 0.02 ** 2 / (0.02 ** 2 + 0.3 / v.numpy() ** 2)
    np.testing.assert_allclose(phi.numpy(), expect, rtol=1e-12)


def test_perpendicular_factor_matches_explicit_basis():
    # Appendix A: |Sigma_perp| from an explicit orthonormal basis U = [d u2 u3]
    rng = np.random.default_rng(5)
    for _ in range(50):
        s = np.exp(rng.normal(-3, 1, 3))
        R = scipy_rot(rng.standard_normal((1, 4)))[0]
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        kv = rng.uniform(1e-5, 1e-2)                       # k / v'^2
        Sig = R @ np.diag(s ** 2) @ R.T
        Sig_hat = Sig + kv * np.eye(3)
        U, _ = np.linalg.qr(np.stack([d, rng.standard_normal(3), rng.standard_normal(3)], 1))
        Pp = lambda M: (U.T @ M @ U)[1:, 1:]
        expect = math.sqrt(np.linalg.det(Pp(Sig)) / np.linalg.det(Pp(Sig_hat)))
        s_t = torch.tensor(s)[None]
        sh = s_t ** 2 + kv
        got = O.perpendicular_factor(s_t, sh, torch.tensor(R)[None], torch.tensor(d)[None]).item()
        assert got == pytest.approx(expect, rel=1e-9)


def test_filter_bounds_and_limits():
    rng = np.random.default_rng(6)
    n = 500
    s = torch.tensor(np.exp(rng.normal(-3, 1.5, (n, 3))))
    R = torch.tensor(scipy_rot(rng.standard_normal((n, 4))))
    d = torch.tensor(rng.standard_normal((n, 3)))
    d = d / d.norm(dim=1, keepdim=True)
    v = torch.tensor(rng.uniform(5, 500, n))
    sh = O.filtered_variances(s, v, 0.3)
    phi = O.perpendicular_factor(s, sh, R, d)
    mip = O.mip_factor(s, sh)
    assert torch.all(phi <= 1 + 1e-15)
    assert torch.all(phi >= mip * (1 - 1e-12))   # Eq. 12 never below the volume factor
    sh0 = O.filtered_variances(s, v, 1e-12)
    assert torch.allclose(O.perpendicular_factor(s, sh0, R, d), torch.ones(n, dtype=torch.float64), atol=1e-6)


def test_smoothed_covariance_is_sum():
    # Sigma_hat - Sigma = (k / v'^2) I  (Sec. 3.1)
    sc = random_scene(40, 7)
    cam = cam_at((0.3, -0.2, -4.0))
    p = O.prepare(sc, cam)
    Sig_hat = torch.linalg.inv(p["Sigma_hat_inv"]).numpy()
    R = scipy_rot(sc.quats)
    s = np.exp(sc.log_scales.astype(np.float64))
    Sig = np.einsum("gij,gj,gkj->gik", R, s ** 2, R)
    kv = 0.3 / p["v_eff"].numpy() ** 2
    np.testing.assert_allclose(Sig_hat - Sig, kv[:, None, None] * np.eye(3), atol=1e-12)


def test_training_sampling_frequency_closed_forms():
    # Eq. 5: max over cameras of f / d among the cameras that see the mean
    eye = np.eye(4, dtype=np.float32)
    cam1 = scenes.Camera(eye, 100.0, 100.0, 32.0, 24.0, 64, 48)            # at the origin, looking +z
    back = eye.copy()
    back[2, 3] = 2.0                                                          # 2 units further back
    cam2 = scenes.Camera(back, 150.0, 150.0, 32.0, 24.0, 64, 48)
    m = np.array([[0.0, 0.0, 4.0],        # seen by both: max(100/4, 150/6)
                  [0.0, 0.0, -1.0],       # behind cam1, in front of cam2 at depth 1
                  [5.0, 0.0, 4.0],        # outside both images
                  [0.0, 0.0, 0.1],        # before cam1's near plane; cam2 at depth 2.1
                  [1.28, 0.0, 4.0]],      # u = 32 + 100 * 0.32 = 64 = W for cam1: on the border
                 np.float32)
    v = O.training_sampling_frequency(m, [cam1, cam2])
    assert v[0] == pytest.approx(max(100 / 4, 150 / 6), rel=1e-12)
    assert v[1] == pytest.approx(150 / 1.0, rel=1e-12)
    assert np.isinf(v[2]) and v[2] > 0
    assert v[3] == pytest.approx(150 / 2.1, rel=1e-6)
    u2 = 32 + 150 * float(np.float32(1.28)) / 6.0                             # cam2 sees it too
    assert u2 < 64 and v[4] == pytest.approx(max(100 / 4, 150 / 6), rel=1e-12)
    assert np.all(np.isinf(O.training_sampling_frequency(m, [])))


def test_sampling_frequency_cases():
    sc = random_scene(30, 8)
    cam = cam_at((0.0, 0.0, -5.0))
    V = cam.viewmat.astype(np.float64)
    z = (sc.means.astype(np.float64) @ V[:3, :3].T + V[:3, 3])[:, 2]
    sc.vhat_train[:] = np.inf
    p = O.prepare(sc, cam)
    np.testing.assert_allclose(p["v_eff"].numpy(), cam.fx / z, rtol=1e-13)   # no clamp
    sc.vhat_train[:] = 1.0                                                   # camera closer than training
    p = O.prepare(sc, cam)
    np.testing.assert_allclose(p["v_eff"].numpy(), 1.0)


# ---------------------------------------------------------------------------
# Sec. 3.1: maximum along the ray
# ---------------------------------------------------------------------------

def ray_quadratic_brute(mu, Sig_hat, o, dw):
    """min over t of (o + t dw - mu)^T Sig_hat^-1 (o + t dw - mu), by dense
    sampling then bounded scalar refinement."""
    Si = np.linalg.inv(Sig_hat)
    f = lambda t: (o + t * dw - mu) @ Si @ (o + t * dw - mu)
    ts = np.linspace(-50, 50, 20001)
    vals = np.array([f(t) for t in ts])
    j = int(np.argmin(vals))
    r = minimize_scalar(f, bounds=(ts[max(j - 1, 0)], ts[min(j + 1, len(ts) - 1)]),
                        method="bounded", options={"xatol": 1e-12})
    return r.fun, r.x


def test_ray_maximum_brute_force():
    sc = random_scene(6, 9, logs=(-1.5, 0.5))
    cam = cam_at((0.2, 0.1, -3.0), W=32, H=24)
    p = O.prepare(sc, cam)
    rng = np.random.default_rng(10)
    px = rng.integers(0, 32, 5)
    py = rng.integers(0, 24, 5)
    rho2, ts = O.ray_maximum(p, px, py)
    R = scipy_rot(sc.quats)
    sh = p["s_hat"].numpy()
    V = cam.viewmat.astype(np.float64)
    Ri = np.linalg.inv(V[:3, :3])
    o = -Ri @ V[:3, 3]
    for i in range(5):
        rv = np.array([(px[i] + 0.5 - cam.cx) / cam.fx, (py[i] + 0.5 - cam.cy) / cam.fy, 1.0])
        dw = Ri @ rv
        for g in range(6):
            Sig_hat = R[g] @ np.diag(sh[g]) @ R[g].T
            v, t = ray_quadratic_brute(sc.means[g].astype(np.float64), Sig_hat, o, dw)
            assert rho2[i, g].item() == pytest.approx(v, rel=1e-7, abs=1e-9)
            assert ts[i, g].item() == pytest.approx(t, rel=1e-5, abs=1e-6)


def test_ray_maximum_isotropic_closed_form():
    rng = np.random.default_rng(11)
    n = 20
    mu = rng.uniform(-1, 1, (n, 3))
    sc = one_gaussian_scene(mu, np.full((n, 3), -2.0), q=rng.standard_normal((n, 4)),
                            logit=np.zeros(n))
    cam = cam_at((0.5, -0.3, -4.0), W=40, H=30)
    p = O.prepare(sc, cam)
    px, py = rng.integers(0, 40, 7), rng.integers(0, 30, 7)
    rho2, ts = O.ray_maximum(p, px, py)
    V = cam.viewmat.astype(np.float64)
    Ri = np.linalg.inv(V[:3, :3])
    o = -Ri @ V[:3, 3]
    sh = p["s_hat"].numpy()[:, 0]
    for i in range(7):
        rv = np.array([(px[i] + 0.5 - cam.cx) / cam.fx, (py[i] + 0.5 - cam.cy) / cam.fy, 1.0])
        dw = Ri @ rv
        w = sc.means.astype(np.float64) - o
        dist2 = np.sum(np.cross(w, dw) ** 2, 1) / (dw @ dw)     # point-line distance^2
        np.testing.assert_allclose(rho2[i].numpy(), dist2 / sh, rtol=1e-10)
        np.testing.assert_allclose(ts[i].numpy(), (w @ dw) / (dw @ dw), rtol=1e-10)


def test_plane_form_equals_ray_form():
    """Eq. 4-5: transform pi_x = (1,0,0,-x), pi_y = (0,1,0,-y) by T'^T with an
    explicit viewport and perspective matrix; the distance from the origin to
    the intersection line (minimum-norm solution) is rho."""
    sc = random_scene(8, 12, logs=(-2.0, 0.7))
    W, H = 48, 36
    cam = cam_at((0.4, 0.3, -3.5), W=W, H=H)
    p = O.prepare(sc, cam)
    rng = np.random.default_rng(13)
    px, py = rng.integers(0, W, 6), rng.integers(0, H, 6)
    rho2, _ = O.ray_maximum(p, px, py)
    n_, f_ = 0.1, 100.0
    P = np.array([[2 * cam.fx / W, 0, 2 * cam.cx / W - 1, 0],
                  [0, 2 * cam.fy / H, 2 * cam.cy / H - 1, 0],
                  [0, 0, (f_ + n_) / (f_ - n_), -2 * f_ * n_ / (f_ - n_)],
                  [0, 0, 1, 0]])
    Mvp = np.array([[W / 2, 0, 0, W / 2], [0, H / 2, 0, H / 2], [0, 0, 1, 0], [0, 0, 0, 1.0]])
    V = cam.viewmat.astype(np.float64)
    R = scipy_rot(sc.quats)
    sp = np.sqrt(p["s_hat"].numpy())
    for g in range(8):
        T = np.eye(4)
        T[:3, :3] = R[g] @ np.diag(sp[g])
        T[:3, 3] = sc.means[g]
        Tp = Mvp @ P @ V @ T
        for i in range(6):
            x, y = px[i] + 0.5, py[i] + 0.5
            a = Tp.T @ np.array([1, 0, 0, -x])
            b = Tp.T @ np.array([0, 1, 0, -y])
            A = np.stack([a[:3], b[:3]])
            u = np.linalg.lstsq(A, -np.array([a[3], b[3]]), rcond=None)[0]
            assert u @ u == pytest.approx(rho2[i, g].item(), rel=1e-7)


# ---------------------------------------------------------------------------
# compositing, discard rules, whole-image pins
# ---------------------------------------------------------------------------

def test_single_gaussian_closed_form():
    # one isotropic Gaussian on the optical axis, pixel ray through its mean
    cam = scenes.Camera(np.eye(4, dtype=np.float32), 50.0, 50.0, 8.5, 6.5, 17, 13,
                        bg=(0.2, 0.4, 0.6))
    sc = one_gaussian_scene([[0.0, 0.0, 5.0]], [[-2.0, -2.0, -2.0]], logit=1.5,
                            sh_dc=(0.5, 0.2, -0.3))
    rgb, alpha = O.render_pixels(sc, cam, [8], [6])
    s2 = math.exp(-4.0)
    v = 50.0 / 5.0
    phi = s2 / (s2 + 0.3 / v ** 2)
    o_hat = phi / (1 + math.exp(-1.5))
    a = min(0.99, o_hat)
    c0 = 0.5 / math.sqrt(math.pi)
    f32 = lambda v: np.asarray(v, np.float32).astype(np.float64)
    col = np.maximum(0.0, c0 * f32([0.5, 0.2, -0.3]) + 0.5)
    expect = col * a + (1 - a) * f32([0.2, 0.4, 0.6])
    np.testing.assert_allclose(rgb[0].numpy(), expect, rtol=1e-12)
    assert alpha[0].item() == pytest.approx(a, rel=1e-12)


def test_two_gaussians_depth_order_and_index_independence():
    cam = scenes.Camera(np.eye(4, dtype=np.float32), 50.0, 50.0, 8.5, 6.5, 17, 13)
    mus = [[0.0, 0.0, 4.0], [0.0, 0.0, 6.0]]
    dcs = np.array([[1.0, 0.0, 0.0], [0.0, 1.0, 0.0]], np.float32)
    def run(order):
        sc = one_gaussian_scene(np.array(mus)[order], np.full((2, 3), -1.5), logit=0.5)
        sc.sh[:, 0, :] = dcs[order]
        return O.render_pixels(sc, cam, [8], [6])[0][0].numpy()
    a, b = run([0, 1]), run([1, 0])
    np.testing.assert_allclose(a, b, atol=1e-15)
    p = O.prepare(one_gaussian_scene(mus, np.full((2, 3), -1.5), logit=0.5), cam)
    al = np.minimum(0.99, p["o_hat"].numpy())
    c0 = 0.5 / math.sqrt(math.pi)
    col = np.maximum(0, c0 * dcs.astype(np.float64) + 0.5)
    np.testing.assert_allclose(a, col[0] * al[0] + col[1] * al[1] * (1 - al[0]), rtol=1e-12)


def test_mean_depth_order_ablation_closed_form():
    # Sort ablation of Sec. 5: blending in the order of the means' depths
    # instead of the maxima.  A is long and tilted in x-z, its mean off the
    # ray, so its maximum along the ray lies in front of B's while its mean
    # lies behind B's; the two orders composite A over B and B over A.
    cam = scenes.Camera(np.eye(4, dtype=np.float32), 50.0, 50.0, 8.5, 6.5, 17, 13, bg=(0.1, 0.2, 0.3))
    h = math.radians(-22.5)
    qs = np.array([[math.cos(h), 0.0, math.sin(h), 0.0], [1.0, 0.0, 0.0, 0.0]], np.float32)
    sc = one_gaussian_scene([[0.3, 0.0, 4.0], [0.0, 0.0, 3.85]], [[0.0, -1.5, -1.5], [-2.5, -2.5, -2.5]],
                            q=qs, logit=1.0)
    sc.sh[:, 0, :] = np.array([[1.0, 0.0, 0.0], [0.0, 0.0, 1.0]], np.float32)
    p = O.prepare(sc, cam)
    rho2, ts = O.ray_maximum(p, np.array([8]), np.array([6]))
    alpha, contrib, _ = O.pixel_alphas(p, rho2, ts)
    assert bool(contrib.all())
    t = ts[0].numpy()
    mz = p["mu_view"][:, 2].numpy()
    assert t[0] < t[1] and mz[0] > mz[1]          # the two orders disagree
    a = alpha[0].numpy()
    col = p["rgb"].numpy()
    bg = np.array([0.1, 0.2, 0.3], np.float32).astype(np.float64)
    a_first = col[0] * a[0] + col[1] * a[1] * (1 - a[0]) + (1 - a[0]) * (1 - a[1]) * bg
    b_first = col[1] * a[1] + col[0] * a[0] * (1 - a[1]) + (1 - a[0]) * (1 - a[1]) * bg
    exact = O.render_pixels(sc, cam, [8], [6])[0][0].numpy()
    mean = O.render_pixels(sc, cam, [8], [6], order="mean")[0][0].numpy()
    np.testing.assert_allclose(exact, a_first, rtol=1e-12)
    np.testing.assert_allclose(mean, b_first, rtol=1e-12)
    assert np.abs(exact - mean).max() > 1e-3


def test_kbuffer_hand_worked_sequence():
    # Bounded buffer of 2 entries, one pixel, four contributors arriving in
    # the order g0 (t* = 3), g1 (t* = 1), g2 (t* = 2), g3 (t* = 0.5):
    #   g0 -> [g0];  g1 -> [g1 g0];  g2 finds it full: g1 is nearer, blended,
    #   g2 enters -> [g2 g0];  g3 finds it full and is nearer than g2: blended
    #   at once;  end: g2, g0.  Blend sequence g1 g3 g2 g0 (exact: g3 g1 g2 g0).
    a = np.array([0.3, 0.5, 0.2, 0.4])
    t = np.array([3.0, 1.0, 2.0, 0.5])
    arrival = np.array([0.1, 0.2, 0.3, 0.4])
    col = np.array([[1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0], [1.0, 1.0, 0.0]])
    bg = np.array([0.1, 0.2, 0.3])

    def by_hand(seq):
        T, C = 1.0, np.zeros(3)
        for g in seq:
            C = C + col[g] * a[g] * T
            T *= 1 - a[g]
        return C + T * bg, T

    f = lambda v: torch.from_numpy(np.asarray(v, np.float64))
    contrib = torch.ones(1, 4, dtype=torch.bool)
    for size, seq in ((2, [1, 3, 2, 0]), (0, [0, 1, 2, 3]), (1, [1, 2, 3, 0]), (4, [3, 1, 2, 0])):
        out, T, n = O.composite_kbuffer(f(a[None]), f(t[None]), arrival, contrib, f(col), f(bg), size)
        C_ref, T_ref = by_hand(seq)
        np.testing.assert_allclose(out[0].numpy(), C_ref, rtol=1e-14, err_msg=str(size))
        assert T[0].item() == pytest.approx(T_ref, rel=1e-14) and int(n[0]) == 4
    # early termination inside the buffer: a = 0.99 layers stop after two
    a2 = np.full(4, 0.99)
    out, T, n = O.composite_kbuffer(f(a2[None]), f(t[None]), arrival, contrib, f(col), f(bg), 2)
    assert int(n[0]) == 2 and T[0].item() == pytest.approx(0.01 ** 2, rel=1e-12)


def test_kbuffer_limits_are_exact_and_mean_orders(small_workload):
    # with room for every contributor the buffer blends in exact depth order;
    # with no room it blends in arrival (mean-depth) order
    sc, cams = small_workload
    cam = cams[1]
    rng = np.random.default_rng(8)
    px, py = rng.integers(0, cam.width, 300), rng.integers(0, cam.height, 300)
    p = O.prepare(sc, cam)
    exact, ea = O.render_pixels(sc, cam, px, py, prep=p)
    big, ba = O.render_pixels(sc, cam, px, py, prep=p, order="kbuffer", kbuffer=1 << 20)
    np.testing.assert_allclose(big.numpy(), exact.numpy(), atol=1e-14)
    np.testing.assert_allclose(ba.numpy(), ea.numpy(), atol=1e-14)
    mean, ma = O.render_pixels(sc, cam, px, py, prep=p, order="mean")
    none, na = O.render_pixels(sc, cam, px, py, prep=p, order="kbuffer", kbuffer=0)
    np.testing.assert_allclose(none.numpy(), mean.numpy(), atol=1e-14)
    # the 16-entry buffer is exact on pixels with at most 16 contributors
    k16, _ = O.render_pixels(sc, cam, px, py, prep=p, order="kbuffer")
    rho2, ts = O.ray_maximum(p, px, py)
    _, contrib, _ = O.pixel_alphas(p, rho2, ts)
    few = contrib.sum(1).numpy() <= 16
    assert few.sum() > 50 and (~few).sum() > 10
    np.testing.assert_allclose(k16.numpy()[few], exact.numpy()[few], atol=1e-14)
    # a buffer of two entries overflows on the crowded pixels: approximate there
    k2, _ = O.render_pixels(sc, cam, px, py, prep=p, order="kbuffer", kbuffer=2)
    few2 = contrib.sum(1).numpy() <= 2
    np.testing.assert_allclose(k2.numpy()[few2], exact.numpy()[few2], atol=1e-14)
    assert np.abs(k2.numpy()[~few2] - exact.numpy()[~few2]).max() > 1e-3


def test_ewa_splat_closed_form():
    # Ablation without 3D evaluation: for an isotropic filtered variance
    # s_hat, Sigma' = s_hat J J^T with J the perspective Jacobian at the mean;
    # for a mean at (x, 0, z): Sigma'_xx = s_hat fx^2 (1/z^2 + x^2/z^4),
    # Sigma'_yy = s_hat fy^2 / z^2, Sigma'_xy = 0.
    cam = scenes.Camera(np.eye(4, dtype=np.float32), 60.0, 50.0, 8.5, 6.5, 17, 13)
    sc = one_gaussian_scene([[0.5, 0.0, 4.0]], [[-1.5, -1.5, -1.5]], logit=1.0)
    p = O.prepare(sc, cam)
    sh = float(p["s_hat"][0, 0])
    assert np.allclose(p["s_hat"].numpy(), sh)
    mean2, cov2 = O.ewa_splats(p)
    x, z = float(np.float32(0.5)), 4.0
    np.testing.assert_allclose(cov2[0].numpy(), [[sh * 60.0 ** 2 * (1 / z ** 2 + x ** 2 / z ** 4), 0.0],
                                                 [0.0, sh * 50.0 ** 2 / z ** 2]], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(mean2[0].numpy(), [60.0 * x / z + 8.5, 6.5], rtol=1e-12)
    # alpha at a pixel: o_hat exp(-rho^2/2) with rho^2 the 2D Mahalanobis distance
    px, py = 13, 9
    d = np.array([px + 0.5 - mean2[0, 0].item(), py + 0.5 - 6.5])
    rho2 = d[0] ** 2 / cov2[0, 0, 0].item() + d[1] ** 2 / cov2[0, 1, 1].item()
    r2, ts = O.splat_maximum(p, np.array([px]), np.array([py]))
    assert r2[0, 0].item() == pytest.approx(rho2, rel=1e-12)
    assert ts[0, 0].item() == pytest.approx(4.0, rel=1e-12)
    rgb, alpha = O.render_pixels(sc, cam, [px], [py], eval2d=True)
    a = min(0.99, p["o_hat"][0].item() * math.exp(-0.5 * rho2))
    assert alpha[0].item() == pytest.approx(a if a >= 1 / 255 else 0.0, rel=1e-12)


def test_early_termination_closed_form():
    # five coaxial Gaussians with o_hat = 0.95 at rho = 0: T = 0.05^k; the
    # fourth would take T below 1e-4, so exactly three are blended
    cam = scenes.Camera(np.eye(4, dtype=np.float32), 50.0, 50.0, 8.5, 6.5, 17, 13)
    n = 5
    mus = [[0.0, 0.0, 3.0 + i] for i in range(n)]
    sc = one_gaussian_scene(mus, np.full((n, 3), -1.0), logit=0.0)
    p = O.prepare(sc, cam)
    # choose opacity logits so that o_hat = 0.95 exactly in float64 terms
    phi = p["phi"].numpy()
    target = 0.95 / phi
    sc.opacity_logits[:] = np.log(target / (1 - target)).astype(np.float32)
    p = O.prepare(sc, cam)
    oh = p["o_hat"].numpy()
    assert bool(p["alive"].all())
    rgb, alpha = O.render_pixels(sc, cam, [8], [6], prep=p)
    T, C = 1.0, 0.0
    for i in range(n):
        if T * (1 - oh[i]) < 1e-4:
            break
        C += oh[i] * T
        T *= 1 - oh[i]
    assert i == 3
    col = 0.5 / math.sqrt(math.pi) * 0.5 + 0.5
    assert rgb[0, 0].item() == pytest.approx(col * C, rel=1e-12)
    assert 1 - alpha[0].item() == pytest.approx(T, rel=1e-12)


def test_camera_inside_discards():
    cam = scenes.Camera(np.eye(4, dtype=np.float32), 50.0, 50.0, 8.5, 6.5, 17, 13)
    # big sphere around the camera and a small one in front
    sc = one_gaussian_scene([[0.0, 0.0, 0.5], [0.0, 0.0, 5.0]], [[0.0] * 3, [-2.0] * 3], logit=3.0)
    p = O.prepare(sc, cam)
    assert bool(p["inside"][0]) and not bool(p["alive"][0])
    assert bool(p["alive"][1])
    # the discarded Gaussian contributes nothing
    rgb, _ = O.render_pixels(sc, cam, [8], [6], prep=p)
    rgb1, _ = O.render_pixels(sc.subset([1]), cam, [8], [6])
    np.testing.assert_allclose(rgb.numpy(), rgb1.numpy(), atol=1e-15)


def test_near_plane_rule_closed_form():
    # Sec. 3.3: a contribution whose ray maximum lies in front of the near
    # plane is dropped.  For an isotropic Gaussian on the optical axis at depth
    # z0 and the ray of direction (x', y', 1), the maximum is the foot of the
    # perpendicular from the mean, t* = z0 / (1 + x'^2 + y'^2): the centre
    # pixels see t* ~ z0 > z_near, the pixels far enough off axis t* < z_near,
    # while alpha stays far above 1/255 on all of them.
    f = 40.0
    cam = scenes.Camera(np.eye(4, dtype=np.float32), f, f, 16.0, 16.0, 32, 32)
    znear = float(np.float32(scenes.ZNEAR))
    assert cam.znear == znear
    z0 = float(np.float32(0.22))
    sc = one_gaussian_scene([[0.0, 0.0, z0]], [[math.log(0.04)] * 3], logit=3.0)
    p = O.prepare(sc, cam)
    assert bool(p["alive"][0])
    px, py = np.arange(16, 32), np.full(16, 16)
    rho2, ts = O.ray_maximum(p, px, py)
    alpha, contrib, raw = O.pixel_alphas(p, rho2, ts)
    xp, yp = (px + 0.5 - 16.0) / f, (py + 0.5 - 16.0) / f
    t_closed = z0 / (1.0 + xp * xp + yp * yp)
    np.testing.assert_allclose(ts[:, 0].numpy(), t_closed, rtol=1e-12)
    bright = raw[:, 0].numpy() >= 10 * O.ALPHA_MIN
    assert bright.all()
    behind = t_closed < znear
    assert 0 < behind.sum() < behind.size          # both sides of the plane occur
    np.testing.assert_array_equal(contrib[:, 0].numpy(), ~behind)
    # straddling z_near by 1e-9 relative: the rule is t* >= z_near
    k = int(np.nonzero(~behind)[0][-1])
    t_k = float(ts[k, 0])
    for zn, expect in ((t_k * (1 + 1e-9), False), (t_k * (1 - 1e-9), True), (t_k, True)):
        p["view"].znear = zn
        _, c, _ = O.pixel_alphas(p, rho2[k:k + 1], ts[k:k + 1])
        assert bool(c[0, 0]) == expect, (zn, t_k)
    # and the image: the pixels behind the plane show the background only
    p["view"].znear = znear
    rgb, a = O.render_pixels(sc, cam, px, py, prep=p)
    assert np.all(a.numpy()[behind] == 0.0) and np.all(a.numpy()[~behind] > 0.01)


def test_cutoff_level_and_camera_inside_flip():
    # tau_rho is the rho^2 at which o_hat exp(-rho^2/2) reaches 1/255
    rng = np.random.default_rng(21)
    oh = rng.uniform(O.ALPHA_MIN * (1 + 1e-6), 0.99, 1000)
    tau = O.cutoff(torch.from_numpy(oh)).numpy()
    np.testing.assert_allclose(oh * np.exp(-tau / 2), O.ALPHA_MIN, rtol=1e-12)
    assert np.all(np.diff(tau[np.argsort(oh)]) > 0)
    # An isotropic Gaussian of scale s on the optical axis at depth D, no
    # training clamp: s_hat = s^2 + k D^2 / f^2 (Eq. 6, 13), o_hat =
    # o s^2 / s_hat (Eq. 12, isotropic), tau = 2 ln(255 o_hat) and
    # |u_cam|^2 = D^2 / s_hat.  The camera-inside discard (Sec. 3.3) must flip
    # where |u_cam|^2 crosses tau, found here by bisection on these closed forms.
    f, k = 50.0, O.K_FILTER
    ls = np.float32(-2.0)
    logit = np.float32(1.0)
    s2 = math.exp(2.0 * float(ls))
    o = 1.0 / (1.0 + math.exp(-float(logit)))

    def closed(D):
        sh = s2 + k * D * D / (f * f)
        t = 2.0 * math.log(255.0 * o * s2 / sh)
        return D * D / sh - t, t

    lo, hi = 0.21, 5.0
    assert closed(lo)[0] < 0 < closed(hi)[0]
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if closed(mid)[0] < 0 else (lo, mid)
    cam = scenes.Camera(np.eye(4, dtype=np.float32), f, f, 8.0, 8.0, 16, 16)
    for rel, inside in ((-1e-6, True), (1e-6, False)):
        D = float(np.float32(lo * (1 + rel)))
        g, t = closed(D)
        assert (g < 0) == inside
        sc = one_gaussian_scene([[0.0, 0.0, D]], [[ls] * 3], logit=logit)
        p = O.prepare(sc, cam)
        assert p["tau"][0].item() == pytest.approx(t, rel=1e-12)
        assert bool(p["inside"][0]) == inside
        assert bool(p["alive"][0]) == (not inside)


def test_transmittance_monotone_and_alpha_range(small_workload):
    sc, cams = small_workload
    p = O.prepare(sc, cams[0])
    rng = np.random.default_rng(14)
    px, py = rng.integers(0, 128, 64), rng.integers(0, 128, 64)
    rho2, ts = O.ray_maximum(p, px, py)
    a, contrib, _ = O.pixel_alphas(p, rho2, ts)
    assert torch.all(a[contrib] >= 1 / 255) and torch.all(a <= 0.99)
    key = torch.where(contrib, ts, torch.full_like(ts, math.inf))
    order = torch.sort(key, dim=1, stable=True).indices
    aa = torch.where(torch.gather(contrib, 1, order), torch.gather(a, 1, order), torch.zeros_like(a))
    T = torch.cumprod(1 - aa, 1)
    assert torch.all(T[:, 1:] <= T[:, :-1])


def test_gradient_matches_finite_differences():
    sc = random_scene(12, 15, spread=0.6, logs=(-2.2, 0.3), deg=2)
    cam = cam_at((0.1, -0.2, -2.5), W=16, H=12)
    st = O.scene_tensors(sc, requires_grad=True)
    rng = np.random.default_rng(16)
    wts = torch.tensor(rng.standard_normal((3, 12, 16)))
    py, px = np.mgrid[0:12, 0:16]

    def loss_of(st_):
        rgb, alpha = O.render_pixels(st_, cam, px.ravel(), py.ravel())
        return (rgb.T.reshape(3, 12, 16) * wts).sum() + 0.3 * alpha.sum()

    loss = loss_of(st)
    loss.backward()
    checked = 0
    for name in ("means", "log_scales", "quats", "opacity_logits", "sh"):
        g = st[name].grad.numpy().ravel()
        base = st[name].detach().clone()
        idx = rng.choice(g.size, size=min(12, g.size), replace=False)
        for j in idx:
            h = 1e-6 * max(1.0, abs(base.view(-1)[j].item()))
            vals = []
            for sgn in (1, -1):
                pert = base.clone()
                pert.view(-1)[j] += sgn * h
                st2 = dict(st)
                st2 = {k: (v.detach() if torch.is_tensor(v) else v) for k, v in st.items()}
                st2[name] = pert
                with torch.no_grad():
                    vals.append(loss_of(st2).item())
            fd = (vals[0] - vals[1]) / (2 * h)
            assert fd == pytest.approx(g[j], rel=1e-4, abs=1e-6), (name, j)
            checked += 1
    assert checked >= 40


# ---------------------------------------------------------------------------
# Sec. 3.3: bounds
# ---------------------------------------------------------------------------

def test_bounds_sphere_closed_form():
    rng = np.random.default_rng(17)
    n = 30
    mu = np.stack([rng.uniform(-1, 1, n), rng.uniform(-0.6, 0.6, n), rng.uniform(3, 6, n)], 1)
    sc = one_gaussian_scene(mu, np.full((n, 3), -2.0), q=rng.standard_normal((n, 4)),
                            logit=np.full(n, 2.0))
    cam = scenes.Camera(np.eye(4, dtype=np.float32), 60.0, 60.0, 40.0, 30.0, 80, 60)
    mu = sc.means.astype(np.float64)
    p = O.prepare(sc, cam)
    b = O.view_space_bounds(p)
    r = np.sqrt(p["tau"].numpy() * p["s_hat"].numpy()[:, 0])
    for ax, i in (("x", 0), ("y", 1)):
        X, Z = mu[:, i], mu[:, 2]
        c = np.arctan2(X, Z)
        half = np.arcsin(r / np.hypot(X, Z))
        np.testing.assert_allclose(b[ax]["a1"].numpy(), c - half, atol=1e-10)
        np.testing.assert_allclose(b[ax]["a2"].numpy(), c + half, atol=1e-10)


def sample_ellipsoid_surface(mu, R, sp, tau, m, rng):
    u = rng.standard_normal((m, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    return mu + (np.sqrt(tau) * u * sp) @ R.T


def test_bounds_contain_sampled_silhouette():
    rng = np.random.default_rng(18)
    sc = random_scene(60, 19, spread=1.2, logs=(-1.8, 0.6))
    cam = cam_at((0.2, 0.1, -2.5), W=64, H=48)
    p = O.prepare(sc, cam)
    b = O.view_space_bounds(p)
    R = scipy_rot(sc.quats)
    sp = np.sqrt(p["s_hat"].numpy())
    V = cam.viewmat.astype(np.float64)
    tested = 0
    for g in range(60):
        if not bool(p["alive"][g]):
            continue
        pts = sample_ellipsoid_surface(sc.means[g].astype(np.float64), R[g], sp[g], p["tau"][g].item(), 4000, rng)
        pv = pts @ V[:3, :3].T + V[:3, 3]
        front = pv[:, 2] > 1e-3
        if not front.any():
            continue
        xs = cam.fx * pv[front, 0] / pv[front, 2] + cam.cx
        ys = cam.fy * pv[front, 1] / pv[front, 2] + cam.cy
        assert xs.min() >= b["x"]["p1"][g].item() - 1e-6 * (1 + abs(xs.min()))
        assert xs.max() <= b["x"]["p2"][g].item() + 1e-6 * (1 + abs(xs.max()))
        assert ys.min() >= b["y"]["p1"][g].item() - 1e-6 * (1 + abs(ys.min()))
        assert ys.max() <= b["y"]["p2"][g].item() + 1e-6 * (1 + abs(ys.max()))
        if (pv[:, 2] > 0.05).all() and not bool(b["x"]["full"][g]):
            # entirely in front: the bound is tight up to sampling density
            w = b["x"]["p2"][g].item() - b["x"]["p1"][g].item()
            assert xs.max() - xs.min() >= 0.97 * w
        tested += 1
    assert tested > 30


def test_bounds_axis_crossing_gives_full_range():
    # an ellipsoid elongated along view x through the optical axis region in
    # front of the camera crosses the view x-axis only if it contains points
    # with y = z = 0: place a long needle along x at y = z = 0 offset behind?
    # Simplest: a big sphere centred on the camera-x axis at x = 1 (y = z = 0).
    cam = scenes.Camera(np.eye(4, dtype=np.float32), 60.0, 60.0, 40.0, 30.0, 80, 60)
    sc = one_gaussian_scene([[1.5, 0.0, 0.0]], [[-1.0, -1.0, -1.0]], logit=3.0)
    p = O.prepare(sc, cam)
    assert bool(p["alive"][0])
    b = O.view_space_bounds(p)
    assert bool(b["y"]["full"][0])            # crosses the x-axis: no y bound
    assert not bool(b["x"]["full"][0])
    # crosses the z = 0 plane at x > 0: the x range reaches the right border
    assert b["x"]["p2"][0].item() >= 80


def test_bounds_behind_camera_is_empty():
    cam = scenes.Camera(np.eye(4, dtype=np.float32), 60.0, 60.0, 40.0, 30.0, 80, 60)
    sc = one_gaussian_scene([[0.3, 0.2, -4.0]], [[-2.0] * 3], logit=3.0)
    p = O.prepare(sc, cam)
    b = O.view_space_bounds(p)
    assert not bool(b["valid"][0])


# ---------------------------------------------------------------------------
# Sec. 3.4: frustum minimum
# ---------------------------------------------------------------------------

def brute_frustum_min(mu, R, sp, cam, x_lo, x_hi, y_lo, y_hi, rng, m=60000, zmax=30.0):
    """Sample points of the near-truncated frustum and take the smallest
    rho^2 (an upper bound of the true minimum that converges to it)."""
    V = cam.viewmat.astype(np.float64)
    xs = rng.uniform(x_lo, x_hi, m)
    ys = rng.uniform(y_lo, y_hi, m)
    zs = np.exp(rng.uniform(np.log(cam.znear), np.log(zmax), m))
    pv = np.stack([(xs - cam.cx) / cam.fx * zs, (ys - cam.cy) / cam.fy * zs, zs], 1)
    pw = (pv - V[:3, 3]) @ np.linalg.inv(V[:3, :3]).T
    u = ((pw - mu) @ R) / sp
    r2 = (u * u).sum(1)
    j = int(np.argmin(r2))
    # local refinement around the best sample
    best = r2[j]
    x0, y0, z0 = xs[j], ys[j], zs[j]
    for scale in (0.3, 0.1, 0.03, 0.01, 0.003):
        xx = np.clip(x0 + scale * (x_hi - x_lo) * rng.uniform(-1, 1, 4000), x_lo, x_hi)
        yy = np.clip(y0 + scale * (y_hi - y_lo) * rng.uniform(-1, 1, 4000), y_lo, y_hi)
        zz = np.clip(z0 * np.exp(scale * rng.uniform(-1, 1, 4000)), cam.znear, zmax)
        pv = np.stack([(xx - cam.cx) / cam.fx * zz, (yy - cam.cy) / cam.fy * zz, zz], 1)
        pw = (pv - V[:3, 3]) @ np.linalg.inv(V[:3, :3]).T
        u = ((pw - mu) @ R) / sp
        rr = (u * u).sum(1)
        k = int(np.argmin(rr))
        if rr[k] < best:
            best, x0, y0, z0 = rr[k], xx[k], yy[k], zz[k]
    return best


def test_frustum_min_brute_force():
    rng = np.random.default_rng(20)
    sc = random_scene(40, 21, spread=1.0, logs=(-1.6, 0.5))
    cam = cam_at((0.0, 0.0, -2.2), W=64, H=64)
    p = O.prepare(sc, cam)
    R = scipy_rot(sc.quats)
    sp = np.sqrt(p["s_hat"].numpy())
    g_idx = np.arange(40)
    tx = rng.integers(0, 4, 40)
    ty = rng.integers(0, 4, 40)
    got = O.tile_min_rho2(p, g_idx, tx, ty).numpy()
    for g in range(40):
        bf = brute_frustum_min(sc.means[g].astype(np.float64), R[g], sp[g], cam,
                               16 * tx[g], 16 * tx[g] + 16, 16 * ty[g], 16 * ty[g] + 16, rng)
        assert got[g] <= bf + 1e-9 * (1 + bf)                       # exact min <= any sample
        assert got[g] >= bf - 2e-3 * (1 + bf)                       # and is attained


def test_frustum_min_bounds_pixel_rays_and_mean_inside():
    sc = random_scene(80, 22, spread=1.0, logs=(-2.2, 0.4))
    cam = cam_at((0.0, 0.0, -2.5), W=64, H=64)
    p = O.prepare(sc, cam)
    G = 80
    tiles = [(tx, ty) for tx in range(4) for ty in range(4)]
    gi = np.repeat(np.arange(G), len(tiles))
    tx = np.tile([t[0] for t in tiles], G)
    ty = np.tile([t[1] for t in tiles], G)
    mins = O.tile_min_rho2(p, gi, tx, ty).numpy().reshape(G, len(tiles))
    py, px = np.mgrid[0:64, 0:64]
    rho2, ts = O.ray_maximum(p, px.ravel(), py.ravel())
    rho2 = rho2.numpy().T.reshape(G, 64, 64)
    ts = ts.numpy().T.reshape(G, 64, 64)
    V = cam.viewmat.astype(np.float64)
    mv = sc.means.astype(np.float64) @ V[:3, :3].T + V[:3, 3]
    for j, (a, b) in enumerate(tiles):
        blk = rho2[:, 16 * b:16 * b + 16, 16 * a:16 * a + 16]
        tb = ts[:, 16 * b:16 * b + 16, 16 * a:16 * a + 16]
        pix_min = np.where(tb >= cam.znear, blk, np.inf).reshape(G, -1).min(1)
        assert np.all(mins[:, j] <= pix_min + 1e-9 * (1 + pix_min))
        xs = cam.fx * mv[:, 0] / mv[:, 2] + cam.cx
        ys = cam.fy * mv[:, 1] / mv[:, 2] + cam.cy
        inside = (mv[:, 2] > cam.znear) & (xs > 16 * a) & (xs < 16 * a + 16) & (ys > 16 * b) & (ys < 16 * b + 16)
        assert np.all(mins[inside, j] == 0.0)
