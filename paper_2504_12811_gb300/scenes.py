"""Seeded synthetic scenes, cameras and request traces.

This module only *draws inputs*: Gaussian parameters, pinhole cameras and
arrival times.  It holds no step of the renderer; both the CUDA path and the
FP64 oracle consume what it returns.  All draws use numpy's PCG64
(`numpy.random.default_rng(seed)`) in a fixed order, so a (workload, seed)
pair always yields bit-identical float32 arrays.

Scene layout (structure of arrays, float32, C-contiguous):
    means           [n, 3]   world-space centres
    log_scales      [n, 3]   per-axis log standard deviations
    quats           [n, 4]   rotation quaternion (w, x, y, z), unnormalised
    opacity_logits  [n]      opacity before the sigmoid
    sh              [n, (deg+1)^2, 3]  real SH colour coefficients
    vhat_train      [n]      training sampling frequency (px per world unit)

Camera: world->view matrix (row-major 4x4; view x right, y down, z forward),
pinhole intrinsics in pixels, image size, near plane and background colour.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

ZNEAR = 0.2


@dataclass
class Camera:
    viewmat: np.ndarray          # [4, 4] float32, world -> view
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    znear: float = ZNEAR
    bg: tuple = (0.0, 0.0, 0.0)

    def __post_init__(self):
        self.viewmat = np.ascontiguousarray(self.viewmat, dtype=np.float32)
        # keep every scalar exactly representable in float32 so both sides
        # see the same camera
        self.fx = float(np.float32(self.fx))
        self.fy = float(np.float32(self.fy))
        self.cx = float(np.float32(self.cx))
        self.cy = float(np.float32(self.cy))
        self.znear = float(np.float32(self.znear))
        self.bg = tuple(float(np.float32(b)) for b in self.bg)

    @property
    def tiles(self):
        return (self.width + 15) // 16, (self.height + 15) // 16


@dataclass
class Scene:
    means: np.ndarray
    log_scales: np.ndarray
    quats: np.ndarray
    opacity_logits: np.ndarray
    sh: np.ndarray
    vhat_train: np.ndarray
    sh_degree: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def subset(self, idx) -> "Scene":
        idx = np.asarray(idx)
        return Scene(self.means[idx].copy(), self.log_scales[idx].copy(),
                     self.quats[idx].copy(), self.opacity_logits[idx].copy(),
                     self.sh[idx].copy(), self.vhat_train[idx].copy(),
                     self.sh_degree, dict(self.meta))

    def nbytes(self) -> int:
        return sum(a.nbytes for a in (self.means, self.log_scales, self.quats,
                                      self.opacity_logits, self.sh, self.vhat_train))


# ----------------------------------------------------------------------------
# cameras
# ----------------------------------------------------------------------------

def look_at(position, target=None, forward=None) -> np.ndarray:
    """World->view matrix for a camera at `position` looking at `target` (or
    along `forward`).  View axes: x right, y down, z forward; world +y is the
    'down' hint, so a camera at (0,0,-d) looking at the origin has the
    identity rotation."""
    p = np.asarray(position, dtype=np.float64)
    if forward is None:
        f = np.asarray(target, dtype=np.float64) - p
    else:
        f = np.asarray(forward, dtype=np.float64)
    f = f / np.linalg.norm(f)
    down = np.array([0.0, 1.0, 0.0])
    if abs(f @ down) > 0.999:
        down = np.array([0.0, 0.0, 1.0])
    x = np.cross(down, f)
    x /= np.linalg.norm(x)
    y = np.cross(f, x)
    rot = np.stack([x, y, f])                # rows: view axes in world coords
    v = np.eye(4)
    v[:3, :3] = rot
    v[:3, 3] = -rot @ p
    return v.astype(np.float32)


def pinhole(width: int, height: int, fov_x_deg: float):
    """Square-pixel pinhole with the horizontal field of view given and the
    principal point at the image centre."""
    fx = (width / 2.0) / math.tan(math.radians(fov_x_deg) / 2.0)
    return fx, fx, width / 2.0, height / 2.0


def make_camera(position, target=None, forward=None, width=128, height=128,
                fov_x_deg=60.0, znear=ZNEAR, bg=(0.0, 0.0, 0.0)) -> Camera:
    fx, fy, cx, cy = pinhole(width, height, fov_x_deg)
    return Camera(look_at(position, target, forward), fx, fy, cx, cy,
                  int(width), int(height), znear, bg)


def _unit_vectors(rng, n):
    v = rng.standard_normal((n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def orbit_cameras(rng, count, radius, width, height, fov_x_deg):
    """Cameras on a sphere of `radius` around the origin, looking at it."""
    dirs = _unit_vectors(rng, count)
    return [make_camera(radius * d, target=(0.0, 0.0, 0.0), width=width,
                        height=height, fov_x_deg=fov_x_deg) for d in dirs]


def interior_cameras(rng, count, half_extent, width, height, fov_x_deg):
    """Cameras placed uniformly in a cube, looking in uniform directions."""
    pos = rng.uniform(-half_extent, half_extent, (count, 3))
    dirs = _unit_vectors(rng, count)
    return [make_camera(p, forward=d, width=width, height=height,
                        fov_x_deg=fov_x_deg) for p, d in zip(pos, dirs)]


def vhat_train_draw(rng, n: int, lo: float, hi: float, unseen: float = 0.0) -> np.ndarray:
    """Synthetic stand-in for the per-Gaussian training sampling frequency
    (the scene input v_train of the 3D smoothing filter, Sec. 3.2): drawn
    log-uniformly in [lo, hi] pixels per world unit, with a random fraction
    `unseen` set to +inf (a Gaussian that no training camera saw: no clamp).
    A draw, not a computation: the renderer only reads the values."""
    v = np.exp(rng.uniform(math.log(lo), math.log(hi), n))
    v[rng.random(n) < unseen] = np.inf
    return v.astype(np.float32)


# ----------------------------------------------------------------------------
# scenes
# ----------------------------------------------------------------------------

def _quats(rng, n):
    return rng.standard_normal((n, 4)).astype(np.float32)


def _sh(rng, n, degree, dc_std=0.3, rest_std=0.05):
    k = (degree + 1) ** 2
    sh = np.empty((n, k, 3), dtype=np.float32)
    sh[:, 0, :] = rng.normal(0.0, dc_std, (n, 3))
    if k > 1:
        sh[:, 1:, :] = rng.normal(0.0, rest_std, (n, k - 1, 3))
    return sh


def uniform_cube_scene(n: int, seed: int = 0, sh_degree: int = 0) -> Scene:
    """Means uniform in [-1,1]^3, log-scales N(-3.5, 0.5) per axis, uniform
    random unit quaternions (normalised N(0, I4), stored unnormalised),
    opacity logits N(0, 1.5), SH DC N(0, 0.3) and higher bands N(0, 0.05);
    training sampling frequency log-uniform in [38, 78] px per unit, the range
    that 128x128, 60-degree training cameras at distance 3 give."""
    rng = np.random.default_rng(seed)
    means = rng.uniform(-1.0, 1.0, (n, 3)).astype(np.float32)
    log_scales = rng.normal(-3.5, 0.5, (n, 3)).astype(np.float32)
    quats = _quats(rng, n)
    opac = rng.normal(0.0, 1.5, n).astype(np.float32)
    sh = _sh(rng, n, sh_degree)
    vt = vhat_train_draw(rng, n, 38.0, 78.0)
    return Scene(means, log_scales, quats, opac, sh, vt, sh_degree,
                 {"kind": "uniform_cube", "seed": seed})


def cluster_scene(n: int = 1_000_000, seed: int = 0, n_clusters: int = 64,
                  shell_fraction: float = 0.1, sh_degree: int = 3) -> Scene:
    """Scene-scale workload: (1 - shell_fraction) * n Gaussians in
    `n_clusters` anisotropic clusters (centres uniform in a 20 m box, per-axis
    std U[0.1, 2] m under a random rotation) plus a background shell at radius
    50 m (+-1%).  log-scales N(-4, 1), opacity logits N(0, 2), SH degree 3 with
    DC N(0, 0.3) and higher bands N(0, 0.05).  Training sampling frequency:
    cluster Gaussians log-uniform in [100, 400] px per unit, shell ones in
    [30, 50], about half of each unseen (+inf), the spread that 16 interior
    1920x1080 training cameras give."""
    rng = np.random.default_rng(seed)
    n_shell = int(round(n * shell_fraction))
    n_cl = n - n_shell
    centres = rng.uniform(-10.0, 10.0, (n_clusters, 3))
    stds = rng.uniform(0.1, 2.0, (n_clusters, 3))
    rots = []
    for _ in range(n_clusters):
        q, r = np.linalg.qr(rng.standard_normal((3, 3)))
        rots.append(q * np.sign(np.diag(r)))
    rots = np.stack(rots)
    which = rng.integers(0, n_clusters, n_cl)
    local = rng.standard_normal((n_cl, 3)) * stds[which]
    pts = centres[which] + np.einsum("nij,nj->ni", rots[which], local)
    shell = _unit_vectors(rng, n_shell) * (50.0 * (1.0 + rng.uniform(-0.01, 0.01, (n_shell, 1))))
    means = np.concatenate([pts, shell]).astype(np.float32)
    log_scales = rng.normal(-4.0, 1.0, (n, 3)).astype(np.float32)
    quats = _quats(rng, n)
    opac = rng.normal(0.0, 2.0, n).astype(np.float32)
    sh = _sh(rng, n, sh_degree)
    vt = np.concatenate([vhat_train_draw(rng, n_cl, 100.0, 400.0, unseen=0.5),
                         vhat_train_draw(rng, n_shell, 30.0, 50.0, unseen=0.4)])
    return Scene(means, log_scales, quats, opac, sh, vt, sh_degree,
                 {"kind": "clusters", "seed": seed, "n_clusters": n_clusters})


def cluster_poses(count: int = 16, seed: int = 1, width=1920, height=1080, fov=60.0):
    """Evaluation poses for the cluster scene: positions uniform in [-8,8]^3,
    look directions uniform on the sphere."""
    rng = np.random.default_rng(seed)
    return interior_cameras(rng, count, 8.0, width, height, fov)


# ----------------------------------------------------------------------------
# named workloads
# ----------------------------------------------------------------------------

def workload(name: str, seed: int | None = None):
    """Return (scene, [cameras]) for a named workload.

    small       4,096 Gaussians (uniform cube, SH 0), camera at distance 3,
                60 deg, 128x128 (plus a seeded orbit pose).
    scene1m     1M Gaussians (64 clusters + 10% shell, SH 3), 16 interior
                1920x1080 poses, 60 deg.
    zoomout     `small` scene seen from distance 24 at 480x270.
    near        `small` scene, camera at z=-0.6 inside the cube, so that many
                Gaussians straddle the near plane.
    widefov     `small` scene, 120 deg at 2048x2048 from distance 3.
    train500k   500k uniform-cube Gaussians with SH 3, 4 orbit views at
                1280x832 (radius 3).
    """
    if name == "small":
        s = uniform_cube_scene(4096, seed=0 if seed is None else seed)
        rng = np.random.default_rng(100)
        cams = [make_camera((0.0, 0.0, -3.0), target=(0, 0, 0))]
        cams += orbit_cameras(rng, 1, 3.0, 128, 128, 60.0)
        return s, cams
    if name == "scene1m":
        s = cluster_scene(1_000_000, seed=0 if seed is None else seed)
        return s, cluster_poses()
    if name == "zoomout":
        s = uniform_cube_scene(4096, seed=0 if seed is None else seed)
        return s, [make_camera((0.0, 0.0, -24.0), target=(0, 0, 0), width=480, height=270)]
    if name == "near":
        s = uniform_cube_scene(4096, seed=0 if seed is None else seed)
        return s, [make_camera((0.0, 0.0, -0.6), forward=(0, 0, 1), width=128, height=128)]
    if name == "widefov":
        s = uniform_cube_scene(4096, seed=0 if seed is None else seed)
        return s, [make_camera((0.0, 0.0, -3.0), target=(0, 0, 0), width=2048, height=2048,
                               fov_x_deg=120.0)]
    if name == "train500k":
        s = uniform_cube_scene(500_000, seed=0 if seed is None else seed, sh_degree=3)
        rng = np.random.default_rng(4)
        return s, orbit_cameras(rng, 4, 3.0, 1280, 832, 60.0)
    raise KeyError(name)


def poisson_arrivals(rate_hz: float, duration_s: float, seed: int = 2) -> np.ndarray:
    """Arrival times (s) of a Poisson process."""
    rng = np.random.default_rng(seed)
    n = int(rate_hz * duration_s * 1.5) + 16
    t = np.cumsum(rng.exponential(1.0 / rate_hz, n))
    return t[t < duration_s]


# ----------------------------------------------------------------------------
# serving workload
# ----------------------------------------------------------------------------

SERVING_SCENES = {"s200k": 200_000, "s1m": 1_000_000, "s3m": 3_000_000}


def serving_scenes(sizes=None, seed: int = 10):
    """Resident scenes of the serving workload: uniform-cube Gaussians with SH
    degree 3 (200k, 1M and 3M by default)."""
    sizes = sizes or SERVING_SCENES
    return {name: uniform_cube_scene(n, seed=seed + i, sh_degree=3)
            for i, (name, n) in enumerate(sizes.items())}


@dataclass
class Request:
    rid: int
    arrival: float          # seconds from the start of the trace
    scene: str
    kind: str               # "vga" | "hd" | "stereo"
    cams: list


def request_cameras(kind: str, rng) -> list:
    """Cameras of one request: a pose inside the scene (position uniform in
    [-0.8, 0.8]^3, uniform look direction); stereo adds a second eye 64 mm
    apart along the view x axis."""
    pos = rng.uniform(-0.8, 0.8, 3)
    d = rng.standard_normal(3)
    d /= np.linalg.norm(d)
    if kind == "vga":
        return [make_camera(pos, forward=d, width=640, height=480, fov_x_deg=60.0)]
    if kind == "hd":
        return [make_camera(pos, forward=d, width=1920, height=1080, fov_x_deg=60.0)]
    left = make_camera(pos, forward=d, width=1832, height=1920, fov_x_deg=110.0)
    x_axis = left.viewmat[0, :3].astype(np.float64)
    right_pos = pos + 0.064 * x_axis
    return [make_camera(pos - 0.032 * x_axis, forward=d, width=1832, height=1920, fov_x_deg=110.0),
            make_camera(right_pos - 0.032 * x_axis, forward=d, width=1832, height=1920, fov_x_deg=110.0)]


def serving_trace(rate_hz: float = 400.0, duration_s: float = 5.0, seed: int = 2,
                  scene_names=None, kinds=("vga", "hd", "stereo")) -> list:
    """Poisson arrivals at `rate_hz`; each request picks a scene and a kind
    uniformly (equal thirds) and a random pose."""
    scene_names = list(scene_names or SERVING_SCENES)
    t = poisson_arrivals(rate_hz, duration_s, seed)
    rng = np.random.default_rng(seed + 1000)
    out = []
    for i, ti in enumerate(t):
        kind = kinds[int(rng.integers(0, len(kinds)))]
        scene = scene_names[int(rng.integers(0, len(scene_names)))]
        out.append(Request(i, float(ti), scene, kind, request_cameras(kind, rng)))
    return out
