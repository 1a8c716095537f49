"""The depth bounds in the pair keys are lower bounds of t*, pinned against
the oracle (CPU, float64).

The per-pixel re-sort releases a queued contributor once the key of the next
pair exceeds its t* (the depth of its ray maximum), so every key must be a
lower bound of t* on every ray its Gaussian contributes to.  Two bounds are
used: the Gaussian's own, from the sphere on which all ray maxima lie (the
maximum u* of a ray from the camera c is the foot of the perpendicular from
the mean, so u*.(u* - c) = 0), and a per-tile one, the smallest t* over the
tile's four corner pixel centres (t* = G.d / |d|^2 with d affine in the pixel
and G = fx fy adj(A) mu_v): with m that value, G.d - m |d|^2 is concave and
non-negative at the corners, hence on the whole tile.  Here both are
evaluated with the oracle's quantities and compared with the oracle's ray
maxima of every pixel, and the corner rule with a fine grid over the tile."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2504_12811_gb300 import scenes


def _frame(wl, size=64):
    scene, cams = scenes.workload(wl)
    cam = cams[0]
    s = size / cam.width
    import dataclasses
    cam = dataclasses.replace(cam, width=size, height=size, fx=cam.fx * s, fy=cam.fy * s, cx=cam.cx * s,
                              cy=cam.cy * s)
    prep = O.prepare(scene, cam)
    py, px = np.mgrid[0:size, 0:size]
    px, py = px.ravel(), py.ravel()
    rho2, ts = O.ray_maximum(prep, px, py)
    _, contrib, _ = O.pixel_alphas(prep, rho2, ts)
    return cam, prep, px, py, ts.numpy(), contrib.numpy()


def _gaussian_bound(prep):
    """mu_z - sqrt(tau) |A3_perp| + min(0, A3.c_hat) tau / |c| (A3_perp: the part
    of the view-z row A3 orthogonal to c_hat, c the camera in normalised space)."""
    T = prep["T_view"].numpy()
    tau = np.clip(prep["tau"].numpy(), 0, None)
    u = prep["u_cam"].numpy()
    A3 = T[:, 2, :3]
    cn = np.linalg.norm(u, axis=1)
    ch = u / cn[:, None]
    a3c = (A3 * ch).sum(1)
    A3p = A3 - a3c[:, None] * ch
    return T[:, 2, 3] - np.sqrt(tau * (A3p ** 2).sum(1)) + np.minimum(a3c, 0) * tau / cn


def _tile_planes(prep, cam, g, tx, ty):
    """G and the affine d = D0 + x Dx + y Dy of Gaussian g over tile (tx, ty)."""
    T = prep["T_view"].numpy()[g]
    t1, t2, t3 = T[0], T[1], T[2]
    A1, A2, T3 = t1[:3], t2[:3], t3[:3]
    cxm, cym = cam.cx - 16 * tx, cam.cy - 16 * ty
    Uv, Wv = cam.fx * A1 + cxm * T3, cam.fy * A2 + cym * T3
    D0, Dx, Dy = np.cross(Uv, Wv), np.cross(Wv, T3), np.cross(T3, Uv)
    G = cam.fx * cam.fy * (t1[3] * np.cross(A2, T3) + t2[3] * np.cross(T3, A1) + t3[3] * np.cross(A1, A2))
    return G, D0, Dx, Dy


def _tile_bound(prep, cam, g, tx, ty):
    """The smallest t* = G.d / |d|^2 over the tile's four corner pixel centres
    (-inf unless G.d > 0 at every corner)."""
    G, D0, Dx, Dy = _tile_planes(prep, cam, g, tx, ty)
    corners = [D0 + x * Dx + y * Dy for x in (0.5, 15.5) for y in (0.5, 15.5)]
    if min(float(G @ d) for d in corners) <= 0:
        return -np.inf
    return min(float(G @ d) / float(d @ d) for d in corners)


@pytest.mark.parametrize("wl", ["small", "near"])
def test_gaussian_depth_bound_is_below_every_contributing_ray(wl):
    cam, prep, px, py, ts, contrib = _frame(wl)
    lo = _gaussian_bound(prep)
    p, g = np.nonzero(contrib)
    assert p.size > 1000
    assert np.all(ts[p, g] >= lo[g] - 1e-9 * (1 + np.abs(lo[g])))
    # and it is not vacuous: within 10% of the nearest contribution for most
    near = np.full(lo.shape, np.inf)
    np.minimum.at(near, g, ts[p, g])
    seen = np.isfinite(near)
    assert np.mean(lo[seen] > 0.9 * near[seen]) > 0.5


def test_plane_form_depth_equals_ray_maximum():
    """t* = G.d / |d|^2 (the render's form) equals the oracle's ray maximum."""
    cam, prep, px, py, ts, contrib = _frame("small", 32)
    rng = np.random.default_rng(3)
    p_idx, g_idx = np.nonzero(contrib)
    for k in rng.choice(p_idx.size, size=200, replace=False):
        p, g = p_idx[k], g_idx[k]
        tx, ty = px[p] // 16, py[p] // 16
        T = prep["T_view"].numpy()[g]
        t1, t2, t3 = T[0], T[1], T[2]
        A1, A2, T3 = t1[:3], t2[:3], t3[:3]
        cxm, cym = cam.cx - 16 * tx, cam.cy - 16 * ty
        Uv, Wv = cam.fx * A1 + cxm * T3, cam.fy * A2 + cym * T3
        x, y = px[p] - 16 * tx + 0.5, py[p] - 16 * ty + 0.5
        d = np.cross(Uv, Wv) + x * np.cross(Wv, T3) + y * np.cross(T3, Uv)
        G = cam.fx * cam.fy * (t1[3] * np.cross(A2, T3) + t2[3] * np.cross(T3, A1) + t3[3] * np.cross(A1, A2))
        assert (G @ d) / (d @ d) == pytest.approx(ts[p, g], rel=1e-9)


@pytest.mark.parametrize("wl", ["small", "near"])
def test_tile_depth_bound_is_below_every_contributing_ray(wl):
    cam, prep, px, py, ts, contrib = _frame(wl)
    tiles = (py // 16) * ((cam.width + 15) // 16) + px // 16
    p, g = np.nonzero(contrib)
    checked = tight = 0
    for tile in np.unique(tiles[p]):
        sel = tiles[p] == tile
        ty, tx = divmod(int(tile), (cam.width + 15) // 16)
        for gg in np.unique(g[sel]):
            b = _tile_bound(prep, cam, gg, tx, ty)
            t_min = ts[p[sel][g[sel] == gg], gg].min()
            assert t_min >= b - 1e-9 * (1 + abs(b)), (wl, tile, gg, t_min, b)
            checked += 1
            tight += b > -np.inf
    assert checked > 500 and tight > 0.5 * checked


@pytest.mark.parametrize("wl", ["small", "near", "widefov"])
def test_tile_depth_bound_is_the_minimum_over_the_tile(wl):
    """The corner rule gives the minimum of t* over the whole tile rectangle:
    a 61 x 61 grid over [0.5, 15.5]^2 (pixel centres and points between them)
    never goes below it, and the grid's minimum is the corner value itself."""
    scene, cams = scenes.workload(wl)
    cam = cams[0]
    prep = O.prepare(scene, cam)
    alive = np.nonzero(prep["alive"].numpy())[0]
    rng = np.random.default_rng(11)
    tiles_x, tiles_y = cam.tiles
    s = np.linspace(0.5, 15.5, 61)
    gx, gy = np.meshgrid(s, s)
    gx, gy = gx.ravel(), gy.ravel()
    checked = 0
    for g in rng.choice(alive, size=min(400, alive.size), replace=False):
        T = prep["T_view"].numpy()[g]
        # tiles near the projected mean, where the Gaussian's rays pass
        z = T[2, 3]
        if z <= cam.znear:
            continue
        u = cam.fx * T[0, 3] / z + cam.cx
        v = cam.fy * T[1, 3] / z + cam.cy
        tx = int(np.clip(u // 16 + rng.integers(-2, 3), 0, tiles_x - 1))
        ty = int(np.clip(v // 16 + rng.integers(-2, 3), 0, tiles_y - 1))
        b = _tile_bound(prep, cam, g, tx, ty)
        if not np.isfinite(b):
            continue
        G, D0, Dx, Dy = _tile_planes(prep, cam, g, tx, ty)
        d = D0[None, :] + gx[:, None] * Dx[None, :] + gy[:, None] * Dy[None, :]
        t = (d @ G) / np.einsum("ij,ij->i", d, d)
        assert t.min() >= b - 1e-12 * abs(b), (wl, g, tx, ty, t.min(), b)
        assert t.min() == pytest.approx(b, rel=1e-12)
        checked += 1
    assert checked > 100


def test_tile_depth_bound_corner_rule_on_random_planes():
    """Random G and affine d (not from a scene, including strongly varying d):
    wherever G.d > 0 at every corner, t* on a fine grid is never below the
    smallest corner value; the rule needs G.d > 0 (m > 0 makes -m |d|^2
    concave)."""
    rng = np.random.default_rng(5)
    s = np.linspace(0.5, 15.5, 41)
    gx, gy = np.meshgrid(s, s)
    gx, gy = gx.ravel(), gy.ravel()
    corners = np.array([[0.5, 0.5], [15.5, 0.5], [0.5, 15.5], [15.5, 15.5]])
    hit = 0
    for _ in range(3000):
        G = rng.standard_normal(3)
        D0 = rng.standard_normal(3) * 10
        Dx, Dy = rng.standard_normal(3) * rng.choice([0.01, 0.3, 3.0]), rng.standard_normal(3) * rng.choice([0.01, 0.3, 3.0])
        dc = D0[None] + corners[:, :1] * Dx[None] + corners[:, 1:] * Dy[None]
        if np.any(dc @ G <= 0):
            continue
        m = np.min((dc @ G) / np.einsum("ij,ij->i", dc, dc))
        d = D0[None] + gx[:, None] * Dx[None] + gy[:, None] * Dy[None]
        t = (d @ G) / np.einsum("ij,ij->i", d, d)
        assert t.min() >= m - 1e-12 * abs(m)
        hit += 1
    assert hit > 500

