"""FP64 oracle: definitions of the AAA-Gaussians forward pass (test infrastructure only).

Every function works on float64 tensors derived exactly from the float32
scene and camera values.  Notation follows the paper: mean mu, scales s,
rotation R (from quaternion q), covariance Sigma = R S S^T R^T (Sec. 3.1,
Eq. 3), filtered variances s_hat (Sec. 3.2, Eq. 12), amplitude factor phi,
cutoff tau_rho, camera origin o.
"""
from __future__ import annotations

import itertools
import math

import numpy as np
import torch

__all__ = [
    "F64", "TILE", "ALPHA_MIN", "ALPHA_MAX", "T_STOP", "K_FILTER", "EPS_ANGLE",
    "t64", "View", "view_of", "rotation_from_quaternion", "sampling_frequency",
    "effective_frequency", "filtered_variances", "perpendicular_factor",
    "mip_factor", "cutoff", "sh_basis", "sh_colour", "prepare", "pixel_rays",
    "ray_maximum", "pixel_alphas", "composite", "render_pixels", "render",
    "view_space_bounds", "frustum_constraints", "frustum_min_rho2",
    "tile_min_rho2", "ambiguous_pixels", "scene_tensors", "training_sampling_frequency",
    "ewa_splats", "splat_maximum", "composite_kbuffer", "KBUFFER_SIZE",
]

F64 = torch.float64
TILE = 16                 # 16x16 pixel tiles (Sec. 3.1 "Tile-Based Rendering")
ALPHA_MIN = 1.0 / 255.0   # smallest alpha that is blended (3DGS convention)
ALPHA_MAX = 0.99          # alpha clamp (3DGS convention)
T_STOP = 1e-4             # early termination threshold on transmittance
K_FILTER = 0.3            # filter size k (Sec. 4, implementation details)
EPS_ANGLE = 1e-3          # epsilon of the angle clamp (Sec. 3.3, Eq. 17)
KBUFFER_SIZE = 16         # entries of the bounded per-pixel buffer (ablation)


def t64(a) -> torch.Tensor:
    """float64 copy of a float32 array / tensor (exact)."""
    if isinstance(a, torch.Tensor):
        return a.detach().to(F64) if not a.requires_grad else a.to(F64)
    return torch.from_numpy(np.ascontiguousarray(a)).to(F64)


class View:
    """Camera in float64: world->view rotation Rv and translation tv (the
    given float32 matrix is the definition, so its exact inverse is used: a
    float32 rotation is orthonormal only to ~1e-7), camera origin
    o = -Rv^-1 tv, pinhole intrinsics, image size, near plane."""

    def __init__(self, cam):
        V = t64(cam.viewmat)
        self.V = V
        self.Rv = V[:3, :3]
        self.tv = V[:3, 3]
        self.Rv_inv = torch.linalg.inv(self.Rv)
        self.o = -(self.Rv_inv @ self.tv)
        self.fx, self.fy = float(cam.fx), float(cam.fy)
        self.cx, self.cy = float(cam.cx), float(cam.cy)
        self.W, self.H = int(cam.width), int(cam.height)
        self.znear = float(cam.znear)
        self.bg = torch.tensor(cam.bg, dtype=F64)


def view_of(cam) -> View:
    return View(cam)


def scene_tensors(scene, requires_grad=False):
    """The differentiable scene parameters as float64 leaf tensors."""
    out = {
        "means": t64(scene.means), "log_scales": t64(scene.log_scales),
        "quats": t64(scene.quats), "opacity_logits": t64(scene.opacity_logits),
        "sh": t64(scene.sh),
    }
    if requires_grad:
        for v in out.values():
            v.requires_grad_(True)
    out["vhat_train"] = t64(scene.vhat_train)
    out["sh_degree"] = int(scene.sh_degree)
    return out


# ---------------------------------------------------------------------------
# Sec. 3.1: Gaussian parameterisation
# ---------------------------------------------------------------------------

def rotation_from_quaternion(q: torch.Tensor) -> torch.Tensor:
    """Rotation matrix R of the unit quaternion q/|q|, q = (w, x, y, z)
    (Sec. 3.1, Eq. 3: 'R is the rotation matrix obtained from q')."""
    q = q / q.norm(dim=-1, keepdim=True)
    w, x, y, z = q.unbind(-1)
    rows = [
        1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
        2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
        2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y),
    ]
    return torch.stack(rows, -1).reshape(q.shape[:-1] + (3, 3))


# ---------------------------------------------------------------------------
# Sec. 3.1 (Eq. 6-7) and Sec. 3.2 (Eq. 8-13): adaptive 3D smoothing filter
# ---------------------------------------------------------------------------

def training_sampling_frequency(means, cams) -> np.ndarray:
    """Sec. 3.2, Eq. 5: v_train = max over the training cameras of f / d, f
    the focal length in pixels (fx), d the view depth of the mean.  Reading:
    a camera counts when the mean lies beyond its near plane and projects
    inside its image (0 <= u <= W, 0 <= v <= H, pixel-centre convention of the
    cameras); +inf when no camera sees the mean (no clamp).  float64."""
    m = np.asarray(means, np.float64)
    best = np.full(m.shape[0], -np.inf)
    for c in cams:
        V = np.asarray(c.viewmat, np.float64)
        p = m @ V[:3, :3].T + V[:3, 3]
        z = p[:, 2]
        front = z > float(c.znear)
        zs = np.where(front, z, 1.0)
        u = float(c.fx) * p[:, 0] / zs + float(c.cx)
        v = float(c.fy) * p[:, 1] / zs + float(c.cy)
        seen = front & (u >= 0) & (u <= c.width) & (v >= 0) & (v <= c.height)
        best = np.maximum(best, np.where(seen, float(c.fx) / zs, -np.inf))
    best[best == -np.inf] = np.inf
    return best


def sampling_frequency(z_view: torch.Tensor, f: float, znear: float) -> torch.Tensor:
    """v_hat = f / d, d = view-space z of the mean (Sec. 3.1, Eq. 6).  The
    paper leaves d <= 0 undefined; d is read as max(z, z_near)."""
    return f / torch.clamp(z_view, min=znear)


def effective_frequency(v_hat: torch.Tensor, v_train: torch.Tensor) -> torch.Tensor:
    """v_hat' = min(v_hat_train, v_hat) (Sec. 3.2, Eq. 13)."""
    return torch.minimum(v_train, v_hat)


def filtered_variances(s: torch.Tensor, v_eff: torch.Tensor, k: float) -> torch.Tensor:
    """s_hat_i = s_i^2 + k / v_hat'^2: the eigenvalues of the smoothed
    covariance Sigma_hat = Sigma + (k / v_hat'^2) I (Sec. 3.1 and Eq. 12)."""
    return s * s + (k / (v_eff * v_eff)).unsqueeze(-1)


def perpendicular_factor(s: torch.Tensor, s_hat: torch.Tensor, R: torch.Tensor,
                         d: torch.Tensor) -> torch.Tensor:
    """Amplitude factor sqrt(|Sigma_perp| / |Sigma_hat_perp|) in the closed
    form of Sec. 3.2, Eq. 12, with d' = R^T d (Eq. 11) and d the unit vector
    from the camera origin to the mean (Appendix A)."""
    dp = torch.einsum("...ji,...j->...i", R, d)          # d' = R^T d
    d2 = dp * dp
    s2 = s * s
    num = (d2[..., 0] * s2[..., 1] * s2[..., 2] + d2[..., 1] * s2[..., 0] * s2[..., 2]
           + d2[..., 2] * s2[..., 0] * s2[..., 1])
    den = (d2[..., 0] * s_hat[..., 1] * s_hat[..., 2] + d2[..., 1] * s_hat[..., 0] * s_hat[..., 2]
           + d2[..., 2] * s_hat[..., 0] * s_hat[..., 1])
    return torch.sqrt(num / den)


def mip_factor(s: torch.Tensor, s_hat: torch.Tensor) -> torch.Tensor:
    """Volume-based factor sqrt(|Sigma| / |Sigma_hat|) of Mip-Splatting
    (Sec. 3.2, Eq. 8); only used to test that Eq. 12 is never smaller."""
    return torch.sqrt(torch.prod(s * s, -1) / torch.prod(s_hat, -1))


def cutoff(o_hat: torch.Tensor) -> torch.Tensor:
    """tau_rho: the rho^2 level at which o_hat * exp(-rho^2 / 2) = 1/255, so
    that rho^2 < tau_rho exactly where alpha >= 1/255 (Sec. 3.3 uses tau_rho as
    the rho^2 cutoff of the ellipsoid; its value is not printed)."""
    return 2.0 * torch.log(o_hat / ALPHA_MIN)


# ---------------------------------------------------------------------------
# View-dependent colour (Sec. 5 'view-dependent encoding'; 3DGS convention)
# ---------------------------------------------------------------------------

def _double_factorial(n: int) -> int:
    out = 1
    while n > 1:
        out *= n
        n -= 2
    return out


def sh_basis(dirs: torch.Tensor, degree: int) -> torch.Tensor:
    """Real orthonormal spherical harmonics with Condon-Shortley phase at unit
    directions, order (l, m) = (0,0), (1,-1), (1,0), (1,1), (2,-2), ...

    Built from the associated Legendre functions: with z = cos(theta),
    sin(theta) e^{i phi} = x + i y, and P_l^m(z) = (1 - z^2)^{m/2} Pbar_l^m(z):
        Y_l^0  = K_l^0 Pbar_l^0(z)
        Y_l^m  = sqrt2 K_l^m Pbar_l^m(z) Re((x + i y)^m)      (m > 0)
        Y_l^-m = sqrt2 K_l^m Pbar_l^m(z) Im((x + i y)^m)      (m > 0)
    K_l^m = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!), Pbar from the standard
    three-term recurrence in l."""
    x, y, z = dirs.unbind(-1)
    L = degree
    # Pbar[l][m]
    pbar = {}
    for m in range(L + 1):
        pmm = ((-1) ** m) * _double_factorial(2 * m - 1) * torch.ones_like(z)
        pbar[(m, m)] = pmm
        if m + 1 <= L:
            pbar[(m + 1, m)] = z * (2 * m + 1) * pmm
        for l in range(m + 2, L + 1):
            pbar[(l, m)] = ((2 * l - 1) * z * pbar[(l - 1, m)]
                            - (l + m - 1) * pbar[(l - 2, m)]) / (l - m)
    # (x + i y)^m
    re = [torch.ones_like(x)]
    im = [torch.zeros_like(x)]
    for m in range(1, L + 1):
        re.append(re[-1] * x - im[-1] * y)
        im.append(re[-2] * y + im[-1] * x)
    out = []
    for l in range(L + 1):
        for m in range(-l, l + 1):
            am = abs(m)
            K = math.sqrt((2 * l + 1) / (4 * math.pi)
                          * math.factorial(l - am) / math.factorial(l + am))
            if m == 0:
                out.append(K * pbar[(l, 0)])
            elif m > 0:
                out.append(math.sqrt(2.0) * K * pbar[(l, am)] * re[am])
            else:
                out.append(math.sqrt(2.0) * K * pbar[(l, am)] * im[am])
    return torch.stack(out, -1)


def sh_colour(sh: torch.Tensor, dirs: torch.Tensor, degree: int) -> torch.Tensor:
    """RGB = max(0, sum_lm k_lm Y_lm(dir) + 0.5) per channel (3DGS colour
    convention; the paper states no colour model beyond 'view-dependent
    encoding', Sec. 5)."""
    Y = sh_basis(dirs, degree)                      # [G, K]
    c = torch.einsum("gk,gkc->gc", Y, sh[:, : Y.shape[-1], :]) + 0.5
    return torch.clamp(c, min=0.0)


# ---------------------------------------------------------------------------
# per-Gaussian preparation for one view
# ---------------------------------------------------------------------------

def prepare(scene, cam, k: float = K_FILTER, params=None):
    """Per-Gaussian quantities for one view.

    `scene` is a `scenes.Scene` or the dict of `scene_tensors` (for autograd).
    Returns a dict with
      mu, R, s, o                  activations (Sec. 3.1; s = exp(log s),
                                   o = sigmoid(logit))
      v_hat, v_eff, s_hat          Eq. 6, 13, 12
      phi, o_hat                   Eq. 12 factor and filtered opacity
      tau                          rho^2 cutoff (see `cutoff`)
      u_cam                        camera origin in normalised Gaussian space
      inside                       camera inside the tau-ellipsoid (Sec. 3.3:
                                   no valid bound, Gaussian discarded)
      alive                        o_hat > 1/255 and not inside
      Sigma_hat_inv                R diag(1/s_hat) R^T (world space)
      mu_view, T_view              view-space mean and the 3x4 top rows of
                                   T_view = V T, T = [R S' mu; 0 1] with
                                   S' = diag(sqrt(s_hat)) (Sec. 3.1, Eq. 4;
                                   Sec. 3.3)
      rgb                          colour for this view
    """
    st = scene if isinstance(scene, dict) else scene_tensors(scene)
    view = View(cam)
    mu = st["means"]
    s = torch.exp(st["log_scales"])
    R = rotation_from_quaternion(st["quats"])
    o = torch.sigmoid(st["opacity_logits"])
    mu_view = mu @ view.Rv.T + view.tv
    v_hat = sampling_frequency(mu_view[:, 2], view.fx, view.znear)
    v_eff = effective_frequency(v_hat, st["vhat_train"])
    s_hat = filtered_variances(s, v_eff, k)
    diff = mu - view.o
    dist = diff.norm(dim=-1, keepdim=True)
    d = diff / dist
    phi = perpendicular_factor(s, s_hat, R, d)
    o_hat = o * phi
    tau = cutoff(o_hat)
    s_prime = torch.sqrt(s_hat)
    # camera origin in normalised Gaussian space: u = S'^-1 R^T (o - mu)
    u_cam = torch.einsum("gji,gj->gi", R, view.o - mu) / s_prime
    with torch.no_grad():
        inside = (u_cam * u_cam).sum(-1) < tau
        alive = (o_hat > ALPHA_MIN) & ~inside
    Sigma_hat_inv = torch.einsum("gij,gj,gkj->gik", R, 1.0 / s_hat, R)
    A = torch.einsum("ij,gjk,gk->gik", view.Rv, R, s_prime)      # Rv R S'
    T_view = torch.cat([A, mu_view.unsqueeze(-1)], -1)          # [G,3,4]
    rgb = sh_colour(st["sh"], d, st["sh_degree"])
    return {
        "mu": mu, "R": R, "s": s, "o": o, "v_hat": v_hat, "v_eff": v_eff,
        "s_hat": s_hat, "phi": phi, "o_hat": o_hat, "tau": tau,
        "u_cam": u_cam, "inside": inside, "alive": alive,
        "Sigma_hat_inv": Sigma_hat_inv, "mu_view": mu_view, "T_view": T_view,
        "rgb": rgb, "view": view, "dir": d,
    }


# ---------------------------------------------------------------------------
# Sec. 3.1: evaluation in 3D, maximum response along the pixel ray
# ---------------------------------------------------------------------------

def pixel_rays(view: View, px, py) -> torch.Tensor:
    """World-space ray directions through the centres (px + 1/2, py + 1/2),
    scaled so that the ray parameter is the view-space depth."""
    x = t64(np.asarray(px, dtype=np.float64)) + 0.5
    y = t64(np.asarray(py, dtype=np.float64)) + 0.5
    rv = torch.stack([(x - view.cx) / view.fx, (y - view.cy) / view.fy,
                      torch.ones_like(x)], -1)
    return rv @ view.Rv_inv.T                         # Rv^-1 rv, row form


def ray_maximum(prep, px, py):
    """Maximum of the Gaussian along each pixel ray (Sec. 3.1, Eq. 1-2 with
    Sigma_hat; 'only the maximum contribution along the ray is considered').

    Along X(t) = o + t d, rho^2(t) = (X - mu)^T Sigma_hat^-1 (X - mu) is the
    quadratic a t^2 + 2 b t + c; its minimum is at t* = -b/a with value
    rho^2* = c - b^2/a.  t is the view depth.  Returns (rho2*, t*) as [P, G]."""
    view = prep["view"]
    dw = pixel_rays(view, px, py)                      # [P,3]
    w = view.o - prep["mu"]                           # [G,3]
    Si = prep["Sigma_hat_inv"]                         # [G,3,3]
    v = torch.einsum("gij,gj->gi", Si, w)
    c = (w * v).sum(-1)                                # [G]
    a = torch.einsum("pi,gij,pj->pg", dw, Si, dw)
    b = dw @ v.T
    tstar = -b / a
    rho2 = c - b * b / a
    return rho2, tstar


def pixel_alphas(prep, rho2, tstar):
    """alpha = min(0.99, o_hat exp(-rho^2/2)); a Gaussian contributes to a
    pixel when it is alive, alpha >= 1/255 and the depth t* of its maximum is
    not closer than the near plane (Sec. 3.3: depth closer than the near plane
    receives no contribution)."""
    G = torch.exp(-0.5 * rho2)
    raw = prep["o_hat"].unsqueeze(0) * G
    alpha = torch.clamp(raw, max=ALPHA_MAX)
    with torch.no_grad():
        contrib = (prep["alive"].unsqueeze(0) & (raw >= ALPHA_MIN)
                   & (tstar >= prep["view"].znear))
    return alpha, contrib, raw


def composite(alpha, tstar, contrib, rgb, bg):
    """Front-to-back compositing in exact per-pixel depth order (the order
    hierarchical sorting approximates, Sec. 3.1 'Blending Sort Order'):
    contributors sorted by (tstar, Gaussian index), tstar being the depth of
    each maximum unless the caller passes another sort key; C = sum c_i a_i T_i,
    T_i = prod_{j<i} (1 - a_j); stop before the contributor that would take T
    below 1e-4.  Returns (RGB + T bg [P,3], final T [P], blended count [P])."""
    with torch.no_grad():
        key = torch.where(contrib, tstar, torch.full_like(tstar, math.inf))
        order = torch.sort(key, dim=1, stable=True).indices
        m = int(contrib.sum(1).max().item()) if contrib.numel() else 0
        order = order[:, :max(m, 1)]
        c_sorted = torch.gather(contrib, 1, order)
    a = torch.gather(alpha, 1, order)
    a = torch.where(c_sorted, a, torch.zeros_like(a))
    one_minus = 1.0 - a
    T_after = torch.cumprod(one_minus, dim=1)
    T_before = torch.cat([torch.ones_like(T_after[:, :1]), T_after[:, :-1]], 1)
    with torch.no_grad():
        blended = c_sorted & (T_after >= T_STOP)
    w = torch.where(blended, a * T_before, torch.zeros_like(a))
    col = rgb[order]                                   # [P,m,3]
    C = (w.unsqueeze(-1) * col).sum(1)
    T = torch.prod(torch.where(blended, one_minus, torch.ones_like(a)), 1)
    out = C + T.unsqueeze(-1) * bg
    return out, T, blended.sum(1)


def composite_kbuffer(alpha, tstar, arrival, contrib, rgb, bg, size=KBUFFER_SIZE, sequences=False):
    """Front-to-back compositing through a bounded per-pixel buffer, the
    approximate per-ray re-sort that hierarchical rasterisation keeps
    (Sec. 3.1 'Blending Sort Order'; the sort ablations of Sec. 5).

    The contributors of a pixel arrive in the order of `arrival` (one key per
    Gaussian, ties by Gaussian index).  The buffer holds up to `size` of them
    ordered by (t*, arrival).  An arrival that finds the buffer full blends the
    nearest of the buffer's entries and itself (the older one on a tie) and
    keeps the others; when every contributor has arrived the buffer is blended
    nearest first.  Blending stops before the contributor that would take T
    below 1e-4.  The order is exact while no pixel holds more than `size`
    contributors at once.  size = 0 blends in arrival order.  Plain float64
    loops over pixels (no autograd).  Returns (RGB + T bg [P,3], final T [P],
    blended count [P]), and with `sequences` also the blended Gaussians of
    every pixel in blend order (a list of index arrays)."""
    a_np = alpha.detach().numpy()
    t_np = tstar.detach().numpy()
    c_np = contrib.detach().numpy()
    col = rgb.detach().numpy()
    bgv = bg.detach().numpy()
    arr = np.asarray(arrival, dtype=np.float64)
    P = a_np.shape[0]
    out = np.zeros((P, 3))
    Tout = np.ones(P)
    nb = np.zeros(P, dtype=np.int64)
    seqs = []
    for p in range(P):
        gs = np.nonzero(c_np[p])[0]
        gs = gs[np.lexsort((gs, arr[gs]))]                # arrival order
        T, C, n = 1.0, np.zeros(3), 0
        done = False
        seq = []

        def blend(g):
            nonlocal T, C, n, done
            Tn = T * (1.0 - a_np[p, g])
            if Tn < T_STOP:
                done = True
                return
            C = C + col[g] * (a_np[p, g] * T)
            T = Tn
            n += 1
            seq.append(g)

        buf = []                                           # sorted (t*, arrival rank, g)
        for rank, g in enumerate(gs):
            if done:
                break
            e = (t_np[p, g], rank, g)
            if size == 0:
                blend(g)
                continue
            if len(buf) == size:
                if e < buf[0]:
                    blend(g)
                    continue
                blend(buf.pop(0)[2])
                if done:
                    break
            lo_, hi_ = 0, len(buf)
            while lo_ < hi_:                               # insert after smaller keys
                mid = (lo_ + hi_) // 2
                if buf[mid] < e:
                    lo_ = mid + 1
                else:
                    hi_ = mid
            buf.insert(lo_, e)
        while buf and not done:
            blend(buf.pop(0)[2])
        out[p] = C + T * bgv
        Tout[p] = T
        nb[p] = n
        seqs.append(np.asarray(seq, dtype=np.int64))
    res = (torch.from_numpy(out), torch.from_numpy(Tout), torch.from_numpy(nb))
    return res + (seqs,) if sequences else res


def ewa_splats(prep):
    """Ablation without 3D evaluation (Sec. 5, 'w/o 3D'): every Gaussian as a
    2D splat.  The filtered world covariance R diag(s_hat) R^T is taken to
    view space (Rv . Rv^T) and projected with the Jacobian J of the
    perspective map (fx x/z + cx, fy y/z + cy) at the view-space mean (the EWA
    local affine approximation); reading: no extra screen-space dilation.
    Returns the projected means [G,2] and the 2D covariances [G,2,2]."""
    view = prep["view"]
    Rv = view.Rv
    S = torch.einsum("gij,gj,gkj->gik", prep["R"], prep["s_hat"], prep["R"])
    Sv = Rv @ S @ Rv.T
    x, y, z = prep["mu_view"].unbind(-1)
    zero = torch.zeros_like(z)
    J = torch.stack([torch.stack([view.fx / z, zero, -view.fx * x / z ** 2], -1),
                     torch.stack([zero, view.fy / z, -view.fy * y / z ** 2], -1)], -2)   # [G,2,3]
    cov2 = J @ Sv @ J.transpose(-1, -2)
    mean2 = torch.stack([view.fx * x / z + view.cx, view.fy * y / z + view.cy], -1)
    return mean2, cov2


def splat_maximum(prep, px, py, splats=None):
    """rho^2 of the 2D splats at the pixel centres [P,G] (squared
    Mahalanobis distance in the 2D covariance) and the depth of each
    contribution, the mean's view depth [P,G]."""
    mean2, cov2 = splats if splats is not None else ewa_splats(prep)
    a, b, c = cov2[:, 0, 0], cov2[:, 0, 1], cov2[:, 1, 1]
    det = a * c - b * b                                  # inverse of [[a, b], [b, c]]
    q = torch.stack([t64(np.asarray(px) + 0.5), t64(np.asarray(py) + 0.5)], -1)   # [P,2]
    dx = q[:, :1] - mean2[:, 0].unsqueeze(0)                                        # [P,G]
    dy = q[:, 1:] - mean2[:, 1].unsqueeze(0)
    rho2 = (c * dx * dx - 2.0 * b * dx * dy + a * dy * dy) / det
    tstar = prep["mu_view"][:, 2].unsqueeze(0).expand_as(rho2)
    return rho2, tstar


def render_pixels(scene, cam, px, py, k: float = K_FILTER, chunk: int = 512,
                  prep=None, order: str = "tstar", eval2d: bool = False, kbuffer: int = KBUFFER_SIZE):
    """RGB [P,3] and alpha [P] of the given pixels (plain definition: every
    Gaussian tested against every pixel).  order="tstar" blends in exact
    per-pixel order of the maxima; order="mean" is the sort ablation of
    Sec. 5 (no per-ray sorting): contributors blended in the order of the view
    depth of their means, clamped to z_near (reading: the same clamp as the
    depth keys), ties by Gaussian index; order="kbuffer" is the bounded-buffer
    re-sort (`composite_kbuffer`, `kbuffer` entries) with contributors arriving
    in that mean-depth order.  eval2d=True is the ablation without
    3D evaluation: alpha from the EWA splats (`ewa_splats`), depth the mean's,
    and (reading) no camera-inside rule: a Gaussian is alive when o_hat >
    1/255 and its mean lies beyond the near plane."""
    if prep is None:
        prep = prepare(scene, cam, k)
    px = np.asarray(px).reshape(-1)
    py = np.asarray(py).reshape(-1)
    G = prep["mu"].shape[0]
    step = max(1, min(chunk, (1 << 24) // max(G, 1)))
    outs, Ts = [], []
    if eval2d:
        splats = ewa_splats(prep)
        p2 = dict(prep)
        p2["alive"] = (prep["o_hat"] > ALPHA_MIN) & (prep["mu_view"][:, 2] >= prep["view"].znear)
    for i in range(0, px.size, step):
        if eval2d:
            rho2, tstar = splat_maximum(prep, px[i:i + step], py[i:i + step], splats)
            alpha, contrib, _ = pixel_alphas(p2, rho2, tstar)
        else:
            rho2, tstar = ray_maximum(prep, px[i:i + step], py[i:i + step])
            alpha, contrib, _ = pixel_alphas(prep, rho2, tstar)
        if order == "kbuffer":
            arrival = torch.clamp(prep["mu_view"][:, 2].detach(), min=prep["view"].znear).numpy()
            out, T, _ = composite_kbuffer(alpha, tstar, arrival, contrib, prep["rgb"], prep["view"].bg, kbuffer)
            outs.append(out)
            Ts.append(T)
            continue
        if order == "mean":
            key = torch.clamp(prep["mu_view"][:, 2].detach(), min=prep["view"].znear).expand_as(tstar)
        elif order == "tstar":
            key = tstar
        else:
            raise ValueError(order)
        out, T, _ = composite(alpha, key, contrib, prep["rgb"], prep["view"].bg)
        outs.append(out)
        Ts.append(T)
    out = torch.cat(outs) if outs else torch.zeros(0, 3, dtype=F64)
    T = torch.cat(Ts) if Ts else torch.zeros(0, dtype=F64)
    return out, 1.0 - T


def render(scene, cam, k: float = K_FILTER, prep=None, order: str = "tstar", eval2d: bool = False,
           kbuffer: int = KBUFFER_SIZE):
    """Full image: RGB [3,H,W] and alpha [H,W] (float64)."""
    W, H = int(cam.width), int(cam.height)
    py, px = np.mgrid[0:H, 0:W]
    out, alpha = render_pixels(scene, cam, px.ravel(), py.ravel(), k, prep=prep, order=order, eval2d=eval2d,
                               kbuffer=kbuffer)
    return out.T.reshape(3, H, W), alpha.reshape(H, W)


# ---------------------------------------------------------------------------
# Sec. 3.3 (Eq. 14-17, Appendix B): view-space angular bounds
# ---------------------------------------------------------------------------

def view_space_bounds(prep, eps: float = EPS_ANGLE):
    """Screen bounds from tangent planes through the camera.

    s_ij = <t, T_i * T_j>, t = (tau, tau, tau, -1), T_i the rows of
    T_view (Eq. 15); tan(theta_12) = (s_13 +- sqrt(s_13^2 - s_11 s_33)) / s_33
    (Eq. 14, the final form of Appendix B); the rotation step places theta_1 in
    (theta_mu - pi, theta_mu) and theta_2 in (theta_mu, theta_mu + pi) with the
    pair chosen so that theta_2 - theta_1 < pi (Eq. 16); the clamp to
    +-(pi/2 - eps) (Eq. 17); a negative discriminant (or s_33 ~ 0) gives the
    whole screen on that axis (Sec. 3.3).  Same for phi with rows 2 and 3.

    Returns a dict with angles, pixel bounds (x1,x2,y1,y2), a validity mask
    (non-empty on both axes) and the inclusive tile rectangle."""
    view = prep["view"]
    T = prep["T_view"]
    tau = prep["tau"]
    tvec = torch.stack([tau, tau, tau, -torch.ones_like(tau)], -1)   # [G,4]

    def sij(i, j):
        return (tvec * T[:, i, :] * T[:, j, :]).sum(-1)

    s33 = sij(2, 2)
    res = {}
    for name, i, f, c, size in (("x", 0, view.fx, view.cx, view.W),
                                ("y", 1, view.fy, view.cy, view.H)):
        sii, si3 = sij(i, i), sij(i, 2)
        disc = si3 * si3 - sii * s33
        full = (disc < 0) | (s33.abs() <= 1e-12 * (sii.abs() + s33.abs()))
        sq = torch.sqrt(torch.clamp(disc, min=0.0))
        s33_safe = torch.where(full, torch.ones_like(s33), s33)
        ra = torch.atan((si3 + sq) / s33_safe)
        rb = torch.atan((si3 - sq) / s33_safe)
        amu = torch.atan2(prep["mu_view"][:, i], prep["mu_view"][:, 2])

        def lo(r):
            return amu - torch.remainder(amu - r, math.pi)

        a1_1, a2_1 = lo(ra), lo(rb) + math.pi
        a1_2, a2_2 = lo(rb), lo(ra) + math.pi
        pick1 = (a2_1 - a1_1) < math.pi
        a1 = torch.where(pick1, a1_1, a1_2)
        a2 = torch.where(pick1, a2_1, a2_2)
        lim = math.pi / 2 - eps
        a1 = torch.where(full, torch.full_like(a1, -lim), torch.clamp(a1, min=-lim))
        a2 = torch.where(full, torch.full_like(a2, lim), torch.clamp(a2, max=lim))
        nonempty = a1 <= a2
        p1 = f * torch.tan(a1) + c
        p2 = f * torch.tan(a2) + c
        ntiles = (size + TILE - 1) // TILE
        t1 = torch.clamp(torch.floor(p1 / TILE), min=0).to(torch.int64)
        t2 = torch.clamp(torch.floor(p2 / TILE), max=ntiles - 1).to(torch.int64)
        onscreen = nonempty & (p2 >= 0) & (p1 <= size) & (t1 <= t2)
        res[name] = {"a1": a1, "a2": a2, "p1": p1, "p2": p2, "full": full,
                     "t1": t1, "t2": t2, "onscreen": onscreen}
    res["valid"] = res["x"]["onscreen"] & res["y"]["onscreen"] & prep["alive"]
    return res


# ---------------------------------------------------------------------------
# Sec. 3.4 (Eq. 18): minimum of rho^2 over a (tile or image) frustum
# ---------------------------------------------------------------------------

def frustum_constraints(prep, x_lo, x_hi, y_lo, y_hi, near: bool = True):
    """Half-spaces n.u + h >= 0 in normalised Gaussian space bounding the
    frustum of the screen rectangle [x_lo,x_hi] x [y_lo,y_hi].

    Screen planes pi_x = (1,0,0,-x), pi_y = (0,1,0,-y) are carried to Gaussian
    space by pi' = T'^T pi with T' = M_vp P V T (Sec. 3.1, Eq. 4-5).  The
    viewport-projection matrix maps view (X,Y,Z) to homogeneous screen
    coordinates (fx X + cx Z, fy Y + cy Z, ., Z).  With `near`, the view-space
    half-space Z >= z_near is added (tiles where the Gaussian lies closer than
    the near plane are culled, Sec. 3.3).  Each (n, h) is normalised so that
    n.u + h is a signed distance.  Inputs x_lo.. are [B] tensors broadcast
    against the Gaussians of `prep` (one rectangle per Gaussian) or scalars."""
    view = prep["view"]
    G = prep["mu"].shape[0]
    Tg = torch.zeros(G, 4, 4, dtype=F64)
    Tg[:, :3, :3] = prep["R"] * torch.sqrt(prep["s_hat"]).unsqueeze(1)   # R S'
    Tg[:, :3, 3] = prep["mu"]
    Tg[:, 3, 3] = 1.0
    KP = torch.tensor([[view.fx, 0, view.cx, 0], [0, view.fy, view.cy, 0],
                       [0, 0, 0, 1], [0, 0, 1, 0]], dtype=F64)
    Tp = KP @ view.V @ Tg                              # T' [G,4,4]
    Tvw = view.V @ Tg                                  # V T
    bx = lambda v: torch.as_tensor(v, dtype=F64).expand(G) if not torch.is_tensor(v) or v.dim() == 0 else v.to(F64)
    x_lo, x_hi, y_lo, y_hi = bx(x_lo), bx(x_hi), bx(y_lo), bx(y_hi)
    one, zero = torch.ones(G, dtype=F64), torch.zeros(G, dtype=F64)

    def plane(pi):                                     # pi [G,4] -> T'^T pi
        return torch.einsum("gji,gj->gi", Tp, pi)

    planes = [
        plane(torch.stack([one, zero, zero, -x_lo], -1)),      # x >= x_lo
        -plane(torch.stack([one, zero, zero, -x_hi], -1)),     # x <= x_hi
        plane(torch.stack([zero, one, zero, -y_lo], -1)),      # y >= y_lo
        -plane(torch.stack([zero, one, zero, -y_hi], -1)),     # y <= y_hi
    ]
    if near:
        zn = torch.full((G,), view.znear, dtype=F64)
        planes.append(torch.einsum("gji,gj->gi", Tvw,
                                   torch.stack([zero, zero, one, -zn], -1)))
    P = torch.stack(planes, 1)                          # [G,m,4]
    nrm = P[..., :3].norm(dim=-1, keepdim=True)
    return P / nrm


def frustum_min_rho2(prep, x_lo, x_hi, y_lo, y_hi, near: bool = True,
                     tol: float = 1e-9):
    """min over the frustum F of rho(x)^2 = |u|^2 (Sec. 3.4, Eq. 18).

    The minimiser of the strictly convex |u|^2 over the polyhedron F is the
    minimum-norm point of the affine hull of some face of F (an active set of
    at most three constraints, or none when the mean is inside).  Every active
    set is enumerated (the paper's 'naive' projection onto all planes and edges,
    here with vertices added for the near-plane corners); a candidate counts
    only if it lies in F.  Returns [G]."""
    P = frustum_constraints(prep, x_lo, x_hi, y_lo, y_hi, near)
    G, m, _ = P.shape
    n, h = P[..., :3], P[..., 3]
    best = torch.full((G,), math.inf, dtype=F64)
    for size in range(0, 4):
        for S in itertools.combinations(range(m), size):
            if size == 0:
                u = torch.zeros(G, 3, dtype=F64)
            else:
                NS = n[:, list(S), :]                   # [G,k,3]
                hS = h[:, list(S)]
                u = -(torch.linalg.pinv(NS) @ hS.unsqueeze(-1)).squeeze(-1)
                on = (torch.einsum("gki,gi->gk", NS, u) + hS).abs().amax(-1) <= 1e-7
            g = torch.einsum("gmi,gi->gm", n, u) + h
            feas = (g >= -tol).all(-1)
            if size > 0:
                feas = feas & on
            val = (u * u).sum(-1)
            best = torch.where(feas & (val < best), val, best)
    return best


def tile_min_rho2(prep, gauss_idx, tile_x, tile_y, near: bool = True):
    """frustum_min_rho2 for (Gaussian, tile) pairs given as index arrays."""
    gi = torch.as_tensor(np.asarray(gauss_idx), dtype=torch.int64)
    sub = {k: (v[gi] if torch.is_tensor(v) and v.dim() > 0 and v.shape[0] == prep["mu"].shape[0] else v)
           for k, v in prep.items()}
    tx = torch.as_tensor(np.asarray(tile_x), dtype=F64)
    ty = torch.as_tensor(np.asarray(tile_y), dtype=F64)
    return frustum_min_rho2(sub, tx * TILE, tx * TILE + TILE, ty * TILE, ty * TILE + TILE, near)


# ---------------------------------------------------------------------------
# pixels where float32 rounding can legitimately flip a discrete decision
# ---------------------------------------------------------------------------

def ambiguous_pixels(prep, px, py, rel_alpha=2e-5, rel_t=2e-6, rel_tau=1e-4, budget=1e-3, eval2d=False):
    """Pixels whose result may depend on a decision that float32 evaluation
    can take differently from float64 (test tolerance logic, not part of the
    method).  Candidate flips at a pixel:
      * a Gaussian whose alpha lies within rel_alpha (relative) of 1/255;
      * a contributor whose depth t* lies within rel_t (relative) of z_near;
      * a Gaussian touching the pixel whose camera-inside test or o_hat > 1/255
        test lies within rel_tau of its threshold;
      * two depth-adjacent contributors whose t* differ by at most rel_t
        (relative), which float32 may blend in either order.
    Front-to-back compositing bounds what each flip can do: a layer of opacity
    a entering or leaving at transmittance T (the product of 1 - alpha of the
    contributors in front of it) moves every output channel by at most
    a T cmax (cmax: the largest colour at the pixel, the background and 1 for
    alpha), and swapping adjacent layers a, b by T_a a_a a_b |c_a - c_b|; a
    flip next to early termination can also move the stopping point, by at
    most T_STOP cmax.  A pixel is flagged when the bounds of its candidate
    flips add up to more than `budget` (half the max-abs tolerance of the
    parity tests), so that in dense content the hundreds of layers hidden
    behind the opaque front do not flag pixels they cannot change.
    eval2d: the same for the 2D-splat ablation (no camera-inside test)."""
    view = prep["view"]
    if eval2d:
        rho2, tstar = splat_maximum(prep, px, py)
        live = ((prep["o_hat"] > ALPHA_MIN) & (prep["mu_view"][:, 2] >= view.znear)).unsqueeze(0)
    else:
        rho2, tstar = ray_maximum(prep, px, py)
        live = prep["alive"].unsqueeze(0)
    with torch.no_grad():
        rho2, tstar = rho2.detach(), tstar.detach()
        o_hat = prep["o_hat"].detach()
        rgb = prep["rgb"].detach()
        raw = o_hat.unsqueeze(0) * torch.exp(-0.5 * rho2)
        a_raw = torch.clamp(raw, max=ALPHA_MAX)
        contrib = live & (raw >= ALPHA_MIN) & (tstar >= view.znear)
        touched = raw >= ALPHA_MIN * (1 - rel_alpha)
        near_alpha = (raw - ALPHA_MIN).abs() < rel_alpha * ALPHA_MIN
        near_z = ((tstar - view.znear).abs() < rel_t * view.znear) & touched
        edge_g = (o_hat - ALPHA_MIN).abs() < rel_tau * ALPHA_MIN
        if not eval2d:
            uu = (prep["u_cam"].detach() ** 2).sum(-1)
            tau = prep["tau"].detach()
            edge_g = edge_g | ((uu - tau).abs() < rel_tau * tau.abs())
        flip = ((near_alpha | near_z) & (live | edge_g.unsqueeze(0))) | (touched & edge_g.unsqueeze(0))
        # transmittance in front of every Gaussian at its own depth
        key = torch.where(contrib, tstar, torch.full_like(tstar, math.inf))
        srt = torch.sort(key, dim=1, stable=True)
        m = max(int(contrib.sum(1).max().item()) if contrib.numel() else 0, 1)
        order = srt.indices[:, :m]
        t_s = srt.values[:, :m].contiguous()
        a_s = torch.where(torch.isfinite(t_s), torch.gather(a_raw, 1, order), torch.zeros_like(t_s))
        T_b = torch.cumprod(torch.cat([torch.ones_like(a_s[:, :1]), 1 - a_s], 1), 1)   # [P, m+1]
        pos = torch.searchsorted(t_s, tstar.contiguous(), side="left")                  # [P, G]
        T_at = torch.gather(T_b, 1, pos)
        c_g = rgb.amax(-1).unsqueeze(0)                                                  # [1, G]
        bgmax = float(view.bg.max().item()) if view.bg.numel() else 0.0
        cmax = torch.where(contrib | flip, c_g, torch.zeros_like(c_g)).amax(1)
        cmax = torch.clamp(cmax, min=max(1.0, bgmax))                                    # [P]
        effect = torch.where(flip, a_raw * T_at, torch.zeros_like(a_raw)).sum(1) * cmax
        effect = effect + torch.where(flip.any(1), T_STOP * cmax, torch.zeros_like(cmax))
        # near-tied adjacent contributors
        if m >= 2:
            valid = torch.isfinite(t_s)
            c_s = rgb[order]                                                             # [P,m,3]
            close = valid[:, 1:] & valid[:, :-1] & \
                ((t_s[:, 1:] - t_s[:, :-1]) <= rel_t * t_s[:, :-1].abs())
            sw = T_b[:, :m - 1] * a_s[:, :-1] * a_s[:, 1:] * \
                (c_s[:, :-1, :] - c_s[:, 1:, :]).abs().amax(-1)
            effect = effect + torch.where(close, sw, torch.zeros_like(sw)).sum(1)
    return effect > budget
