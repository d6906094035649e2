"""Seeded synthetic scenes shaped like the paper's indoor RGB-D mapping workloads.

The paper evaluates on Replica (1200x680), TUM-RGBD (640x480) and VECtor
(Sec. IV-A); none of these datasets is used here. These generators stand in
for them with the same image sizes, Gaussian counts (Tables I-II report
38k-2M Gaussians) and structure (Gaussians on the walls and floor of a room,
an inward-looking camera trajectory). Everything is drawn from
``numpy.random.default_rng(seed)`` (PCG64) and stored as float32.

This module only draws and lays out random numbers. It holds none of the
method's arithmetic: target images are rendered by whoever consumes the scene
(the CUDA path in the benchmark, the oracle in tests).

Parameter layout (one flat float32 vector, group after group, Sec. III-B
lists the per-primitive attributes p, q, s, sigma, SH):

    means[n][3] | log_scales[n][3] | quats[n][4] (w, x, y, z) |
    opacity_logits[n] | sh_dc[n][3] | sh_rest[n][K-1][3]

with K = (degree + 1)^2 SH coefficients per colour channel.

Camera layout (float32[V][20]): R[9] (world->camera rotation, row-major),
t[3] (world->camera translation), fx, fy, cx, cy, loss weight, 3 x padding.
Camera frame: x right, y down, z forward (pinhole, pixel (x, y) centred on
integer coordinates).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

CAM_FLOATS = 20

# Standard deviation of the degree-0 SH coefficient that makes the DC colour
# N(0.5, 0.2): the zeroth real SH basis function is the constant 1/(2 sqrt(pi)).
_Y00 = 0.28209479177387814

CONFIG_NAMES = {
    1: "single_view_2k_sh0_160x120",
    2: "single_view_100k_sh3_1200x680",
    3: "diffcheck_5k_sh1_320x240",
    4: "window8_200k_sh3_640x480",
    5: "window16_300k_sh3_1200x680",
}


def param_layout(n: int, sh_degree: int) -> dict:
    """Offsets (in floats) of each parameter group in the flat vector."""
    K = (sh_degree + 1) ** 2
    lay = {
        "means": 0,
        "log_scales": 3 * n,
        "quats": 6 * n,
        "opacity": 10 * n,
        "sh_dc": 11 * n,
        "sh_rest": 14 * n,
        "total": 14 * n + 3 * (K - 1) * n,
    }
    return lay


@dataclass
class Scene:
    name: str
    n: int
    sh_degree: int
    width: int
    height: int
    tile: int
    params: np.ndarray          # float32 flat, see module docstring
    params_target: np.ndarray   # seed-perturbed copy used to render targets
    cams: np.ndarray            # float32 [V, 20]
    lr: tuple = (1e-3,) * 6     # per group: means, log_scales, quats, opacity, sh_dc, sh_rest
    meta: dict = field(default_factory=dict)

    @property
    def views(self) -> int:
        return int(self.cams.shape[0])

    def group(self, name: str, params: np.ndarray | None = None) -> np.ndarray:
        """View of one parameter group, shaped [n, ...]."""
        p = self.params if params is None else params
        lay = param_layout(self.n, self.sh_degree)
        K = (self.sh_degree + 1) ** 2
        shapes = {"means": (3,), "log_scales": (3,), "quats": (4,), "opacity": (),
                  "sh_dc": (3,), "sh_rest": (K - 1, 3)}
        width = int(np.prod(shapes[name])) if shapes[name] else 1
        a = p[lay[name]: lay[name] + width * self.n]
        return a.reshape((self.n,) + shapes[name])


def _camera_row(R: np.ndarray, t: np.ndarray, fx, fy, cx, cy, weight=1.0) -> np.ndarray:
    row = np.zeros(CAM_FLOATS, dtype=np.float64)
    row[0:9] = R.reshape(-1)
    row[9:12] = t
    row[12:17] = (fx, fy, cx, cy, weight)
    return row.astype(np.float32)


def look_at(pos, target, world_up=(0.0, 1.0, 0.0)):
    """World->camera (R, t) for a camera at `pos` looking at `target`.

    Camera axes: x right, y down, z forward; world y is up.
    """
    pos = np.asarray(pos, np.float64)
    f = np.asarray(target, np.float64) - pos
    f /= np.linalg.norm(f)
    down = -np.asarray(world_up, np.float64)
    right = np.cross(down, f)
    right /= np.linalg.norm(right)
    down = np.cross(f, right)
    R = np.stack([right, down, f])
    t = -R @ pos
    return R, t


def _gaussian_attributes(rng, n, sh_degree, opacity_mean=0.0, opacity_std=1.0,
                         log_scale_mean=-3.5, log_scale_std=0.5, rest_std=0.05):
    log_scales = rng.normal(log_scale_mean, log_scale_std, size=(n, 3))
    q = rng.normal(0.0, 1.0, size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    opac = rng.normal(opacity_mean, opacity_std, size=n)
    sh_dc = rng.normal(0.0, 0.2 / _Y00, size=(n, 3))
    K = (sh_degree + 1) ** 2
    sh_rest = rng.normal(0.0, rest_std, size=(n, K - 1, 3))
    return log_scales, q, opac, sh_dc, sh_rest


def _pack(means, log_scales, quats, opac, sh_dc, sh_rest) -> np.ndarray:
    parts = [means.reshape(-1), log_scales.reshape(-1), quats.reshape(-1),
             opac.reshape(-1), sh_dc.reshape(-1), sh_rest.reshape(-1)]
    return np.concatenate(parts).astype(np.float32)


def _perturbed(rng, params: np.ndarray, n: int, std=0.01) -> np.ndarray:
    out = params.copy()
    out[: 3 * n] += rng.normal(0.0, std, size=3 * n).astype(np.float32)
    return out


def _room_means(rng, n):
    """70% on the floor and four walls of a 6x5x3 m room (area-weighted, N(0, 0.02) m
    jitter along the normal), 30% uniform in the interior.  World y is up; the room spans
    x in [-3, 3], y in [0, 3], z in [-2.5, 2.5]."""
    n_surf = int(round(0.7 * n))
    n_int = n - n_surf
    areas = np.array([6 * 5, 5 * 3, 5 * 3, 6 * 3, 6 * 3], np.float64)
    which = rng.choice(5, size=n_surf, p=areas / areas.sum())
    a = rng.uniform(0.0, 1.0, size=n_surf)
    b = rng.uniform(0.0, 1.0, size=n_surf)
    jit = rng.normal(0.0, 0.02, size=n_surf)
    pts = np.zeros((n_surf, 3))
    # floor y = 0
    m = which == 0
    pts[m] = np.stack([-3 + 6 * a[m], jit[m], -2.5 + 5 * b[m]], 1)
    for k, xs in ((1, -3.0), (2, 3.0)):          # walls x = +-3
        m = which == k
        pts[m] = np.stack([xs + jit[m], 3 * a[m], -2.5 + 5 * b[m]], 1)
    for k, zs in ((3, -2.5), (4, 2.5)):          # walls z = +-2.5
        m = which == k
        pts[m] = np.stack([-3 + 6 * a[m], 3 * b[m], zs + jit[m]], 1)
    interior = np.stack([rng.uniform(-3, 3, n_int), rng.uniform(0, 3, n_int),
                         rng.uniform(-2.5, 2.5, n_int)], 1)
    allp = np.concatenate([pts, interior], 0)
    return allp[rng.permutation(n)]


def _ellipse_cams(V, W, H, f, cx, cy, start=0):
    """Cameras on an ellipse (2.0 x 1.5 m, height 1.4 m) looking at the room centre."""
    rows = []
    for i in range(V):
        th = 2.0 * np.pi * (start + i) / max(V, 1)
        pos = (2.0 * np.cos(th), 1.4, 1.5 * np.sin(th))
        R, t = look_at(pos, (0.0, 1.5, 0.0))
        rows.append(_camera_row(R, t, f, f, cx, cy))
    return np.stack(rows)


# The 8-view window's path (2 m along the room's long axis z, 1.6 m high, pitched down by
# 0.15): it starts 2.35 m behind the back wall (z = -2.5; the cameras look into the room
# over it) and ends 0.35 m behind it, while the yaw turns from straight down the room
# (0) to 1.5 rad (a side wall).  Chosen once by a search over the start and the yaw span
# so that the per-view visible counts of the 200k-Gaussian room fall from about 150k to
# about 20k: 151.7k, 130.7k, 108.8k, 86.1k, 65.3k, 44.0k, 28.5k, 20.9k.
_PATH_Z0, _PATH_LEN, _PATH_Y, _PATH_PITCH, _PATH_YAW_END = -4.85, 2.0, 1.6, -0.15, 1.5


def _path_cams(V, W, H, f, cx, cy):
    """Cameras on the 2 m straight path with the yaw sweep above (evenly spaced)."""
    rows = []
    for i in range(V):
        a = i / max(V - 1, 1)
        pos = np.array([0.0, _PATH_Y, _PATH_Z0 + _PATH_LEN * a])
        yaw = _PATH_YAW_END * a
        fwd = np.array([np.sin(yaw), _PATH_PITCH, np.cos(yaw)])
        R, t = look_at(pos, pos + fwd)
        rows.append(_camera_row(R, t, f, f, cx, cy))
    return np.stack(rows)


def _box_scene(rng, n, sh_degree, name, W, H, f, cx, cy, tile):
    means = np.stack([rng.uniform(-2, 2, n), rng.uniform(-1.5, 1.5, n),
                      rng.uniform(1, 4, n)], 1)
    attrs = _gaussian_attributes(rng, n, sh_degree)
    params = _pack(means, *attrs)
    target = _perturbed(rng, params, n)
    cams = np.stack([_camera_row(np.eye(3), np.zeros(3), f, f, cx, cy)])
    return Scene(name, n, sh_degree, W, H, tile, params, target, cams)


def make_scene(config: int, seed: int = 0, n: int | None = None, views: int | None = None) -> Scene:
    """The five workload shapes (1-5). `n` / `views` override the size for scaled-down
    parity cases that keep the same distributions."""
    rng = np.random.default_rng(seed)
    name = CONFIG_NAMES[config]
    if config == 1:
        return _box_scene(rng, n or 2000, 0, name, 160, 120, 150.0, 80.0, 60.0, 16)
    if config == 3:
        return _box_scene(rng, n or 5000, 1, name, 320, 240, 300.0, 159.5, 119.5, 16)
    if config == 2:
        n = n or 100_000
        W, H, f = 1200, 680, 600.0
        means = _room_means(rng, n)
        attrs = _gaussian_attributes(rng, n, 3)
        params = _pack(means, *attrs)
        target = _perturbed(rng, params, n)
        cams = _ellipse_cams(1, W, H, f, 599.5, 339.5)
        lr = _room_lr()
        return Scene(name, n, 3, W, H, 16, params, target, cams, lr)
    if config == 4:
        n = n or 200_000
        V = views or 8
        W, H, f = 640, 480, 525.0
        means = _room_means(rng, n)
        attrs = _gaussian_attributes(rng, n, 3)
        params = _pack(means, *attrs)
        target = _perturbed(rng, params, n)
        cams = _path_cams(V, W, H, f, 319.5, 239.5)
        return Scene(name, n, 3, W, H, 16, params, target, cams, _room_lr())
    if config == 5:
        n = n or 300_000
        V = views or 16
        W, H, f = 1200, 680, 600.0
        means = _room_means(rng, n)
        attrs = _gaussian_attributes(rng, n, 3, opacity_mean=-1.0, opacity_std=1.5)
        params = _pack(means, *attrs)
        target = _perturbed(rng, params, n)
        cams = _ellipse_cams(V, W, H, f, 599.5, 339.5)
        return Scene(name, n, 3, W, H, 16, params, target, cams, _room_lr())
    raise ValueError(f"unknown config {config}")


def _room_lr():
    """Per-group learning rates in the 3DGS defaults' proportions (the paper keeps most
    3DGS hyper-parameters, Sec. IV-A): means, log_scales, quats, opacity, sh_dc, sh_rest."""
    return (1.6e-4, 5e-3, 1e-3, 2.5e-2, 2.5e-3, 2.5e-3 / 20.0)


def make_tiny_scene(seed: int = 0, n: int = 40, sh_degree: int = 1, W: int = 32, H: int = 24,
                    views: int = 2, tile: int = 8, opacity_mean: float = 0.0) -> Scene:
    """A few dozen Gaussians seen by `views` small cameras (finite-difference scale)."""
    rng = np.random.default_rng(seed)
    means = np.stack([rng.uniform(-1.0, 1.0, n), rng.uniform(-0.75, 0.75, n),
                      rng.uniform(2.0, 4.0, n)], 1)
    attrs = _gaussian_attributes(rng, n, sh_degree, opacity_mean=opacity_mean,
                                 log_scale_mean=-1.8, log_scale_std=0.3, rest_std=0.2)
    params = _pack(means, *attrs)
    target = _perturbed(rng, params, n, std=0.05)
    f = 0.9 * W
    rows = []
    for v in range(views):
        # small sideways offsets and yaw so the views differ
        yaw = 0.08 * v
        pos = np.array([0.15 * v, -0.05 * v, 0.0])
        fwd = np.array([np.sin(yaw), 0.0, np.cos(yaw)])
        R, t = look_at(pos, pos + fwd, world_up=(0.0, -1.0, 0.0))
        rows.append(_camera_row(R, t, f, f, W / 2.0 - 0.5, H / 2.0 - 0.5))
    return Scene(f"tiny_{n}_sh{sh_degree}_{W}x{H}_v{views}", n, sh_degree, W, H, tile,
                 params, target, np.stack(rows))


def make_records(seed: int, views: int, n: int, W: int, H: int, cull_frac: float = 0.2,
                 max_radius: int = 40, depth_ties: float = 0.05):
    """Synthetic projected positions, radii and depths for testing the binning sort on
    its own: u, v spread over the image plus a margin, integer radii, fp32 depths with
    a share of exact ties and a share of positions on tile boundaries."""
    rng = np.random.default_rng(seed)
    m = views * n
    u = rng.uniform(-2 * max_radius, W + 2 * max_radius, m).astype(np.float32)
    v = rng.uniform(-2 * max_radius, H + 2 * max_radius, m).astype(np.float32)
    snap = rng.uniform(0, 1, m) < 0.05
    u[snap] = np.round(u[snap] / 16.0) * 16.0
    v[snap] = np.round(v[snap] / 16.0) * 16.0
    radius = rng.integers(1, max_radius + 1, m).astype(np.int32)
    radius[rng.uniform(0, 1, m) < cull_frac] = 0
    z = rng.uniform(0.25, 10.0, m).astype(np.float32)
    tie = rng.uniform(0, 1, m) < depth_ties
    z[tie] = z[0] if m else 1.0
    return u, v, radius, z


def make_conics(seed: int, radius, opacity_low: float = 0.002):
    """Per record an inverse covariance (A, B, C), float32: an ellipse whose larger
    3-sigma half-axis is about the record's radius, random aspect (0.05-1) and rotation;
    and an opacity, uniform in [opacity_low, 0.99] (some below 1/255)."""
    rng = np.random.default_rng(seed)
    r = np.maximum(np.asarray(radius, np.float64), 1.0)
    m = r.size
    lmax = (r / 3.0) ** 2
    lmin = lmax * rng.uniform(0.05, 1.0, m)
    th = rng.uniform(0, np.pi, m)
    c, s = np.cos(th), np.sin(th)
    sxx = c * c * lmax + s * s * lmin
    syy = s * s * lmax + c * c * lmin
    sxy = c * s * (lmax - lmin)
    det = sxx * syy - sxy * sxy
    conic = np.stack([syy / det, -sxy / det, sxx / det], 1).astype(np.float32)
    opacity = rng.uniform(opacity_low, 0.99, m).astype(np.float32)
    return conic, opacity


def make_point_cloud(seed: int, m: int, dup_frac: float = 0.01, outliers: int = 2):
    """A keyframe's coloured point cloud for geometric densification: m points of the
    6x5x3 m room (surfaces and interior as the room scenes), float32 xyz and rgb in [0, 1].
    A share of points repeats another point exactly (as quantised depth back-projects
    neighbouring pixels onto one point), and a few lie far outside the room."""
    rng = np.random.default_rng(seed)
    xyz = _room_means(rng, m)
    rgb = rng.uniform(0.0, 1.0, (m, 3))
    nd = int(dup_frac * m) if m > 1 else 0
    if nd:
        src = rng.integers(0, m, nd)
        dst = rng.integers(0, m, nd)
        xyz[dst] = xyz[src]
    for i in range(min(outliers, m)):
        xyz[rng.integers(0, m)] = rng.uniform(-40.0, 40.0, 3)
    return xyz.astype(np.float32), rgb.astype(np.float32)
