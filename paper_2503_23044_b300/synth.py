"""Seeded synthetic workloads for the RGB-Depth-Normal training step.

This module only *produces inputs*: Gaussian / anchor parameters, decoder
weights, cameras, target images and depth priors, and random image-space
gradients for backward tests.  It holds none of the rendering method's
arithmetic (no decoding, projection, blending or loss); both the CUDA path and
the FP64 oracle take what it returns as plain arrays.

Workload shapes follow the paper's captures as restated for one GPU:

* ``explicit_scene``: plain splatting of N explicit Gaussians in front of one
  camera (means uniform in [-1,1]^2 x [2,6] in camera space, log-scales
  N(-3, 0.5), normalised N(0,1) quaternions, opacity logits N(0,1), RGB
  U[0,1]; 256x256 pinhole with fx = fy = 256 and centred principal point).
* ``anchor_scene``: the hybrid anchor representation of Sec. 3.2 -- voxel
  anchors on a K-level grid (Eq. 2 voxelisation of points sampled from a
  synthetic terrain heightfield z = 0.1 * sum_k sin(w_k . (x, y) + phi_k)),
  each with a 32-dim feature ~ N(0, 0.1), a 3-dim log-scale equal to the log
  of its voxel size, and n = 10 offsets ~ N(0, 0.01) (second argument is the
  standard deviation); a 2-layer decoder 35 -> 32 -> 110 with He-uniform
  weights and zero biases.
* aerial and street camera rigs and the analytic ray-marched targets.

All arrays are float32 (int32 for levels); callers upcast for the oracle.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

N_OFFSETS = 10
FEAT_DIM = 32
HIDDEN = 32
IN_DIM = 35            # feature (32) + unit view direction (3)
OUT_DIM = 110          # 10 x (opacity 1 + colour 3 + scale 3 + rotation 4)


@dataclasses.dataclass
class Camera:
    """Pinhole camera, OpenCV frame (x right, y down, z forward).

    ``R`` maps world to camera (row-major 3x3), ``t`` is the translation so
    that x_cam = R x_world + t.
    """

    R: np.ndarray
    t: np.ndarray
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int

    def center(self) -> np.ndarray:
        return (-(self.R.astype(np.float64).T @ self.t.astype(np.float64))).astype(np.float32)


def _f32(x) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(x, dtype=np.float32))


# ---------------------------------------------------------------- cameras
def look_camera(position, yaw: float, pitch_down: float, width: int, height: int,
                hfov_deg: float = 60.0) -> Camera:
    """Camera at ``position`` (world, z up) looking along ``yaw`` and pitched
    ``pitch_down`` radians below the horizon; centred principal point."""
    fwd = np.array([math.cos(pitch_down) * math.cos(yaw),
                    math.cos(pitch_down) * math.sin(yaw),
                    -math.sin(pitch_down)], dtype=np.float64)
    up = np.array([0.0, 0.0, 1.0])
    right = np.cross(fwd, up)
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    R = np.stack([right, down, fwd], axis=0)           # rows: camera axes in world
    pos = np.asarray(position, dtype=np.float64)
    t = -R @ pos
    fx = (width / 2.0) / math.tan(math.radians(hfov_deg) / 2.0)
    return Camera(R=_f32(R), t=_f32(t), fx=float(np.float32(fx)), fy=float(np.float32(fx)),
                  cx=width / 2.0, cy=height / 2.0, width=width, height=height)


def identity_camera(width: int, height: int, f: float) -> Camera:
    return Camera(R=np.eye(3, dtype=np.float32), t=np.zeros(3, np.float32), fx=f, fy=f,
                  cx=width / 2.0, cy=height / 2.0, width=width, height=height)


# ---------------------------------------------------------------- explicit Gaussians
def explicit_scene(n: int = 10_000, seed: int = 0, width: int = 256, height: int = 256,
                   f: float = 256.0, z_range=(2.0, 6.0), log_scale_mean: float = -3.0,
                   log_scale_std: float = 0.5) -> dict:
    rng = np.random.default_rng(seed)
    means = np.concatenate([rng.uniform(-1.0, 1.0, (n, 2)),
                            rng.uniform(z_range[0], z_range[1], (n, 1))], axis=1)
    log_scales = rng.normal(log_scale_mean, log_scale_std, (n, 3))
    q = rng.normal(0.0, 1.0, (n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    opacity_logits = rng.normal(0.0, 1.0, (n,))
    colors = rng.uniform(0.0, 1.0, (n, 3))
    cam = identity_camera(width, height, f)
    return dict(kind="explicit", means=_f32(means), log_scales=_f32(log_scales), quats=_f32(q),
                opacity_logits=_f32(opacity_logits), colors=_f32(colors), cameras=[cam])


# ---------------------------------------------------------------- terrain + anchors
@dataclasses.dataclass
class Terrain:
    omega: np.ndarray      # (8, 2)
    phase: np.ndarray      # (8,)
    amplitude: float = 0.1

    @staticmethod
    def make(rng: np.random.Generator, n_waves: int = 8) -> "Terrain":
        mag = rng.uniform(0.5, 4.0, n_waves)
        ang = rng.uniform(0.0, 2 * math.pi, n_waves)
        omega = np.stack([mag * np.cos(ang), mag * np.sin(ang)], axis=1)
        phase = rng.uniform(0.0, 2 * math.pi, n_waves)
        return Terrain(omega=omega, phase=phase)

    def height(self, x, y):
        xp = np if isinstance(x, np.ndarray) else _torch()
        h = 0.0
        for k in range(self.omega.shape[0]):
            h = h + xp.sin(float(self.omega[k, 0]) * x + float(self.omega[k, 1]) * y + float(self.phase[k]))
        return self.amplitude * h

    def grad(self, x, y):
        """(dh/dx, dh/dy) of the heightfield."""
        xp = np if isinstance(x, np.ndarray) else _torch()
        gx, gy = 0.0, 0.0
        for k in range(self.omega.shape[0]):
            c = xp.cos(float(self.omega[k, 0]) * x + float(self.omega[k, 1]) * y + float(self.phase[k]))
            gx = gx + float(self.omega[k, 0]) * c
            gy = gy + float(self.omega[k, 1]) * c
        return self.amplitude * gx, self.amplitude * gy


def _torch():
    import torch
    return torch


def _round_half_away(v: np.ndarray) -> np.ndarray:
    return np.sign(v) * np.floor(np.abs(v) + 0.5)


def voxelize(points: np.ndarray, voxel: float) -> np.ndarray:
    """Eq. 2 (Sec. 3.2): round P / voxel to the nearest integer (half away
    from zero) and scale back; duplicates removed.  Input construction only."""
    idx = _round_half_away(points / voxel).astype(np.int64)
    idx = np.unique(idx, axis=0)
    return idx.astype(np.float64) * voxel


@dataclasses.dataclass
class SceneSpec:
    name: str
    n_anchors: int
    extent: float
    voxel_sizes: Sequence[float]          # coarse -> fine, level k = index
    lod_d0: float
    views: str                            # "aerial1" | "aerial" | "street" | "close"
    resolutions: Sequence[tuple]
    seed: int = 0


SPECS = {
    # 1 view 1920x1080, 50k anchors on a 0.01 grid (single level).
    "anchor_1080p": SceneSpec("anchor_1080p", 50_000, 2.24, [0.01], 1e9, "aerial1", [(1920, 1080)]),
    # 8 views 1600x1064, 200k anchors x 10 = 2M Gaussians, 3 LoD levels 0.04/0.02/0.01.
    "batch8_1600": SceneSpec("batch8_1600", 200_000, 4.0, [0.04, 0.02, 0.01], 6.0, "aerial",
                             [(1600, 1064)] * 8),
    # 4 views 3840x2160, 500k anchors.
    "batch4_4k": SceneSpec("batch4_4k", 500_000, 6.2, [0.04, 0.02, 0.01], 6.0, "aerial",
                           [(3840, 2160)] * 4),
    # 16 mixed street views, 1M anchors.
    "street16_mixed": SceneSpec("street16_mixed", 1_000_000, 8.8, [0.04, 0.02, 0.01], 0.5, "street",
                                [(960, 540)] * 4 + [(1600, 1064)] * 4 + [(1920, 1080)] * 4
                                + [(3840, 2160)] * 4),
}


def he_uniform(rng: np.random.Generator, fan_out: int, fan_in: int) -> np.ndarray:
    bound = math.sqrt(6.0 / fan_in)
    return rng.uniform(-bound, bound, (fan_out, fan_in))


def make_mlp(rng: np.random.Generator, in_dim: int = IN_DIM) -> dict:
    return dict(W1=_f32(he_uniform(rng, HIDDEN, in_dim)), b1=np.zeros(HIDDEN, np.float32),
                W2=_f32(he_uniform(rng, OUT_DIM, HIDDEN)), b2=np.zeros(OUT_DIM, np.float32))


def _terrain_anchors(rng, terrain: Terrain, extent: float, voxel_sizes, n_anchors: int):
    finest = min(voxel_sizes)
    step = finest / 2.0                       # 2 samples per finest cell per axis (4 per cell)
    m = int(round(extent / step))
    g = (np.arange(m) + 0.5) * step - extent / 2.0
    X, Y = np.meshgrid(g, g, indexing="xy")
    Z = terrain.height(X, Y)
    P = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    per_level = [voxelize(P, v) for v in voxel_sizes]
    counts = np.array([len(c) for c in per_level], dtype=np.float64)
    if counts.sum() < n_anchors:
        raise ValueError(f"terrain yields {int(counts.sum())} voxels < {n_anchors} requested")
    take = np.floor(n_anchors * counts / counts.sum()).astype(np.int64)
    take[-1] += n_anchors - take.sum()
    xs, levels = [], []
    for k, (cells, nk) in enumerate(zip(per_level, take)):
        sel = rng.choice(len(cells), size=int(nk), replace=False)
        sel.sort()
        xs.append(cells[sel])
        levels.append(np.full(int(nk), k, np.int32))
    return np.concatenate(xs, 0), np.concatenate(levels, 0)


def aerial_cameras(rng, terrain: Terrain, extent: float, resolutions, altitude: float = 1.5,
                   grid=(4, 2), pitch_deg=(45.0, 60.0), single: bool = False) -> List[Camera]:
    cams = []
    if single:
        centers = [(0.0, -0.6 * extent / 2.0)]
        pitches = [math.radians(50.0)]
        yaws = [math.pi / 2.0]
    else:
        gx, gy = grid
        centers = [((i + 0.5) / gx * extent - extent / 2.0, (j + 0.5) / gy * extent - extent / 2.0)
                   for j in range(gy) for i in range(gx)]
        pitches = [math.radians(rng.uniform(*pitch_deg)) for _ in centers]
        # views 2i and 2i+1 (neighbours on the grid) fly the same heading within
        # +-15 degrees, like consecutive frames of a sweep, so the view pairs of the
        # batch overlap
        yaws = []
        for k in range(len(centers)):
            yaws.append(rng.uniform(0.0, 2 * math.pi) if k % 2 == 0 else
                        yaws[-1] + rng.uniform(-math.pi / 12.0, math.pi / 12.0))
    for (cx, cy), p, yw, (w, h) in zip(centers, pitches, yaws, resolutions):
        ground = float(terrain.height(np.array(cx), np.array(cy)))
        cams.append(look_camera((cx, cy, ground + altitude), yw, p, w, h))
    return cams


def street_cameras(rng, terrain: Terrain, extent: float, resolutions, height: float = 0.02) -> List[Camera]:
    cams = []
    for (w, h) in resolutions:
        cx, cy = rng.uniform(-0.35 * extent, 0.35 * extent, 2)
        yaw = rng.uniform(0.0, 2 * math.pi)
        pitch = math.radians(rng.uniform(-10.0, 10.0))
        ground = float(terrain.height(np.array(cx), np.array(cy)))
        cams.append(look_camera((cx, cy, ground + height), yaw, pitch, w, h))
    return cams


def anchor_scene(spec: SceneSpec | str, n_anchors: Optional[int] = None, seed: Optional[int] = None,
                 resolutions: Optional[Sequence[tuple]] = None, offset_std: float = 0.01,
                 in_dim: int = IN_DIM) -> dict:
    if isinstance(spec, str):
        spec = SPECS[spec]
    seed = spec.seed if seed is None else seed
    n_anchors = spec.n_anchors if n_anchors is None else n_anchors
    rng = np.random.default_rng(seed)
    terrain = Terrain.make(rng)
    x, level = _terrain_anchors(rng, terrain, spec.extent, spec.voxel_sizes, n_anchors)
    vox = np.asarray(spec.voxel_sizes, dtype=np.float64)[level]
    log_l = np.repeat(np.log(vox)[:, None], 3, axis=1)
    offsets = rng.normal(0.0, offset_std, (n_anchors, N_OFFSETS, 3))
    feat = rng.normal(0.0, 0.1, (n_anchors, FEAT_DIM))
    mlp = make_mlp(rng, in_dim)
    res = list(resolutions if resolutions is not None else spec.resolutions)
    if spec.views == "aerial1":
        cams = aerial_cameras(rng, terrain, spec.extent, res, single=True)
    elif spec.views == "aerial":
        cams = aerial_cameras(rng, terrain, spec.extent, res)
    elif spec.views == "street":
        cams = street_cameras(rng, terrain, spec.extent, res)
    else:
        raise ValueError(spec.views)
    return dict(kind="anchor", x=_f32(x), level=np.ascontiguousarray(level.astype(np.int32)),
                log_l=_f32(log_l), offsets=_f32(offsets), feat=_f32(feat), mlp=mlp, cameras=cams,
                n_levels=len(spec.voxel_sizes), lod_d0=float(spec.lod_d0), terrain=terrain,
                extent=float(spec.extent), name=spec.name)


def tiny_anchor_scene(n_anchors: int = 4, seed: int = 0, width: int = 24, height: int = 20,
                      offset_std: float = 0.3, n_views: int = 1, in_dim: int = IN_DIM) -> dict:
    """A handful of anchors hovering in front of the camera(s): used for the
    finite-difference checks of the oracle and for the smallest GPU cases."""
    rng = np.random.default_rng(seed)
    x = np.concatenate([rng.uniform(-0.25, 0.25, (n_anchors, 2)), rng.uniform(1.6, 2.4, (n_anchors, 1))], 1)
    level = np.zeros(n_anchors, np.int32)
    log_l = np.log(rng.uniform(0.05, 0.09, (n_anchors, 1))).repeat(3, 1)
    offsets = rng.normal(0.0, offset_std, (n_anchors, N_OFFSETS, 3))
    feat = rng.normal(0.0, 1.0, (n_anchors, FEAT_DIM))
    mlp = make_mlp(rng, in_dim)
    f = 0.9 * width
    cams = []
    for v in range(n_views):
        yaw = 0.05 * v
        R = np.array([[math.cos(yaw), 0.0, -math.sin(yaw)], [0.0, 1.0, 0.0], [math.sin(yaw), 0.0, math.cos(yaw)]])
        cams.append(Camera(R=_f32(R), t=_f32([0.03 * v, -0.02 * v, 0.0]), fx=f, fy=f, cx=width / 2.0,
                           cy=height / 2.0, width=width, height=height))
    return dict(kind="anchor", x=_f32(x), level=level, log_l=_f32(log_l), offsets=_f32(offsets),
                feat=_f32(feat), mlp=mlp, cameras=cams, n_levels=1, lod_d0=1e9, terrain=None,
                name="tiny")


# ---------------------------------------------------------------- targets
def texture(x, y):
    xp = np if isinstance(x, np.ndarray) else _torch()
    r = 0.5 + 0.4 * xp.sin(7.0 * x) * xp.cos(5.0 * y)
    g = 0.5 + 0.4 * xp.sin(3.0 * x + 11.0 * y)
    b = 0.5 + 0.4 * xp.cos(13.0 * x - 2.0 * y)
    return r, g, b


def march_targets(terrain: Terrain, cam: Camera, stride: int = 4, t_max: float = 40.0,
                  dt: float = 0.02, device: str = "cpu", seed: int = 0) -> dict:
    """Analytic ray-march of the heightfield (independent of both renderers).

    Returns target RGB [3,H,W], true z-depth [H,W], depth prior
    z * (1 + N(0, 0.02)) [H,W], a {0,1} mask of rays that hit and the unit
    surface normal in the camera frame, facing the camera [3,H,W] (0 where
    the ray misses).  Rays are
    marched at every ``stride``-th pixel and the result is held over the
    stride x stride block (the target only shapes the loss workload).
    """
    import torch
    W, H = cam.width, cam.height
    ws, hs = (W + stride - 1) // stride, (H + stride - 1) // stride
    us = (torch.arange(ws, device=device, dtype=torch.float64) * stride + 0.5)
    vs = (torch.arange(hs, device=device, dtype=torch.float64) * stride + 0.5)
    V, U = torch.meshgrid(vs, us, indexing="ij")
    dcam = torch.stack([(U - cam.cx) / cam.fx, (V - cam.cy) / cam.fy, torch.ones_like(U)], -1)
    R = torch.tensor(cam.R, dtype=torch.float64, device=device)
    o = torch.tensor(cam.center(), dtype=torch.float64, device=device)
    dw = dcam @ R                                   # world direction (per unit camera z)
    n = dw.shape[0] * dw.shape[1]
    dw = dw.reshape(n, 3)
    t_hit = torch.full((n,), float("nan"), dtype=torch.float64, device=device)
    prev_t = torch.zeros(n, dtype=torch.float64, device=device)
    prev_s = o[2] - terrain.height(o[0].expand(n), o[1].expand(n))
    active = torch.ones(n, dtype=torch.bool, device=device)
    t = 0.0
    while t < t_max and bool(active.any()):
        t += dt
        p = o + t * dw
        s = p[:, 2] - terrain.height(p[:, 0], p[:, 1])
        hit = active & (s <= 0)
        if bool(hit.any()):
            lo, hi = prev_t[hit], torch.full_like(prev_t[hit], t)
            for _ in range(30):
                mid = 0.5 * (lo + hi)
                pm = o + mid[:, None] * dw[hit]
                sm = pm[:, 2] - terrain.height(pm[:, 0], pm[:, 1])
                below = sm <= 0
                hi = torch.where(below, mid, hi)
                lo = torch.where(below, lo, mid)
            t_hit[hit] = hi
            active = active & ~hit
        prev_t = torch.full_like(prev_t, t)
        prev_s = s
    mask = ~torch.isnan(t_hit)
    th = torch.where(mask, t_hit, torch.zeros_like(t_hit))
    P = o + th[:, None] * dw
    r, g, b = texture(P[:, 0], P[:, 1])
    rgb = torch.stack([r, g, b], 0) * mask
    depth = th                                      # dcam has unit camera z, so t is z-depth
    gen = torch.Generator(device="cpu").manual_seed(seed)
    noise = torch.randn(n, generator=gen, dtype=torch.float64).to(device)
    prior = depth * (1.0 + 0.02 * noise) * mask
    gx, gy = terrain.grad(P[:, 0], P[:, 1])
    nw = torch.stack([-gx, -gy, torch.ones_like(gx)], 1)
    nc = (nw / nw.norm(dim=1, keepdim=True)) @ R.T          # camera frame
    nc = torch.where(((nc * dcam.reshape(n, 3)).sum(1) > 0)[:, None], -nc, nc)
    normal = nc.T * mask

    def up(a):
        a = a.reshape(-1, hs, ws)
        a = a.repeat_interleave(stride, 1).repeat_interleave(stride, 2)
        return a[:, :H, :W]

    return dict(rgb=up(rgb).float().contiguous(), depth=up(depth * mask)[0].float().contiguous(),
                prior=up(prior)[0].float().contiguous(), mask=up(mask.double())[0].float().contiguous(),
                normal=up(normal).float().contiguous())


def constant_targets(cam: Camera, rgb: float = 0.5, depth: float = 4.0) -> dict:
    import torch
    H, W = cam.height, cam.width
    return dict(rgb=torch.full((3, H, W), rgb), depth=torch.full((H, W), depth),
                prior=torch.full((H, W), depth), mask=torch.ones(H, W))


def random_image_grads(cams: Sequence[Camera], seed: int, scale: float = 1e-3,
                       crops: Optional[Sequence[tuple]] = None) -> List[dict]:
    """Seeded dL/d(RGB, depth, normal) per view for backward tests; optional
    crop (x0, y0, w, h) per view zeroes everything outside it."""
    import torch
    gen = torch.Generator().manual_seed(seed)
    out = []
    for i, cam in enumerate(cams):
        H, W = cam.height, cam.width
        g = dict(rgb=torch.randn(3, H, W, generator=gen) * scale,
                 depth=torch.randn(H, W, generator=gen) * scale,
                 normal=torch.randn(3, H, W, generator=gen) * scale)
        if crops is not None:
            x0, y0, w, h = crops[i]
            m = torch.zeros(H, W)
            m[y0:y0 + h, x0:x0 + w] = 1.0
            g = {k: v * m for k, v in g.items()}
        out.append(g)
    return out


def random_maps(cams: Sequence[Camera], seed: int) -> List[dict]:
    """Random rendered-like maps (RGB, unbiased depth, raw distance, normal)
    for loss tests: depth ~ U[1, 5], normals facing the camera."""
    import torch
    gen = torch.Generator().manual_seed(seed)
    out = []
    for cam in cams:
        H, W = cam.height, cam.width
        rgb = torch.rand(3, H, W, generator=gen)
        depth = 1.0 + 4.0 * torch.rand(H, W, generator=gen)
        n = torch.randn(3, H, W, generator=gen) * 0.3
        n[2] = -1.0 + n[2] * 0.1
        out.append(dict(rgb=rgb, depth=depth, normal=n))
    return out


# ---------------------------------------------------------------- depth-prior inputs (Sec. 3.4, Step 2)
def sparse_points(terrain: Terrain, extent: float, n: int, seed: int = 0, noise: float = 0.0) -> np.ndarray:
    """Stand-in for the sparse SfM cloud: n points on the heightfield over the
    scene extent (optionally jittered by N(0, noise) per axis), float32 [n, 3]."""
    rng = np.random.default_rng(seed)
    xy = rng.uniform(-extent / 2.0, extent / 2.0, (n, 2))
    z = terrain.height(xy[:, 0], xy[:, 1])
    p = np.concatenate([xy, z[:, None]], 1)
    if noise > 0:
        p = p + rng.normal(0.0, noise, p.shape)
    return _f32(p)


def pseudo_depth(true_depth, valid, seed: int = 0, noise: float = 5e-4, n_blobs: int = 3,
                 blob_radius=(0.05, 0.12), blob_factor=(1.3, 1.8)):
    """Stand-in for a monocular depth estimate of one view: the true z-depth with
    relative noise N(0, noise), wrong by a factor U[blob_factor] inside n_blobs
    discs (radius a fraction of the image width), then expressed in an unknown
    affine frame, D_p = (z - t) / s with s ~ U[0.5, 2], t ~ U[-0.5, 0.5]; 0 where
    there is no depth.  Returns (D_p [H, W] float32 tensor, s, t, blob mask)."""
    import torch
    gen = torch.Generator().manual_seed(seed)
    z = torch.as_tensor(true_depth, dtype=torch.float64).cpu()
    ok = torch.as_tensor(valid).cpu().bool()
    H, W = z.shape
    z = z * (1.0 + noise * torch.randn(H, W, generator=gen, dtype=torch.float64))
    blob = torch.zeros(H, W, dtype=torch.bool)
    vv, uu = torch.meshgrid(torch.arange(H, dtype=torch.float64), torch.arange(W, dtype=torch.float64), indexing="ij")
    for _ in range(n_blobs):
        cx = float(torch.rand(1, generator=gen)) * W
        cy = float(torch.rand(1, generator=gen)) * H
        r = (blob_radius[0] + (blob_radius[1] - blob_radius[0]) * float(torch.rand(1, generator=gen))) * W
        f = blob_factor[0] + (blob_factor[1] - blob_factor[0]) * float(torch.rand(1, generator=gen))
        disc = (uu - cx) ** 2 + (vv - cy) ** 2 <= r * r
        z = torch.where(disc, z * f, z)
        blob |= disc
    s = 0.5 + 1.5 * float(torch.rand(1, generator=gen))
    t = -0.5 + float(torch.rand(1, generator=gen))
    dp = torch.where(ok, (z - t) / s, torch.zeros_like(z))
    dp = torch.where(ok & (dp > 0), dp, torch.zeros_like(dp))
    return dp.float(), s, t, blob & ok
