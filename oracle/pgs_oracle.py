"""Plain FP64 CPU oracle of the batch-level RGB-Depth-Normal training step.

TEST INFRASTRUCTURE ONLY: imported by tests/, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline leg; never by the product path.

What it computes (CityGS-X, Sec. 3.1-3.4), in the paper's order and without
tiling, blocking or fusion:

1. LoD selection of anchors by observation distance (Sec. 3.1, Octree-GS
   paragraph), with the cumulative rule ``level <= clamp(floor(log2(d0/d)),
   0, K-1)``.  No frustum pre-cull: every LoD-active anchor is decoded.
2. The shared Gaussian decoder F_de (Eq. 4): mu_n = x_v + O_n * l_v and
   {alpha, c, Sigma} = F_de(F_v, view direction).
3. EWA projection of every Gaussian (3DGS, cited in Sec. 3.1), the normal as
   the smallest-scale axis in the camera frame facing the camera (Eq. 6) and
   the plane distance d = n . mu_c (Eq. 7).
4. For every pixel centre, all surviving Gaussians of the view in (depth,
   index) order, blended front to back (Eq. 1 / Eq. 5) into RGB, D and N
   (Eq. 6-7), then the unbiased depth D_hat = D / (N . K^-1 p~) (Eq. 7).
5. The batch losses: RGB L1 (Eq. 8), depth L1 against a prior (Eq. 9) and a
   normal-depth consistency term.
6. Gradients: reverse-mode differentiation of steps 2-5 by torch.autograd
   in FP64 (the exact derivative of this definition, not a hand derivation).
7. The enhanced depth prior of Step 2 (Sec. 3.4): least-squares scale and
   shift of a pseudo depth to sparse points, the round-trip re-projection
   error through the nearest batch views and the tau_d filter.
8. The batch geometric NCC of Step 3 (Eq. 10): view pairs, 7 x 7 patches
   warped by the plane homography of the rendered depth and normal, 1 - NCC,
   with the stop-gradient on the partner (autograd, as in 6).
9. The projective TSDF fusion of rendered depth and colour (supplementary,
   mesh reconstruction).
Each of 7-9 states its reading of the paper in its own section below.

Readings of the paper where it is silent (all parameters of ``RenderParams``):
EWA with 0.3 px^2 dilation and J clamped at 1.3 * tan(fov/2); alpha =
min(0.99, o * exp(power)); pairs with alpha < 1/255 or power > 0 skipped; a
pixel stops before the Gaussian that would take T below 1e-4; background 0;
decoder outputs blocked [alpha x10 | colour x30 | scale x30 | quat x40] with
sigmoid / sigmoid / l * sigmoid / normalise; quaternions (w, x, y, z).

Besides images and gradients the oracle returns *ambiguity flags*: pixels
where an FP32 evaluation may legitimately take another branch of one of the
discrete rules above (a value within rounding of a threshold, or two
contributing depths within rounding of each other).  Parity tests compare
only unflagged pixels and report the flagged fraction.

The integer helpers at the end (tile sets, stable sort, exclusive scan, tile
ranges) are the textbook definitions the GPU's binning and sort must equal.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional, Sequence

import numpy as np
import torch

DT = torch.float64
N_OFF = 10
# Relative reach of an FP32 evaluation around the alpha thresholds, the
# transmittance stop and the per-Gaussian discrete choices: pixels with a
# decision inside it are flagged ambiguous.
AMB_ALPHA = 5e-5
AMB_T = 1e-4
AMB_GAUSS = 1e-6


@dataclasses.dataclass
class RenderParams:
    decode: str = "fp64"            # decoder arithmetic: "fp64", "bf16" or "bf16_1pass" (see ``decode``)
    near: float = 0.01
    dilation: float = 0.3
    alpha_min: float = 1.0 / 255.0
    alpha_max: float = 0.99
    t_min: float = 1e-4
    jclamp: float = 1.3
    tile: int = 16
    tile_pad: float = 1e-3          # padding of the tile-list level set, in ln units
    lod_d0: float = 1e9
    n_levels: int = 1
    bg: float = 0.0


@dataclasses.dataclass
class LossParams:
    lambda_depth: float = 1.0
    lambda_normal: float = 0.1


def _t(a) -> torch.Tensor:
    if isinstance(a, torch.Tensor):
        return a.cpu().to(DT)
    return torch.as_tensor(np.asarray(a), dtype=DT)


def camera(cam) -> dict:
    R = _t(cam.R).reshape(3, 3)
    t = _t(cam.t).reshape(3)
    return dict(R=R, t=t, fx=float(cam.fx), fy=float(cam.fy), cx=float(cam.cx), cy=float(cam.cy),
                W=int(cam.width), H=int(cam.height), center=-(R.T @ t))


# ------------------------------------------------------------------ rotations
def normalize_quat(q: torch.Tensor) -> torch.Tensor:
    """Unit quaternion; a (near-)zero vector maps to the identity rotation."""
    n = torch.linalg.norm(q, dim=-1, keepdim=True)
    ident = torch.zeros_like(q)
    ident[..., 0] = 1.0
    small = n < 1e-12
    return torch.where(small, ident, q / torch.where(small, torch.ones_like(n), n))


def quat_to_rotmat(q: torch.Tensor) -> torch.Tensor:
    """Rotation matrix of a unit quaternion (w, x, y, z); columns are the
    Gaussian's local axes expressed in world coordinates."""
    w, x, y, z = q.unbind(-1)
    R = torch.stack([
        1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
        2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
        2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1)
    return R.reshape(q.shape[:-1] + (3, 3))


# ------------------------------------------------------------------ LoD (Sec. 3.1)
def lod_active(x: torch.Tensor, level: torch.Tensor, cam: dict, rp: RenderParams):
    """Anchor at level k is active for this camera iff k <= L(d),
    L(d) = clamp(floor(log2(d0 / d)), 0, K-1), d = |x - camera centre|.
    Written as comparisons against the exact thresholds d0 / 2^m.
    Returns (active, ambiguous): ambiguous marks d within 1e-5 relative of a
    threshold, where an FP32 distance may fall on the other side."""
    d = torch.linalg.norm(x - cam["center"], dim=-1)
    L = torch.zeros_like(level)
    amb = torch.zeros_like(level, dtype=torch.bool)
    for m in range(1, rp.n_levels):
        thr = rp.lod_d0 / (2.0 ** m)
        L = L + (d <= thr).to(level.dtype)
        amb |= (d - thr).abs() <= 1e-5 * thr
    return level <= L, amb


# ------------------------------------------------------------------ decoder (Eq. 4)
def bf16_round(x: torch.Tensor) -> torch.Tensor:
    """Round to the nearest BF16 value (8 significant bits, ties to even),
    computed in FP64 as the definition: x = m 2^e with 0.5 <= |m| < 1, keep
    round(m 2^8) / 2^8.  The gradient passes straight through (d round(x)/dx
    taken as 1), which is the gradient of the rounded forward's arithmetic."""
    xd = x.detach()
    m, e = torch.frexp(xd)
    r = torch.ldexp(torch.round(m * 256.0) / 256.0, e)       # torch.round: half to even
    return x + (r - xd)


def decode(anchors: dict, mlp: dict, cam: dict, idx: torch.Tensor, in_dim: int = 35,
           precision: str = "fp64") -> dict:
    """Decode the anchors ``idx`` into n = 10 neural Gaussians each.

    Input X = [F_v (32), unit direction (x_v - o_c)/|.| (3)] (+ distance if
    ``in_dim`` = 36); H = ReLU(W1 X + b1); Z = W2 H + b2 (110).

    The paper states no precision for F_de.  ``precision`` selects the
    arithmetic the GPU's decoder forms define, emulated in FP64:
    "fp64" exact; "bf16" the colour outputs Z[10:40] from BF16-rounded H and
    W2 (one BF16 pass), everything else exact; "bf16_1pass" X, W1, H and W2
    all rounded to BF16 before their products (biases exact)."""
    x = anchors["x"][idx]
    F = anchors["feat"][idx]
    l = torch.exp(anchors["log_l"][idx])
    O = anchors["offsets"][idx]
    dvec = x - cam["center"]
    dist = torch.linalg.norm(dvec, dim=-1, keepdim=True)
    parts = [F, dvec / dist]
    if in_dim == 36:
        parts.append(dist)
    X = torch.cat(parts, -1)
    if precision == "bf16_1pass":
        H = torch.relu(bf16_round(X) @ bf16_round(mlp["W1"]).T + mlp["b1"])
        Z = bf16_round(H) @ bf16_round(mlp["W2"]).T + mlp["b2"]
    else:
        H = torch.relu(X @ mlp["W1"].T + mlp["b1"])
        Z = H @ mlp["W2"].T + mlp["b2"]
        if precision == "bf16":
            Zc = bf16_round(H) @ bf16_round(mlp["W2"][10:40]).T + mlp["b2"][10:40]
            Z = torch.cat([Z[:, :10], Zc, Z[:, 40:]], 1)
        elif precision != "fp64":
            raise ValueError(f"decoder precision {precision!r}")
    A = x.shape[0]
    opacity = torch.sigmoid(Z[:, 0:10])
    color = torch.sigmoid(Z[:, 10:40]).reshape(A, N_OFF, 3)
    scale = l[:, None, :] * torch.sigmoid(Z[:, 40:70]).reshape(A, N_OFF, 3)
    quat = normalize_quat(Z[:, 70:110].reshape(A, N_OFF, 4))
    mu = x[:, None, :] + O * l[:, None, :]
    return dict(mu=mu.reshape(-1, 3), opacity=opacity.reshape(-1), color=color.reshape(-1, 3),
                scale=scale.reshape(-1, 3), quat=quat.reshape(-1, 4), X=X, H=H, Z=Z)


# ------------------------------------------------------------------ projection
def project(mu, scale, quat, opacity, color, cam: dict, rp: RenderParams) -> dict:
    """EWA splatting of 3D Gaussians (3DGS): 2D mean, 2D covariance with
    dilation, its inverse (conic), view depth z, camera-frame normal facing
    the camera (Eq. 6 reading) and plane distance d = n . mu_c (Eq. 7)."""
    R, t = cam["R"], cam["t"]
    fx, fy, cx, cy, W, H = cam["fx"], cam["fy"], cam["cx"], cam["cy"], cam["W"], cam["H"]
    mu_c = mu @ R.T + t
    x, y, z = mu_c.unbind(-1)
    lim_x = rp.jclamp * 0.5 * W / fx
    lim_y = rp.jclamp * 0.5 * H / fy
    txz = torch.clamp(x / z, -lim_x, lim_x)
    tyz = torch.clamp(y / z, -lim_y, lim_y)
    zero = torch.zeros_like(z)
    J = torch.stack([torch.stack([fx / z, zero, -fx * txz / z], -1),
                     torch.stack([zero, fy / z, -fy * tyz / z], -1)], -2)        # [G,2,3]
    Rg = quat_to_rotmat(quat)                                                     # [G,3,3]
    M = Rg * scale[:, None, :]
    Sigma = M @ M.transpose(-1, -2)
    T = J @ R
    cov = T @ Sigma @ T.transpose(-1, -2)
    a = cov[:, 0, 0] + rp.dilation
    b = cov[:, 0, 1]
    c = cov[:, 1, 1] + rp.dilation
    det = a * c - b * b
    conic = torch.stack([c / det, -b / det, a / det], -1)
    mean2d = torch.stack([fx * x / z + cx, fy * y / z + cy], -1)
    k = torch.argmin(scale.detach(), dim=-1)                                     # first minimum on ties
    n_w = torch.gather(Rg, 2, k[:, None, None].expand(-1, 3, 1))[..., 0]
    n_c = n_w @ R.T
    facing = (n_c * mu_c).sum(-1)
    sgn = torch.where(facing.detach() > 0, -torch.ones_like(facing), torch.ones_like(facing))
    n_c = n_c * sgn[:, None]
    dist = (n_c * mu_c).sum(-1)
    valid = (z.detach() >= rp.near) & (det.detach() > 0) & (opacity.detach() >= rp.alpha_min)
    with torch.no_grad():
        zd = z.detach()
        z32 = zd.to(torch.float32)
        zkey = z32.to(DT)
        zulp = torch.from_numpy(np.spacing(np.abs(z32.numpy())).astype(np.float64))
        # exact depth within 1e-9 (relative) of the midpoint between two FP32 values
        zmid = ((zd - zkey).abs() - 0.5 * zulp).abs() <= 1e-9 * zd.abs()
        s_sorted = torch.sort(scale, dim=-1).values
        # Gaussian-level decisions within FP32 reach: near plane, the facing
        # flip of the normal (edge-on), the smallest-scale axis (near ties)
        amb = ((z - rp.near).abs() <= 1e-5 * rp.near)
        amb |= facing.abs() <= AMB_GAUSS * torch.linalg.norm(mu_c, dim=-1)
        amb |= (s_sorted[:, 1] - s_sorted[:, 0]) <= AMB_GAUSS * s_sorted[:, 1]
        amb |= (opacity - rp.alpha_min).abs() <= 1e-5 * rp.alpha_min
    return dict(mean2d=mean2d, cov=torch.stack([a, b, c], -1), conic=conic, z=z, normal=n_c,
                dist=dist, opacity=opacity, color=color, valid=valid, ambiguous=amb, mu_c=mu_c,
                zkey=zkey, zulp=zulp, zmid=zmid)


# ------------------------------------------------------------------ blending (Eq. 1, 5-7)
def _reject_rect(proj: dict, keep: torch.Tensor, x0, x1, y0, y1, rp: RenderParams) -> torch.Tensor:
    """Gaussians that can reach alpha >= alpha_min somewhere in the pixel-centre
    rectangle [x0,x1]x[y0,y1].  Provable bound: power <= -|delta|^2 /
    (2 lambda_max(cov)), so o * exp(that) < alpha_min (with a 1e-6 margin)
    rules the Gaussian out everywhere in the rectangle."""
    with torch.no_grad():
        m = proj["mean2d"]
        a, b, c = proj["cov"].unbind(-1)
        lam = 0.5 * (a + c) + torch.sqrt(torch.clamp(0.25 * (a - c) ** 2 + b * b, min=0.0))
        ddx = torch.clamp(torch.maximum(x0 - m[:, 0], m[:, 0] - x1), min=0.0)
        ddy = torch.clamp(torch.maximum(y0 - m[:, 1], m[:, 1] - y1), min=0.0)
        bound = proj["opacity"] * torch.exp(-0.5 * (ddx * ddx + ddy * ddy) / lam)
        return keep & (bound >= rp.alpha_min * (1.0 - 1e-6))


def blend_pixels(proj: dict, order: torch.Tensor, px: torch.Tensor, py: torch.Tensor, rp: RenderParams,
                 cam: dict) -> dict:
    """Front-to-back compositing of the Gaussians ``order`` (already sorted by
    depth, index) at pixel centres (px, py).  Eq. 5 (RGB), Eq. 6 (normal),
    Eq. 7 (distance D and unbiased depth D_hat)."""
    m = proj["mean2d"][order]
    A, B, C = proj["conic"][order].unbind(-1)
    o = proj["opacity"][order]
    col = proj["color"][order]
    d = proj["dist"][order]
    n = proj["normal"][order]
    dx = px[:, None] - m[None, :, 0]
    dy = py[:, None] - m[None, :, 1]
    power = -0.5 * (A * dx * dx + C * dy * dy) - B * dx * dy
    a_raw = o * torch.exp(power)
    skip = (power.detach() > 0) | (a_raw.detach() < rp.alpha_min)
    alpha = torch.where(skip, torch.zeros_like(a_raw), torch.clamp(a_raw, max=rp.alpha_max))
    om = 1.0 - alpha
    T_incl = torch.cumprod(om, dim=1)
    T_excl = torch.cat([torch.ones_like(T_incl[:, :1]), T_incl[:, :-1]], 1)
    included = (T_incl.detach() >= rp.t_min)
    w = alpha * T_excl * included
    rgb = w @ col if w.shape[1] else torch.zeros(px.shape[0], 3, dtype=DT)
    D = w @ d if w.shape[1] else torch.zeros(px.shape[0], dtype=DT)
    N = w @ n if w.shape[1] else torch.zeros(px.shape[0], 3, dtype=DT)
    T_final = torch.prod(torch.where(included, om, torch.ones_like(om)), dim=1)
    rgb = rgb + T_final[:, None] * rp.bg
    # Eq. 7: D_hat = D / (N . K^-1 p~), guarded [reading]
    r = torch.stack([(px - cam["cx"]) / cam["fx"], (py - cam["cy"]) / cam["fy"], torch.ones_like(px)], -1)
    ndr = (N * r).sum(-1)
    ok = (ndr.detach().abs() >= 1e-8) & ((1.0 - T_final.detach()) >= 1e-6)
    depth = torch.where(ok, D / torch.where(ok, ndr, torch.ones_like(ndr)), torch.zeros_like(D))
    with torch.no_grad():
        contrib = included & ~skip
        n_contrib = contrib.sum(1)
        evaluated = T_excl >= rp.t_min
        ev_ns = evaluated & ~skip
        # a decision within the FP32 evaluation's reach of its threshold
        flag = ((a_raw - rp.alpha_min).abs() <= AMB_ALPHA * rp.alpha_min) & evaluated
        flag |= ((a_raw - rp.alpha_max).abs() <= AMB_ALPHA * rp.alpha_max) & evaluated
        flag |= ((T_incl - rp.t_min).abs() <= AMB_T * rp.t_min) & ev_ns
        flag |= proj["ambiguous"][order][None, :] & ev_ns
        pix_flag = flag.any(1)
        # two contributors whose FP32 depth keys are adjacent while one exact
        # depth sits within rounding of an FP32 midpoint: either order is valid
        key = proj["zkey"][order]
        mid = proj["zmid"][order]
        big = contrib & (w.detach() > 1e-7)
        G = big.shape[1]
        pos = torch.where(big, torch.arange(G)[None, :].expand_as(big), torch.full_like(big, -1, dtype=torch.long))
        prev = torch.cummax(torch.cat([torch.full_like(pos[:, :1], -1), pos[:, :-1]], 1), dim=1).values
        has_prev = big & (prev >= 0)
        pc = prev.clamp(min=0)
        close = (key[None, :] - key[pc]).abs() <= 1.5 * proj["zulp"][order][None, :]
        tie = has_prev & close & (mid[None, :] | mid[pc])
        pix_flag |= tie.any(1)
        pix_flag |= ((1.0 - T_final - 1e-6).abs() <= 1e-3 * 1e-6)
        pix_flag |= ((ndr.abs() - 1e-8).abs() <= 0.5e-8)
    return dict(rgb=rgb, D=D, normal=N, depth=depth, T_final=T_final, n_contrib=n_contrib, flag=pix_flag)


def sort_order(proj: dict, keep: torch.Tensor) -> torch.Tensor:
    """Surviving Gaussians ordered by (view depth z as an FP32 key, Gaussian
    index).  The paper leaves the key's precision open; the order is an
    integer decision taken from a float, so it is taken in the kernel's
    precision: z rounded to the nearest FP32 value, ties by index."""
    idx = torch.nonzero(keep).flatten()
    z = proj["zkey"][idx]
    perm = torch.sort(z, stable=True).indices
    return idx[perm]


def render_view(proj: dict, cam: dict, rp: RenderParams, crop=None, block: int = 32,
                image_grads: Optional[dict] = None) -> dict:
    """Render one view (or the crop (x0, y0, w, h)) pixel by pixel.

    Pixels are processed in independent blocks only to bound memory; each
    block sees every surviving Gaussian that can reach alpha >= alpha_min in
    it.  If ``image_grads`` (dL/d rgb, depth, normal over the crop) is given,
    the vector-Jacobian product is accumulated into the leaves' ``.grad``."""
    W, H = cam["W"], cam["H"]
    x0, y0, w, h = crop if crop is not None else (0, 0, W, H)
    keep_all = proj["valid"] | proj["ambiguous"]
    out = {k: torch.zeros(sh, dtype=DT) for k, sh in
           dict(rgb=(3, h, w), depth=(h, w), normal=(3, h, w), D=(h, w), T_final=(h, w)).items()}
    out["n_contrib"] = torch.zeros(h, w, dtype=torch.long)
    out["flag"] = torch.zeros(h, w, dtype=torch.bool)
    valid_order = sort_order(proj, proj["valid"])
    amb_only = proj["ambiguous"] & ~proj["valid"]
    for by in range(0, h, block):
        for bx in range(0, w, block):
            bh, bw = min(block, h - by), min(block, w - bx)
            ys = torch.arange(y0 + by, y0 + by + bh, dtype=DT) + 0.5
            xs = torch.arange(x0 + bx, x0 + bx + bw, dtype=DT) + 0.5
            PY, PX = torch.meshgrid(ys, xs, indexing="ij")
            px, py = PX.reshape(-1), PY.reshape(-1)
            near = _reject_rect(proj, keep_all, xs[0], xs[-1], ys[0], ys[-1], rp)
            order = valid_order[near[valid_order]]
            res = blend_pixels(proj, order, px, py, rp, cam)
            # an ambiguous Gaussian the oracle culled may still be kept in FP32
            amb_idx = torch.nonzero(amb_only & near).flatten()
            if amb_idx.numel():
                with torch.no_grad():
                    m = proj["mean2d"][amb_idx]
                    A, B, C = proj["conic"][amb_idx].unbind(-1)
                    ddx = px[:, None] - m[None, :, 0]
                    ddy = py[:, None] - m[None, :, 1]
                    pw = -0.5 * (A * ddx * ddx + C * ddy * ddy) - B * ddx * ddy
                    hit = (proj["opacity"][amb_idx] * torch.exp(pw) >= rp.alpha_min * 0.5).any(1)
                    res["flag"] = res["flag"] | hit
            sl = (slice(by, by + bh), slice(bx, bx + bw))
            if image_grads is not None:
                g_rgb = image_grads["rgb"][:, sl[0], sl[1]].reshape(3, -1).T
                g_d = image_grads["depth"][sl].reshape(-1)
                g_n = image_grads["normal"][:, sl[0], sl[1]].reshape(3, -1).T
                tot = (res["rgb"] * g_rgb).sum() + (res["depth"] * g_d).sum() + (res["normal"] * g_n).sum()
                if tot.requires_grad:
                    tot.backward(retain_graph=True)
            out["rgb"][:, sl[0], sl[1]] = res["rgb"].detach().T.reshape(3, bh, bw)
            out["normal"][:, sl[0], sl[1]] = res["normal"].detach().T.reshape(3, bh, bw)
            for k in ("depth", "D", "T_final", "n_contrib", "flag"):
                out[k][sl] = res[k].detach().reshape(bh, bw)
    return out


# ------------------------------------------------------------------ full step
def leaves_explicit(scene: dict) -> dict:
    return {k: _t(scene[k]).clone().requires_grad_(True)
            for k in ("means", "log_scales", "quats", "opacity_logits", "colors")}


def leaves_anchor(scene: dict) -> dict:
    p = {k: _t(scene[k]).clone().requires_grad_(True) for k in ("x", "log_l", "offsets", "feat")}
    for k, v in scene["mlp"].items():
        p[k] = _t(v).clone().requires_grad_(True)
    return p


def gaussians_for_view(scene: dict, leaves: dict, cam: dict, rp: RenderParams, in_dim: int = 35,
                       exclude: Optional[torch.Tensor] = None) -> dict:
    """Per-view 3D Gaussians: explicit ones as given, or the decoded ones of
    every LoD-active anchor (Eq. 4).  Index = anchor * 10 + j."""
    if scene["kind"] == "explicit":
        return dict(mu=leaves["means"], scale=torch.exp(leaves["log_scales"]),
                    quat=normalize_quat(leaves["quats"]), opacity=torch.sigmoid(leaves["opacity_logits"]),
                    color=leaves["colors"], lod_amb=None)
    level = torch.as_tensor(np.asarray(scene["level"]), dtype=torch.long)
    active, amb = lod_active(leaves["x"].detach(), level, cam, rp)
    if exclude is not None:
        active &= ~exclude
    idx = torch.nonzero(active).flatten()
    anchors = dict(x=leaves["x"], feat=leaves["feat"], log_l=leaves["log_l"], offsets=leaves["offsets"])
    mlp = {k: leaves[k] for k in ("W1", "b1", "W2", "b2")}
    dec = decode(anchors, mlp, cam, idx, in_dim, rp.decode)
    dec["anchor_idx"] = idx
    dec["lod_amb"] = amb
    return dec


def render(scene: dict, rp: RenderParams, leaves: Optional[dict] = None, crops=None,
           image_grads: Optional[Sequence[dict]] = None, views: Optional[Sequence[int]] = None,
           exclude: Optional[torch.Tensor] = None, block: int = 32, in_dim: int = 35) -> dict:
    """Render every view (optionally a crop per view).  With ``image_grads``
    the VJP lands in ``leaves[*].grad``.  Returns per-view dicts."""
    if leaves is None:
        leaves = leaves_explicit(scene) if scene["kind"] == "explicit" else leaves_anchor(scene)
    views = list(range(len(scene["cameras"]))) if views is None else list(views)
    outs = []
    for v in views:
        cam = camera(scene["cameras"][v])
        g = gaussians_for_view(scene, leaves, cam, rp, in_dim, exclude)
        proj = project(g["mu"], g["scale"], g["quat"], g["opacity"], g["color"], cam, rp)
        crop = crops[v] if crops is not None else None
        ig = image_grads[v] if image_grads is not None else None
        if ig is not None:
            ig = {k: _t(val) for k, val in ig.items()}
        out = render_view(proj, cam, rp, crop, block, ig)
        out["n_gaussians"] = int(proj["valid"].sum())
        out["proj"] = {k: (val.detach() if isinstance(val, torch.Tensor) else val) for k, val in proj.items()}
        out["lod_amb"] = g.get("lod_amb")
        out["anchor_idx"] = g.get("anchor_idx")
        outs.append(out)
    return dict(views=outs, leaves=leaves)


# ------------------------------------------------------------------ losses (Eq. 8-9 + consistency)
def depth_normal(depth: torch.Tensor, cam: dict):
    """Normal of the surface implied by a depth map: back-project pixel
    centres P = D_hat * K^-1 [u+.5, v+.5, 1], cross product of the central
    differences along x and y, normalised and turned to face the camera.
    Returns (normal [3,H,W], valid [H,W]) -- valid needs an interior pixel
    with positive depth at itself and its four neighbours."""
    H, W = depth.shape
    v, u = torch.meshgrid(torch.arange(H, dtype=DT) + 0.5, torch.arange(W, dtype=DT) + 0.5, indexing="ij")
    r = torch.stack([(u - cam["cx"]) / cam["fx"], (v - cam["cy"]) / cam["fy"], torch.ones_like(u)], 0)
    P = depth[None] * r
    Nd = torch.zeros(3, H, W, dtype=DT)
    valid = torch.zeros(H, W, dtype=torch.bool)
    if H >= 3 and W >= 3:
        ex = P[:, 1:-1, 2:] - P[:, 1:-1, :-2]
        ey = P[:, 2:, 1:-1] - P[:, :-2, 1:-1]
        cr = torch.cross(ex, ey, dim=0)
        nrm = torch.linalg.norm(cr, dim=0)
        pos = depth > 0
        ok = pos[1:-1, 1:-1] & pos[1:-1, 2:] & pos[1:-1, :-2] & pos[2:, 1:-1] & pos[:-2, 1:-1] & (nrm > 1e-20)
        nd = cr / torch.where(nrm > 0, nrm, torch.ones_like(nrm))
        face = (nd * P[:, 1:-1, 1:-1]).sum(0)
        nd = torch.where(face > 0, -nd, nd)
        Nd[:, 1:-1, 1:-1] = nd
        valid[1:-1, 1:-1] = ok
    return Nd, valid


def loss_view(rgb, depth, normal, target: dict, cam: dict, lp: LossParams) -> dict:
    """Per-view loss terms (before the 1/B batch mean):
    RGB L1 mean over pixels and channels (Eq. 8); depth L1 over the prior's
    mask, normalised by the mask count (Eq. 9); normal-depth consistency
    mean(1 - N_d . N/|N|) over valid pixels with N_d under stop-gradient."""
    I = _t(target["rgb"])
    prior = _t(target["prior"])
    mask = _t(target["mask"])
    l_rgb = (rgb - I).abs().mean()
    l_depth = (mask * (depth - prior).abs()).sum() / torch.clamp(mask.sum(), min=1.0)
    with torch.no_grad():
        Nd, valid = depth_normal(depth.detach(), cam)
    nn_ = torch.linalg.norm(normal, dim=0)
    valid = valid & (nn_.detach() > 1e-8)
    cosang = (Nd * normal).sum(0) / torch.where(valid, nn_, torch.ones_like(nn_))
    cnt = max(int(valid.sum()), 1)
    l_normal = torch.where(valid, 1.0 - cosang, torch.zeros_like(cosang)).sum() / cnt
    total = l_rgb + lp.lambda_depth * l_depth + lp.lambda_normal * l_normal
    return dict(total=total, rgb=l_rgb, depth=l_depth, normal=l_normal, n_valid=int(valid.sum()))


def batch_loss(maps: Sequence[dict], targets: Sequence[dict], cams: Sequence, lp: LossParams) -> dict:
    """L = (1/B) sum_b [L_rgb + lambda_d L_depth + lambda_n L_normal]."""
    B = len(maps)
    terms = [loss_view(m["rgb"], m["depth"], m["normal"], t, camera(c), lp) for m, t, c in zip(maps, targets, cams)]
    total = sum(t["total"] for t in terms) / B
    return dict(total=total, terms=terms)


def loss_and_image_grads(maps: Sequence[dict], targets: Sequence[dict], cams: Sequence, lp: LossParams):
    """Loss value and dL/d(rgb, depth, normal) per view (FP64 autograd)."""
    leaves = [{k: _t(m[k]).clone().requires_grad_(True) for k in ("rgb", "depth", "normal")} for m in maps]
    L = batch_loss(leaves, targets, cams, lp)
    L["total"].backward()
    grads = [{k: lv[k].grad.detach().clone() for k in lv} for lv in leaves]
    return float(L["total"].detach()), grads, L


def loss_ambiguity(maps: Sequence[dict], targets: Sequence[dict], tol: float = 1e-5):
    """Pixels where the sign of an L1 residual is decided within rounding."""
    flags = []
    for m, t in zip(maps, targets):
        f = ((_t(m["rgb"]) - _t(t["rgb"])).abs() <= tol).any(0)
        f |= ((_t(m["depth"]) - _t(t["prior"])).abs() <= tol) & (_t(t["mask"]) > 0)
        flags.append(f)
    return flags


# ------------------------------------------------------------------ integer definitions
def tile_set(mean2d, conic, opacity, W: int, H: int, rp: RenderParams, margin: float = 0.0):
    """Tiles of one view whose pixel-centre rectangle meets the level set
    1/2 delta^T Q delta <= ln(255 * o) + pad of a Gaussian (the set on which
    alpha >= 1/255, padded in the exponent).  Decided by the exact minimum of
    the quadratic over the rectangle (convex: the unconstrained minimiser if
    inside, else the best point of the four edges).

    Returns (tiles, ambiguous) as python lists of global-in-view tile ids;
    ``ambiguous`` holds tiles whose minimum lies within ``margin`` (relative)
    of the level."""
    tile = rp.tile
    tx_n, ty_n = (W + tile - 1) // tile, (H + tile - 1) // tile
    mx, my = float(mean2d[0]), float(mean2d[1])
    A, B, C = (float(v) for v in conic)
    o = float(opacity)
    if o < rp.alpha_min:
        return [], []
    lvl = math.log(255.0 * o) + rp.tile_pad
    det = A * C - B * B
    cov_xx, cov_yy = C / det, A / det
    rx = math.sqrt(max(2.0 * lvl * cov_xx, 0.0)) * (1 + 4 * margin) + 1e-9
    ry = math.sqrt(max(2.0 * lvl * cov_yy, 0.0)) * (1 + 4 * margin) + 1e-9

    def q(dx, dy):
        return A * dx * dx + 2 * B * dx * dy + C * dy * dy

    def seg_min_v(dx, lo, hi):                      # edge with fixed dx, dy in [lo, hi]
        dy = -B * dx / C
        dy = min(max(dy, lo), hi)
        return q(dx, dy)

    def seg_min_h(dy, lo, hi):
        dx = -B * dy / A
        dx = min(max(dx, lo), hi)
        return q(dx, dy)

    tiles, amb = [], []
    t0x = max(0, int(math.floor((mx - rx - 0.5) / tile)))
    t1x = min(tx_n - 1, int(math.floor((mx + rx - 0.5) / tile)))
    t0y = max(0, int(math.floor((my - ry - 0.5) / tile)))
    t1y = min(ty_n - 1, int(math.floor((my + ry - 0.5) / tile)))
    for ty in range(t0y, t1y + 1):
        y0 = ty * tile + 0.5 - my
        y1 = min(ty * tile + tile - 0.5, H - 0.5) - my
        for tx in range(t0x, t1x + 1):
            x0 = tx * tile + 0.5 - mx
            x1 = min(tx * tile + tile - 0.5, W - 0.5) - mx
            if x0 <= 0 <= x1 and y0 <= 0 <= y1:
                mn = 0.0
            else:
                mn = min(seg_min_v(x0, y0, y1), seg_min_v(x1, y0, y1), seg_min_h(y0, x0, x1), seg_min_h(y1, x0, x1))
            val = 0.5 * mn
            if val <= lvl:
                tiles.append(ty * tx_n + tx)
            if abs(val - lvl) <= margin * max(lvl, 1.0):
                amb.append(ty * tx_n + tx)
    return tiles, amb


def exclusive_scan(counts: np.ndarray) -> np.ndarray:
    counts = np.asarray(counts, dtype=np.uint64)
    out = np.zeros_like(counts)
    if len(counts) > 1:
        out[1:] = np.cumsum(counts[:-1])
    return out


def stable_sort(keys: np.ndarray, values: np.ndarray):
    perm = np.argsort(keys, kind="stable")
    return keys[perm], values[perm]


def tile_ranges(sorted_tiles: np.ndarray, n_tiles: int) -> np.ndarray:
    """ranges[t] = [first, last+1) of tile t in the sorted list, [0,0) if absent."""
    r = np.zeros((n_tiles, 2), dtype=np.int64)
    prev = None
    for i, t in enumerate(sorted_tiles.tolist()):
        if t != prev:
            r[t, 0] = i
            if prev is not None:
                r[prev, 1] = i
            prev = t
    if prev is not None:
        r[prev, 1] = len(sorted_tiles)
    return r


# ------------------------------------------------------------------ enhanced depth prior (Sec. 3.4, Step 2)
# Reading of the paper's description (it gives the steps, not the formulas):
# the pseudo depth D_p of view v is brought to the sparse points' scale by the
# least-squares scale and shift (s_v, t_v) of z_k ~ s D_p(u_k) + t over the
# points k that project into v (D_p sampled bilinearly at u_k, pixel centres at
# +1/2); the re-projection error E(p) of pixel p of view a is the pixel
# distance after the round trip a -> b -> a through the rescaled pseudo depths
# of a and of b (b read bilinearly), minimised over the k batch views nearest
# to a by camera centre; the filtered prior keeps D~_p(p) where E(p) <= tau_d
# (1 in the supplementary) or where no neighbour could check p, and is 0
# elsewhere or where D_p(p) <= 0.
# E is a difference of pixel positions of order 10^3 carried through ~20 FP32
# operations: its FP32 reach is about 10 ulp of 10^3, i.e. a few 1e-3 px.
AMB_PRIOR_E = 2e-2      # px: decisions with E this close to tau_d are flagged
AMB_PRIOR_EDGE = 1e-3   # px: a bilinear footprint this close to the frame edge may be in or out in FP32
# On a steep footprint (the four samples differ by more than PRIOR_STEEP of the
# value, e.g. across the edge of a wrong region of the pseudo depth) the read
# depth moves by (jump / 1 px) per pixel of position error, so FP32 rounding of
# the projected position can move E by a tenth of a pixel: the reach there is
# AMB_PRIOR_E_STEEP.
PRIOR_STEEP = 0.02
AMB_PRIOR_E_STEEP = 0.25


def _prior_bilinear(dp: torch.Tensor, x: torch.Tensor, y: torch.Tensor):
    """Bilinear read of dp [H, W] at pixel coordinates (centres at +1/2).
    Returns (value, defined, near_edge, steep)."""
    H, W = dp.shape
    u, w = x - 0.5, y - 0.5
    fu, fw = torch.floor(u), torch.floor(w)
    inside = (fu >= 0) & (fw >= 0) & (fu + 1 <= W - 1) & (fw + 1 <= H - 1)
    near = ((u.abs() < AMB_PRIOR_EDGE) | (w.abs() < AMB_PRIOR_EDGE) | ((u - (W - 1)).abs() < AMB_PRIOR_EDGE)
            | ((w - (H - 1)).abs() < AMB_PRIOR_EDGE))
    i0 = fu.clamp(0, W - 2).long()
    j0 = fw.clamp(0, H - 2).long()
    a, b = dp[j0, i0], dp[j0, i0 + 1]
    c, d = dp[j0 + 1, i0], dp[j0 + 1, i0 + 1]
    au, aw = u - fu, w - fw
    val = (1 - aw) * ((1 - au) * a + au * b) + aw * ((1 - au) * c + au * d)
    ok = inside & (a > 0) & (b > 0) & (c > 0) & (d > 0)
    hi = torch.maximum(torch.maximum(a, b), torch.maximum(c, d))
    lo = torch.minimum(torch.minimum(a, b), torch.minimum(c, d))
    steep = (hi - lo) > PRIOR_STEEP * val.abs()
    return val, ok, near, steep


def _to_cam(cam: dict, x: torch.Tensor) -> torch.Tensor:
    return x @ cam["R"].T + cam["t"]


def _to_world(cam: dict, c: torch.Tensor) -> torch.Tensor:
    return (c - cam["t"]) @ cam["R"]


def prior_scale_shift(cam: dict, dp: torch.Tensor, points: torch.Tensor, near: float):
    """Least-squares (s, t) of the points' view depths against the bilinear pseudo depth
    (a library least-squares solve on [D_p, 1]); (1, 0) with fewer than two points."""
    c = _to_cam(cam, points)
    front = c[:, 2] > near
    zc = torch.where(front, c[:, 2], torch.ones_like(c[:, 2]))
    px = cam["fx"] * c[:, 0] / zc + cam["cx"]
    py = cam["fy"] * c[:, 1] / zc + cam["cy"]
    d, ok, _, _ = _prior_bilinear(dp, px, py)
    use = front & ok
    if int(use.sum()) < 2:
        return 1.0, 0.0, int(use.sum())
    A = torch.stack([d[use], torch.ones_like(d[use])], 1)
    sol = torch.linalg.lstsq(A, c[use, 2:3]).solution
    s, t = float(sol[0, 0]), float(sol[1, 0])
    if not math.isfinite(s) or float(d[use].var(unbiased=False)) <= 0.0:
        return 1.0, 0.0, int(use.sum())
    return s, t, int(use.sum())


def nearest_views(cams: Sequence[dict], k: int) -> List[List[int]]:
    """The k other views nearest by camera centre (ties by index)."""
    out = []
    for a, ca in enumerate(cams):
        d = sorted((float(((ca["center"] - cb["center"]) ** 2).sum()), b) for b, cb in enumerate(cams) if b != a)
        out.append([b for _, b in d[:min(k, len(cams) - 1)]])
    return out


def filter_depth_prior(cams_in: Sequence, pseudo: Sequence[torch.Tensor], points, tau_d: float = 1.0, k: int = 2,
                       near: float = 0.01) -> dict:
    """Enhanced depth prior of a batch (see the reading above).  pseudo[v]: [H, W]
    pseudo depth (<= 0 = none); points: [n, 3] world.  Returns per view the
    filtered prior, mask, error E (-1 = unchecked), ambiguity flags, the
    steep-footprint map (E ill-conditioned there), and (s, t)."""
    cams = [camera(c) for c in cams_in]
    pts = _t(points).reshape(-1, 3)
    dps = [_t(p) for p in pseudo]
    st = [prior_scale_shift(c, dp, pts, near) for c, dp in zip(cams, dps)]
    nbr = nearest_views(cams, k)
    views = []
    for a, ca in enumerate(cams):
        H, W = ca["H"], ca["W"]
        s, t, _ = st[a]
        dp = dps[a]
        d = s * dp + t
        have = (dp > 0) & (d > 0)
        vv, uu = torch.meshgrid(torch.arange(H, dtype=DT) + 0.5, torch.arange(W, dtype=DT) + 0.5, indexing="ij")
        pc = torch.stack([d * (uu - ca["cx"]) / ca["fx"], d * (vv - ca["cy"]) / ca["fy"], d], -1)
        xw = _to_world(ca, pc.reshape(-1, 3))
        best = torch.full((H * W,), float("inf"), dtype=DT)
        checked = torch.zeros(H * W, dtype=torch.bool)
        amb = torch.zeros(H * W, dtype=torch.bool)
        steep = torch.zeros(H * W, dtype=torch.bool)
        for b in nbr[a]:
            cb = cams[b]
            sb, tb, _ = st[b]
            c1 = _to_cam(cb, xw)
            front1 = c1[:, 2] > near
            z1 = torch.where(front1, c1[:, 2], torch.ones_like(c1[:, 2]))
            qx = cb["fx"] * c1[:, 0] / z1 + cb["cx"]
            qy = cb["fy"] * c1[:, 1] / z1 + cb["cy"]
            rb, okb, nearb, steepb = _prior_bilinear(dps[b], qx, qy)
            db = sb * rb + tb
            pb = torch.stack([db * (qx - cb["cx"]) / cb["fx"], db * (qy - cb["cy"]) / cb["fy"], db], -1)
            c2 = _to_cam(ca, _to_world(cb, pb))
            front2 = c2[:, 2] > near
            z2 = torch.where(front2, c2[:, 2], torch.ones_like(c2[:, 2]))
            rx = ca["fx"] * c2[:, 0] / z2 + ca["cx"] - uu.reshape(-1)
            ry = ca["fy"] * c2[:, 1] / z2 + ca["cy"] - vv.reshape(-1)
            e = torch.sqrt(rx * rx + ry * ry)
            valid = front1 & okb & (db > 0) & front2
            best = torch.where(valid, torch.minimum(best, e), best)
            checked |= valid
            steep |= valid & steepb
            amb |= front1 & nearb
        have_f = have.reshape(-1)
        keep = have_f & (~checked | (best <= tau_d))
        amb |= have_f & checked & ((best - tau_d).abs() <= AMB_PRIOR_E)
        amb |= have_f & checked & steep & ((best - tau_d).abs() <= AMB_PRIOR_E_STEEP)
        E = torch.where(checked & have_f, best, torch.full_like(best, -1.0))
        views.append(dict(prior=torch.where(keep, d.reshape(-1), torch.zeros_like(best)).reshape(H, W),
                          mask=keep.to(DT).reshape(H, W), err=E.reshape(H, W), amb=amb.reshape(H, W),
                          steep=steep.reshape(H, W),
                          scale=s, shift=t, n_points=st[a][2]))
    return dict(views=views, neighbours=nbr)


# ------------------------------------------------------------------ batch geometric NCC (Sec. 3.4, Step 3, Eq. 10)
# Reading of Eq. 10 and the text around it:
# * the rendered batch is split into pairs (views 2i-1, 2i counted from 1); in
#   0-based indices pair i has the reference view 2i+1, whose patches are
#   compared, and the partner view 2i, sampled through the homography;
# * every pair draws N patch centres p (the random draw is an input here); a
#   7 x 7 patch of reference pixels around p is mapped into the partner by the
#   homography of the plane through the back-projected centre, with the
#   rendered unbiased depth D_hat(p) and normal N_hat(p) of the reference view:
#   plane m . X = 1 with m = N_hat / (D_hat (N_hat . r_p)), r_p = K_r^-1 p~,
#   H = K_s (R + t m^T) K_r^-1 where X_s = R X_r + t maps reference to partner
#   camera coordinates;
# * NCC (zero-normalised cross-correlation) of the BT.601 luma of the two
#   patches: the reference's at its 49 pixels, the partner's read bilinearly
#   (pixel centres at +1/2) at the 49 warped positions,
#   NCC = S_ab / sqrt((S_aa + eps)(S_bb + eps)) over centred sums, eps = 1e-6;
# * a patch counts only if it lies inside the reference frame, the plane is
#   defined (D_hat(p) > 0, |N_hat(p) . r_p| >= 1e-8), and every warped sample
#   has the plane in front of both cameras and its whole bilinear footprint
#   inside the partner frame;
# * L_ncc = (1 / (B/2)) sum_i mean over pair i's valid patches of (1 - NCC),
#   a pair without valid patches adding 0;
# * sg[.]: with geo=True the partner image is a constant while the sampling
#   positions keep their dependence on D_hat(p) and N_hat(p) (so Step 3 reaches
#   the geometry); with geo=False the whole sampled partner patch is constant
#   (gradients reach the reference colours only, the formula taken literally).
NCC_HALF = 3
NCC_EPS = 1e-6
LUMA = (0.299, 0.587, 0.114)
# an FP32 evaluation reaches the warped positions to ~1e-4 px (positions of
# order 10^3 through a 3 x 3 product and a division): a sample this close to
# the edge of the bilinear area may be in or out, and a sample this close to a
# cell boundary may take the other cell's bilinear slope (the geometric
# gradient jumps there; the sampled value does not)
AMB_NCC_EDGE = 1e-3
AMB_NCC_CELL = 1e-3
AMB_NCC_FRONT = 1e-6    # relative: m . r_q or h_z this close to 0
# Conditioning of the NCC of a patch under errors db in the partner samples:
# |dNCC| <= sqrt((1 - NCC^2) / S_bb) |db|_2 (the gradient of NCC with respect
# to b has that norm for eps -> 0), and |db|_2 <= 7 (max_k |grad b_k| du +
# d_luma) for position errors du and luma rounding d_luma.  ``ncc_patches``
# returns S_bb and max_k |grad b_k| so that a comparison can take that bound.


def ncc_pairs(n_views: int) -> List[tuple]:
    """(reference, partner) view indices of the pairs of Eq. 10."""
    return [(2 * i + 1, 2 * i) for i in range(n_views // 2)]


def luma(rgb: torch.Tensor) -> torch.Tensor:
    """BT.601 luma of a [3, ...] colour array."""
    return LUMA[0] * rgb[0] + LUMA[1] * rgb[1] + LUMA[2] * rgb[2]


def _kmat(cam: dict) -> torch.Tensor:
    return torch.tensor([[cam["fx"], 0.0, cam["cx"]], [0.0, cam["fy"], cam["cy"]], [0.0, 0.0, 1.0]], dtype=DT)


def plane_homography(cr: dict, cs: dict, m: torch.Tensor) -> torch.Tensor:
    """Homographies [n, 3, 3] from reference pixels to partner pixels induced by
    the planes m . X = 1 (m [n, 3], reference camera frame)."""
    R = cs["R"] @ cr["R"].T
    t = cs["t"] - R @ cr["t"]
    A = R.unsqueeze(0) + t.view(1, 3, 1) * m.view(-1, 1, 3)
    return _kmat(cs) @ A @ torch.linalg.inv(_kmat(cr))


def _bilinear_area(x: torch.Tensor, y: torch.Tensor, W: int, H: int):
    """(inside, near_edge, near_cell) of bilinear reads at pixel coordinates."""
    u, w = x - 0.5, y - 0.5
    inside = (torch.floor(u) >= 0) & (torch.floor(w) >= 0) & (torch.floor(u) + 1 <= W - 1) & \
             (torch.floor(w) + 1 <= H - 1)
    near = ((u.abs() < AMB_NCC_EDGE) | (w.abs() < AMB_NCC_EDGE) | ((u - (W - 1)).abs() < AMB_NCC_EDGE)
            | ((w - (H - 1)).abs() < AMB_NCC_EDGE))
    fu, fw = u - torch.floor(u), w - torch.floor(w)
    cell = (fu < AMB_NCC_CELL) | (fu > 1 - AMB_NCC_CELL) | (fw < AMB_NCC_CELL) | (fw > 1 - AMB_NCC_CELL)
    return inside, near, cell


def _bilinear(img: torch.Tensor, x: torch.Tensor, y: torch.Tensor) -> torch.Tensor:
    """Bilinear read of img [H, W] at pixel coordinates (centres at +1/2); the
    caller guarantees the footprint is inside (indices are clamped only so that
    invalid samples stay addressable)."""
    H, W = img.shape
    u, w = x - 0.5, y - 0.5
    fu, fw = torch.floor(u), torch.floor(w)
    i0 = fu.clamp(0, W - 2).long()
    j0 = fw.clamp(0, H - 2).long()
    au, aw = u - fu, w - fw
    a, b = img[j0, i0], img[j0, i0 + 1]
    c, d = img[j0 + 1, i0], img[j0 + 1, i0 + 1]
    return (1 - aw) * ((1 - au) * a + au * b) + aw * ((1 - au) * c + au * d)


def _bilinear_slope(img: torch.Tensor, x: torch.Tensor, y: torch.Tensor) -> torch.Tensor:
    """|grad| of the bilinear interpolant of img at pixel coordinates (per-cell slopes)."""
    H, W = img.shape
    u, w = x - 0.5, y - 0.5
    fu, fw = torch.floor(u), torch.floor(w)
    i0 = fu.clamp(0, W - 2).long()
    j0 = fw.clamp(0, H - 2).long()
    au, aw = u - fu, w - fw
    a, b = img[j0, i0], img[j0, i0 + 1]
    c, d = img[j0 + 1, i0], img[j0 + 1, i0 + 1]
    gx = (1 - aw) * (b - a) + aw * (d - c)
    gy = (1 - au) * (c - a) + au * (d - b)
    return torch.sqrt(gx * gx + gy * gy)


def ncc(a: torch.Tensor, b: torch.Tensor, eps: float = NCC_EPS) -> torch.Tensor:
    """Zero-normalised cross-correlation along the last axis, eps added to each
    centred sum of squares."""
    da = a - a.mean(-1, keepdim=True)
    db = b - b.mean(-1, keepdim=True)
    return (da * db).sum(-1) / torch.sqrt(((da * da).sum(-1) + eps) * ((db * db).sum(-1) + eps))


def ncc_patches(cr: dict, cs: dict, ref: dict, part_rgb: torch.Tensor, centers: torch.Tensor, geo: bool = True,
                eps: float = NCC_EPS) -> dict:
    """Eq. 10 for one pair: NCC of the 7 x 7 reference patches at `centers`
    (local pixel indices y W + x) against the partner read through the plane
    homography.  ref: dict(rgb [3,H,W], depth [H,W] = D_hat, normal [3,H,W] =
    N_hat) of the reference view (tensors may require grad); part_rgb [3,H,W]
    the partner's colour.  Returns dict(ncc [n], valid [n], amb [n], cell [n],
    warped [n, 49, 2])."""
    W, H = cr["W"], cr["H"]
    centers = torch.as_tensor(centers, dtype=torch.long).reshape(-1)
    n = centers.numel()
    cy, cx = centers // W, centers % W
    inframe = (cx >= NCC_HALF) & (cx <= W - 1 - NCC_HALF) & (cy >= NCC_HALF) & (cy <= H - 1 - NCC_HALF)
    cxc = cx.clamp(NCC_HALF, W - 1 - NCC_HALF)
    cyc = cy.clamp(NCC_HALF, H - 1 - NCC_HALF)
    d = ref["depth"][cyc, cxc]
    nr = ref["normal"][:, cyc, cxc].T                                    # [n, 3]
    rp = torch.stack([(cxc.to(DT) + 0.5 - cr["cx"]) / cr["fx"], (cyc.to(DT) + 0.5 - cr["cy"]) / cr["fy"],
                      torch.ones(n, dtype=DT)], 1)
    c = (nr * rp).sum(1)
    plane = inframe & (d > 0) & (c.abs() >= 1e-8)
    den = torch.where(plane, d * c, torch.ones_like(c))
    m = nr / den.unsqueeze(1)                                            # m . X = 1
    Hm = plane_homography(cr, cs, m)                                     # [n, 3, 3]
    off = torch.arange(-NCC_HALF, NCC_HALF + 1)
    oy, ox = torch.meshgrid(off, off, indexing="ij")
    qx = (cxc.view(-1, 1) + ox.reshape(1, -1))                            # [n, 49] reference pixels
    qy = (cyc.view(-1, 1) + oy.reshape(1, -1))
    q = torch.stack([qx.to(DT) + 0.5, qy.to(DT) + 0.5, torch.ones(n, qx.shape[1], dtype=DT)], -1)
    h = torch.einsum("nij,nkj->nki", Hm, q)                              # [n, 49, 3]
    rq = torch.stack([(q[..., 0] - cr["cx"]) / cr["fx"], (q[..., 1] - cr["cy"]) / cr["fy"], q[..., 2]], -1)
    mr = (m.unsqueeze(1) * rq).sum(-1)
    hz = torch.where(h[..., 2] > 0, h[..., 2], torch.ones_like(h[..., 2]))
    ux, uy = h[..., 0] / hz, h[..., 1] / hz
    Ws, Hs = cs["W"], cs["H"]
    inside, near, cell = _bilinear_area(ux.detach(), uy.detach(), Ws, Hs)
    front = (mr > 0) & (h[..., 2] > 0)
    valid = plane & (front & inside).all(1)
    a = luma(ref["rgb"][:, qy, qx])                                      # [n, 49]
    g = luma(part_rgb).detach()
    if geo:
        b = _bilinear(g, ux, uy)
    else:
        b = _bilinear(g, ux.detach(), uy.detach()).detach()
    val = ncc(a, b, eps)
    bd = b.detach()
    sbb = ((bd - bd.mean(-1, keepdim=True)) ** 2).sum(-1)
    slope = _bilinear_slope(g, ux.detach(), uy.detach()).amax(1)
    scale_mr = mr.detach().abs().amax(1).clamp(min=1e-30)
    amb = plane & (near | (mr.detach().abs() < AMB_NCC_FRONT * scale_mr.unsqueeze(1))
                   | (h[..., 2].detach().abs() < AMB_NCC_FRONT * h[..., 2].detach().abs().amax(1, keepdim=True))).any(1)
    return dict(ncc=val, valid=valid, amb=amb, cell=plane & cell.any(1), warped=torch.stack([ux, uy], -1),
                sbb=sbb, slope=slope)


def ncc_loss(cams_in: Sequence, maps: Sequence[dict], centers, geo: bool = True, eps: float = NCC_EPS,
             lam: float = 1.0, grad: bool = True) -> dict:
    """L_ncc of Eq. 10 over the batch (reading above) and, with grad=True, its
    gradients with respect to every view's rgb, depth (D_hat) and normal
    (N_hat), scaled by lam (torch.autograd in FP64).  maps[v]: dict(rgb
    [3,H,W], depth [H,W], normal [3,H,W]); centers: [B/2, N] local pixel
    indices of the reference views."""
    cams = [camera(c) for c in cams_in]
    pairs = ncc_pairs(len(cams))
    leaves = [{k: _t(mp[k]).clone().requires_grad_(grad) for k in ("rgb", "depth", "normal")} for mp in maps]
    centers = torch.as_tensor(np.asarray(centers), dtype=torch.long).reshape(len(pairs), -1) if pairs else None
    per = []
    total = torch.zeros((), dtype=DT)
    for i, (r, s) in enumerate(pairs):
        out = ncc_patches(cams[r], cams[s], leaves[r], leaves[s]["rgb"], centers[i], geo, eps)
        nv = int(out["valid"].sum())
        li = ((1.0 - out["ncc"]) * out["valid"]).sum() / nv if nv > 0 else torch.zeros((), dtype=DT)
        total = total + li
        per.append(dict(ncc=out["ncc"].detach(), valid=out["valid"], amb=out["amb"], cell=out["cell"],
                        sbb=out["sbb"], slope=out["slope"], n_valid=nv, loss=float(li.detach())))
    L = total / len(pairs) if pairs else total
    res = dict(loss=float(L.detach()), pairs=per)
    if grad and pairs:
        (lam * L).backward()
        res["grads"] = [{k: (lf[k].grad if lf[k].grad is not None else torch.zeros_like(lf[k])).detach()
                         for k in ("rgb", "depth", "normal")} for lf in leaves]
    return res


# ------------------------------------------------------------------ TSDF fusion of rendered depth (supplementary)
# The supplementary fuses rendered colour and depth maps into a projective TSDF
# volume (Zeng et al.'s fusion; voxel 0.01 and truncation 0.04 for the aerial
# scenes).  Reading of the steps, which the paper does not spell out:
# * volume: an axis-aligned grid, voxel (i, j, k) centred at origin + (i + 1/2,
#   j + 1/2, k + 1/2) * voxel, x fastest in memory;
# * a voxel centre X is projected into each view in batch order: camera point
#   R X + t with depth z > near, pixel (floor(u), floor(v)) of u = fx x / z + cx,
#   v = fy y / z + cy (pixel centres at +1/2, so the nearest pixel), inside the
#   frame, with a rendered depth D > 0 there;
# * projective signed distance sdf = D - z; views with sdf < -trunc (behind the
#   surface beyond the band) leave the voxel alone; otherwise the observation
#   tsdf = min(1, sdf / trunc) enters a running average with unit weight,
#   T <- (T W + tsdf) / (W + 1), W <- W + 1, and the pixel's colour likewise.
AMB_TSDF_PIX = 1e-3     # px: a projection this close to a pixel boundary may pick the neighbour in FP32
AMB_TSDF_SDF = 1e-5     # sdf this close to -trunc may fall on either side in FP32
AMB_TSDF_NEAR = 1e-6    # relative: depth this close to the near plane


def voxel_centres(origin, voxel: float, dims, index=None) -> torch.Tensor:
    """World centres [n, 3] of the voxels with linear indices `index` (default all),
    x fastest."""
    nx, ny, nz = dims
    if index is None:
        index = torch.arange(nx * ny * nz)
    index = torch.as_tensor(index, dtype=torch.long)
    i = index % nx
    j = (index // nx) % ny
    k = index // (nx * ny)
    o = _t(origin).reshape(3)
    return o + (torch.stack([i, j, k], 1).to(DT) + 0.5) * voxel


def tsdf_fuse(cams_in: Sequence, depths: Sequence[torch.Tensor], origin, voxel: float, dims, trunc: float,
              colors: Optional[Sequence[torch.Tensor]] = None, index=None, near: float = 0.01,
              state: Optional[dict] = None) -> dict:
    """Fuse the views' depth maps [H, W] (and colours [3, H, W]) into the voxels
    `index` (default all) of the volume, in view order, starting from `state`
    (tsdf, weight, color of those voxels; default empty).  Returns the new state
    and `amb`: voxels where an FP32 evaluation may take another branch."""
    cams = [camera(c) for c in cams_in]
    X = voxel_centres(origin, voxel, dims, index)
    n = X.shape[0]
    T = torch.zeros(n, dtype=DT) if state is None else _t(state["tsdf"]).clone()
    Wt = torch.zeros(n, dtype=DT) if state is None else _t(state["weight"]).clone()
    Cl = torch.zeros(n, 3, dtype=DT) if state is None else _t(state["color"]).clone()
    amb = torch.zeros(n, dtype=torch.bool)
    for v, c in enumerate(cams):
        D = _t(depths[v])
        H, W = D.shape
        pc = _to_cam(c, X)
        z = pc[:, 2]
        front = z > near
        zs = torch.where(front, z, torch.ones_like(z))
        u = c["fx"] * pc[:, 0] / zs + c["cx"]
        w = c["fy"] * pc[:, 1] / zs + c["cy"]
        px, py = torch.floor(u), torch.floor(w)
        inside = front & (px >= 0) & (py >= 0) & (px <= W - 1) & (py <= H - 1)
        ix = px.clamp(0, W - 1).long()
        iy = py.clamp(0, H - 1).long()
        d = D[iy, ix]
        sdf = d - z
        upd = inside & (d > 0) & (sdf >= -trunc)
        obs = torch.clamp(sdf / trunc, max=1.0)
        T = torch.where(upd, (T * Wt + obs) / (Wt + 1), T)
        if colors is not None:
            col = _t(colors[v])[:, iy, ix].T
            Cl = torch.where(upd[:, None], (Cl * Wt[:, None] + col) / (Wt[:, None] + 1), Cl)
        Wt = torch.where(upd, Wt + 1, Wt)
        fu, fw = u - px, w - py
        amb |= front & (((fu < AMB_TSDF_PIX) | (fu > 1 - AMB_TSDF_PIX) | (fw < AMB_TSDF_PIX)
                         | (fw > 1 - AMB_TSDF_PIX)) & (u > -1) & (w > -1) & (u < W + 1) & (w < H + 1))
        amb |= inside & (d > 0) & ((sdf + trunc).abs() < AMB_TSDF_SDF)
        amb |= (z - near).abs() < AMB_TSDF_NEAR * max(1.0, near)
    return dict(tsdf=T, weight=Wt, color=Cl, amb=amb)
