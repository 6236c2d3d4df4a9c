"""Helpers shared by the GPU parity tests: build CUDA scenes from the seeded
generator's output and compare them with the oracle.  Both sides get only the
generator's inputs."""
from __future__ import annotations

import numpy as np
import torch

import oracle as O
from paper_2503_23044_b300 import binding as B


def oracle_params(p: B.RenderParams) -> O.RenderParams:
    return O.RenderParams(near=p.near_plane, dilation=p.dilation, alpha_min=p.alpha_min, alpha_max=p.alpha_max,
                          t_min=p.t_min, jclamp=p.jclamp, tile=p.tile_w, tile_pad=p.tile_pad, lod_d0=p.lod_d0,
                          n_levels=p.n_levels, bg=p.bg)


def npix(cams):
    return sum(int(c.width) * int(c.height) for c in cams)


def explicit_gpu(sc, params=None, cap_pairs=None):
    N = len(sc["means"])
    cams = sc["cameras"]
    params = params if params is not None else B.default_params()
    cap_pairs = cap_pairs or max(1 << 16, 400 * N * len(cams))
    scene = B.Scene(B.MODE_EXPLICIT, N, len(cams), npix(cams), min(cap_pairs, (1 << 30) - 1), params=params)
    t = {k: torch.tensor(np.asarray(sc[k], np.float32), device="cuda").contiguous()
         for k in ("means", "log_scales", "quats", "opacity_logits", "colors")}
    scene.bind_explicit(t["means"], t["log_scales"], t["quats"], t["opacity_logits"], t["colors"])
    return scene, t


def anchor_params(sc, **kw):
    return B.default_params(lod_d0=float(sc["lod_d0"]), n_levels=int(sc["n_levels"]), **kw)


def anchor_gpu(sc, params=None, cap_rows=None, cap_pairs=None):
    cams = sc["cameras"]
    Na = len(sc["x"])
    params = params if params is not None else anchor_params(sc)
    cap_rows = cap_rows or Na * len(cams)
    cap_pairs = cap_pairs or (1 << 28)
    scene = B.Scene(B.MODE_ANCHOR, Na, len(cams), npix(cams), cap_pairs, capacity_rows=cap_rows, params=params)
    t = {k: torch.tensor(np.asarray(sc[k]), device="cuda").contiguous() for k in ("x", "level", "log_l", "offsets", "feat")}
    for k, v in sc["mlp"].items():
        t[k] = torch.tensor(np.asarray(v, np.float32), device="cuda").contiguous()
    scene.bind_anchors(t["x"], t["level"], t["log_l"], t["offsets"], t["feat"], t["W1"], t["b1"], t["W2"], t["b2"])
    return scene, t


def rel_l2(a: torch.Tensor, b: torch.Tensor) -> float:
    a = a.double().cpu()
    b = b.double().cpu()
    den = float(torch.linalg.norm(b))
    return float(torch.linalg.norm(a - b)) / max(den, 1e-30)


def crop_view(img: dict, crop):
    x0, y0, w, h = crop
    return {k: v[..., y0:y0 + h, x0:x0 + w] for k, v in img.items()}


def image_errors(gpu: dict, orc: dict, flag: torch.Tensor) -> dict:
    """Max errors over unflagged pixels: colour / normal absolute, depth relative."""
    ok = ~flag
    g_rgb, o_rgb = gpu["rgb"].double().cpu(), orc["rgb"]
    g_n, o_n = gpu["normal"].double().cpu(), orc["normal"]
    g_d, o_d = gpu["depth"].double().cpu(), orc["depth"]
    e_rgb = (g_rgb - o_rgb).abs().amax(0)[ok]
    e_n = (g_n - o_n).abs().amax(0)[ok]
    e_d = ((g_d - o_d).abs() / o_d.abs().clamp(min=1e-6))[ok & (o_d.abs() > 0)]
    e_t = (gpu["t_final"].double().cpu() - orc["T_final"]).abs()[ok]
    nc = gpu["n_contrib"].cpu().long()
    mx = lambda e: float(e.max()) if e.numel() else 0.0
    return dict(rgb=mx(e_rgb), normal=mx(e_n), depth_rel=mx(e_d), t_final=mx(e_t),
                n_contrib_mismatch=int((nc != orc["n_contrib"])[ok].sum()), flagged=float(flag.float().mean()))
