"""Pins of the oracle's TSDF fusion of rendered depth (supplementary, mesh
reconstruction) against closed forms: a camera looking straight down at a flat
ground gives tsdf = min(1, h / trunc) by world height h, two views average
their observations (depths and colours), the nearest pixel is the one read,
voxels behind the truncation band or outside every frustum stay empty, and
fusing a batch at once equals fusing its views one after the other."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2503_23044_b300 import synth

F, W, H = 50.0, 40, 30
DOWN = np.array([[1, 0, 0], [0, -1, 0], [0, 0, -1]], np.float64)   # camera looking along world -z


def cam_at(cx, cy, h):
    c = np.array([cx, cy, h], np.float64)
    return synth.Camera(R=DOWN.astype(np.float32), t=(-DOWN @ c).astype(np.float32), fx=F, fy=F,
                        cx=W / 2.0, cy=H / 2.0, width=W, height=H)


# a small volume under the cameras: 16 x 12 x 20 voxels of 0.01 around the ground z = 0
ORIGIN, VOXEL, DIMS, TRUNC = (-0.08, -0.06, -0.1), 0.01, (16, 12, 20), 0.04


def test_voxel_layout_is_x_fastest():
    idx = torch.tensor([0, 1, 16, 16 * 12, 16 * 12 * 3 + 16 * 5 + 7])
    c = O.voxel_centres(ORIGIN, VOXEL, DIMS, idx)
    ijk = torch.tensor([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [7, 5, 3]], dtype=torch.float64)
    assert torch.allclose(c, torch.tensor(ORIGIN, dtype=torch.float64) + (ijk + 0.5) * VOXEL, atol=1e-15)


def test_flat_ground_seen_from_above():
    """Depth Z everywhere (the ground z = 0 from height Z): a voxel at world
    height h has projective distance h, so tsdf = min(1, h / trunc) for
    h >= -trunc and no update below."""
    Z = 1.0
    cam = cam_at(0.0, 0.0, Z)
    out = O.tsdf_fuse([cam], [torch.full((H, W), Z, dtype=torch.float64)], ORIGIN, VOXEL, DIMS, TRUNC)
    X = O.voxel_centres(ORIGIN, VOXEL, DIMS)
    h = X[:, 2]
    z_cam = Z - h                                                        # camera depth of the voxel centre
    expect_w = (h >= -TRUNC - 1e-12).double()
    # every voxel of this volume projects inside the frame (|x| <= 0.08 at depth >= 0.9: |u - cx| <= 4.5 px)
    assert torch.equal(out["weight"], expect_w)
    exp_t = torch.clamp((Z - z_cam) / TRUNC, max=1.0)
    assert torch.allclose(out["tsdf"][expect_w > 0], exp_t[expect_w > 0], atol=1e-12)
    assert bool((out["tsdf"][expect_w == 0] == 0).all())
    # the zero crossing lies at the ground: tsdf changes sign between the layers at h = -0.005 and +0.005
    layer = lambda k: out["tsdf"].view(20, 12, 16)[k]
    assert bool((layer(9) < 0).all()) and bool((layer(10) > 0).all())


def test_two_views_average_depths_and_colours():
    Z = 1.0
    cams = [cam_at(0.0, 0.0, Z), cam_at(0.02, 0.01, Z)]
    d0 = torch.full((H, W), Z, dtype=torch.float64)
    d1 = torch.full((H, W), Z + 0.01, dtype=torch.float64)       # the second view sees the ground 0.01 lower
    c0 = torch.tensor([0.2, 0.4, 0.6], dtype=torch.float64).view(3, 1, 1).expand(3, H, W)
    c1 = torch.tensor([0.6, 0.0, 0.2], dtype=torch.float64).view(3, 1, 1).expand(3, H, W)
    out = O.tsdf_fuse(cams, [d0, d1], ORIGIN, VOXEL, DIMS, TRUNC, colors=[c0, c1])
    X = O.voxel_centres(ORIGIN, VOXEL, DIMS)
    h = X[:, 2]
    both = (h >= -TRUNC + 0.01 + 1e-9)                            # inside both truncation bands
    assert bool((out["weight"][both] == 2).all())
    o0 = torch.clamp(h / TRUNC, max=1.0)
    o1 = torch.clamp((h + 0.01) / TRUNC, max=1.0)
    assert torch.allclose(out["tsdf"][both], (0.5 * (o0 + o1))[both], atol=1e-6)
    assert torch.allclose(out["color"][both], torch.tensor([0.4, 0.2, 0.4], dtype=torch.float64).expand(int(both.sum()), 3),
                          atol=1e-12)
    only1 = (h < -TRUNC - 1e-9) & (h >= -TRUNC - 0.01 + 1e-9)     # in the second view's band only
    assert bool((out["weight"][only1] == 1).all())
    assert torch.allclose(out["color"][only1], c1[:, 0, 0].expand(int(only1.sum()), 3), atol=1e-12)


def test_nearest_pixel_is_read():
    """A depth map that changes along x: each voxel reads the pixel its centre
    projects into (floor of u), not an interpolation."""
    Z = 1.0
    cam = cam_at(0.0, 0.0, Z)
    depth = (Z + 0.003 * torch.arange(W, dtype=torch.float64)).expand(H, W).clone()
    out = O.tsdf_fuse([cam], [depth], ORIGIN, VOXEL, DIMS, TRUNC)
    X = O.voxel_centres(ORIGIN, VOXEL, DIMS)
    c = O.camera(cam)
    pc = X @ c["R"].T + c["t"]
    u = c["fx"] * pc[:, 0] / pc[:, 2] + c["cx"]
    d = Z + 0.003 * torch.floor(u)
    sdf = d - pc[:, 2]
    upd = sdf >= -TRUNC
    assert torch.equal(out["weight"] > 0, upd)
    assert torch.allclose(out["tsdf"][upd], torch.clamp(sdf / TRUNC, max=1.0)[upd], atol=1e-12)


def test_outside_frustum_and_missing_depth_stay_empty():
    Z = 1.0
    far = cam_at(5.0, 0.0, Z)                                     # looks at other ground
    out = O.tsdf_fuse([far], [torch.full((H, W), Z, dtype=torch.float64)], ORIGIN, VOXEL, DIMS, TRUNC)
    assert float(out["weight"].abs().max()) == 0.0
    out = O.tsdf_fuse([cam_at(0.0, 0.0, Z)], [torch.zeros(H, W, dtype=torch.float64)], ORIGIN, VOXEL, DIMS, TRUNC)
    assert float(out["weight"].abs().max()) == 0.0


def test_batch_equals_sequential_fusion():
    rng = np.random.default_rng(0)
    cams = [cam_at(0.01 * k, -0.01 * k, 1.0 + 0.05 * k) for k in range(3)]
    depths = [torch.tensor(1.0 + 0.05 * k + rng.normal(0, 0.01, (H, W))) for k in range(3)]
    cols = [torch.tensor(rng.uniform(0, 1, (3, H, W))) for _ in range(3)]
    all3 = O.tsdf_fuse(cams, depths, ORIGIN, VOXEL, DIMS, TRUNC, colors=cols)
    st = None
    for k in range(3):
        st = O.tsdf_fuse(cams[k:k + 1], depths[k:k + 1], ORIGIN, VOXEL, DIMS, TRUNC, colors=cols[k:k + 1], state=st)
    for key in ("tsdf", "weight", "color"):
        assert torch.allclose(all3[key], st[key], atol=1e-15)
    assert float(all3["weight"].max()) == 3.0
