"""Pins of the oracle's enhanced depth prior (Sec. 3.4, Step 2) against
closed forms: exact recovery of a known scale and shift, zero re-projection
error for consistent depths, the two-view disparity formula for a depth error,
and the handling of unverifiable pixels and missing priors."""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2503_23044_b300 import synth

F, W, H = 100.0, 64, 48
DOWN = np.array([[1, 0, 0], [0, -1, 0], [0, 0, -1]], np.float64)   # camera looking along world -z


def cam_at(cx, cy, h, width=W, height=H, f=F):
    c = np.array([cx, cy, h], np.float64)
    return synth.Camera(R=DOWN.astype(np.float32), t=(-DOWN @ c).astype(np.float32), fx=f, fy=f,
                        cx=width / 2.0, cy=height / 2.0, width=width, height=height)


def plane_depth(cam, h, alpha=0.0):
    """z-depth of the plane z = alpha * x seen by a downward camera centred at (x0, y0, h)."""
    c = O.camera(cam)
    vv, uu = torch.meshgrid(torch.arange(cam.height, dtype=torch.float64) + 0.5,
                            torch.arange(cam.width, dtype=torch.float64) + 0.5, indexing="ij")
    xn = (uu - c["cx"]) / c["fx"]
    x0 = float(c["center"][0])
    # ray point (x0 + lam xn, ., h - lam) on z = alpha x:  h - lam = alpha (x0 + lam xn)
    return (h - alpha * x0) / (1.0 + alpha * xn)


def pixel_points(cam, depth, step=5):
    """World points at pixel centres (interior pixels, every step-th) at the given z-depth."""
    c = O.camera(cam)
    pts = []
    for j in range(2, cam.height - 2, step):
        for i in range(2, cam.width - 2, step):
            z = float(depth[j, i])
            pc = torch.tensor([z * (i + 0.5 - c["cx"]) / c["fx"], z * (j + 0.5 - c["cy"]) / c["fy"], z],
                              dtype=torch.float64)
            pts.append(((pc - c["t"]) @ c["R"]).numpy())
    return np.array(pts)


def test_scale_shift_recovered_exactly():
    cam = cam_at(0.3, 0.1, 2.0)
    z = plane_depth(cam, 2.0, alpha=0.4)
    s, t = 1.7, -0.35
    pseudo = (z - t) / s
    st = O.prior_scale_shift(O.camera(cam), pseudo, torch.tensor(pixel_points(cam, z)), 0.01)
    assert abs(st[0] - s) < 1e-9 and abs(st[1] - t) < 1e-9 and st[2] > 50


def test_consistent_depths_have_zero_error_and_are_all_kept():
    cams = [cam_at(0.0, 0.0, 2.0), cam_at(0.15, 0.0, 2.0), cam_at(0.0, 0.12, 2.0)]
    pseudo = [plane_depth(c, 2.0) for c in cams]
    out = O.filter_depth_prior(cams, pseudo, np.zeros((0, 3)), tau_d=1.0, k=2)
    for v in out["views"]:
        chk = v["err"] >= 0
        assert int(chk.sum()) > 0.5 * W * H
        assert float(v["err"][chk].max()) < 1e-9
        assert bool((v["mask"] == 1).all())
        assert torch.allclose(v["prior"], torch.full_like(v["prior"], 2.0))
        assert v["scale"] == 1.0 and v["shift"] == 0.0      # constant depth: no spread, identity fit


@pytest.mark.parametrize("delta", [0.05, 0.3])
def test_depth_error_gives_the_disparity_closed_form(delta):
    """Parallel cameras with baseline b along x over a fronto-parallel plane at Z:
    a depth error delta at a pixel of view 0 moves its round trip by
    f b delta / (Z (Z + delta)) pixels."""
    Z, b = 2.0, 0.2
    cams = [cam_at(0.0, 0.0, Z), cam_at(b, 0.0, Z)]
    pseudo = [plane_depth(c, Z).clone() for c in cams]
    j0, i0 = 20, 40                       # a 3 x 3 block of view 0, away from the frame edges
    pseudo[0][j0 - 1:j0 + 2, i0 - 1:i0 + 2] += delta
    out = O.filter_depth_prior(cams, pseudo, np.zeros((0, 3)), tau_d=1.0, k=1)
    e = float(out["views"][0]["err"][j0, i0])
    b_stored = float(np.float32(b))       # the cameras hold t in FP32
    expect = F * b_stored * delta / (Z * (Z + delta))
    assert abs(e - expect) < 1e-9 * max(1.0, expect)
    assert float(out["views"][0]["mask"][j0, i0]) == (1.0 if expect <= 1.0 else 0.0)
    # the unperturbed pixels of view 0 that view 1 sees round-trip exactly
    other = out["views"][0]["err"].clone()
    other[j0 - 3:j0 + 4, i0 - 3:i0 + 4] = -1
    assert float(other[other >= 0].max()) < 1e-9


def test_unverifiable_pixels_kept_and_missing_prior_masked():
    cams = [cam_at(0.0, 0.0, 2.0), cam_at(5.0, 0.0, 2.0)]     # no overlap
    pseudo = [plane_depth(c, 2.0).clone() for c in cams]
    pseudo[0][:5, :] = 0.0                                   # no prior in the top rows of view 0
    out = O.filter_depth_prior(cams, pseudo, np.zeros((0, 3)), tau_d=1.0, k=1)
    v = out["views"][0]
    assert bool((v["err"][5:] == -1).all())
    assert bool((v["mask"][5:] == 1).all()) and bool((v["mask"][:5] == 0).all())
    assert bool((v["prior"][:5] == 0).all())


def test_nearest_views_by_camera_centre():
    cams = [O.camera(cam_at(x, 0.0, 2.0)) for x in (0.0, 1.0, 0.3, 5.0)]
    assert O.nearest_views(cams, 2) == [[2, 1], [2, 0], [0, 1], [1, 2]]
