"""Pins of the oracle's small helpers against textbook facts (CPU):
bilinear reads (exact at pixel centres and on bilinear data), the slope of the
bilinear interpolant, BT.601 luma weights, quaternion normalisation and the
L1-sign ambiguity flags."""
import math

import torch

import oracle as O
from oracle import pgs_oracle as P

D = torch.float64


def _grid(H, W, f):
    y, x = torch.meshgrid(torch.arange(H, dtype=D) + 0.5, torch.arange(W, dtype=D) + 0.5, indexing="ij")
    return f(x, y)


def test_bilinear_is_exact_at_pixel_centres():
    img = torch.arange(20, dtype=D).reshape(4, 5) ** 1.5
    y, x = torch.meshgrid(torch.arange(1, 3, dtype=D) + 0.5, torch.arange(1, 4, dtype=D) + 0.5, indexing="ij")
    assert torch.equal(P._bilinear(img, x, y), img[1:3, 1:4])


def test_bilinear_reproduces_bilinear_data():
    # a + b x + c y + d x y is reproduced exactly by bilinear interpolation
    f = lambda x, y: 0.3 + 1.7 * x - 0.6 * y + 0.25 * x * y
    img = _grid(6, 7, f)
    g = torch.Generator().manual_seed(0)
    x = 0.5 + torch.rand(200, generator=g, dtype=D) * 5.999
    y = 0.5 + torch.rand(200, generator=g, dtype=D) * 4.999
    assert torch.allclose(P._bilinear(img, x, y), f(x, y), rtol=0, atol=1e-12)


def test_bilinear_worked_case():
    img = torch.tensor([[0.0, 1.0], [2.0, 3.0]], dtype=D)
    # the point midway between the four centres averages them; a quarter of the way along x
    assert float(P._bilinear(img, torch.tensor([1.0], dtype=D), torch.tensor([1.0], dtype=D))) == 1.5
    assert float(P._bilinear(img, torch.tensor([0.75], dtype=D), torch.tensor([0.5], dtype=D))) == 0.25


def test_bilinear_slope_of_an_affine_image():
    img = _grid(5, 6, lambda x, y: 2.0 - 3.0 * x + 4.0 * y)
    x = torch.tensor([1.2, 2.7, 4.9], dtype=D)
    y = torch.tensor([0.9, 2.2, 3.6], dtype=D)
    assert torch.allclose(P._bilinear_slope(img, x, y), torch.full((3,), 5.0, dtype=D), atol=1e-12)


def test_luma_uses_bt601_weights():
    rgb = torch.eye(3, dtype=D).reshape(3, 3, 1)
    assert torch.allclose(O.luma(rgb)[:, 0], torch.tensor([0.299, 0.587, 0.114], dtype=D), atol=1e-15)
    grey = torch.full((3, 2, 2), 0.37, dtype=D)
    assert torch.allclose(O.luma(grey), torch.full((2, 2), 0.37, dtype=D), atol=1e-15)


def test_normalize_quat_unit_identity_and_sign():
    g = torch.Generator().manual_seed(1)
    q = torch.randn(50, 4, generator=g, dtype=D)
    n = O.normalize_quat(q)
    assert torch.allclose(n.norm(dim=-1), torch.ones(50, dtype=D), atol=1e-14)
    assert torch.equal(O.normalize_quat(torch.zeros(1, 4, dtype=D)), torch.tensor([[1.0, 0.0, 0.0, 0.0]], dtype=D))
    R1, R2 = O.quat_to_rotmat(n), O.quat_to_rotmat(-n)
    assert torch.allclose(R1, R2, atol=1e-14)
    eye = torch.eye(3, dtype=D).expand(50, 3, 3)
    assert torch.allclose(R1.transpose(-1, -2) @ R1, eye, atol=1e-13)
    assert torch.allclose(torch.linalg.det(R1), torch.ones(50, dtype=D), atol=1e-13)


def test_quarter_turn_about_z_maps_x_to_y():
    h = math.sqrt(0.5)
    R = O.quat_to_rotmat(O.normalize_quat(torch.tensor([[h, 0.0, 0.0, h]], dtype=D)))[0]
    assert torch.allclose(R @ torch.tensor([1.0, 0.0, 0.0], dtype=D), torch.tensor([0.0, 1.0, 0.0], dtype=D),
                          atol=1e-15)


def test_loss_ambiguity_flags_residuals_within_tolerance():
    H, W = 2, 3
    m = dict(rgb=torch.zeros(3, H, W, dtype=D), depth=torch.full((H, W), 2.0, dtype=D))
    t = dict(rgb=torch.full((3, H, W), 0.5, dtype=D), prior=torch.full((H, W), 1.0, dtype=D),
             mask=torch.ones(H, W, dtype=D))
    t["rgb"][1, 0, 0] = 1e-7                        # colour residual within tolerance
    t["prior"][1, 2] = 2.0 + 5e-6                   # masked depth residual within tolerance
    t["prior"][0, 2] = 2.0                          # same, but the pixel is outside the mask
    t["mask"][0, 2] = 0.0
    f = O.loss_ambiguity([m], [t], tol=1e-5)[0]
    expect = torch.zeros(H, W, dtype=torch.bool)
    expect[0, 0] = True
    expect[1, 2] = True
    assert torch.equal(f, expect)
