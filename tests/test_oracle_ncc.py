"""Pins of the oracle's batch geometric NCC (Sec. 3.4, Step 3, Eq. 10) against
closed forms and independent constructions: the homography against a
ray-plane intersection done in world coordinates, the pure shift of
fronto-parallel stereo, NCC against the Pearson correlation of numpy, its
invariance to an affine change of brightness, the pairing of the batch, the
validity rules, the stop-gradient, finite differences of the gradients and the
behaviour on true against wrong geometry of a textured terrain."""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2503_23044_b300 import synth

F, W, H = 60.0, 48, 40
DOWN = np.array([[1, 0, 0], [0, -1, 0], [0, 0, -1]], np.float64)   # camera looking along world -z


def cam_at(cx, cy, h, R=DOWN, width=W, height=H, f=F):
    c = np.array([cx, cy, h], np.float64)
    return synth.Camera(R=R.astype(np.float32), t=(-R @ c).astype(np.float32), fx=f, fy=f,
                        cx=width / 2.0, cy=height / 2.0, width=width, height=height)


def rot(axis, ang):
    a = np.asarray(axis, np.float64) / np.linalg.norm(axis)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * K @ K


def plane_maps(cam, h, alpha, tex):
    """D_hat, N_hat and colour of the plane z = alpha x (world) seen by a camera
    at height h looking down; colour = tex(world x, world y) at pixel centres."""
    c = O.camera(cam)
    vv, uu = torch.meshgrid(torch.arange(cam.height, dtype=torch.float64) + 0.5,
                            torch.arange(cam.width, dtype=torch.float64) + 0.5, indexing="ij")
    xn, yn = (uu - c["cx"]) / c["fx"], (vv - c["cy"]) / c["fy"]
    x0, y0 = float(c["center"][0]), float(c["center"][1])
    z = (h - alpha * x0) / (1.0 + alpha * xn)                       # camera z-depth
    xw, yw = x0 + z * xn, y0 - z * yn
    nw = torch.tensor([-alpha, 0.0, 1.0], dtype=torch.float64)
    ncam = c["R"] @ (nw / nw.norm())
    normal = ncam.view(3, 1, 1).expand(3, cam.height, cam.width).clone()
    return dict(rgb=tex(xw, yw), depth=z, normal=normal)


def smooth_tex(xw, yw):
    return torch.stack([0.5 + 0.3 * torch.sin(7 * xw + 2 * yw), 0.5 + 0.3 * torch.cos(5 * yw - 3 * xw),
                        0.5 + 0.2 * torch.sin(4 * xw) * torch.cos(6 * yw)], 0)


def test_pairs_of_the_batch():
    assert O.ncc_pairs(8) == [(1, 0), (3, 2), (5, 4), (7, 6)]
    assert O.ncc_pairs(3) == [(1, 0)]
    assert O.ncc_pairs(1) == []


def test_homography_matches_ray_plane_intersection():
    """H q must land where the ray of q meets the plane, carried to the partner
    through world coordinates (no relative pose is formed)."""
    rng = np.random.default_rng(0)
    cr = O.camera(cam_at(0.1, -0.2, 2.0, R=rot([0.3, 1, 0.2], 0.4) @ DOWN))
    cs = O.camera(cam_at(0.6, 0.1, 2.3, R=rot([1, -0.4, 0.5], -0.3) @ DOWN))
    m = torch.tensor(rng.normal(0, 0.1, (5, 3)) + np.array([0, 0, 0.5]))
    Hm = O.plane_homography(cr, cs, m)
    for k in range(5):
        for _ in range(10):
            q = np.array([rng.uniform(0, W), rng.uniform(0, H)])
            r = np.array([(q[0] - cr["cx"]) / cr["fx"], (q[1] - cr["cy"]) / cr["fy"], 1.0])
            lam = 1.0 / float(m[k].numpy() @ r)
            X = lam * r                                           # on m . X = 1, reference frame
            Xw = cr["R"].numpy().T @ (X - cr["t"].numpy())
            Xs = cs["R"].numpy() @ Xw + cs["t"].numpy()
            u = np.array([cs["fx"] * Xs[0] / Xs[2] + cs["cx"], cs["fy"] * Xs[1] / Xs[2] + cs["cy"]])
            h = Hm[k].numpy() @ np.array([q[0], q[1], 1.0])
            assert np.allclose(h[:2] / h[2], u, rtol=0, atol=1e-9), (k, h[:2] / h[2], u)


def test_fronto_parallel_stereo_is_a_shift():
    """Parallel cameras with baseline b along x over the plane z = 0 seen from
    height Z: the reference camera sits at x = b, the partner at x = 0, so
    every warped sample moves by +f b / Z along x."""
    Z, b = 2.0, 0.25
    cams = [cam_at(0.0, 0.0, Z), cam_at(b, 0.0, Z)]
    ref = plane_maps(cams[1], Z, 0.0, smooth_tex)
    part = plane_maps(cams[0], Z, 0.0, smooth_tex)
    centers = torch.tensor([20 * W + 30, 10 * W + 24])
    out = O.ncc_patches(O.camera(cams[1]), O.camera(cams[0]), ref, part["rgb"], centers)
    shift = F * float(np.float32(b)) / Z                          # the cameras hold t in FP32
    for j, c in enumerate(centers.tolist()):
        cy, cx = divmod(c, W)
        off = torch.arange(-3, 4, dtype=torch.float64)
        qy, qx = torch.meshgrid(off + cy + 0.5, off + cx + 0.5, indexing="ij")
        wx, wy = out["warped"][j, :, 0].view(7, 7), out["warped"][j, :, 1].view(7, 7)
        assert torch.allclose(wx, qx + shift, atol=1e-9)
        assert torch.allclose(wy, qy, atol=1e-9)
    assert bool(out["valid"].all())


def test_ncc_is_the_pearson_correlation():
    rng = np.random.default_rng(1)
    a, b = rng.normal(size=(20, 49)), rng.normal(size=(20, 49))
    b[:5] = 0.3 * a[:5] + 0.1 * b[:5]
    v = O.ncc(torch.tensor(a), torch.tensor(b), eps=0.0).numpy()
    ref = np.array([np.corrcoef(a[i], b[i])[0, 1] for i in range(20)])
    assert np.allclose(v, ref, atol=1e-12)


@pytest.mark.parametrize("alpha,beta", [(0.6, 0.2), (-1.5, 0.9)])
def test_affine_brightness_change_gives_plus_or_minus_one(alpha, beta):
    """Disparity of exactly 3 pixels: the warped samples fall on pixel centres
    of the partner, whose luma is alpha * (reference luma) + beta."""
    Z = 2.5
    b = 3.0 * Z / F                                               # 0.125: exact in FP32
    cams = [cam_at(0.0, 0.0, Z), cam_at(b, 0.0, Z)]
    cr, cs = O.camera(cams[1]), O.camera(cams[0])
    assert (float(cs["t"][0]) - float(cr["t"][0])) * F / Z == 3.0
    rng = np.random.default_rng(2)
    g_ref = torch.tensor(rng.uniform(0, 1, (H, W)))
    ref = dict(rgb=g_ref.expand(3, H, W).clone(), depth=torch.full((H, W), Z, dtype=torch.float64),
               normal=torch.tensor([0.0, 0.0, -1.0], dtype=torch.float64).view(3, 1, 1).expand(3, H, W).clone())
    g_part = torch.zeros(H, W, dtype=torch.float64)
    g_part[:, 3:] = alpha * g_ref[:, :-3] + beta                  # partner pixel x + 3 shows reference pixel x
    centers = torch.tensor([y * W + x for y in (8, 20, 31) for x in (6, 20, 40)])
    out = O.ncc_patches(cr, cs, ref, g_part.expand(3, H, W), centers, eps=0.0)
    assert bool(out["valid"].all())
    assert torch.allclose(out["ncc"], torch.full_like(out["ncc"], math.copysign(1.0, alpha)), atol=1e-12)


def test_validity_rules():
    Z, b = 2.0, 0.25
    cams = [cam_at(0.0, 0.0, Z), cam_at(b, 0.0, Z)]
    ref = plane_maps(cams[1], Z, 0.0, smooth_tex)
    part = plane_maps(cams[0], Z, 0.0, smooth_tex)
    cr, cs = O.camera(cams[1]), O.camera(cams[0])
    # the shift is +7.5 px: the last warped sample of a patch at x sits at x + 11,
    # and its bilinear footprint needs it below W - 1/2
    cases = {2 * W + 20: False,           # patch leaves the reference frame (y = 2 < 3)
             20 * W + 45: False,          # x = 45 > W - 4
             20 * W + 37: False,          # x + 11 = 48 > 47.5: leaves the partner on the right
             20 * W + 36: True,
             20 * W + 3: True}
    out = O.ncc_patches(cr, cs, ref, part["rgb"], torch.tensor(list(cases)))
    assert out["valid"].tolist() == list(cases.values())
    no_depth = dict(ref, depth=ref["depth"].clone())
    no_depth["depth"][20, 30] = 0.0
    out = O.ncc_patches(cr, cs, no_depth, part["rgb"], torch.tensor([20 * W + 30, 20 * W + 31]))
    assert out["valid"].tolist() == [False, True]
    # a pair with no valid patch adds 0; the batch mean still divides by B/2
    res = O.ncc_loss([cams[0], cams[1], cams[0], cam_at(9.0, 0.0, Z)],
                     [part, ref, part, plane_maps(cam_at(9.0, 0.0, Z), Z, 0.0, smooth_tex)],
                     [[20 * W + 30], [20 * W + 30]], grad=False)
    assert res["pairs"][1]["n_valid"] == 0
    assert abs(res["loss"] - res["pairs"][0]["loss"] / 2) < 1e-15


def _two_view_case(alpha=0.3):
    Z = 2.0
    cams = [cam_at(0.0, 0.05, Z), cam_at(0.12, -0.03, Z + 0.1)]
    maps = [plane_maps(cams[0], Z, alpha, smooth_tex), plane_maps(cams[1], Z + 0.1, alpha, smooth_tex)]
    # move the reference geometry off the truth so the loss has a slope
    maps[1]["depth"] = maps[1]["depth"] * 1.02
    maps[1]["normal"] = maps[1]["normal"] + torch.tensor([0.05, -0.03, 0.0], dtype=torch.float64).view(3, 1, 1)
    return cams, maps


def test_gradients_match_finite_differences():
    cams, maps = _two_view_case()
    cr, cs = O.camera(cams[1]), O.camera(cams[0])
    cand = torch.tensor([y * W + x for y in range(6, H - 6, 5) for x in range(10, W - 6, 6)])
    chk = O.ncc_patches(cr, cs, maps[1], maps[0]["rgb"], cand)
    centers = cand[chk["valid"] & ~chk["cell"]][:6]
    assert centers.numel() == 6
    res = O.ncc_loss(cams, maps, [centers.tolist()], geo=True, lam=1.0)
    g = res["grads"]
    assert float(g[0]["rgb"].abs().max()) == 0.0                 # partner colour under stop-gradient
    assert float(g[0]["depth"].abs().max()) == 0.0 and float(g[0]["normal"].abs().max()) == 0.0

    def L(mod):
        mp = [{k: v.clone() for k, v in m.items()} for m in maps]
        mod(mp)
        return O.ncc_loss(cams, mp, [centers.tolist()], grad=False)["loss"]

    h = 1e-6
    c0 = int(centers[0])
    cy, cx = divmod(c0, W)
    probes = [("depth", (cy, cx)), ("normal", (0, cy, cx)), ("normal", (1, cy, cx)), ("normal", (2, cy, cx)),
              ("rgb", (0, cy, cx)), ("rgb", (1, cy + 2, cx - 1)), ("rgb", (2, cy - 3, cx + 3))]
    for key, idx in probes:
        def plus(mp, s=1.0):
            mp[1][key][idx] += s * h
        fd = (L(lambda mp: plus(mp, 1.0)) - L(lambda mp: plus(mp, -1.0))) / (2 * h)
        an = float(g[1][key][idx])
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)) + 1e-9, (key, idx, fd, an)
    # NCC ignores a brightness offset of the reference patch, so each patch's colour gradient sums to zero
    for ch in range(3):
        assert abs(float(g[1]["rgb"][ch].sum())) <= 1e-12 * float(g[1]["rgb"][ch].abs().sum())
    # the literal stop-gradient: the same colour gradient, no geometric one
    lit = O.ncc_loss(cams, maps, [centers.tolist()], geo=False)["grads"]
    assert float(lit[1]["depth"].abs().max()) == 0.0 and float(lit[1]["normal"].abs().max()) == 0.0
    assert torch.allclose(lit[1]["rgb"], g[1]["rgb"], atol=1e-15)


@pytest.mark.parametrize("pos,yaw", [((0.0, -1.0), math.pi / 2), ((0.5, 0.5), 0.3), ((-1.0, 0.2), 2.0)])
def test_true_geometry_correlates_and_wrong_geometry_does_not(pos, yaw):
    """An aerial view of the textured terrain and a partner displaced by 0.3
    along its image x axis (disparity ~20 px): with the true depth and normal
    the warped patches match (NCC near 1); a 60% depth error moves them by
    ~8 px and raises the loss by more than 0.2."""
    sc = synth.anchor_scene("batch8_1600", n_anchors=1000, resolutions=[(160, 106)] * 8)
    ter = sc["terrain"]
    g = float(ter.height(np.array(pos[0]), np.array(pos[1])))
    c1 = synth.look_camera((pos[0], pos[1], g + 1.5), yaw, math.radians(50.0), 160, 106)
    R = c1.R.astype(np.float64)
    centre = c1.center().astype(np.float64) + 0.3 * R[0]
    c0 = synth.Camera(R=c1.R, t=(-R @ centre).astype(np.float32), fx=c1.fx, fy=c1.fy, cx=c1.cx, cy=c1.cy,
                      width=c1.width, height=c1.height)
    pair_cams = [c0, c1]
    maps = []
    for v, c in enumerate(pair_cams):
        tg = synth.march_targets(ter, c, stride=1, seed=v)
        maps.append(dict(rgb=tg["rgb"].double(), depth=tg["depth"].double(), normal=tg["normal"].double()))
    centers = np.random.default_rng(0).integers(0, 160 * 106, 3000)
    good = O.ncc_loss(pair_cams, maps, [centers], grad=False)
    gp = good["pairs"][0]
    assert gp["n_valid"] > 1000
    assert float(gp["ncc"][gp["valid"]].median()) > 0.999
    assert float(gp["ncc"][gp["valid"]].mean()) > 0.99
    bad = O.ncc_loss(pair_cams, [maps[0], dict(maps[1], depth=maps[1]["depth"] * 1.6)], [centers], grad=False)
    assert bad["loss"] > good["loss"] + 0.2
