"""Pins of the FP64 oracle against closed forms, invariants and textbook
special cases (no GPU).  Each test names the passage of the paper whose
arithmetic it pins; a plausible slip in the oracle (dropped term, wrong sign
or index, transposed operand) fails at least one of them."""
import math

import numpy as np
import pytest
import torch
from scipy.spatial.transform import Rotation

import oracle as O
from paper_2503_23044_b300 import synth

RP = O.RenderParams()


def logit(p):
    return math.log(p / (1 - p))


def explicit(means, log_scales, quats, opac, colors, cam):
    return dict(kind="explicit", means=np.asarray(means, np.float64), log_scales=np.asarray(log_scales, np.float64),
                quats=np.asarray(quats, np.float64), opacity_logits=np.asarray([logit(o) for o in opac]),
                colors=np.asarray(colors, np.float64), cameras=[cam])


def quat_wxyz(rot: Rotation):
    x, y, z, w = rot.as_quat()
    return [w, x, y, z]


# ----------------------------------------------------------------- Eq. 1 / Eq. 5
def test_single_gaussian_peak_and_onaxis_ewa():
    """On-axis isotropic Gaussian: mean2D = principal point, cov2D = ((f s/z)^2
    + 0.3) I, and the pixel at the mean gets alpha = min(0.99, o)."""
    f, z, s = 40.0, 3.0, 0.05
    cam = synth.identity_camera(33, 33, f)                       # cx = cy = 16.5, a pixel centre
    for o in (0.6, 0.995):
        sc = explicit([[0, 0, z]], [[math.log(s)] * 3], [[1, 0, 0, 0]], [o], [[0.2, 0.5, 0.9]], cam)
        out = O.render(sc, RP)["views"][0]
        p = out["proj"]
        assert torch.allclose(p["mean2d"][0], torch.tensor([16.5, 16.5], dtype=O.DT), atol=1e-12)
        var = (f * s / z) ** 2 + 0.3
        assert abs(p["cov"][0, 0].item() - var) < 1e-12 and abs(p["cov"][0, 2].item() - var) < 1e-12
        assert abs(p["cov"][0, 1].item()) < 1e-15
        a = min(0.99, o)
        rgb = out["rgb"][:, 16, 16]
        assert torch.allclose(rgb, torch.tensor([0.2, 0.5, 0.9], dtype=O.DT) * a, atol=1e-12)
        assert abs(out["T_final"][16, 16].item() - (1 - a)) < 1e-12
        # a pixel one step away follows the Gaussian profile
        a1 = o * math.exp(-0.5 * 1.0 / var)
        assert abs(out["rgb"][0, 16, 17].item() - 0.2 * min(a1, 0.99)) < 1e-12


def test_two_gaussian_hand_calculation():
    """C = c1 a1 + c2 a2 (1 - a1) with the nearer Gaussian first (Eq. 5);
    swapping the depths swaps the roles."""
    f = 40.0
    cam = synth.identity_camera(33, 33, f)
    o1, o2 = 0.7, 0.5
    c1, c2 = [1.0, 0.0, 0.25], [0.0, 1.0, 0.75]
    for z1, z2 in ((2.0, 4.0), (4.0, 2.0)):
        sc = explicit([[0, 0, z1], [0, 0, z2]], [[math.log(0.05)] * 3] * 2, [[1, 0, 0, 0]] * 2,
                      [o1, o2], [c1, c2], cam)
        out = O.render(sc, RP)["views"][0]
        rgb = out["rgb"][:, 16, 16].numpy()
        (ca, aa), (cb, ab) = ((c1, o1), (c2, o2)) if z1 < z2 else ((c2, o2), (c1, o1))
        want = np.asarray(ca) * aa + np.asarray(cb) * ab * (1 - aa)
        assert np.allclose(rgb, want, atol=1e-12)
        assert abs(out["T_final"][16, 16].item() - (1 - aa) * (1 - ab)) < 1e-12
        assert out["n_contrib"][16, 16].item() == 2


def test_weights_plus_transmittance_is_one():
    """Telescoping: sum_i w_i + T_final = 1 at every pixel (Eq. 1 weights)."""
    sc = synth.explicit_scene(n=300, seed=3, width=48, height=40, f=48.0)
    sc["colors"] = np.ones_like(sc["colors"])
    out = O.render(sc, RP)["views"][0]
    s = out["rgb"] + out["T_final"][None]
    assert torch.allclose(s, torch.ones_like(s), atol=1e-12)
    assert out["n_contrib"].max() > 3


def test_order_invariance_for_disjoint_splats():
    """Permuting the storage order of non-overlapping splats leaves the image unchanged."""
    cam = synth.identity_camera(64, 64, 64.0)
    rng = np.random.default_rng(0)
    g = np.stack(np.meshgrid(np.linspace(-0.6, 0.6, 4), np.linspace(-0.6, 0.6, 4)), -1).reshape(-1, 2)
    n = len(g)
    means = np.concatenate([g * 3.0, rng.uniform(2.5, 3.5, (n, 1))], 1)
    ls = np.full((n, 3), math.log(0.03))
    q = rng.normal(size=(n, 4))
    op = rng.uniform(0.3, 0.9, n)
    col = rng.uniform(0, 1, (n, 3))
    a = O.render(explicit(means, ls, q, op, col, cam), RP)["views"][0]
    perm = rng.permutation(n)
    b = O.render(explicit(means[perm], ls[perm], q[perm], op[perm], col[perm], cam), RP)["views"][0]
    assert torch.equal(a["rgb"], b["rgb"]) or torch.allclose(a["rgb"], b["rgb"], atol=1e-15)
    assert a["rgb"].max() > 0.2


# ----------------------------------------------------------------- EWA projection (3DGS)
def test_quaternion_matches_scipy():
    rng = np.random.default_rng(1)
    q = rng.normal(size=(20, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    R = O.quat_to_rotmat(torch.tensor(q)).numpy()
    ref = Rotation.from_quat(q[:, [1, 2, 3, 0]]).as_matrix()
    assert np.allclose(R, ref, atol=1e-13)


def test_ewa_covariance_matches_fd_jacobian():
    """cov2D = J W Sigma W^T J^T + 0.3 I with J the Jacobian of the pinhole map,
    here obtained by central differences and Sigma from scipy's rotation."""
    rng = np.random.default_rng(2)
    cam = synth.look_camera((0.3, -0.2, 1.0), 0.7, 0.4, 80, 60)
    c = O.camera(cam)
    n = 12
    mu_c = np.concatenate([rng.uniform(-0.3, 0.3, (n, 2)), rng.uniform(1.5, 3.0, (n, 1))], 1)
    R = c["R"].numpy()
    mu = (mu_c - c["t"].numpy()) @ R                             # world points
    mu_c = mu @ R.T + c["t"].numpy()                              # R is FP32-rounded, not exactly orthogonal
    s = np.exp(rng.normal(-3, 0.4, (n, 3)))
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    p = O.project(torch.tensor(mu), torch.tensor(s), torch.tensor(q), torch.full((n,), 0.5, dtype=O.DT),
                  torch.zeros(n, 3, dtype=O.DT), c, RP)

    def pin(X):
        return np.array([c["fx"] * X[0] / X[2] + c["cx"], c["fy"] * X[1] / X[2] + c["cy"]])

    for i in range(n):
        h = 1e-6
        J = np.stack([(pin(mu_c[i] + h * e) - pin(mu_c[i] - h * e)) / (2 * h) for e in np.eye(3)], 1)
        Rg = Rotation.from_quat(q[i, [1, 2, 3, 0]]).as_matrix()
        Sig = Rg @ np.diag(s[i] ** 2) @ Rg.T
        cov = J @ R @ Sig @ R.T @ J.T + 0.3 * np.eye(2)
        got = p["cov"][i].numpy()
        assert np.allclose([cov[0, 0], cov[0, 1], cov[1, 1]], got, rtol=1e-7, atol=1e-9)
        inv = np.linalg.inv(cov)
        assert np.allclose([inv[0, 0], inv[0, 1], inv[1, 1]], p["conic"][i].numpy(), rtol=1e-7)
        assert np.allclose(pin(mu_c[i]), p["mean2d"][i].numpy(), atol=1e-10)
        assert abs(p["z"][i].item() - mu_c[i, 2]) < 1e-12


# ----------------------------------------------------------------- Eq. 6-7
def _plane_gaussians(cam, n_plane, p0, k, rng, tiny=1e-7, spread=0.15):
    """k Gaussians lying in the plane through p0 with normal n_plane (world)."""
    n_plane = n_plane / np.linalg.norm(n_plane)
    a = np.cross(n_plane, [0.3, 0.9, 0.1])
    a /= np.linalg.norm(a)
    b = np.cross(n_plane, a)
    basis = np.stack([a, b, n_plane], 1)                          # columns: local x, y, z(normal)
    rot = Rotation.from_matrix(basis)
    uv = rng.uniform(-spread, spread, (k, 2))
    means = p0[None] + uv[:, :1] * a + uv[:, 1:] * b
    ls = np.log(np.stack([rng.uniform(0.05, 0.1, k), rng.uniform(0.05, 0.1, k), np.full(k, tiny)], 1))
    q = np.tile(quat_wxyz(rot), (k, 1))
    return means, ls, q


def test_coplanar_gaussians_give_exact_plane_depth_and_normal():
    """Eq. 7 invariant: for Gaussians sharing one plane, D_hat is the ray-plane
    z-depth and N/|N| the plane normal facing the camera, whatever the opacities."""
    rng = np.random.default_rng(4)
    cam = synth.look_camera((0.0, 0.0, 2.0), 0.3, 0.9, 40, 32)
    c = O.camera(cam)
    n_world = np.array([0.2, -0.1, 1.0])
    p0 = c["center"].numpy() + 2.2 * c["R"].numpy()[2]            # 2.2 along the optical axis
    means, ls, q = _plane_gaussians(cam, n_world, p0, 60, rng, spread=0.3)
    op = rng.uniform(0.2, 0.95, 60)
    sc = explicit(means, ls, q, op, rng.uniform(0, 1, (60, 3)), cam)
    out = O.render(sc, RP)["views"][0]
    R = c["R"].numpy()
    n_c = R @ (n_world / np.linalg.norm(n_world))
    p0_c = R @ p0 + c["t"].numpy()
    if n_c @ p0_c > 0:
        n_c = -n_c
    H, W = out["depth"].shape
    v, u = np.meshgrid(np.arange(H) + 0.5, np.arange(W) + 0.5, indexing="ij")
    r = np.stack([(u - c["cx"]) / c["fx"], (v - c["cy"]) / c["fy"], np.ones_like(u)], 0)
    want = (n_c @ p0_c) / np.einsum("k,khw->hw", n_c, r)
    covered = (1 - out["T_final"].numpy()) > 1e-3
    assert covered.sum() > 150
    got = out["depth"].numpy()
    assert np.allclose(got[covered], want[covered], rtol=1e-9)
    N = out["normal"].numpy()
    Nn = N / np.linalg.norm(N, axis=0, keepdims=True)
    assert np.allclose(Nn[:, covered], n_c[:, None], atol=1e-6)


def test_camera_looking_down_at_flat_gaussians_sees_minus_z_normal():
    rng = np.random.default_rng(5)
    cam = synth.look_camera((0.0, 0.0, 2.0), 0.0, math.pi / 2 - 1e-9, 24, 24)
    means, ls, q = _plane_gaussians(cam, np.array([0, 0, 1.0]), np.array([0, 0, 0.0]), 10, rng)
    out = O.render(explicit(means, ls, q, [0.8] * 10, np.ones((10, 3)), cam), RP)["views"][0]
    N = out["normal"][:, 12, 12].numpy()
    assert np.allclose(N / np.linalg.norm(N), [0, 0, -1], atol=1e-6)
    assert abs(out["depth"][12, 12].item() - 2.0) < 1e-6


# ----------------------------------------------------------------- Eq. 4 decoder, LoD
def test_decoder_matches_textbook_loops():
    sc = synth.tiny_anchor_scene(n_anchors=3, seed=7)
    lv = O.leaves_anchor(sc)
    cam = O.camera(sc["cameras"][0])
    idx = torch.arange(3)
    dec = O.decode(dict(x=lv["x"], feat=lv["feat"], log_l=lv["log_l"], offsets=lv["offsets"]),
                   {k: lv[k] for k in ("W1", "b1", "W2", "b2")}, cam, idx)
    W1, b1, W2, b2 = (sc["mlp"][k].astype(np.float64) for k in ("W1", "b1", "W2", "b2"))
    sig = lambda v: 1.0 / (1.0 + math.exp(-v))
    oc = cam["center"].numpy()
    for a in range(3):
        x = sc["x"][a].astype(np.float64)
        d = x - oc
        dist = math.sqrt(sum(t * t for t in d))
        X = list(sc["feat"][a].astype(np.float64)) + [t / dist for t in d]
        H = []
        for i in range(32):
            acc = b1[i]
            for j in range(35):
                acc += W1[i, j] * X[j]
            H.append(max(acc, 0.0))
        Z = []
        for i in range(110):
            acc = b2[i]
            for j in range(32):
                acc += W2[i, j] * H[j]
            Z.append(acc)
        l = [math.exp(v) for v in sc["log_l"][a]]
        for j in range(10):
            g = a * 10 + j
            assert abs(dec["opacity"][g].item() - sig(Z[j])) < 1e-12
            for ch in range(3):
                assert abs(dec["color"][g, ch].item() - sig(Z[10 + 3 * j + ch])) < 1e-12
                assert abs(dec["scale"][g, ch].item() - l[ch] * sig(Z[40 + 3 * j + ch])) < 1e-12
                assert abs(dec["mu"][g, ch].item() - (x[ch] + float(sc["offsets"][a, j, ch]) * l[ch])) < 1e-12
            qv = Z[70 + 4 * j: 74 + 4 * j]
            qn = math.sqrt(sum(t * t for t in qv))
            assert np.allclose(dec["quat"][g].detach().numpy(), [t / qn for t in qv], atol=1e-12)


def test_lod_rule_special_cases():
    """level <= clamp(floor(log2(d0/d)), 0, K-1), checked with math.log2."""
    rp = O.RenderParams(lod_d0=8.0, n_levels=3)
    cam = O.camera(synth.identity_camera(8, 8, 8.0))
    ds = np.array([0.5, 1.0, 1.5, 2.5, 3.0, 4.5, 7.9, 8.5, 30.0])
    x = torch.tensor(np.stack([np.zeros_like(ds), np.zeros_like(ds), ds], 1))
    for k in range(3):
        act, amb = O.lod_active(x, torch.full((len(ds),), k), cam, rp)
        want = [k <= min(max(math.floor(math.log2(8.0 / d)), 0), 2) for d in ds]
        assert act.tolist() == want
    act, amb = O.lod_active(torch.tensor([[0.0, 0.0, 4.0]]), torch.tensor([1]), cam, rp)
    assert amb.item()                                              # exactly on d0/2


# ----------------------------------------------------------------- losses (Eq. 8-9)
def test_losses_on_constant_maps():
    cam = synth.identity_camera(10, 8, 10.0)
    H, W = 8, 10
    tgt = dict(rgb=torch.full((3, H, W), 0.5), prior=torch.full((H, W), 3.0), mask=torch.zeros(H, W))
    tgt["mask"][:, :5] = 1.0
    c = O.camera(cam)
    # a fronto-parallel plane at depth 2: its depth-normal is (0, 0, -1)
    rgb = torch.full((3, H, W), 0.3, dtype=O.DT)
    depth = torch.full((H, W), 2.0, dtype=O.DT)
    normal = torch.zeros(3, H, W, dtype=O.DT)
    normal[2] = -2.0
    L = O.loss_view(rgb, depth, normal, tgt, c, O.LossParams())
    assert abs(L["rgb"].item() - 0.2) < 1e-12
    assert abs(L["depth"].item() - 1.0) < 1e-12
    assert abs(L["normal"].item()) < 1e-12 and L["n_valid"] == (H - 2) * (W - 2)
    normal[2] = 2.0
    L = O.loss_view(rgb, depth, normal, tgt, c, O.LossParams())
    assert abs(L["normal"].item() - 2.0) < 1e-12
    val, grads, _ = O.loss_and_image_grads([dict(rgb=rgb, depth=depth, normal=normal)], [tgt], [cam], O.LossParams())
    assert abs(val - (0.2 + 1.0 + 0.1 * 2.0)) < 1e-12
    assert torch.allclose(grads[0]["rgb"], torch.full((3, H, W), -1.0 / (3 * H * W), dtype=O.DT))
    gd = grads[0]["depth"]
    assert torch.allclose(gd[:, :5], torch.full((H, 5), -1.0 / (H * 5), dtype=O.DT)) and gd[:, 5:].abs().max() == 0


# ----------------------------------------------------------------- integer definitions
def test_tile_set_axis_aligned_closed_form_and_superset_of_pixels():
    rng = np.random.default_rng(6)
    W, H = 70, 45
    rp = O.RenderParams(tile_pad=0.0)
    for _ in range(200):
        m = rng.uniform(-10, 80, 2)
        A, C = rng.uniform(0.002, 0.5, 2)
        o = rng.uniform(0.01, 1.0)
        tiles, _ = O.tile_set(m, (A, 0.0, C), o, W, H, rp)
        lvl = math.log(255 * o)
        want = []
        for ty in range((H + 15) // 16):
            for tx in range((W + 15) // 16):
                x0, x1 = tx * 16 + 0.5, min(tx * 16 + 15.5, W - 0.5)
                y0, y1 = ty * 16 + 0.5, min(ty * 16 + 15.5, H - 0.5)
                ddx = max(x0 - m[0], 0, m[0] - x1)
                ddy = max(y0 - m[1], 0, m[1] - y1)
                if 0.5 * (A * ddx * ddx + C * ddy * ddy) <= lvl:
                    want.append(ty * ((W + 15) // 16) + tx)
        assert sorted(tiles) == want
    # general ellipses: every pixel with alpha >= 1/255 lies in a listed tile
    for _ in range(100):
        m = rng.uniform(0, 70, 2)
        L = rng.normal(size=(2, 2))
        cov = L @ L.T * rng.uniform(1, 60) + 0.3 * np.eye(2)
        Q = np.linalg.inv(cov)
        o = rng.uniform(0.01, 1.0)
        tiles, _ = O.tile_set(m, (Q[0, 0], Q[0, 1], Q[1, 1]), o, W, H, rp)
        v, u = np.meshgrid(np.arange(H) + 0.5, np.arange(W) + 0.5, indexing="ij")
        dx, dy = u - m[0], v - m[1]
        a = o * np.exp(-0.5 * (Q[0, 0] * dx * dx + 2 * Q[0, 1] * dx * dy + Q[1, 1] * dy * dy))
        ys, xs = np.nonzero(a >= 1 / 255)
        need = set((ys // 16) * ((W + 15) // 16) + xs // 16)
        assert need <= set(tiles)


def test_integer_helpers_textbook():
    rng = np.random.default_rng(7)
    c = rng.integers(0, 9, 57)
    s = O.exclusive_scan(c)
    acc = 0
    for i in range(57):
        assert s[i] == acc
        acc += c[i]
    keys = rng.integers(0, 5, 300).astype(np.uint32)
    vals = np.arange(300, dtype=np.uint32)
    k, v = O.stable_sort(keys, vals)
    want = sorted(zip(keys.tolist(), vals.tolist()))
    assert list(zip(k.tolist(), v.tolist())) == want
    r = O.tile_ranges(k.astype(np.int64), 7)
    for t in range(7):
        idx = [i for i, kk in enumerate(k.tolist()) if kk == t]
        assert (r[t, 0], r[t, 1]) == ((idx[0], idx[-1] + 1) if idx else (0, 0))


def test_stop_and_skip_rules():
    """Stacked opaque splats: with o = 0.95 the transmittance runs 0.05^k, so the
    4th would take T to 6.25e-6 < 1e-4 and the pixel stops before it (3
    contributors, T_final = 1.25e-4).  A splat whose alpha at the pixel is
    below 1/255 adds nothing; one with o < 1/255 is dropped everywhere."""
    cam = synth.identity_camera(33, 33, 40.0)
    n = 5
    cols = [[0.1 * (i + 1), 0.5, 1.0 - 0.1 * i] for i in range(n)]
    sc = explicit([[0, 0, 2.0 + i] for i in range(n)], [[math.log(0.05)] * 3] * n, [[1, 0, 0, 0]] * n,
                  [0.95] * n, cols, cam)
    out = O.render(sc, RP)["views"][0]
    assert out["n_contrib"][16, 16].item() == 3
    assert abs(out["T_final"][16, 16].item() - 0.05 ** 3) < 1e-15
    want = sum(np.asarray(cols[i]) * 0.95 * 0.05 ** i for i in range(3))
    assert np.allclose(out["rgb"][:, 16, 16].numpy(), want, atol=1e-14)
    # skip: on-axis splat whose alpha two pixels from its centre is just under 1/255
    var = (40.0 * 0.05 / 2.0) ** 2 + 0.3
    o = math.exp(4.0 / (2 * var)) / (255.0 * 1.001)
    sc = explicit([[0, 0, 2.0]], [[math.log(0.05)] * 3], [[1, 0, 0, 0]], [o], [[1, 1, 1]], cam)
    out = O.render(sc, RP)["views"][0]
    assert out["rgb"][0, 16, 18].item() == 0.0 and out["rgb"][0, 18, 16].item() == 0.0
    assert abs(out["rgb"][0, 16, 17].item() - o * math.exp(-0.5 / var)) < 1e-15
    sc = explicit([[0, 0, 2.0]], [[math.log(0.05)] * 3], [[1, 0, 0, 0]], [0.0035], [[1, 1, 1]], cam)
    out = O.render(sc, RP)["views"][0]
    assert out["rgb"].abs().max().item() == 0.0 and out["n_gaussians"] == 0


# ----------------------------------------------------------------- depth-normal (consistency term) and block cull
def test_depth_normal_of_a_tilted_plane_seen_off_axis():
    """The depth map of the plane n . X = d (camera frame) seen by a camera
    with fx != fy and an off-centre principal point is D(u, v) = d / (n . r),
    r = ((u + 1/2 - cx) / fx, (v + 1/2 - cy) / fy, 1).  Back-projecting it and
    crossing the central differences must give the plane normal (facing the
    camera) at every interior pixel.  Dropping the depth factor, the +1/2
    pixel centre, or using fx for fy bends the back-projected surface and
    fails."""
    n = np.array([0.3, -0.5, -0.8])
    n /= np.linalg.norm(n)
    d = -3.0                                    # n . X = d with X in front of the camera (n . X < 0: faces it)
    H, W = 23, 31
    cam = dict(fx=41.0, fy=29.0, cx=9.3, cy=15.8, W=W, H=H)
    v, u = np.meshgrid(np.arange(H) + 0.5, np.arange(W) + 0.5, indexing="ij")
    r = np.stack([(u - cam["cx"]) / cam["fx"], (v - cam["cy"]) / cam["fy"], np.ones_like(u)], 0)
    D = d / np.einsum("i,ijk->jk", n, r)
    assert (D > 0).all()
    Nd, valid = O.depth_normal(torch.tensor(D, dtype=O.DT), cam)
    assert bool(valid[1:-1, 1:-1].all()) and not bool(valid[0].any()) and not bool(valid[:, -1].any())
    err = (Nd[:, 1:-1, 1:-1] - torch.tensor(n, dtype=O.DT)[:, None, None]).abs().max().item()
    assert err < 1e-9, err

    def wrong(fn_r):
        P = D[None] * fn_r
        ex = P[:, 1:-1, 2:] - P[:, 1:-1, :-2]
        ey = P[:, 2:, 1:-1] - P[:, :-2, 1:-1]
        c = np.cross(ex, ey, axis=0)
        c /= np.linalg.norm(c, axis=0)
        return np.abs(np.abs(c) - np.abs(n)[:, None, None]).max()
    # the same construction with each plausible slip is far from the normal (the test can see them)
    r_no_half = np.stack([(u - 0.5 - cam["cx"]) / cam["fx"], (v - 0.5 - cam["cy"]) / cam["fy"], np.ones_like(u)], 0)
    r_fx = np.stack([(u - cam["cx"]) / cam["fx"], (v - cam["cy"]) / cam["fx"], np.ones_like(u)], 0)
    assert wrong(r_no_half) > 1e-3 and wrong(r_fx) > 1e-2 and wrong(r / D[None]) > 1e-2


def _anisotropic_scene(seed=11):
    """Rotated needle-like Gaussians (axis ratios 10-30) scattered over a
    96 x 80 frame, so that many 32 x 32 blocks see only a long tail."""
    rng = np.random.default_rng(seed)
    n = 60
    W, H, f = 96, 80, 90.0
    cam = synth.identity_camera(W, H, f)
    z = rng.uniform(2.0, 4.0, n)
    means = np.stack([rng.uniform(-1.2, 1.2, n) * z / 2.5, rng.uniform(-1.0, 1.0, n) * z / 2.5, z], 1)
    big = rng.uniform(-1.6, -1.0, n)
    ratio = np.log(rng.uniform(10.0, 30.0, n))
    log_scales = np.stack([big, big - ratio, big - ratio - rng.uniform(0, 0.5, n)], 1)
    quats = np.array([quat_wxyz(Rotation.from_euler("zyx", rng.uniform(-math.pi, math.pi, 3))) for _ in range(n)])
    opac = rng.uniform(0.3, 0.99, n)
    colors = rng.uniform(0.0, 1.0, (n, 3))
    return explicit(means, log_scales, quats, opac, colors, cam)


def test_block_cull_keeps_every_contributor_of_anisotropic_gaussians(monkeypatch):
    """The oracle processes pixels in 32 x 32 blocks and keeps, per block, the
    Gaussians whose bound o exp(-|delta|^2 / (2 lambda_max)) can reach
    alpha >= 1/255 there.  Rendering the same rotated, strongly anisotropic
    scene with that cull and with no cull at all (every Gaussian kept in every
    block) must give the same FP64 images and contributor counts.  The same
    bound taken with the smaller eigenvalue culls contributors and must show."""
    import oracle.pgs_oracle as OP
    sc = _anisotropic_scene()
    culled = O.render(sc, RP)["views"][0]
    kept_per_block = []
    real = OP._reject_rect

    def count(proj, keep, x0, x1, y0, y1, rp):
        k = real(proj, keep, x0, x1, y0, y1, rp)
        kept_per_block.append((int(k.sum()), int(keep.sum())))
        return k
    monkeypatch.setattr(OP, "_reject_rect", count)
    O.render(sc, RP)
    assert any(a < b for a, b in kept_per_block), "the cull removed nothing: the scene does not exercise it"
    monkeypatch.setattr(OP, "_reject_rect", lambda proj, keep, *a: keep)
    full = O.render(sc, RP)["views"][0]
    for k in ("rgb", "normal", "depth", "D", "T_final"):
        assert (culled[k] - full[k]).abs().max().item() <= 1e-12, k
    assert torch.equal(culled["n_contrib"], full["n_contrib"])
    assert int(full["n_contrib"].sum()) > 0

    def lam_min_cull(proj, keep, x0, x1, y0, y1, rp):     # the plausible slip: the smaller eigenvalue
        with torch.no_grad():
            m = proj["mean2d"]
            a, b, c = proj["cov"].unbind(-1)
            lam = 0.5 * (a + c) - torch.sqrt(torch.clamp(0.25 * (a - c) ** 2 + b * b, min=0.0))
            ddx = torch.clamp(torch.maximum(x0 - m[:, 0], m[:, 0] - x1), min=0.0)
            ddy = torch.clamp(torch.maximum(y0 - m[:, 1], m[:, 1] - y1), min=0.0)
            bound = proj["opacity"] * torch.exp(-0.5 * (ddx * ddx + ddy * ddy) / lam)
            return keep & (bound >= rp.alpha_min * (1.0 - 1e-6))
    monkeypatch.setattr(OP, "_reject_rect", lam_min_cull)
    slip = O.render(sc, RP)["views"][0]
    assert not torch.equal(slip["n_contrib"], full["n_contrib"])
    assert (slip["rgb"] - full["rgb"]).abs().max().item() > 1e-3
