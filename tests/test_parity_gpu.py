"""GPU (CUDA, through the C ABI) against the FP64 oracle on the same seeded
inputs.  Integer work bit-exact; FP32 images within 1e-4 (colour and normal
max-abs, depth relative) on pixels the oracle does not flag as ambiguous;
gradients within relative L2 1e-3."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2503_23044_b300 import binding as B
from paper_2503_23044_b300 import synth
from tests.gpu_util import anchor_gpu, crop_view, explicit_gpu, image_errors, rel_l2

pytestmark = pytest.mark.gpu

TOL_RGB = 1e-4
TOL_DEPTH_REL = 1e-4
TOL_NORMAL = 1e-4
TOL_GRAD = 1e-3
MAX_FLAGGED = 0.01


# ------------------------------------------------------------------ integer stages
@pytest.mark.parametrize("n", [0, 1, 31, 4095, 4096, 4097, 100_003, 1 << 20])
@pytest.mark.parametrize("bits", [(0, 32), (0, 16), (0, 17), (0, 18), (3, 29), (5, 29)])
def test_sort_pairs_bitexact(n, bits):
    """8-bit digits for 32, 16, 24 and 26 bits; two 9-bit digits (one pass fewer) for 17 and 18 bits."""
    rng = np.random.default_rng(n + bits[1])
    keys = rng.integers(0, 1 << 32, n, dtype=np.uint64).astype(np.uint32)
    if n > 100:                                       # many equal digits exercise stability
        keys[: n // 3] = keys[n // 3: 2 * (n // 3)]
    vals = np.arange(n, dtype=np.uint32)
    kt = torch.tensor(keys.view(np.int32), device="cuda")
    vt = torch.tensor(vals.view(np.int32), device="cuda")
    kk, vv, err = B.sort_pairs(kt, vt, *bits)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    mask = np.uint64(((1 << bits[1]) - 1) ^ ((1 << bits[0]) - 1))
    _, perm_vals = O.stable_sort(keys.astype(np.uint64) & mask, vals)
    assert np.array_equal(vv.cpu().numpy().view(np.uint32), perm_vals)
    assert np.array_equal(kk.cpu().numpy().view(np.uint32), keys[perm_vals])


@pytest.mark.parametrize("n", [0, 1, 4096, 4097, 1_000_003])
def test_exclusive_scan_bitexact(n):
    rng = np.random.default_rng(n)
    x = rng.integers(0, 50, n).astype(np.uint32)
    xt = torch.tensor(x.view(np.int32), device="cuda")
    out, total = B.exclusive_scan(xt)
    assert np.array_equal(out.cpu().numpy().view(np.uint32).astype(np.uint64), O.exclusive_scan(x))
    assert int(total.item()) == int(x.sum())
    if n:
        idx = rng.permutation(n).astype(np.uint32)
        out, total = B.exclusive_scan(xt, torch.tensor(idx.view(np.int32), device="cuda"))
        assert np.array_equal(out.cpu().numpy().view(np.uint32).astype(np.uint64), O.exclusive_scan(x[idx]))


# ------------------------------------------------------------------ explicit Gaussians (plain splatting)
def _render_explicit(sc, params=None):
    scene, t = explicit_gpu(sc, params)
    img = scene.render(sc["cameras"])
    scene.read_status()
    return scene, t, img


@pytest.fixture(scope="module")
def cfg1():
    sc = synth.explicit_scene(n=10_000, seed=0)
    return sc, O.render(sc, O.RenderParams())


def test_explicit_forward_matches_oracle(cfg1):
    sc, orc = cfg1
    scene, t, img = _render_explicit(sc)
    ov = orc["views"][0]
    e = image_errors(img.view(0), ov, ov["flag"])
    print("explicit 10k 256x256:", e)
    assert e["flagged"] < MAX_FLAGGED
    assert e["rgb"] <= TOL_RGB and e["normal"] <= TOL_NORMAL and e["depth_rel"] <= TOL_DEPTH_REL
    assert e["n_contrib_mismatch"] == 0


def test_explicit_tile_lists_match_oracle(cfg1):
    """Per Gaussian, the set of tiles it is listed in equals the oracle's FP64
    ellipse-rectangle test except on tiles within rounding of the level; the
    lists are sorted by tile, then FP32 depth, then index; ranges match the
    textbook boundary scan."""
    sc, orc = cfg1
    scene, t, img = _render_explicit(sc)
    P = int(scene.stats().pairs)
    tiles = scene.buffer(2, P).cpu().numpy().view(np.uint32)
    gids = scene.buffer(3, P).cpu().numpy().view(np.uint32)
    rec = scene.buffer(0, len(sc["means"]) * 16, "<f4").view(-1, 16).cpu().numpy()
    assert np.all(np.diff(tiles.astype(np.int64)) >= 0)
    same = np.diff(tiles.astype(np.int64)) == 0
    z = rec[gids, 15]
    dz = np.diff(z)
    assert np.all(dz[same] >= 0)
    tie = same & (dz == 0)
    assert np.all(np.diff(gids.astype(np.int64))[tie] > 0)
    proj = orc["views"][0]["proj"]
    rp = O.RenderParams()
    gpu_sets = {}
    for tt, g in zip(tiles.tolist(), gids.tolist()):
        gpu_sets.setdefault(g, set()).add(tt)
    n_amb = 0
    for g in range(len(sc["means"])):
        if not bool(proj["valid"][g]):
            assert g not in gpu_sets
            continue
        ts, amb = O.tile_set(proj["mean2d"][g].numpy(), proj["conic"][g].numpy(), float(proj["opacity"][g]), 256, 256,
                             rp, margin=1e-5)
        diff = set(ts) ^ gpu_sets.get(g, set())
        assert diff <= set(amb), (g, diff, amb)
        n_amb += len(diff)
    print("ambiguous tile decisions that differ:", n_amb, "of", P)
    assert n_amb <= 5
    ranges = scene.buffer(4, 2 * 256).view(-1, 2).cpu().numpy()
    assert np.array_equal(ranges.astype(np.int64), O.tile_ranges(tiles.astype(np.int64), 256))


def test_explicit_backward_matches_oracle(cfg1):
    sc, orc0 = cfg1
    rp = O.RenderParams()
    flag = orc0["views"][0]["flag"]
    grads = synth.random_image_grads(sc["cameras"], seed=11, scale=1e-2)
    # pixels flagged as ambiguous carry no gradient on either side
    grads = [{k: v * (~flag).float() for k, v in grads[0].items()}]
    leaves = O.leaves_explicit(sc)
    O.render(sc, rp, leaves=leaves, image_grads=grads)
    scene, t, img = _render_explicit(sc)
    pg = {k: torch.zeros_like(v) for k, v in t.items()}
    scene.backward(sc["cameras"], img, B.ImageGrads.from_views(grads), pg)
    scene.read_status()
    for k in pg:
        err = rel_l2(pg[k], leaves[k].grad)
        print(k, err)
        assert err <= TOL_GRAD, (k, err)


@pytest.mark.parametrize("shape", [(8, 32), (32, 8)])
def test_tile_shapes_give_identical_images(cfg1, shape):
    """A pixel's contributors are the same ordered subsequence whatever the
    tile shape, so the images are bit-identical."""
    sc, _ = cfg1
    _, _, a = _render_explicit(sc)
    _, _, b = _render_explicit(sc, B.default_params(tile_w=shape[0], tile_h=shape[1]))
    assert torch.equal(a.rgb, b.rgb) and torch.equal(a.depth, b.depth) and torch.equal(a.normal, b.normal)
    assert torch.equal(a.n_contrib, b.n_contrib)


def test_ragged_image_and_multi_view_batch():
    """Non-multiple-of-16 image sizes and a batch of views of different sizes."""
    sc = synth.explicit_scene(n=3000, seed=4, width=250, height=170, f=200.0)
    c2 = synth.Camera(R=np.array([[0.995, 0, -0.0998], [0, 1, 0], [0.0998, 0, 0.995]], np.float32),
                      t=np.array([0.05, 0.0, 0.1], np.float32), fx=150.0, fy=150.0, cx=65.5, cy=40.0,
                      width=131, height=77)
    sc["cameras"] = [sc["cameras"][0], c2]
    orc = O.render(sc, O.RenderParams())
    scene, t, img = _render_explicit(sc)
    for v in range(2):
        e = image_errors(img.view(v), orc["views"][v], orc["views"][v]["flag"])
        print(v, e)
        assert e["rgb"] <= TOL_RGB and e["depth_rel"] <= TOL_DEPTH_REL and e["normal"] <= TOL_NORMAL
        assert e["n_contrib_mismatch"] == 0 and e["flagged"] < MAX_FLAGGED


def test_empty_scene_and_capacity_overflow():
    sc = synth.explicit_scene(n=500, seed=5)
    sc["means"] = sc["means"].copy()
    sc["means"][:, 2] = -3.0                                    # everything behind the camera
    scene, t, img = _render_explicit(sc)
    assert float(img.rgb.abs().max()) == 0.0 and int(scene.stats().pairs) == 0
    assert float(img.t_final.min()) == 1.0
    sc = synth.explicit_scene(n=2000, seed=6)
    scene, t = explicit_gpu(sc, cap_pairs=100)
    scene.render(sc["cameras"])
    with pytest.raises(B.PGSError) as ei:
        scene.read_status()
    assert ei.value.status == B.PGS_ERR_CAPACITY
    scene.read_status()                                          # cleared


# ------------------------------------------------------------------ loss
@pytest.mark.parametrize("sizes", [((40, 30), (23, 17)), ((40, 30), (24, 16))],
                         ids=["scalar-form (width 23)", "quad-form (widths % 4 == 0)"])
def test_loss_matches_oracle(sizes):
    """Both loss forms: per pixel when a width is not a multiple of 4, four
    pixels per thread with 16-byte accesses otherwise."""
    (w0, h0), (w1, h1) = sizes
    cams = [synth.identity_camera(w0, h0, 40.0), synth.identity_camera(w1, h1, 20.0)]
    maps = synth.random_maps(cams, seed=7)
    tv = synth.random_maps(cams, seed=8)
    gen = torch.Generator().manual_seed(9)
    tgts = [dict(rgb=t["rgb"], prior=t["depth"], mask=(torch.rand(c.height, c.width, generator=gen) > 0.2).float())
            for t, c in zip(tv, cams)]
    val, grads, _ = O.loss_and_image_grads(maps, tgts, cams, O.LossParams())
    scene = B.Scene(B.MODE_EXPLICIT, 1, 2, sum(c.width * c.height for c in cams), 1024)
    img = B.Images.empty(cams)
    img.rgb.copy_(torch.cat([m["rgb"].reshape(-1) for m in maps]))
    img.depth.copy_(torch.cat([m["depth"].reshape(-1) for m in maps]))
    img.normal.copy_(torch.cat([m["normal"].reshape(-1) for m in maps]))
    loss, g = scene.loss_grad(cams, img, B.Targets.from_views(tgts))
    scene.read_status()
    assert abs(float(loss[0]) - val) <= 1e-5 * abs(val)
    amb = O.loss_ambiguity(maps, tgts)
    for v, c in enumerate(cams):
        a, b_ = img.offsets[v], img.offsets[v + 1]
        H, W = c.height, c.width
        ok = ~amb[v]
        gr = g.rgb[3 * a:3 * b_].view(3, H, W).cpu().double()
        assert (gr - grads[v]["rgb"]).abs().amax(0)[ok].max() <= 1e-6 * grads[v]["rgb"].abs().max()
        gd = g.depth[a:b_].view(H, W).cpu().double()
        assert (gd - grads[v]["depth"]).abs()[ok].max() <= 1e-5 * grads[v]["depth"].abs().max()
        gn = g.normal[3 * a:3 * b_].view(3, H, W).cpu().double()
        assert (gn - grads[v]["normal"]).abs().max() <= 1e-4 * grads[v]["normal"].abs().max()


# ------------------------------------------------------------------ anchors (decoder + representation)
@pytest.mark.parametrize("n_views", [1, 3])
def test_tiny_anchor_step_matches_oracle(n_views):
    sc = synth.tiny_anchor_scene(n_anchors=6, seed=3, n_views=n_views, width=48, height=40)
    rp = O.RenderParams()
    orc0 = O.render(sc, rp)
    grads = synth.random_image_grads(sc["cameras"], seed=5, scale=1e-2)
    grads = [{k: v * (~ov["flag"]).float() for k, v in g.items()} for g, ov in zip(grads, orc0["views"])]
    leaves = O.leaves_anchor(sc)
    orc = O.render(sc, rp, leaves=leaves, image_grads=grads)
    scene, t = anchor_gpu(sc)
    img = scene.render(sc["cameras"])
    for v in range(n_views):
        e = image_errors(img.view(v), orc["views"][v], orc["views"][v]["flag"])
        print(v, e)
        assert e["flagged"] < MAX_FLAGGED
        assert e["rgb"] <= TOL_RGB and e["depth_rel"] <= TOL_DEPTH_REL and e["normal"] <= TOL_NORMAL
    pg = {k: torch.zeros_like(v, dtype=torch.float32) for k, v in t.items() if k != "level"}
    scene.backward(sc["cameras"], img, B.ImageGrads.from_views(grads), pg)
    scene.read_status()
    for k in pg:
        err = rel_l2(pg[k], leaves[k].grad)
        print(k, err)
        assert err <= TOL_GRAD, (k, err)


def test_decode_matches_oracle_decoder():
    sc = synth.anchor_scene("anchor_1080p", n_anchors=4000, resolutions=[(640, 360)])
    scene, t = anchor_gpu(sc)
    dec = scene.decode(sc["cameras"], capacity_rows=len(sc["x"]))
    rows = dec["rows"].cpu().numpy().view(np.uint32)
    anchors = (rows & ((1 << 27) - 1)).astype(np.int64)
    assert len(anchors) > 100
    assert np.all(np.diff(anchors) > 0)                       # compaction keeps anchor order
    cam = O.camera(sc["cameras"][0])
    leaves = O.leaves_anchor(sc)
    od = O.decode(dict(x=leaves["x"], feat=leaves["feat"], log_l=leaves["log_l"], offsets=leaves["offsets"]),
                  {k: leaves[k] for k in ("W1", "b1", "W2", "b2")}, cam, torch.tensor(anchors))
    for k in ("mu", "opacity", "color", "scale", "quat"):
        e = (dec[k].cpu().double().reshape(od[k].shape) - od[k].detach()).abs().max()
        assert e <= 1e-5, (k, float(e))


def _crops(cam, k, size=64, seed=0):
    rng = np.random.default_rng(seed)
    W, H = cam.width, cam.height
    return [(int(rng.integers(0, W - size)), int(rng.integers(H // 3, H - size)), size, size) for _ in range(k)]


def _crop_grads(g, crop):
    x0, y0, w, h = crop
    return {k: v[..., y0:y0 + h, x0:x0 + w] for k, v in g.items()}


@pytest.mark.parametrize("seed", [1, 2])
def test_anchor_1080p_full_render_on_crops(seed):
    """Full-size 1-view 1920x1080 frame of 50k anchors (500k neural Gaussians),
    compared with the oracle on a sampled 64x64 crop: images and gradients."""
    sc = synth.anchor_scene("anchor_1080p")
    cam = sc["cameras"][0]
    crop = _crops(cam, 1, seed=seed)[0]
    rp = O.RenderParams()
    orc0 = O.render(sc, rp, crops=[crop])
    ov = orc0["views"][0]
    scene, t = anchor_gpu(sc, cap_rows=len(sc["x"]))
    img = scene.render([cam])
    scene.read_status()
    e = image_errors(crop_view(img.view(0), crop), ov, ov["flag"])
    print("anchor 1080p crop", crop, e, "pairs", scene.stats().pairs)
    assert e["flagged"] < MAX_FLAGGED
    assert e["rgb"] <= TOL_RGB and e["depth_rel"] <= TOL_DEPTH_REL and e["normal"] <= TOL_NORMAL
    assert e["n_contrib_mismatch"] == 0
    # gradients of a seeded image-space gradient on the crop (flagged pixels carry none)
    fl = torch.ones(cam.height, cam.width, dtype=torch.bool)
    fl[crop[1]:crop[1] + 64, crop[0]:crop[0] + 64] = ov["flag"]
    g = synth.random_image_grads([cam], seed=3 + seed, scale=1e-2)[0]
    g = {k: v * (~fl).float() for k, v in g.items()}
    leaves = O.leaves_anchor(sc)
    O.render(sc, rp, leaves=leaves, crops=[crop], image_grads=[_crop_grads(g, crop)])
    pg = {k: torch.zeros_like(v, dtype=torch.float32) for k, v in t.items() if k != "level"}
    scene.backward([cam], img, B.ImageGrads.from_views([g]), pg)
    scene.read_status()
    for k in pg:
        err = rel_l2(pg[k], leaves[k].grad)
        print(k, err)
        assert err <= TOL_GRAD, (k, err)
