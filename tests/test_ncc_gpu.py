"""Batch geometric NCC loss (Sec. 3.4, Step 3, Eq. 10) on the GPU, through the
C ABI, against the FP64 oracle: patch validity (exact outside patches the
oracle flags as within rounding of the partner's edge), the NCC of every used
patch, the loss, and the gradients with respect to the reference colours and,
in the geometric form, to D_hat and N_hat at the patch centres.  Inputs: the
aerial terrain batches (analytic ray-march: colour, z-depth and surface normal
per pixel) with a seeded smooth error on the depth and the normal, so that the
loss has a slope."""
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2503_23044_b300 import binding as B
from paper_2503_23044_b300 import synth
from tests.gpu_util import rel_l2

pytestmark = pytest.mark.gpu

# NCC of a patch: the FP32 warped positions are good to ~1e-4 px (coordinates of
# order 10^3 through a few roundings) and the luma to ~1e-7, so |dNCC| <=
# sqrt((1 - NCC^2) / S_bb) * 7 * (max |grad b| * DU + DL) (the oracle's
# conditioning bound), taken with DU = 5e-4 px, DL = 2e-7 and a factor 2, plus
# a floor of 1e-5 for the sums.
DU, DL, TOL_NCC = 5e-4, 2e-7, 1e-5


def ncc_allowed(pr, sel):
    n = pr["ncc"][sel]
    return TOL_NCC + 2.0 * torch.sqrt((1 - n * n).clamp(min=0) / pr["sbb"][sel].clamp(min=1e-30)) * 7.0 * \
        (pr["slope"][sel] * DU + DL)
TOL_LOSS = 1e-5      # loss, relative
TOL_GRAD = 1e-3      # gradients, rel-L2


def _maps(sc, cams, seed, perturb=True):
    gen = torch.Generator().manual_seed(seed)
    out = []
    for v, c in enumerate(cams):
        tg = synth.march_targets(sc["terrain"], c, stride=1, device="cuda", seed=seed + v)
        depth, normal = tg["depth"].cpu().double(), tg["normal"].cpu().double()
        if perturb:
            H, W = depth.shape
            yy, xx = torch.meshgrid(torch.arange(H, dtype=torch.float64), torch.arange(W, dtype=torch.float64),
                                    indexing="ij")
            ph = torch.rand(4, generator=gen, dtype=torch.float64) * 2 * math.pi
            depth = depth * (1.0 + 0.03 * torch.sin(xx / 23.0 + ph[0]) * torch.cos(yy / 17.0 + ph[1]))
            normal = normal + 0.05 * torch.stack([torch.sin(yy / 29.0 + ph[2]), torch.cos(xx / 31.0 + ph[3]),
                                                  torch.zeros_like(xx)], 0) * (tg["mask"].cpu() > 0)
        out.append(dict(rgb=tg["rgb"].cpu().float(), depth=depth.float(), normal=normal.float()))
    return out


def _images(cams, maps):
    img = B.Images.empty(cams, stats=False)
    for v, m in enumerate(maps):
        a, b = img.offsets[v], img.offsets[v + 1]
        img.rgb[3 * a:3 * b] = m["rgb"].reshape(-1).cuda()
        img.depth[a:b] = m["depth"].reshape(-1).cuda()
        img.normal[3 * a:3 * b] = m["normal"].reshape(-1).cuda()
    return img


def _centers(cams, n, seed):
    gen = torch.Generator().manual_seed(seed)
    return torch.stack([torch.randperm(cams[2 * i + 1].width * cams[2 * i + 1].height, generator=gen)[:n]
                        for i in range(len(cams) // 2)]).to(torch.int32)


def _run(cams, maps, centers, geometric=True, lam=0.2, eps=1e-6):
    npix = sum(c.width * c.height for c in cams)
    scene = B.Scene(B.MODE_EXPLICIT, 1, len(cams), npix, 1024)
    img = _images(cams, maps)
    grads = B.ImageGrads.empty(npix)
    out = scene.ncc_loss_grad(cams, img, centers.cuda(), grads, lambda_ncc=lam, eps=eps, geometric=geometric)
    scene.read_status()
    return img, grads, out


def _split(img, grads, cams):
    res = []
    for v, c in enumerate(cams):
        a, b = img.offsets[v], img.offsets[v + 1]
        res.append(dict(rgb=grads.rgb[3 * a:3 * b].view(3, c.height, c.width).cpu(),
                        depth=grads.depth[a:b].view(c.height, c.width).cpu(),
                        normal=grads.normal[3 * a:3 * b].view(3, c.height, c.width).cpu()))
    return res


def _compare(cams, maps, centers, geometric=True, lam=0.2):
    img, grads, out = _run(cams, maps, centers, geometric, lam)
    orc = O.ncc_loss(cams, maps, centers.numpy(), geo=geometric, lam=lam)
    g_ncc = out["ncc"].cpu().double()
    stats, flips, nmin = [], 0, 1 << 30
    for i, pr in enumerate(orc["pairs"]):
        gv = g_ncc[i] != -2.0
        ok = ~pr["amb"]
        assert torch.equal(gv[ok], pr["valid"][ok]), (i, int((gv[ok] != pr["valid"][ok]).sum()))
        flips += int((gv != pr["valid"]).sum())
        both = gv & pr["valid"] & ok
        if bool(both.any()):
            e = (g_ncc[i][both] - pr["ncc"][both]).abs()
            allowed = ncc_allowed(pr, both)
            assert bool((e <= allowed).all()), (i, float(e.max()), float((e / allowed).max()))
            err = (float(e.max()), float((e / allowed).max()))
        else:
            err = (0.0, 0.0)
        nmin = min(nmin, max(1, pr["n_valid"]))
        stats.append((pr["n_valid"], round(float(pr["ncc"][pr["valid"]].mean()), 4) if pr["n_valid"] else None, err))
    slack = 2.0 * flips / nmin                       # a patch that changed sides moves its pair's 1 / count
    gl = out["loss"].cpu().double()
    assert abs(float(gl[1]) - orc["loss"]) <= (TOL_LOSS + slack) * max(1e-3, abs(orc["loss"])), (float(gl[1]), orc["loss"])
    assert abs(float(gl[0]) - lam * float(gl[1])) <= 1e-6 * abs(float(gl[0])) + 1e-12
    gg = _split(img, grads, cams)
    og = orc["grads"]
    e_rgb = rel_l2(torch.cat([g["rgb"].reshape(-1) for g in gg]), torch.cat([g["rgb"].reshape(-1) for g in og]))
    assert e_rgb <= TOL_GRAD + slack, e_rgb
    e_geo = None
    if geometric:
        # at the centres of used patches no sample of which sits within rounding of a cell boundary
        sel_g, sel_o = [], []
        for i, (r, s) in enumerate(O.ncc_pairs(len(cams))):
            pr = orc["pairs"][i]
            keep = pr["valid"] & ~pr["amb"] & ~pr["cell"] & (g_ncc[i] != -2.0)
            cen = centers[i][keep].long()
            W = cams[r].width
            yy, xx = cen // W, cen % W
            sel_g.append(torch.cat([gg[r]["depth"][yy, xx].double(), gg[r]["normal"][:, yy, xx].reshape(-1).double()]))
            sel_o.append(torch.cat([og[r]["depth"][yy, xx], og[r]["normal"][:, yy, xx].reshape(-1)]))
        e_geo = rel_l2(torch.cat(sel_g), torch.cat(sel_o))
        assert e_geo <= TOL_GRAD + slack, e_geo
    else:
        for g in gg:
            assert float(g["depth"].abs().max()) == 0.0 and float(g["normal"].abs().max()) == 0.0
    # views outside every pair and partner views receive nothing
    for v in range(len(cams)):
        if v % 2 == 0 or v == len(cams) - 1 and len(cams) % 2 == 1:
            assert float(gg[v]["rgb"].abs().max()) == 0.0
            assert float(gg[v]["depth"].abs().max()) == 0.0
    return dict(pairs=stats, flips=flips, e_rgb=e_rgb, e_geo=e_geo, loss=orc["loss"])


def test_ncc_reduced_aerial_batch():
    sc = synth.anchor_scene("batch8_1600", n_anchors=1000, resolutions=[(200, 133)] * 8)
    cams = sc["cameras"]
    maps = _maps(sc, cams, seed=1)
    r = _compare(cams, maps, _centers(cams, 3000, seed=2))
    print(r)
    assert all(n > 300 for n, _, _ in r["pairs"])       # the batch's pairs overlap


def test_ncc_literal_stop_gradient():
    sc = synth.anchor_scene("batch8_1600", n_anchors=1000, resolutions=[(120, 80)] * 8)
    cams = sc["cameras"][:4]
    maps = _maps(sc, cams, seed=3)
    print(_compare(cams, maps, _centers(cams, 2000, seed=4), geometric=False, lam=1.0))


def test_ncc_ragged_odd_batch():
    """Five views of mixed sizes: pairs (1, 0) and (3, 2) with different reference
    and partner resolutions; view 4 is unpaired."""
    res = [(250, 170), (131, 77), (96, 64), (200, 133), (150, 100)]
    sc = synth.anchor_scene("batch8_1600", n_anchors=1000, resolutions=res + [(64, 48)] * 3)
    cams = sc["cameras"][:5]
    maps = _maps(sc, cams, seed=5)
    print(_compare(cams, maps, _centers(cams, 1500, seed=6)))


def test_ncc_edge_cases():
    sc = synth.anchor_scene("batch8_1600", n_anchors=1000, resolutions=[(64, 48)] * 8)
    cams = sc["cameras"][:2]
    maps = _maps(sc, cams, seed=7)
    W, H = 64, 48
    # no patches: loss 0, gradients untouched
    img, grads, out = _run(cams, maps, torch.zeros(1, 0, dtype=torch.int32))
    assert out["loss"].abs().max().item() == 0.0 and grads.rgb.abs().max().item() == 0.0
    # patches that leave the reference frame, or centres past its pixels, are unused
    bad = torch.tensor([[0, W + 2, 3 * W - 1, W * H - 1, W * H, 2 ** 31 - 1]], dtype=torch.int32)
    img, grads, out = _run(cams, maps, bad)
    assert bool((out["ncc"].cpu() == -2.0).all())
    assert out["loss"].abs().max().item() == 0.0 and grads.rgb.abs().max().item() == 0.0
    # one view: no pair
    img, grads, out = _run(cams[:1], maps[:1], torch.zeros(0, 5, dtype=torch.int32))
    assert out["loss"].abs().max().item() == 0.0
    # gradients accumulate
    cen = _centers(cams, 500, seed=8).cuda()
    npix = sum(c.width * c.height for c in cams)
    scene = B.Scene(B.MODE_EXPLICIT, 1, 2, npix, 1024)
    img = _images(cams, maps)
    grads = B.ImageGrads.empty(npix)
    scene.ncc_loss_grad(cams, img, cen, grads)
    once = grads.rgb.clone()
    scene.ncc_loss_grad(cams, img, cen, grads)
    scene.read_status()
    assert rel_l2(grads.rgb, 2 * once) < 1e-6
    with pytest.raises(B.PGSError):
        scene.ncc_loss_grad(cams, img, cen, grads, eps=-1.0)


def test_ncc_full_size_training_batch():
    """The 8-view 1600x1064 batch of the benchmark, 4,096 patches per pair, every patch compared."""
    sc = synth.anchor_scene("batch8_1600", n_anchors=1000)
    cams = sc["cameras"]
    maps = _maps(sc, cams, seed=9)
    r = _compare(cams, maps, _centers(cams, 4096, seed=10))
    print(r)


def test_ncc_full_size_benchmark_patch_count():
    """The benchmark's launch: 65,536 patches per pair on the full-size batch.
    The NCC of 2,000 sampled patches per pair and the loss over all of them
    against the oracle (forward only, in chunks)."""
    sc = synth.anchor_scene("batch8_1600", n_anchors=1000)
    cams = sc["cameras"]
    maps = _maps(sc, cams, seed=11)
    centers = _centers(cams, 65536, seed=12)
    img, grads, out = _run(cams, maps, centers)
    g_ncc = out["ncc"].cpu().double()
    oc = [O.camera(c) for c in cams]
    total = 0.0
    for i, (r, s) in enumerate(O.ncc_pairs(len(cams))):
        ref = {k: maps[r][k].double() for k in ("rgb", "depth", "normal")}
        part = maps[s]["rgb"].double()
        parts = []
        for c0 in range(0, centers.shape[1], 16384):
            o = O.ncc_patches(oc[r], oc[s], ref, part, centers[i, c0:c0 + 16384])
            parts.append({k: o[k].detach() for k in ("ncc", "valid", "amb", "sbb", "slope")})
        pr = {k: torch.cat([q[k] for q in parts]) for k in parts[0]}
        vals, valid, amb = pr["ncc"], pr["valid"], pr["amb"]
        gv = g_ncc[i] != -2.0
        assert torch.equal(gv[~amb], valid[~amb])
        pick = torch.nonzero(valid & gv & ~amb).reshape(-1)[:2000]
        assert bool(((g_ncc[i][pick] - vals[pick]).abs() <= ncc_allowed(pr, pick)).all())
        n = int(valid.sum())
        total += float(((1 - vals) * valid).sum()) / n if n else 0.0
    L = total / (len(cams) // 2)
    assert abs(float(out["loss"][1]) - L) <= 1e-4 * max(1e-3, abs(L)), (float(out["loss"][1]), L)
    assert bool(torch.isfinite(grads.rgb).all()) and bool(torch.isfinite(grads.depth).all())
