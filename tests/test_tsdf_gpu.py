"""TSDF fusion of rendered depth and colour (supplementary, mesh
reconstruction) on the GPU, through the C ABI, against the FP64 oracle: voxel
weights exact and the fused signed distance and colour within FP32 rounding,
outside voxels the oracle flags as within rounding of a pixel boundary or of
the truncation band.  Inputs: the aerial terrain batches' analytic depth and
colour maps (independent of the renderer)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2503_23044_b300 import binding as B
from paper_2503_23044_b300 import synth

pytestmark = pytest.mark.gpu

TOL_T = 2e-5     # tsdf: (D - z) / trunc with D, z ~ 2 in FP32 (~2e-7 / 0.04) through a running mean of <= 8 terms
TOL_C = 1e-6     # colour: a running mean of <= 8 values in [0, 1]


def _maps(sc, cams, seed):
    out = []
    for v, c in enumerate(cams):
        tg = synth.march_targets(sc["terrain"], c, stride=1, device="cuda", seed=seed + v)
        out.append(dict(rgb=tg["rgb"].float(), depth=tg["depth"].float()))
    return out


def _arena(cams, maps):
    off = B.arena_offsets(cams)
    depth = torch.zeros(off[-1], device="cuda")
    rgb = torch.zeros(3 * off[-1], device="cuda")
    for v, m in enumerate(maps):
        depth[off[v]:off[v + 1]] = m["depth"].reshape(-1)
        rgb[3 * off[v]:3 * off[v + 1]] = m["rgb"].reshape(-1)
    return depth, rgb


def _volume(origin, voxel, dims, trunc, color=True):
    n = dims[0] * dims[1] * dims[2]
    vol = dict(origin=origin, voxel=voxel, dims=dims, trunc=trunc, tsdf=torch.zeros(n, device="cuda"),
               weight=torch.zeros(n, device="cuda"))
    if color:
        vol["color"] = torch.zeros(n, 3, device="cuda")
    return vol


def _compare(cams, maps, vol, index=None, state=None, extra_amb=None):
    sel = slice(None) if index is None else torch.as_tensor(index, device="cuda")
    orc = O.tsdf_fuse(cams, [m["depth"].cpu() for m in maps], vol["origin"], vol["voxel"], vol["dims"], vol["trunc"],
                      colors=[m["rgb"].cpu() for m in maps], index=index, state=state)
    amb = orc["amb"] if extra_amb is None else orc["amb"] | extra_amb
    ok = ~amb
    gw = vol["weight"][sel].cpu().double()
    gt = vol["tsdf"][sel].cpu().double()
    gc = vol["color"][sel].cpu().double()
    assert torch.equal(gw[ok], orc["weight"][ok]), int((gw[ok] != orc["weight"][ok]).sum())
    upd = ok & (orc["weight"] > 0)
    et = float((gt[upd] - orc["tsdf"][upd]).abs().max()) if bool(upd.any()) else 0.0
    ec = float((gc[upd] - orc["color"][upd]).abs().max()) if bool(upd.any()) else 0.0
    assert et <= TOL_T and ec <= TOL_C, (et, ec)
    return dict(flagged=float(amb.double().mean()), observed=float((orc["weight"] > 0).double().mean()),
                max_w=float(orc["weight"].max()), e_tsdf=et, e_color=ec, orc=orc)


def test_tsdf_reduced_aerial_batch():
    sc = synth.anchor_scene("batch8_1600", n_anchors=1000, resolutions=[(200, 133)] * 8)
    cams = sc["cameras"]
    maps = _maps(sc, cams, seed=1)
    depth, rgb = _arena(cams, maps)
    vol = _volume((-2.0, -2.0, -0.8), 0.04, (100, 100, 40), 0.16)
    scene = B.Scene(B.MODE_EXPLICIT, 1, len(cams), depth.numel(), 1024)
    scene.tsdf_integrate(cams, depth, vol, rgb=rgb)
    scene.read_status()
    r = _compare(cams, maps, vol)
    print({k: v for k, v in r.items() if k != "orc"})
    assert r["flagged"] < 0.05 and r["observed"] > 0.05 and r["max_w"] >= 4


def test_tsdf_ragged_views_and_repeated_calls():
    """Views of mixed sizes fused in two calls (the second continues the first's
    state); the same views fused without colour give the same weights."""
    res = [(250, 170), (131, 77), (96, 64), (200, 133), (150, 100), (64, 48), (64, 48), (64, 48)]
    sc = synth.anchor_scene("batch8_1600", n_anchors=1000, resolutions=res)
    cams = sc["cameras"][:5]
    maps = _maps(sc, cams, seed=2)
    vol = _volume((-2.0, -1.0, -0.6), 0.05, (80, 40, 24), 0.2)
    scene = B.Scene(B.MODE_EXPLICIT, 1, 5, sum(c.width * c.height for c in cams), 1024)
    d1, c1 = _arena(cams[:2], maps[:2])
    d2, c2 = _arena(cams[2:], maps[2:])
    scene.tsdf_integrate(cams[:2], d1, vol, rgb=c1)
    state = O.tsdf_fuse(cams[:2], [m["depth"].cpu() for m in maps[:2]], vol["origin"], vol["voxel"], vol["dims"],
                        vol["trunc"], colors=[m["rgb"].cpu() for m in maps[:2]])
    scene.tsdf_integrate(cams[2:], d2, vol, rgb=c2)
    scene.read_status()
    r = _compare(cams[2:], maps[2:], vol, state=state, extra_amb=state["amb"])
    print({k: v for k, v in r.items() if k != "orc"})
    assert r["flagged"] < 0.05
    # without colour
    vol2 = _volume((-2.0, -1.0, -0.6), 0.05, (80, 40, 24), 0.2, color=False)
    d, _ = _arena(cams, maps)
    scene.tsdf_integrate(cams, d, vol2)
    scene.read_status()
    assert torch.equal(vol2["weight"], vol["weight"])


def test_tsdf_argument_errors():
    sc = synth.anchor_scene("batch8_1600", n_anchors=1000, resolutions=[(64, 48)] * 8)
    cams = sc["cameras"][:1]
    depth = torch.ones(64 * 48, device="cuda")
    scene = B.Scene(B.MODE_EXPLICIT, 1, 1, 64 * 48, 1024)
    for bad in (dict(dims=(0, 4, 4)), dict(voxel=0.0), dict(trunc=-1.0)):
        v = dict(origin=(0.0, 0.0, 0.0), voxel=0.1, dims=(4, 4, 4), trunc=0.2)
        v.update(bad)
        n = max(1, v["dims"][0] * v["dims"][1] * v["dims"][2])
        v.update(tsdf=torch.zeros(n, device="cuda"), weight=torch.zeros(n, device="cuda"))
        with pytest.raises(B.PGSError):
            scene.tsdf_integrate(cams, depth, v)
    v = _volume((0.0, 0.0, 0.0), 0.1, (4, 4, 4), 0.2)
    with pytest.raises(B.PGSError):                    # colour state without colour input is fine, not the reverse
        scene.tsdf_integrate(cams, depth, dict(v, color=None), rgb=torch.zeros(3 * 64 * 48, device="cuda"))


def test_tsdf_full_size_batch():
    """The benchmark's 8 x 1600x1064 batch into a 400 x 400 x 200 volume of 0.01
    (truncation 0.04, as for the aerial scenes), 200,000 seeded voxels compared
    and invariants over the whole volume."""
    sc = synth.anchor_scene("batch8_1600", n_anchors=1000)
    cams = sc["cameras"]
    maps = _maps(sc, cams, seed=3)
    depth, rgb = _arena(cams, maps)
    vol = _volume((-2.0, -2.0, -1.0), 0.01, (400, 400, 200), 0.04)
    scene = B.Scene(B.MODE_EXPLICIT, 1, len(cams), depth.numel(), 1024)
    scene.tsdf_integrate(cams, depth, vol, rgb=rgb)
    scene.read_status()
    n = 400 * 400 * 200
    w = vol["weight"]
    assert bool((w >= 0).all()) and bool((w <= 8).all()) and bool((w == torch.round(w)).all())
    assert bool((vol["tsdf"] <= 1).all()) and bool((vol["tsdf"] >= -1.0001).all())
    # sample half from the observed voxels, half anywhere
    gen = torch.Generator().manual_seed(4)
    obs = torch.nonzero(w > 0).reshape(-1).cpu()
    idx = torch.cat([obs[torch.randperm(obs.numel(), generator=gen)[:100_000]],
                     torch.randperm(n, generator=gen)[:100_000]])
    r = _compare(cams, maps, vol, index=idx)
    print({k: v for k, v in r.items() if k != "orc"}, "observed voxels", obs.numel())
    assert r["flagged"] < 0.05
