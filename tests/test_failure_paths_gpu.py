"""Failure paths, graph replay and the autograd wrapper, all through the C ABI.

- A bounded device wait that runs out: the only spin-waits of the step are
  the onesweep sorts' look-backs.  A test hook withholds one sort tile's
  status so the next tile's wait (a few polls) runs out; the step must return,
  pgs_read_status must report PGS_ERR_TIMEOUT, and the next step on the same
  scene (default limits) must be correct again.  No GPU fault is involved:
  the wait gives up and the kernels carry on with safe stand-ins.
- Non-finite inputs (an opacity logit, a target pixel) raise PGS_ERR_NONFINITE.
- The whole training step captured in a CUDA graph and replayed gives the
  eager step's images bit for bit and its gradients to atomic-order noise.
- torch.autograd through RenderFunction gives the oracle's parameter
  gradients (relative L2 <= 1e-3)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2503_23044_b300 import binding as B
from paper_2503_23044_b300 import synth
from tests.gpu_util import anchor_gpu, anchor_params, explicit_gpu, rel_l2

pytestmark = pytest.mark.gpu

TOL_GRAD = 1e-3


def _constant_targets(cams):
    return B.Targets.from_views([synth.constant_targets(c) for c in cams])


def _step(scene, cams, img, tg, grads, pg, packed=None):
    scene.render(cams, img, packed=packed)
    scene.loss_grad(cams, img, tg, grads=grads, packed=packed)
    for v in pg.values():
        v.zero_()
    scene.backward(cams, img, grads, pg, packed=packed)


@pytest.mark.parametrize("mode", ["explicit", "anchor"])
def test_sort_wait_that_runs_out_is_reported_and_the_scene_recovers(mode):
    if mode == "explicit":
        sc = synth.explicit_scene(n=10_000, seed=0)
        scene, t = explicit_gpu(sc)
    else:
        sc = synth.anchor_scene("batch8_1600", n_anchors=20_000, resolutions=[(320, 213)] * 2)
        scene, t = anchor_gpu(sc)
    cams = sc["cameras"]
    tg = _constant_targets(cams)
    pg = {k: torch.zeros_like(v, dtype=torch.float32) for k, v in t.items() if k != "level"}
    ref = B.Images.empty(cams)
    _step(scene, cams, ref, tg, B.ImageGrads.empty(ref.offsets[-1]), pg)
    scene.read_status()
    st = scene.stats()
    assert st.gaussian_views > 2 * 4096 and st.pairs > 2 * 4096   # both sorts span several onesweep tiles
    # tile 0 never publishes; tile 1 gives up after 64 polls
    scene.set_wait_limits(spin_limit=64, withhold_tile=0)
    img = B.Images.empty(cams)
    _step(scene, cams, img, tg, B.ImageGrads.empty(img.offsets[-1]), pg)
    torch.cuda.synchronize()                                     # the step returned
    with pytest.raises(B.PGSError) as ei:
        scene.read_status()
    assert ei.value.status == B.PGS_ERR_TIMEOUT
    # the stand-ins: no pairs, so every pixel is background with T = 1, and the gradients are zero
    assert float(img.rgb.abs().max()) == 0.0 and float(img.t_final.min()) == 1.0
    assert all(bool(torch.isfinite(v).all()) for v in pg.values())
    # default limits again: the same scene renders the reference images
    scene.set_wait_limits()
    img2 = B.Images.empty(cams)
    _step(scene, cams, img2, tg, B.ImageGrads.empty(img2.offsets[-1]), pg)
    scene.read_status()
    for k in ("rgb", "depth", "normal", "t_final", "last"):
        assert torch.equal(getattr(img2, k), getattr(ref, k)), k


def test_nonfinite_opacity_logit_and_target_pixel_are_reported():
    sc = synth.explicit_scene(n=2000, seed=8, width=96, height=80, f=96.0)
    scene, t = explicit_gpu(sc)
    cams = sc["cameras"]
    scene.render(cams)
    scene.read_status()
    t["opacity_logits"][17] = float("nan")
    scene.render(cams)
    with pytest.raises(B.PGSError) as ei:
        scene.read_status()
    assert ei.value.status == B.PGS_ERR_NONFINITE
    t["opacity_logits"][17] = 0.5
    img = scene.render(cams)
    scene.read_status()                                          # clean again
    tv = synth.constant_targets(cams[0])
    tv["rgb"][1, 40, 50] = float("nan")
    scene.loss_grad(cams, img, B.Targets.from_views([tv]))
    with pytest.raises(B.PGSError) as ei:
        scene.read_status()
    assert ei.value.status == B.PGS_ERR_NONFINITE


def test_graph_replay_equals_the_eager_step():
    """The benchmarked form: BF16 tensor-core decoder, render + loss + backward
    captured once and replayed."""
    sc = synth.anchor_scene("batch8_1600", n_anchors=30_000, resolutions=[(400, 266)] * 4)
    cams = sc["cameras"]
    packed = B.pack_cameras(cams)
    scene, t = anchor_gpu(sc, params=anchor_params(sc, decode_precision=B.DECODE_BF16))
    tg = _constant_targets(cams)
    img = B.Images.empty(cams, stats=False)
    grads = B.ImageGrads.empty(img.offsets[-1])
    pg = {k: torch.zeros_like(v, dtype=torch.float32) for k, v in t.items() if k != "level"}
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        _step(scene, cams, img, tg, grads, pg, packed)
    scene.read_status(stream)
    eager_img = {k: getattr(img, k).clone() for k in ("rgb", "depth", "normal", "dist", "t_final", "last")}
    eager_pg = {k: v.clone() for k, v in pg.items()}
    assert float(eager_img["rgb"].abs().max()) > 0
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(stream):
        stream.synchronize()
        with torch.cuda.graph(graph, stream=stream):
            _step(scene, cams, img, tg, grads, pg, packed)
    for _ in range(2):
        img.rgb.fill_(-1.0)
        with torch.cuda.stream(stream):
            graph.replay()
        scene.read_status(stream)
        for k, v in eager_img.items():
            assert torch.equal(getattr(img, k), v), k
        for k, v in eager_pg.items():
            e = rel_l2(pg[k], v)
            assert e <= 1e-6, (k, e)


@pytest.mark.parametrize("mode", ["explicit", "anchor"])
def test_autograd_through_render_function_matches_oracle(mode):
    if mode == "explicit":
        sc = synth.explicit_scene(n=400, seed=21, width=64, height=48, f=60.0)
        scene, t = explicit_gpu(sc)
        names = ("means", "log_scales", "quats", "opacity_logits", "colors")
        leaves = O.leaves_explicit(sc)
    else:
        sc = synth.tiny_anchor_scene(n_anchors=6, seed=3, n_views=2, width=48, height=40)
        scene, t = anchor_gpu(sc)
        names = ("x", "log_l", "offsets", "feat", "W1", "b1", "W2", "b2")
        leaves = O.leaves_anchor(sc)
    cams = sc["cameras"]
    rp = O.RenderParams(lod_d0=float(sc.get("lod_d0", 1e9)), n_levels=int(sc.get("n_levels", 1)))
    orc0 = O.render(sc, rp)
    grads = synth.random_image_grads(cams, seed=5, scale=1e-2)
    grads = [{k: g * (~orc0["views"][v]["flag"]).float() for k, g in gv.items()} for v, gv in enumerate(grads)]
    O.render(sc, rp, leaves=leaves, image_grads=grads)
    params = [t[n].requires_grad_(True) for n in names]
    rgb, depth, normal = B.RenderFunction.apply(scene, cams, names, *params)
    gi = B.ImageGrads.from_views(grads)
    loss = (rgb * gi.rgb).sum() + (depth * gi.depth).sum() + (normal * gi.normal).sum()
    loss.backward()
    scene.read_status()
    for n, p in zip(names, params):
        assert p.grad is not None, n
        e = rel_l2(p.grad, leaves[n].grad)
        print(mode, n, e)
        assert e <= TOL_GRAD, (n, e)
