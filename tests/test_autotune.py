"""Launch-shape autotuner: every (tile shape, shared-memory batch) combination
renders the same images bit for bit (so the tuner may pick any of them), the
tuner times all nine, keeps the fastest, and serves a repeated workload from
its cache.  The backward under each combination matches the default one."""
import numpy as np
import pytest
import torch

from paper_2503_23044_b300 import binding as B
from paper_2503_23044_b300 import synth
from tests.gpu_util import explicit_gpu

pytestmark = pytest.mark.gpu


def _grads(img, seed=0):
    g = torch.Generator(device="cuda").manual_seed(seed)
    return B.ImageGrads(torch.randn(img.rgb.shape, device="cuda", generator=g) * 1e-3,
                        torch.randn(img.depth.shape, device="cuda", generator=g) * 1e-3,
                        torch.randn(img.normal.shape, device="cuda", generator=g) * 1e-3)


def _pg(t):
    return {k: torch.zeros_like(v) for k, v in t.items()}


@pytest.fixture(scope="module")
def scene2():
    sc = synth.explicit_scene(n=6000, seed=11, width=200, height=136)
    c2 = synth.Camera(R=np.eye(3, dtype=np.float32), t=np.array([0.02, -0.01, 0.05], np.float32), fx=180.0, fy=180.0,
                      cx=70.0, cy=45.0, width=150, height=90)
    sc["cameras"] = [sc["cameras"][0], c2]
    return sc


@pytest.mark.parametrize("shape,nb", [((16, 16), 128), ((16, 16), 512), ((8, 32), 256), ((32, 8), 512)])
def test_every_launch_shape_gives_identical_images_and_gradients(scene2, shape, nb):
    sc = scene2
    ref_scene, t0 = explicit_gpu(sc)
    ref = ref_scene.render(sc["cameras"])
    g = _grads(ref)
    pg0 = _pg(t0)
    ref_scene.backward(sc["cameras"], ref, g, pg0)
    ref_scene.read_status()
    scene, t1 = explicit_gpu(sc, B.default_params(tile_w=shape[0], tile_h=shape[1], blend_batch=nb))
    img = scene.render(sc["cameras"])
    pg1 = _pg(t1)
    scene.backward(sc["cameras"], img, g, pg1)
    scene.read_status()
    for k in ("rgb", "depth", "normal", "t_final", "n_contrib"):
        assert torch.equal(getattr(ref, k), getattr(img, k)), k
    # gradients: same sums in a different atomic order
    for k in pg0:
        a, b = pg0[k], pg1[k]
        rel = float((a - b).norm() / a.norm().clamp_min(1e-30))
        assert rel <= 1e-5, (k, rel)


def test_autotune_times_all_combinations_and_caches(scene2):
    sc = scene2
    scene, t = explicit_gpu(sc)
    img = scene.render(sc["cameras"])
    g = _grads(img)
    res = scene.autotune(sc["cameras"], img, g, _pg(t), reps=2)
    print(res)
    assert len(res) == 9
    assert {(r["tile_w"], r["tile_h"]) for r in res} == {(16, 16), (8, 32), (32, 8)}
    assert {r["blend_batch"] for r in res} == {128, 256, 512}
    assert all(r["ms"] > 0 for r in res)
    best = min(res, key=lambda r: r["ms"])
    p = scene.params()
    assert (p["tile_w"], p["tile_h"], p["blend_batch"]) == (best["tile_w"], best["tile_h"], best["blend_batch"])
    # the chosen shape renders the same images as the default one
    img2 = scene.render(sc["cameras"])
    scene.read_status()
    ref_scene, _ = explicit_gpu(sc)
    ref = ref_scene.render(sc["cameras"])
    assert torch.equal(ref.rgb, img2.rgb) and torch.equal(ref.depth, img2.depth)
    # same workload signature: served from the cache, no timing
    other, t2 = explicit_gpu(sc)
    res2 = other.autotune(sc["cameras"], img, g, _pg(t2), reps=2)
    assert len(res2) == 1 and res2[0]["ms"] < 0
    p2 = other.params()
    assert (p2["tile_w"], p2["tile_h"], p2["blend_batch"]) == (best["tile_w"], best["tile_h"], best["blend_batch"])
