"""The decoder of Eq. 4 on the tensor cores (BF16 operands, FP32 accumulation):
its outputs against the FP32 decoder, and BF16-decoded images against the
FP64 oracle (exact decoder) with the stated bar: colour max-abs <= 5e-3."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2503_23044_b300 import binding as B
from paper_2503_23044_b300 import synth
from tests.gpu_util import anchor_gpu, anchor_params, crop_view, image_errors

pytestmark = pytest.mark.gpu

TOL_BF16_RGB = 5e-3


def _decode(sc, precision):
    scene, t = anchor_gpu(sc, params=anchor_params(sc, decode_precision=precision))
    out = scene.decode(sc["cameras"], capacity_rows=len(sc["x"]) * len(sc["cameras"]))
    scene.read_status()
    return out


@pytest.mark.parametrize("n_anchors", [300, 4000])
def test_tensor_core_decoder_matches_fp32_decoder(n_anchors):
    """Same rows, same Gaussian means (not decoded by the MLP); activations
    within BF16 rounding of the FP32 decoder.  Covers a partial 128-row tile."""
    sc = synth.anchor_scene("anchor_1080p", n_anchors=n_anchors, resolutions=[(640, 360)])
    a = _decode(sc, B.DECODE_FP32)
    b = _decode(sc, B.DECODE_BF16)
    print("visible rows", len(a["rows"]))
    assert len(a["rows"]) > 0
    assert torch.equal(a["rows"], b["rows"])
    assert torch.equal(a["mu"], b["mu"])
    for k, tol in (("opacity", 2e-2), ("color", 2e-2), ("scale", 2e-2), ("quat", 5e-2)):
        d = (a[k] - b[k]).abs()
        print(k, float(d.max()), float(d.mean()))
        assert float(d.max()) <= tol * max(1.0, float(a[k].abs().max())), k
        assert float(d.mean()) <= tol / 10 * max(1.0, float(a[k].abs().max())), k


def test_bf16_images_against_fp64_oracle_tiny():
    sc = synth.tiny_anchor_scene(n_anchors=6, seed=3, n_views=2, width=48, height=40)
    orc = O.render(sc, O.RenderParams(lod_d0=float(sc["lod_d0"]), n_levels=int(sc["n_levels"])))
    scene, t = anchor_gpu(sc, params=anchor_params(sc, decode_precision=B.DECODE_BF16))
    img = scene.render(sc["cameras"])
    scene.read_status()
    for v in range(2):
        e = image_errors(img.view(v), orc["views"][v], orc["views"][v]["flag"])
        print("bf16 tiny view", v, e)
        assert e["rgb"] <= TOL_BF16_RGB


@pytest.mark.parametrize("seed", [1, 2])
def test_bf16_images_against_fp64_oracle_1080p_crop(seed):
    sc = synth.anchor_scene("anchor_1080p")
    cam = sc["cameras"][0]
    rng = np.random.default_rng(seed)
    crop = (int(rng.integers(0, cam.width - 64)), int(rng.integers(cam.height // 3, cam.height - 64)), 64, 64)
    rp = O.RenderParams(lod_d0=float(sc["lod_d0"]), n_levels=int(sc["n_levels"]))
    orc = O.render(sc, rp, crops=[crop])["views"][0]
    scene, t = anchor_gpu(sc, params=anchor_params(sc, decode_precision=B.DECODE_BF16), cap_rows=len(sc["x"]))
    img = scene.render([cam])
    scene.read_status()
    e = image_errors(crop_view(img.view(0), crop), orc, orc["flag"])
    print("bf16 1080p crop", crop, e)
    assert e["rgb"] <= TOL_BF16_RGB
