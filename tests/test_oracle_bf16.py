"""Pins of the oracle's emulation of the decoder's BF16 arithmetic (Eq. 4 with
the rounding points of the GPU's BF16 forms), against library routines and
textbook loops (no GPU).

- ``bf16_round`` (round to nearest BF16, ties to even, written from the
  definition in FP64) equals torch's own float32 -> bfloat16 conversion bit
  for bit, including exact ties.
- ``decode(precision="bf16")`` keeps every output exact except the colour
  heads, which are a textbook sum of products of BF16-rounded H and W2;
  ``"bf16_1pass"`` rounds X, W1, H and W2 before their products.
- The gradient passes straight through the rounding: d Z_colour / d W2_colour
  is the rounded H that the forward multiplied."""
import numpy as np
import torch

import oracle as O
from paper_2503_23044_b300 import synth


def _lib_bf16(x64: torch.Tensor) -> torch.Tensor:
    return x64.to(torch.float32).to(torch.bfloat16).to(torch.float64)


def test_bf16_round_equals_the_library_conversion_including_ties():
    rng = np.random.default_rng(0)
    x = torch.tensor(rng.normal(0, 1, 20000) * np.exp(rng.uniform(-20, 20, 20000)), dtype=torch.float32).double()
    assert torch.equal(O.bf16_round(x), _lib_bf16(x))
    # exact midpoints between adjacent BF16 values: mantissa (2k + 1) / 2^9 with 128 <= k < 256, i.e. k + 1/2
    # units of the last place; ties go to the even mantissa
    k = torch.arange(128, 256, dtype=torch.float64)
    for e in (-7, 0, 3):
        mid = (2 * k + 1) / 512.0 * 2.0 ** e
        r = O.bf16_round(mid)
        assert torch.equal(r, _lib_bf16(mid))
        m = torch.frexp(r)[0] * 256
        assert bool((torch.remainder(m, 2) == 0).all())          # even mantissa
    assert float(O.bf16_round(torch.zeros(1, dtype=torch.float64))) == 0.0


def _decode(sc, precision, leaves=None):
    lv = leaves if leaves is not None else O.leaves_anchor(sc)
    cam = O.camera(sc["cameras"][0])
    idx = torch.arange(len(sc["x"]))
    return O.decode(dict(x=lv["x"], feat=lv["feat"], log_l=lv["log_l"], offsets=lv["offsets"]),
                    {k: lv[k] for k in ("W1", "b1", "W2", "b2")}, cam, idx, 35, precision), lv


def test_bf16_decode_rounds_only_the_colour_heads():
    sc = synth.tiny_anchor_scene(n_anchors=5, seed=2)
    ex, _ = _decode(sc, "fp64")
    bf, lv = _decode(sc, "bf16")
    assert torch.equal(bf["Z"][:, :10], ex["Z"][:, :10]) and torch.equal(bf["Z"][:, 40:], ex["Z"][:, 40:])
    assert torch.equal(bf["opacity"], ex["opacity"]) and torch.equal(bf["scale"], ex["scale"])
    assert torch.equal(bf["quat"], ex["quat"]) and torch.equal(bf["mu"], ex["mu"])
    H = ex["H"].detach()
    W2, b2 = lv["W2"].detach(), lv["b2"].detach()
    for r in range(H.shape[0]):
        for o in range(10, 40):
            want = float(b2[o]) + sum(float(_lib_bf16(H[r, k:k + 1])) * float(_lib_bf16(W2[o, k:k + 1]))
                                      for k in range(H.shape[1]))
            assert abs(float(bf["Z"][r, o]) - want) <= 1e-12 * (1 + abs(want))
    assert float((bf["Z"][:, 10:40] - ex["Z"][:, 10:40]).abs().max()) > 1e-5      # the rounding is there


def test_bf16_1pass_decode_rounds_every_operand():
    sc = synth.tiny_anchor_scene(n_anchors=3, seed=4)
    bf, lv = _decode(sc, "bf16_1pass")
    X = bf["X"].detach()
    W1, b1, W2, b2 = (lv[k].detach() for k in ("W1", "b1", "W2", "b2"))
    for r in range(X.shape[0]):
        h = [max(0.0, float(b1[i]) + sum(float(_lib_bf16(X[r, k:k + 1])) * float(_lib_bf16(W1[i, k:k + 1]))
                                         for k in range(X.shape[1]))) for i in range(W1.shape[0])]
        hb = [float(_lib_bf16(torch.tensor([v], dtype=torch.float64))) for v in h]
        for o in (0, 11, 45, 77, 109):
            want = float(b2[o]) + sum(hb[k] * float(_lib_bf16(W2[o, k:k + 1])) for k in range(len(hb)))
            assert abs(float(bf["Z"][r, o]) - want) <= 1e-12 * (1 + abs(want))


def test_bf16_rounding_passes_the_gradient_straight_through():
    sc = synth.tiny_anchor_scene(n_anchors=4, seed=6)
    bf, lv = _decode(sc, "bf16")
    bf["Z"][:, 10:40].sum().backward()
    Hb = _lib_bf16(bf["H"].detach())
    # d sum(Z_colour) / d W2[o, k] = sum over rows of the rounded H[r, k] the forward used
    assert torch.allclose(lv["W2"].grad[10:40], Hb.sum(0).expand(30, -1), rtol=0, atol=1e-12)
    assert float(lv["W2"].grad[:10].abs().max()) == 0.0 and float(lv["W2"].grad[40:].abs().max()) == 0.0
