"""The binding's argument checks (CPU): the C entry points receive bare device
pointers, so the binding refuses tensors whose element type or length does
not match what the call will read or write, before any device work.  A
refusal is an ArgumentError, which is both a PGSError (status
PGS_ERR_INVALID_ARG) and a ValueError."""
import numpy as np
import pytest
import torch

from paper_2503_23044_b300 import binding as B
from paper_2503_23044_b300 import synth

N = 5
IN_DIM = 35


def _anchor_tensors(n=N, in_dim=IN_DIM):
    f = lambda *s: torch.zeros(*s, dtype=torch.float32)
    return dict(x=f(n, 3), level=torch.zeros(n, dtype=torch.int32), log_l=f(n, 3), offsets=f(n, 10, 3),
                feat=f(n, 32), W1=f(32, in_dim), b1=f(32), W2=f(110, 32), b2=f(110))


def _explicit_tensors(n=N):
    f = lambda *s: torch.zeros(*s, dtype=torch.float32)
    return dict(means=f(n, 3), log_scales=f(n, 3), quats=f(n, 4), opacity_logits=f(n), colors=f(n, 3))


def test_argument_error_is_a_pgs_error_and_a_value_error():
    e = B.ArgumentError("x")
    assert isinstance(e, B.PGSError) and isinstance(e, ValueError) and e.status == B.PGS_ERR_INVALID_ARG


def test_anchor_tensors_of_the_documented_shapes_pass():
    B.check_anchor_tensors(N, IN_DIM, **_anchor_tensors())
    B.check_anchor_tensors(N, 36, **_anchor_tensors(in_dim=36))


@pytest.mark.parametrize("name", ["x", "level", "log_l", "offsets", "feat", "W1", "b1", "W2", "b2"])
def test_anchor_tensor_of_wrong_length_or_type_is_refused(name):
    t = _anchor_tensors()
    short = dict(t, **{name: t[name].reshape(-1)[:-1]})
    with pytest.raises(B.ArgumentError, match=name):
        B.check_anchor_tensors(N, IN_DIM, **short)
    other = torch.float32 if t[name].dtype == torch.int32 else torch.float64
    wrong = dict(t, **{name: t[name].to(other)})
    with pytest.raises(B.ArgumentError, match=name):
        B.check_anchor_tensors(N, IN_DIM, **wrong)


def test_w1_must_match_the_scene_input_width():
    with pytest.raises(B.ArgumentError, match="W1"):
        B.check_anchor_tensors(N, 36, **_anchor_tensors(in_dim=35))


@pytest.mark.parametrize("name", ["means", "log_scales", "quats", "opacity_logits", "colors"])
def test_explicit_tensor_of_wrong_length_or_type_is_refused(name):
    t = _explicit_tensors()
    B.check_explicit_tensors(N, **t)
    with pytest.raises(B.ArgumentError, match=name):
        B.check_explicit_tensors(N, **dict(t, **{name: torch.zeros(t[name].numel() + 1)}))
    with pytest.raises(B.ArgumentError, match=name):
        B.check_explicit_tensors(N, **dict(t, **{name: t[name].double()}))


def _cams():
    return [synth.identity_camera(8, 6, 8.0), synth.identity_camera(5, 4, 5.0)]


def test_images_must_be_laid_out_for_the_views():
    cams = _cams()
    img = B.Images.empty(cams, device="cpu")
    img.check(cams)
    with pytest.raises(B.ArgumentError, match="arena"):
        img.check(cams[:1])
    with pytest.raises(B.ArgumentError, match="images.last"):
        B.Images(**dict(img.__dict__, last=img.last.float())).check(cams)
    with pytest.raises(B.ArgumentError, match="images.rgb"):
        B.Images(**dict(img.__dict__, rgb=img.rgb[:-3])).check(cams)
    img.without_stats().check(cams)            # the diagnostic counts are optional


def test_image_grads_and_targets_sizes():
    n = B.arena_offsets(_cams())[-1]
    g = B.ImageGrads.empty(n, device="cpu")
    g.check(n)
    with pytest.raises(B.ArgumentError, match="grads.normal"):
        B.ImageGrads(g.rgb, g.depth, g.normal[:-1]).check(n)
    tg = B.Targets(torch.zeros(3 * n), torch.zeros(n), torch.zeros(n))
    tg.check(n)
    with pytest.raises(B.ArgumentError, match="targets.prior"):
        B.Targets(tg.rgb, torch.zeros(n + 1), tg.mask).check(n)
    with pytest.raises(B.ArgumentError, match="targets.mask"):
        B.Targets(tg.rgb, tg.prior, torch.zeros(n, dtype=torch.float64)).check(n)


def test_host_tensors_are_refused_before_any_device_call():
    with pytest.raises(B.ArgumentError, match="CUDA"):
        B._ptr(torch.zeros(4))
