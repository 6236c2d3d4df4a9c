"""The oracle's analytic (autograd FP64) gradients against FP64 central finite
differences on tiny scenes: explicit Gaussians (means, log-scales,
quaternions, opacity logits, colours), anchors with the 35->32->110 decoder
(Eq. 4: features, offsets, log-scales, positions and all MLP weights) and the
batch loss (Eq. 8-9 + normal-depth consistency).  No GPU."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2503_23044_b300 import synth

RP = O.RenderParams()


def _objective(scene, leaves, grads):
    with torch.no_grad():
        out = O.render(scene, RP, leaves=leaves)
    tot = 0.0
    for v, g in zip(out["views"], grads):
        tot += float((v["rgb"] * g["rgb"].double()).sum() + (v["depth"] * g["depth"].double()).sum()
                     + (v["normal"] * g["normal"].double()).sum())
    return tot, out


def _analytic(scene, leaves, grads):
    for t in leaves.values():
        t.grad = None
    out = O.render(scene, RP, leaves=leaves, image_grads=grads)
    return {k: (t.grad.clone() if t.grad is not None else torch.zeros_like(t)) for k, t in leaves.items()}, out


def _fd_dir(scene, leaves, grads, name, direction, h):
    base = leaves[name].detach().clone()
    lp = {k: v.detach().clone() for k, v in leaves.items()}
    lp[name] = base + h * direction
    fp, op = _objective(scene, lp, grads)
    lp[name] = base - h * direction
    fm, om = _objective(scene, lp, grads)
    for a, b in zip(op["views"], om["views"]):          # no discrete decision may flip under +-h
        assert torch.equal(a["n_contrib"], b["n_contrib"])
    return (fp - fm) / (2 * h)


def test_explicit_gradients_match_central_fd():
    sc = synth.explicit_scene(n=8, seed=11, width=16, height=16, f=16.0, log_scale_mean=-2.2)
    leaves = O.leaves_explicit(sc)
    grads = synth.random_image_grads(sc["cameras"], seed=1, scale=1.0)
    an, out = _analytic(sc, leaves, grads)
    assert out["views"][0]["flag"].sum() == 0
    assert out["views"][0]["n_contrib"].max() >= 3
    for name, t in leaves.items():
        fd = torch.zeros_like(t)
        flat = fd.view(-1)
        for i in range(flat.numel()):
            e = torch.zeros_like(t).view(-1)
            e[i] = 1.0
            h = 1e-6 * max(1.0, abs(float(t.detach().view(-1)[i])))
            flat[i] = _fd_dir(sc, leaves, grads, name, e.view_as(t), h)
        err = torch.linalg.norm(fd - an[name]) / max(torch.linalg.norm(fd), 1e-30)
        assert err <= 1e-6, (name, float(err))
        assert torch.linalg.norm(fd) > 0, name


@pytest.mark.parametrize("n_views", [1, 2])
def test_anchor_gradients_match_central_fd(n_views):
    sc = synth.tiny_anchor_scene(n_anchors=3, seed=5, n_views=n_views)
    leaves = O.leaves_anchor(sc)
    grads = synth.random_image_grads(sc["cameras"], seed=2, scale=1.0)
    an, out = _analytic(sc, leaves, grads)
    for v in out["views"]:
        assert v["flag"].sum() == 0
    rng = np.random.default_rng(0)
    for name, t in leaves.items():
        for _ in range(3):
            d = torch.tensor(rng.normal(size=tuple(t.shape)), dtype=O.DT)
            d /= torch.linalg.norm(d)
            h = 1e-6 * max(1.0, float(t.detach().abs().max()))
            fd = _fd_dir(sc, leaves, grads, name, d, h)
            ad = float((an[name] * d).sum())
            assert abs(fd - ad) <= 1e-6 * max(abs(fd), 1e-3 * float(torch.linalg.norm(an[name]))), (name, fd, ad)
        assert torch.linalg.norm(an[name]) > 0, name


def test_loss_gradients_match_central_fd():
    cam = synth.identity_camera(12, 10, 12.0)
    maps = synth.random_maps([cam], seed=3)
    tgt = synth.random_maps([cam], seed=4)[0]
    tgt = dict(rgb=tgt["rgb"], prior=tgt["depth"], mask=(torch.rand(10, 12, generator=torch.Generator().manual_seed(0)) > 0.3).float())
    rng = np.random.default_rng(1)
    for k in ("rgb", "depth", "normal"):
        # the depth-derived normal is under stop-gradient, so FD in depth holds that term out
        lp = O.LossParams(lambda_normal=0.0) if k == "depth" else O.LossParams()
        val, grads, _ = O.loss_and_image_grads(maps, [tgt], [cam], lp)
        for _ in range(3):
            d = torch.tensor(rng.normal(size=tuple(maps[0][k].shape)), dtype=O.DT)
            h = 1e-7
            mp = {kk: vv.double().clone() for kk, vv in maps[0].items()}
            mm = {kk: vv.double().clone() for kk, vv in maps[0].items()}
            mp[k] += h * d
            mm[k] -= h * d
            fp = float(O.batch_loss([mp], [tgt], [cam], lp)["total"])
            fm = float(O.batch_loss([mm], [tgt], [cam], lp)["total"])
            fd = (fp - fm) / (2 * h)
            ad = float((grads[0][k] * d).sum())
            assert abs(fd - ad) <= 1e-6 * max(1.0, abs(ad)), (k, fd, ad)
