"""Checkpoint and resume (CPU): the parameter tensors, render parameters,
step count and optimiser state come back exactly; the write replaces the
target atomically and leaves no temporary file; other files are refused."""
import os

import pytest
import torch

from paper_2503_23044_b300 import binding as B
from paper_2503_23044_b300 import checkpoint as ck


def _params():
    g = torch.Generator().manual_seed(0)
    return dict(x=torch.randn(7, 3, generator=g), log_l=torch.randn(7, 3, generator=g),
                offsets=torch.randn(7, 10, 3, generator=g), feat=torch.randn(7, 32, generator=g),
                W1=torch.randn(32, 35, generator=g), b1=torch.randn(32, generator=g),
                W2=torch.randn(110, 32, generator=g), b2=torch.randn(110, generator=g))


def _render_params():
    p = B.RenderParams()
    p.near_plane, p.dilation, p.alpha_min, p.alpha_max, p.t_min = 0.01, 0.3, 1.0 / 255.0, 0.99, 1e-4
    p.tile_w, p.tile_h, p.blend_batch, p.in_dim, p.n_levels, p.lod_d0 = 16, 16, 256, 35, 3, 4.0
    return p


def test_round_trip_is_exact(tmp_path):
    params = _params()
    leaves = [v.clone().requires_grad_(True) for v in params.values()]
    opt = torch.optim.Adam(leaves, lr=1e-3)
    sum((v * v).sum() for v in leaves).backward()
    opt.step()
    path = str(tmp_path / "state.pt")
    ck.save(path, params, _render_params(), step=1234, optimizer_state=opt.state_dict(), extra=dict(seed=5))
    st = ck.load(path, device="cpu")
    assert st["step"] == 1234 and st["extra"] == dict(seed=5)
    for k, v in params.items():
        assert torch.equal(st["params"][k], v), k
    rp = ck.render_params_from_dict(st["render_params"])
    assert ck.render_params_dict(rp) == ck.render_params_dict(_render_params())
    opt2 = torch.optim.Adam([v.clone().requires_grad_(True) for v in params.values()], lr=1e-3)
    opt2.load_state_dict(st["optimizer_state"])
    for a, b in zip(opt.state_dict()["state"].values(), opt2.state_dict()["state"].values()):
        assert torch.equal(a["exp_avg"], b["exp_avg"]) and torch.equal(a["exp_avg_sq"], b["exp_avg_sq"])


def test_save_replaces_atomically_and_leaves_no_temporary(tmp_path):
    path = str(tmp_path / "state.pt")
    ck.save(path, _params(), _render_params(), step=1)
    ck.save(path, _params(), _render_params(), step=2)
    assert ck.load(path, device="cpu")["step"] == 2
    assert sorted(os.listdir(tmp_path)) == ["state.pt"]


def test_failed_write_keeps_the_previous_checkpoint(tmp_path):
    path = str(tmp_path / "state.pt")
    ck.save(path, _params(), _render_params(), step=1)

    class Unpicklable:
        def __reduce__(self):
            raise RuntimeError("cannot pickle")

    with pytest.raises(RuntimeError):
        ck.save(path, _params(), _render_params(), step=2, extra=dict(bad=Unpicklable()))
    assert ck.load(path, device="cpu")["step"] == 1
    assert sorted(os.listdir(tmp_path)) == ["state.pt"]


def test_other_files_and_unknown_fields_are_refused(tmp_path):
    path = str(tmp_path / "other.pt")
    torch.save(dict(format=99), path)
    with pytest.raises(ValueError):
        ck.load(path, device="cpu")
    with pytest.raises(KeyError):
        ck.render_params_from_dict(dict(not_a_field=1))
