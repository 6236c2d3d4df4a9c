"""Enhanced depth prior (Sec. 3.4, Step 2) on the GPU, through the C ABI,
against the FP64 oracle: per-view scale and shift, the filter mask (bit-exact
except pixels the oracle flags as within rounding of tau_d or of the frame
edge), the kept prior values and the re-projection error E.  Inputs: the
aerial terrain batches (true z-depth by an analytic ray-march), a pseudo depth
in an unknown affine frame with noise and wrong blobs, and sparse surface
points."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2503_23044_b300 import binding as B
from paper_2503_23044_b300 import synth

pytestmark = pytest.mark.gpu

TOL_ST = 1e-4        # scale and shift, relative (FP32 normal equations over ~10^4 points)
TOL_PRIOR = 1e-5     # kept prior value, relative
TOL_E = 1e-2         # re-projection error, px: a difference of ~10^3 px positions in FP32 (unflagged, smooth footprints)


def _inputs(name, res, n_points, seed):
    sc = synth.anchor_scene(name, n_anchors=2000, resolutions=res)
    cams = sc["cameras"]
    pseudo = []
    for v, c in enumerate(cams):
        tg = synth.march_targets(sc["terrain"], c, stride=1, device="cuda", seed=seed + v)
        dp, _, _, _ = synth.pseudo_depth(tg["depth"], tg["mask"] > 0, seed=100 * seed + v)
        pseudo.append(dp)
    pts = synth.sparse_points(sc["terrain"], sc["extent"], n_points, seed=seed)
    return cams, pseudo, pts


def _compare(cams, pseudo, pts, k=2, tau=1.0):
    orc = O.filter_depth_prior(cams, pseudo, pts, tau_d=tau, k=k, near=0.01)
    npix = sum(c.width * c.height for c in cams)
    scene = B.Scene(B.MODE_EXPLICIT, 1, len(cams), npix, 1024)
    arena = torch.cat([p.reshape(-1) for p in pseudo]).cuda()
    out = scene.filter_depth_prior(cams, arena, torch.tensor(pts).cuda(), tau_d=tau, k_neighbors=k, with_error=True)
    scene.read_status()
    st = out["scale_shift"].cpu().double()
    off, stats = 0, []
    for v, c in enumerate(cams):
        ov = orc["views"][v]
        n = c.width * c.height
        s_ref, t_ref = ov["scale"], ov["shift"]
        assert abs(float(st[v, 0]) - s_ref) <= TOL_ST * abs(s_ref), (v, float(st[v, 0]), s_ref)
        assert abs(float(st[v, 1]) - t_ref) <= TOL_ST * max(1.0, abs(t_ref)), (v, float(st[v, 1]), t_ref)
        gm = out["mask"][off:off + n].view(c.height, c.width).cpu().double()
        gp = out["prior"][off:off + n].view(c.height, c.width).cpu().double()
        ge = out["err"][off:off + n].view(c.height, c.width).cpu().double()
        ok = ~ov["amb"]
        assert torch.equal(gm[ok], ov["mask"][ok]), (v, int((gm[ok] != ov["mask"][ok]).sum()))
        both = ok & (gm > 0) & (ov["mask"] > 0)
        rel = ((gp - ov["prior"]).abs() / ov["prior"].abs().clamp(min=1e-6))[both]
        assert float(rel.max()) <= TOL_PRIOR, (v, float(rel.max()))
        chk = ok & (ge >= 0) & (ov["err"] >= 0)
        assert torch.equal(ge[ok] >= 0, ov["err"][ok] >= 0)
        smooth = chk & ~ov["steep"]                       # E is ill-conditioned on steep footprints
        if bool(smooth.any()):                            # a view may share no pixels with its neighbours
            de = (ge - ov["err"]).abs()[smooth]
            assert float(de.max()) <= TOL_E, (v, float(de.max()))
        de_steep = float((ge - ov["err"]).abs()[chk & ov["steep"]].max()) if bool((chk & ov["steep"]).any()) else 0.0
        stats.append((float(ov["amb"].double().mean()), float(gm.mean()), float((ge >= 0).double().mean()),
                      round(de_steep, 4)))
        off += n
    return stats


def test_depth_prior_reduced_aerial_batch():
    cams, pseudo, pts = _inputs("batch8_1600", [(200, 133)] * 8, 20_000, seed=3)
    stats = _compare(cams, pseudo, pts, k=2)
    print("flagged / kept / checked / max E difference on steep footprints, per view:", stats)
    assert all(a < 0.01 for a, _, _, _ in stats)
    assert sum(chk for _, _, chk, _ in stats) > 0.5              # the batch's views overlap
    assert any(kept < 0.999 for _, kept, _, _ in stats)          # the wrong blobs are filtered somewhere


@pytest.mark.parametrize("k", [1, 3])
def test_depth_prior_neighbour_counts(k):
    cams, pseudo, pts = _inputs("batch8_1600", [(120, 80)] * 8, 8_000, seed=5)
    _compare(cams, pseudo, pts, k=k)


def test_depth_prior_full_size_training_batch():
    """The 8-view 1600x1064 batch of the benchmark, every pixel compared."""
    cams, pseudo, pts = _inputs("batch8_1600", None, 50_000, seed=7)
    stats = _compare(cams, pseudo, pts, k=2)
    print("flagged / kept / checked / max E difference on steep footprints, per view:", stats)
    assert all(a < 0.01 for a, _, _, _ in stats)
    assert sum(chk for _, _, chk, _ in stats) > 0.5              # the batch's views overlap
