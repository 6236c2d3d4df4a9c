"""Writes the regression fixtures of this folder from the FP64 oracle alone
(no value comes from the CUDA path).  The paper prints no worked example, so
these fixtures are not the paper's numbers: they freeze the oracle's results
on three tiny seeded cases of the rows it pins against closed forms (the
enhanced depth prior, the batch geometric NCC and the TSDF fusion), so that an
unintended change of the oracle's arithmetic shows in a test.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle as O                                       # noqa: E402
from paper_2503_23044_b300 import synth                  # noqa: E402


def cases():
    sc = synth.anchor_scene("batch8_1600", n_anchors=1000, resolutions=[(40, 30)] * 8)
    cams = sc["cameras"][:2]
    maps = [synth.march_targets(sc["terrain"], c, stride=1, seed=v) for v, c in enumerate(cams)]
    pseudo = [synth.pseudo_depth(m["depth"], m["mask"] > 0, seed=v)[0] for v, m in enumerate(maps)]
    pts = synth.sparse_points(sc["terrain"], sc["extent"], 500, seed=0)
    centers = [[int(x) for x in np.random.default_rng(0).integers(0, 40 * 30, 64)]]
    return sc, cams, maps, pseudo, pts, centers


def compute():
    sc, cams, maps, pseudo, pts, centers = cases()
    pr = O.filter_depth_prior(cams, pseudo, pts, tau_d=1.0, k=1, near=0.01)
    nc = O.ncc_loss(cams, [{k: m[k] for k in ("rgb", "depth", "normal")} for m in maps], centers, geo=True, lam=1.0)
    ts = O.tsdf_fuse(cams, [m["depth"] for m in maps], (-2.0, -2.0, -0.8), 0.1, (40, 40, 16), 0.4,
                     colors=[m["rgb"] for m in maps])
    return dict(
        prior=dict(scale=[v["scale"] for v in pr["views"]], shift=[v["shift"] for v in pr["views"]],
                   kept=[float(v["mask"].sum()) for v in pr["views"]],
                   prior_sum=[float(v["prior"].sum()) for v in pr["views"]]),
        ncc=dict(loss=nc["loss"], n_valid=nc["pairs"][0]["n_valid"],
                 ncc_sum=float(nc["pairs"][0]["ncc"][nc["pairs"][0]["valid"]].sum()),
                 grad_rgb_abs_sum=float(nc["grads"][1]["rgb"].abs().sum()),
                 grad_depth_sum=float(nc["grads"][1]["depth"].sum())),
        tsdf=dict(weight_sum=float(ts["weight"].sum()), tsdf_sum=float(ts["tsdf"].sum()),
                  color_sum=float(ts["color"].sum())))


if __name__ == "__main__":
    out = dict(source="FP64 oracle, tests/golden/make_golden.py (regression fixtures; the paper prints no worked "
                      "example)", values=compute())
    with open(os.path.join(HERE, "oracle_rows.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out["values"], indent=1))
