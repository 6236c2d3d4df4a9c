"""Throughput of the batch-level RGB-Depth-Normal training step on one B300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl pgs|reference]

A step is one pass of the whole hot path over one batch: the enhanced depth
prior of the batch (Step 2), LoD/frustum cull, decoder, projection, depth sort,
tile binning, tile sort, forward blend, losses, the batch geometric NCC of the
view pairs (Step 3, Eq. 10), backward blend, projection/decoder backward and
the decoder's weight gradients.  Workload: 8 aerial views of 1600x1064 over 200k anchors (2M
neural Gaussians) on a 3-level LoD hierarchy, seeded synthetic terrain.

Batched form (the headline): all views in one call sequence, captured once in
a CUDA graph and replayed.  Plain form: one view per call sequence, eager.
Under torchrun each rank renders its own batch (weak scaling, no collective
on the data path).  ``--impl reference`` times the FP64 CPU oracle instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "train views/s fwd+bwd RGB-D-N, 2M Gaussians @1600x1064, batched vs plain"
FP32_LANES_PER_SM = 128
# FP32 op model of the blend kernels (per pixel-Gaussian evaluation): the
# power of the Gaussian costs 12 flops (4 sub, 4 mul, 2 fma); a contributing
# pair adds 18 in the forward (alpha, transmittance, weight, 7 fma) and ~70 in
# the backward (transmittance undo, dL/dalpha over 7 channels, suffix sums,
# 13 per-pair gradients).
FWD_FLOPS_EVAL, FWD_FLOPS_CONTRIB = 12, 18
BWD_FLOPS_EVAL, BWD_FLOPS_CONTRIB = 12, 70
# the coarser op model the scope table states: ~30 FP32 ops per evaluation forward, ~70 backward
FWD_FLOPS_8D, BWD_FLOPS_8D = 30, 70


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return dict(hbm_gbs=float(d["hbm_gbs"]), sm_max_mhz=float(d.get("sm_max_mhz", 2032.0)), src="measured")
    return dict(hbm_gbs=6400.0, sm_max_mhz=2032.0, src="fallback")


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not self.path or not os.path.exists(self.path):
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["nvidia-smi unavailable"])
        rows = [l.strip().split(",") for l in open(self.path) if l.strip()]
        os.unlink(self.path)
        sm, mx, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
            except ValueError:
                continue
            for n, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return dict(sm_mhz=float(np.median(sm)) if sm else None, sm_max_mhz=mx, reasons=sorted(reasons),
                    samples=len(sm))


# ------------------------------------------------------------------ workload
def resolution_desc(cams) -> str:
    from collections import Counter
    cnt = Counter(f"{c.width}x{c.height}" for c in cams)
    return ", ".join(k if n == 1 else f"{n}x {k}" for k, n in cnt.items())


N_SPARSE = 50_000   # sparse-cloud stand-in for the depth-prior scale/shift fit
N_PATCH = 65_536    # patch centres per view pair for the batch geometric NCC (Eq. 10)
TSDF_REPS = 10      # timed TSDF fusions of the rendered batch
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one ncu capture of the kernel on
# that workload; drop an entry whenever its kernel changes
MEASURED_TRAFFIC = {("batch8_1600", "blend_bwd"): 913.8e6 + 85.1e6,
                    ("batch8_1600", "blend_fwd"): 137.0e6 + 491.3e6}
LAMBDA_NCC = 0.2    # NCC weight at the end of the paper's schedule


def make_workload(name: str, seed: int, device: str):
    """Scene, per-view targets (analytic ray-march at every pixel: RGB, true depth, mask),
    per-view pseudo depth in an unknown affine frame with wrong regions (the monocular
    prior of Step 2) and the sparse cloud."""
    from paper_2503_23044_b300 import synth
    sc = synth.anchor_scene(name, seed=seed)
    targets = []
    for i, c in enumerate(sc["cameras"]):
        tg = synth.march_targets(sc["terrain"], c, stride=1, device=device, seed=seed * 100 + i)
        tg["pseudo"] = synth.pseudo_depth(tg["depth"], tg["mask"] > 0, seed=seed * 100 + i)[0].to(device)
        targets.append(tg)
    sc["sparse"] = synth.sparse_points(sc["terrain"], sc["extent"], N_SPARSE, seed=seed)
    return sc, targets


def build_scene(sc, B, device, cap_pairs=None, cap_rows=None, precision=None):
    cams = sc["cameras"]
    Na = len(sc["x"])
    params = B.default_params(lod_d0=float(sc["lod_d0"]), n_levels=int(sc["n_levels"]),
                              decode_precision=B.DECODE_FP32 if precision is None else precision)
    npix = sum(c.width * c.height for c in cams)
    scene = B.Scene(B.MODE_ANCHOR, Na, len(cams), npix, cap_pairs or (1 << 29),
                    capacity_rows=cap_rows or Na * len(cams), params=params)
    t = {k: torch.tensor(np.asarray(sc[k]), device=device).contiguous() for k in ("x", "level", "log_l", "offsets", "feat")}
    for k, v in sc["mlp"].items():
        t[k] = torch.tensor(np.asarray(v, np.float32), device=device).contiguous()
    scene.bind_anchors(t["x"], t["level"], t["log_l"], t["offsets"], t["feat"], t["W1"], t["b1"], t["W2"], t["b2"])
    pg = {k: torch.zeros_like(v, dtype=torch.float32) for k, v in t.items() if k != "level"}
    return scene, t, pg


# ------------------------------------------------------------------ CPU oracle baseline
CPU_CROP = 128   # oracle crop side: 8 views x (setup + 128^2 crop fwd+bwd) is about 10-15 s of CPU work


def cpu_oracle_sample(sc, targets, view: int, crop_size: int = CPU_CROP):
    """FP64 oracle on one view: decode + project every LoD-active anchor, then a
    crop_size^2 crop forward + backward (seeded image gradient).  Returns
    (seconds of the whole-view setup, seconds of the crop, crop pixels)."""
    import oracle as O
    from paper_2503_23044_b300 import synth
    cam = sc["cameras"][view]
    rp = O.RenderParams(lod_d0=float(sc["lod_d0"]), n_levels=int(sc["n_levels"]))
    x0, y0 = cam.width // 2 - crop_size // 2, cam.height * 2 // 3 - crop_size // 2
    crop = (x0, y0, crop_size, crop_size)
    g = synth.random_image_grads([cam], seed=view, scale=1e-2, crops=[crop])[0]
    g = {k: v[..., y0:y0 + crop_size, x0:x0 + crop_size] for k, v in g.items()}
    leaves = O.leaves_anchor(sc)
    t0 = time.perf_counter()
    c = O.camera(cam)
    gs = O.gaussians_for_view(sc, leaves, c, rp)
    proj = O.project(gs["mu"], gs["scale"], gs["quat"], gs["opacity"], gs["color"], c, rp)
    t1 = time.perf_counter()
    O.render_view(proj, c, rp, crop, 32, {k: v.double() for k, v in g.items()})
    t2 = time.perf_counter()
    return t1 - t0, t2 - t1, crop_size * crop_size


def cpu_views_per_s(sc, targets, views, crop_size=CPU_CROP):
    total_t, parts = 0.0, []
    for v in views:
        ts, tc, npx = cpu_oracle_sample(sc, targets, v, crop_size)
        cam = sc["cameras"][v]
        t_view = ts + tc * (cam.width * cam.height / npx)
        total_t += t_view
        parts.append((ts, tc))
    return len(views) / total_t, parts


def cpu_prior_seconds(sc, pseudo):
    """FP64 oracle of the batch's enhanced depth prior (k = 2, tau_d = 1 px): seconds."""
    import oracle as O
    t0 = time.perf_counter()
    O.filter_depth_prior(sc["cameras"], [p.cpu() for p in pseudo], sc["sparse"], tau_d=1.0, k=2, near=0.01)
    return time.perf_counter() - t0


NCC_SAMPLE = 4096   # oracle NCC patches per pair timed; the cost is scaled to N_PATCH


def cpu_ncc_seconds(sc, maps):
    """FP64 oracle of the batch's NCC loss and gradients on NCC_SAMPLE patches per
    pair (seeded centres), scaled to N_PATCH patches per pair: seconds."""
    import oracle as O
    cams = sc["cameras"]
    gen = torch.Generator().manual_seed(7)
    centers = [torch.randperm(cams[2 * i + 1].width * cams[2 * i + 1].height, generator=gen)[:NCC_SAMPLE].numpy()
               for i in range(len(cams) // 2)]
    t0 = time.perf_counter()
    O.ncc_loss(cams, maps, centers, geo=True, lam=LAMBDA_NCC)
    return (time.perf_counter() - t0) * N_PATCH / NCC_SAMPLE


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    torch.set_num_threads(max(1, len(os.sched_getaffinity(0))))
    from paper_2503_23044_b300 import synth
    sc = synth.anchor_scene(args.workload, seed=0)
    V = len(sc["cameras"])
    # the batch's pseudo depths from a stride-4 march (values held over 4x4 blocks: the
    # oracle filter's cost per pixel does not depend on them) and the sparse cloud
    marched = [synth.march_targets(sc["terrain"], c, stride=4, seed=i) for i, c in enumerate(sc["cameras"])]
    pseudo = [synth.pseudo_depth(tg["depth"], tg["mask"] > 0, seed=i)[0] for i, tg in enumerate(marched)]
    sc["sparse"] = synth.sparse_points(sc["terrain"], sc["extent"], N_SPARSE, seed=0)
    t_prior = cpu_prior_seconds(sc, pseudo)
    t_ncc = cpu_ncc_seconds(sc, marched)
    full, ran, crop_px, frame_px = [], [], 0, 0
    for s in range(args.warmup + args.steps):
        v = s % V
        ts, tc, npx = cpu_oracle_sample(sc, None, v)
        cam = sc["cameras"][v]
        scale = cam.width * cam.height / npx
        # measured: the view's setup and one crop; extrapolated: the crop's per-pixel cost over the frame
        ran.append(ts + tc)
        full.append(ts + tc * scale + (t_prior + t_ncc) / V)
        if s >= args.warmup:
            crop_px += npx
            frame_px += cam.width * cam.height
    timed, timed_ran = full[args.warmup:], ran[args.warmup:]
    value = len(timed) / sum(timed)
    cores = torch.get_num_threads()
    sample = (f"per step one of the {V} views ({resolution_desc(sc['cameras'])}): FP64 decode+projection of every "
              "LoD-active anchor, then a "
              f"{CPU_CROP}x{CPU_CROP} crop fwd+bwd; per-pixel cost extrapolated to the full frame; plus 1/{V} of the "
              f"batch's FP64 enhanced depth-prior filter ({t_prior:.2f} s for all views, timed once) and of its FP64 "
              f"NCC loss + gradients ({NCC_SAMPLE} patches per pair timed once, scaled to {N_PATCH}: {t_ncc:.2f} s)")
    # ms_per_step is what each step actually ran (one view's decode + projection and one crop fwd+bwd);
    # value is the full-view rate those samples extrapolate to (see "extrapolation")
    line = dict(metric=METRIC, value=value, unit="views/s", n_gpus=args.gpus, steps=args.steps, warmup=args.warmup,
                ms_per_step=1e3 * sum(timed_ran) / len(timed_ran), higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="f64", data="synthetic", impl="reference",
                extrapolation=dict(what="value is extrapolated: per step one view's decode+projection and one "
                                        f"{CPU_CROP}x{CPU_CROP} crop fwd+bwd were run; the crop's per-pixel cost is "
                                        "scaled to the full frame and 1/V of the batch's prior filter and NCC (each "
                                        "timed once) is added",
                                   measured_s_per_step=sum(timed_ran) / len(timed_ran),
                                   extrapolated_s_per_full_view=sum(timed) / len(timed),
                                   crop_pixels_per_step=crop_px // max(1, len(timed)),
                                   frame_pixels_per_step=frame_px // max(1, len(timed)),
                                   pixel_scale=frame_px / max(1, crop_px),
                                   prior_s_all_views=t_prior, ncc_s_all_views_scaled=t_ncc),
                config=dict(workload=args.workload, views=V, anchors=len(sc["x"]), gaussians=10 * len(sc["x"]),
                            resolution=resolution_desc(sc["cameras"]), l2="n/a (CPU)"),
                cpu_baseline=dict(value=value, unit="views/s", cores=cores, kind="oracle", sample=sample),
                e2e=dict(value=value, unit="views/s", h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ ranks
def max_over_ranks(ms: float, dist, device) -> float:
    """The slowest rank's time for a region every rank brackets with barriers (no-op on one rank)."""
    if dist is None:
        return ms
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, n_ranks: int, ms: float) -> float:
    """Whole-job throughput: every rank processes its own batch (weak scaling), the job takes the slowest time."""
    return n_ranks * units_per_rank / (ms / 1e3)


# ------------------------------------------------------------------ GPU arm
def arena_slice(B, img, grads, v0: int, v1: int):
    """Images and image gradients of views v0 .. v1 - 1 as views of a batch arena."""
    a, b = img.offsets[v0], img.offsets[v1]
    s1 = lambda x: None if x is None else x[a:b]
    s3 = lambda x: x[3 * a:3 * b]
    im = B.Images(s3(img.rgb), s1(img.depth), s3(img.normal), s1(img.dist), s1(img.t_final), s1(img.last),
                  s1(img.n_contrib), s1(img.n_eval), [o - a for o in img.offsets[v0:v1 + 1]], img.shapes[v0:v1])
    return im, B.ImageGrads(s3(grads.rgb), s1(grads.depth), s3(grads.normal))


def run_pgs(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    device = f"cuda:{local}"
    from paper_2503_23044_b300 import binding as B
    sc, tviews = make_workload(args.workload, seed=rank, device=device)
    cams = sc["cameras"]
    V = len(cams)
    packed = B.pack_cameras(cams)
    res_desc = resolution_desc(cams)
    precision = B.DECODE_BF16 if args.decode == "bf16" else B.DECODE_FP32
    scene, t, pg = build_scene(sc, B, device, args.cap_pairs, args.cap_rows, precision)
    targets = B.Targets.from_views(tviews, device=device)
    pseudo = torch.cat([tv["pseudo"].reshape(-1) for tv in tviews]).to(device).contiguous()
    sparse = torch.tensor(sc["sparse"], device=device)
    scale_shift = torch.zeros(V, 2, device=device)
    prior_out = dict(prior=targets.prior, mask=targets.mask, scale_shift=scale_shift)
    images = B.Images.empty(cams, device=device)
    n_pix = images.offsets[-1]
    grads = B.ImageGrads.empty(n_pix, device=device)
    loss = torch.zeros(4, device=device)
    # NCC patch centres: a seeded draw (without repetition) over each pair's reference view
    gen = torch.Generator().manual_seed(1000 + rank)
    centers = torch.stack([torch.randperm(cams[2 * i + 1].width * cams[2 * i + 1].height, generator=gen)[:N_PATCH]
                           for i in range(V // 2)]).to(torch.int32).to(device)
    ncc_buf = torch.empty(max(1, centers.numel()), device=device)
    ncc_loss = torch.zeros(2, device=device)
    stream = torch.cuda.Stream(device=device)

    def step(tg=None, ps=None):
        # tg / ps: the step's input buffers (target colour, pseudo depth); the e2e run alternates two sets
        tg = targets if tg is None else tg
        ps = pseudo if ps is None else ps
        # enhanced depth prior of the batch -> the loss's depth prior and mask (Step 2)
        scene.filter_depth_prior(cams, ps, sparse, tau_d=1.0, k_neighbors=2, packed=packed, out=prior_out)
        scene.render(cams, images, packed=packed)
        scene.loss_grad(cams, images, tg, loss=loss, grads=grads, packed=packed)
        # batch geometric NCC (Step 3): pairs (2i+1, 2i), gradients added to the image gradients
        scene.ncc_loss_grad(cams, images, centers, grads, lambda_ncc=LAMBDA_NCC, ncc_out=ncc_buf, loss=ncc_loss,
                            packed=packed)
        for v in pg.values():
            v.zero_()
        scene.backward(cams, images, grads, pg, packed=packed)

    # eager warm-up, counts and launch accounting
    with torch.cuda.stream(stream):
        step()
    scene.read_status(stream)
    st0 = scene.stats(stream)
    with torch.cuda.stream(stream):
        step()
    st1 = scene.stats(stream)
    launches_per_step = int(st1.launches - st0.launches)
    scene.read_status(stream)
    n_eval = float(images.n_eval.double().sum())
    n_contrib = float(images.n_contrib.double().sum())
    images = images.without_stats()     # the timed step renders without the diagnostic counts

    # launch-shape autotuner (tile shape x shared-memory batch), outside the timed region
    tune = []
    if not args.no_tune:
        with torch.cuda.stream(stream):
            tune = scene.autotune(cams, images, grads, pg, reps=3, stream=stream, packed=packed)
        scene.read_status(stream)
    tp = scene.params()
    tile_desc = f"{tp['tile_w']}x{tp['tile_h']}"

    # capture the whole step in one CUDA graph, with the stage events inside it
    scene.set_profiling(True)
    graph = torch.cuda.CUDAGraph()
    use_graph = True
    try:
        with torch.cuda.stream(stream):
            stream.synchronize()
            with torch.cuda.graph(graph, stream=stream):
                step()
    except Exception as e:  # pragma: no cover - reported, not hidden
        print(f"graph capture failed ({e}); timing the eager step", file=sys.stderr)
        use_graph = False
    run = graph.replay if use_graph else step

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=device)   # > 126 MB L2
    for _ in range(args.warmup):
        with torch.cuda.stream(stream):
            run()
    stream.synchronize()
    scene.read_status(stream)
    stage_sum = {k: 0.0 for k in B.STAGES}
    step_ms = []
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(1.0)                      # evict L2 between timed steps
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                run()
                e1.record(stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            for k, v in scene.stage_times().items():
                stage_sum[k] += max(v, 0.0)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if dist is not None:
        dist.barrier()
    scene.read_status(stream)
    tot_ms = max_over_ranks(float(sum(step_ms)), dist, device)
    ms_per_step = tot_ms / args.steps
    value = job_rate(V * args.steps, world, tot_ms)
    stage_ms = {k: v / args.steps for k, v in stage_sum.items()}
    stats = scene.stats(stream)
    scene.set_profiling(False)

    # plain form: one view per call sequence, eager, no graph, FP32 decoder
    plain_vps, plain_stage, plain_counts = None, None, None
    if not args.no_plain:
        pscene, _, _ = build_scene(sc, B, device, 1 << 26, len(sc["x"]), B.DECODE_FP32)
        pscene.bind_anchors(t["x"], t["level"], t["log_l"], t["offsets"], t["feat"], t["W1"], t["b1"], t["W2"], t["b2"])
        pimg_all = B.Images.empty(cams, device=device)
        pgr_all = B.ImageGrads.empty(pimg_all.offsets[-1], device=device)
        pimgs, pgr = zip(*[arena_slice(B, pimg_all, pgr_all, v, v + 1) for v in range(V)])
        ppairs = [arena_slice(B, pimg_all, pgr_all, 2 * i, 2 * i + 2) for i in range(V // 2)]
        pkp = [B.pack_cameras(cams[2 * i:2 * i + 2]) for i in range(V // 2)]
        pncc = torch.empty_like(ncc_buf)
        # per-view targets as slices of batch buffers, so the batch-level depth-prior
        # filter writes every view's prior and mask in one call
        pbatch = B.Targets(targets.rgb.clone(), torch.empty_like(targets.prior), torch.empty_like(targets.mask))
        pprior = dict(prior=pbatch.prior, mask=pbatch.mask, scale_shift=torch.zeros(V, 2, device=device))
        ptg, off = [], 0
        for c in cams:
            n = c.width * c.height
            ptg.append(B.Targets(pbatch.rgb[3 * off:3 * (off + n)], pbatch.prior[off:off + n], pbatch.mask[off:off + n]))
            off += n
        pk = [B.pack_cameras([c]) for c in cams]

        def plain_step():
            pscene.filter_depth_prior(cams, pseudo, sparse, tau_d=1.0, k_neighbors=2, packed=packed, out=pprior)
            for i, c in enumerate(cams):
                pscene.render([c], pimgs[i], packed=pk[i])
                pscene.loss_grad([c], pimgs[i], ptg[i], loss=loss, grads=pgr[i], packed=pk[i])
                if i % 2 == 1:      # reference view of the pair (i, i - 1), whose partner is rendered
                    q = i // 2
                    pscene.ncc_loss_grad(cams[i - 1:i + 1], ppairs[q][0], centers[q:q + 1], ppairs[q][1],
                                         lambda_ncc=LAMBDA_NCC, ncc_out=pncc[q * N_PATCH:(q + 1) * N_PATCH],
                                         loss=ncc_loss, packed=pkp[q])
                pscene.backward([c], pimgs[i], pgr[i], pg, packed=pk[i])

        with torch.cuda.stream(stream):
            plain_step()
        stream.synchronize()
        ks = max(1, min(args.steps, 5))
        pm = 0.0
        for _ in range(ks):
            with torch.cuda.stream(stream):
                flush.fill_(1.0)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                plain_step()
                e1.record(stream)
            e1.synchronize()
            pm += e0.elapsed_time(e1)
        pscene.read_status(stream)
        plain_vps = job_rate(V * ks, world, max_over_ranks(pm, dist, device))
        # one more plain step with the stage events on, read view by view (outside the timed region):
        # per-stage time of the plain step and the pixel-Gaussian counts of its own renders
        pscene.set_profiling(True)
        plain_stage = {k: 0.0 for k in B.STAGES}
        with torch.cuda.stream(stream):
            pscene.filter_depth_prior(cams, pseudo, sparse, tau_d=1.0, k_neighbors=2, packed=packed, out=pprior)
        for k, v in pscene.stage_times().items():
            plain_stage[k] += max(v, 0.0)
        for i, c in enumerate(cams):
            with torch.cuda.stream(stream):
                pscene.render([c], pimgs[i], packed=pk[i])
                pscene.loss_grad([c], pimgs[i], ptg[i], loss=loss, grads=pgr[i], packed=pk[i])
                if i % 2 == 1:
                    q = i // 2
                    pscene.ncc_loss_grad(cams[i - 1:i + 1], ppairs[q][0], centers[q:q + 1], ppairs[q][1],
                                         lambda_ncc=LAMBDA_NCC, ncc_out=pncc[q * N_PATCH:(q + 1) * N_PATCH],
                                         loss=ncc_loss, packed=pkp[q])
                pscene.backward([c], pimgs[i], pgr[i], pg, packed=pk[i])
            for k, v in pscene.stage_times().items():
                if k != "prior":
                    plain_stage[k] += max(v, 0.0)
        pscene.set_profiling(False)
        pscene.read_status(stream)
        plain_counts = dict(n_eval=float(pimg_all.n_eval.double().sum()), n_contrib=float(pimg_all.n_contrib.double().sum()))
        pscene.close()

    # end to end through the public API: every step's inputs (target colour, pseudo depth)
    # from pinned host memory in, its loss values out.  Two input buffer sets, each with
    # its own captured graph, so the copy of step k+1's inputs (copy stream) overlaps
    # step k (main stream), as a training loop's loader would; 218 MB per step, larger
    # than L2, so no flush is needed between steps.
    host_t = [x.cpu().pin_memory() for x in (targets.rgb, pseudo)]
    host_loss = torch.zeros(6).pin_memory()
    h2d = sum(x.numel() * x.element_size() for x in host_t)
    d2h = host_loss.numel() * 4
    ke = max(2, min(args.steps, 50))
    sets = [(targets, pseudo),
            (B.Targets(torch.empty_like(targets.rgb), targets.prior, targets.mask), torch.empty_like(pseudo))]
    runs = [run]
    if use_graph:
        g2 = torch.cuda.CUDAGraph()
        with torch.cuda.stream(stream):
            stream.synchronize()
            with torch.cuda.graph(g2, stream=stream):
                step(*sets[1])
        runs.append(g2.replay)
    else:
        runs.append(lambda: step(*sets[1]))
    copy_stream = torch.cuda.Stream(device=device)
    ev_copied = [torch.cuda.Event(), torch.cuda.Event()]
    ev_free = [torch.cuda.Event(), torch.cuda.Event()]

    def h2d_copy(i):
        sets[i][0].rgb.copy_(host_t[0], non_blocking=True)
        sets[i][1].copy_(host_t[1], non_blocking=True)

    with torch.cuda.stream(stream):
        runs[1]()                                   # warm the second graph
    stream.synchronize()
    if dist is not None:
        dist.barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    copy_stream.wait_event(e0)
    with torch.cuda.stream(copy_stream):
        h2d_copy(0)
        ev_copied[0].record(copy_stream)
    for k in range(ke):
        cur, nxt = k % 2, 1 - k % 2
        if k + 1 < ke:
            with torch.cuda.stream(copy_stream):
                if k >= 1:
                    copy_stream.wait_event(ev_free[nxt])    # the step that read set nxt has finished
                h2d_copy(nxt)
                ev_copied[nxt].record(copy_stream)
        stream.wait_event(ev_copied[cur])
        with torch.cuda.stream(stream):
            runs[cur]()
            ev_free[cur].record(stream)
            host_loss[:4].copy_(loss, non_blocking=True)
            host_loss[4:].copy_(ncc_loss, non_blocking=True)
    e1.record(stream)
    e1.synchronize()
    em = max_over_ranks(e0.elapsed_time(e1), dist, device)
    e2e_vps = job_rate(V * ke, world, em)

    # TSDF fusion of the rendered batch (mesh reconstruction; not part of the training step):
    # a 400 x 400 x 200 volume of 0.01 with truncation 0.04, fused TSDF_REPS times
    tsdf = None
    if not args.no_tsdf:
        dims = (400, 400, 200)
        nvox = dims[0] * dims[1] * dims[2]
        vol = dict(origin=(-2.0, -2.0, -1.0), voxel=0.01, dims=dims, trunc=0.04,
                   tsdf=torch.zeros(nvox, device=device), weight=torch.zeros(nvox, device=device),
                   color=torch.zeros(nvox, 3, device=device))
        with torch.cuda.stream(stream):
            scene.tsdf_integrate(cams, images.depth, vol, rgb=images.rgb, stream=stream, packed=packed)
        stream.synchronize()
        n_upd = int((vol["weight"] > 0).sum())
        tm = 0.0
        for _ in range(TSDF_REPS):
            with torch.cuda.stream(stream):
                flush.fill_(1.0)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                scene.tsdf_integrate(cams, images.depth, vol, rgb=images.rgb, stream=stream, packed=packed)
                e1.record(stream)
            e1.synchronize()
            tm += e0.elapsed_time(e1)
        scene.read_status(stream)
        t_ms = tm / TSDF_REPS
        nbytes = 20 * nvox + 20 * n_upd + 16 * int(n_pix)
        tsdf = dict(ms=t_ms, voxels=nvox, updated_voxels=n_upd, views=V, voxel_views_per_s=nvox * V / (t_ms / 1e3),
                    bytes_per_launch=nbytes, achieved_gbs=nbytes / (t_ms / 1e3) / 1e9,
                    volume="400x400x200 voxels of 0.01, truncation 0.04, rendered depth and colour of the batch")
        del vol

    # roofline of the dominant kernel (batched form, and the plain form's own)
    peaks = _peaks()
    sm_count = torch.cuda.get_device_properties(local).multi_processor_count
    clocks = clk.summary()
    P = int(stats.pairs)

    def roofline(stages, ne, nc, traffic_ok):
        dom = max(("blend_bwd", "blend_fwd", "tile_sort", "depth_sort", "project", "project_bwd", "wgrad", "bin",
                   "loss", "prior", "ncc"), key=lambda k: stages.get(k, 0.0))
        fp32_peak = sm_count * FP32_LANES_PER_SM * 2 * peaks["sm_max_mhz"] * 1e6 / 1e12
        if dom in ("blend_bwd", "blend_fwd"):
            bwd = dom == "blend_bwd"
            fl = (BWD_FLOPS_EVAL * ne + BWD_FLOPS_CONTRIB * nc) if bwd else (FWD_FLOPS_EVAL * ne + FWD_FLOPS_CONTRIB * nc)
            fl8 = (BWD_FLOPS_8D if bwd else FWD_FLOPS_8D) * ne
            sec = stages[dom] / 1e3
            ach, ach8 = fl / sec / 1e12, fl8 / sec / 1e12
            r = dict(bound="alu", kernel=f"k_{dom}", achieved=ach, peak=fp32_peak, unit="TFLOP/s", frac=ach / fp32_peak,
                     traffic=MEASURED_TRAFFIC.get((args.workload, dom)) if traffic_ok else None,
                     flops_per_launch=fl, ms=stages[dom],
                     op_model=f"{BWD_FLOPS_EVAL if bwd else FWD_FLOPS_EVAL} flops per evaluation + "
                              f"{BWD_FLOPS_CONTRIB if bwd else FWD_FLOPS_CONTRIB} per contribution",
                     achieved_scope_model=ach8, frac_scope_model=ach8 / fp32_peak,
                     scope_model=f"{BWD_FLOPS_8D if bwd else FWD_FLOPS_8D} flops per pixel-Gaussian evaluation",
                     peak_src=f"{sm_count} SMs x 128 FP32 lanes x 2 x {peaks['sm_max_mhz']:.0f} MHz")
            if clocks.get("sm_mhz"):
                r["frac_at_median_clock"] = r["frac"] * peaks["sm_max_mhz"] / clocks["sm_mhz"]
                r["frac_scope_model_at_median_clock"] = r["frac_scope_model"] * peaks["sm_max_mhz"] / clocks["sm_mhz"]
        else:
            nb = {"tile_sort": 2 * 16 * P * math.ceil(max(1, math.log2(max(2, stats.tiles))) / 8) + 4 * P,
                  "depth_sort": 4 * 16 * stats.gaussian_views + 4 * stats.gaussian_views}.get(dom, 64 * stats.gaussian_views)
            ach = nb / (stages[dom] / 1e3) / 1e9
            r = dict(bound="hbm", kernel=dom, achieved=ach, peak=peaks["hbm_gbs"], unit="GB/s",
                     frac=ach / peaks["hbm_gbs"], traffic=None, bytes_per_launch=nb, ms=stages[dom])
        r["peak_source"] = peaks["src"]
        return r

    roof = roofline(stage_ms, n_eval, n_contrib, True)
    plain_roof = roofline(plain_stage, plain_counts["n_eval"], plain_counts["n_contrib"], False) if plain_stage else None

    # CPU oracle baseline on a bounded sample (rank 0, N = 1 only)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        torch.set_num_threads(max(1, len(os.sched_getaffinity(0))))
        vps, parts = cpu_views_per_s(sc, tviews, list(range(V)))
        t_prior = cpu_prior_seconds(sc, [tv["pseudo"] for tv in tviews])
        t_ncc = cpu_ncc_seconds(sc, [{k: tv[k].cpu() for k in ("rgb", "depth", "normal")} for tv in tviews])
        vps = V / (V / vps + t_prior + t_ncc)
        cpu = dict(value=vps, unit="views/s", cores=torch.get_num_threads(), kind="oracle",
                   sample=f"all {V} views: the batch's FP64 enhanced depth-prior filter, FP64 decode+projection of "
                          f"every LoD-active anchor, then one {CPU_CROP}x{CPU_CROP} crop fwd+bwd per view (per-pixel "
                          f"cost extrapolated to the full frame), and the FP64 NCC loss + gradients on {NCC_SAMPLE} "
                          f"patches per pair (cost scaled to {N_PATCH}) on the synthetic colour, depth and normal maps",
                   seconds=dict(prior=t_prior, ncc_scaled=t_ncc, setup=sum(p[0] for p in parts),
                                crops=sum(p[1] for p in parts)))

    if rank == 0:
        line = dict(metric=METRIC, value=value, unit="views/s", n_gpus=world, steps=args.steps, warmup=args.warmup,
                    ms_per_step=ms_per_step, higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f32",
                    data="synthetic",
                    config=dict(workload=args.workload, views=V, anchors=len(sc["x"]), gaussians=10 * len(sc["x"]),
                                resolution=res_desc, form="batched: all views per call, CUDA graph" if use_graph
                                else "batched: all views per call, eager", decode="BF16 tcgen05, FP32 accumulate (colour heads one pass; layer 1, opacity, scale, rotation "
                                                          "three-piece split)" if args.decode == "bf16" else "FP32 SIMT",
                                tile=tile_desc, blend_batch=tp["blend_batch"],
                                autotune=[f"{e['tile_w']}x{e['tile_h']}/{e['blend_batch']}: {e['ms']:.3f} ms" for e in tune]
                                if tune else "off",
                                depth_prior=f"enhanced filter every step (Step 2): {N_SPARSE} sparse points, k=2 "
                                            "nearest views, tau_d=1 px -> the loss's prior and mask",
                                ncc=f"batch geometric NCC every step (Step 3, Eq. 10): {V // 2} view pairs x {N_PATCH} "
                                    f"7x7 patches (seeded centres), lambda={LAMBDA_NCC}, geometric gradients",
                                l2="flushed between timed steps (256 MB write)",
                                parallelism=f"replicas x{world}"),
                    plain=dict(value=plain_vps, unit="views/s", form="batch depth-prior filter, then one view per call "
                                                                       "sequence, eager, FP32 decoder",
                               roofline=plain_roof, stage_ms=plain_stage),
                    e2e=dict(value=e2e_vps, unit="views/s", h2d_bytes_per_step=h2d, d2h_bytes_per_step=d2h,
                             steps=ke, form="inputs copied from pinned host memory on a copy stream, one step "
                                         "ahead (two input sets, two graphs); losses read back every step"),
                    gpu_launches=launches_per_step * args.steps,
                    roofline=roof, stage_ms=stage_ms, cpu_baseline=cpu, clocks=clocks,
                    tsdf=(dict(tsdf, frac_of_hbm=tsdf["achieved_gbs"] / peaks["hbm_gbs"]) if tsdf else None),
                    counts=dict(rows=int(stats.rows), gaussian_views=int(stats.gaussian_views), pairs=P,
                                tiles=int(stats.tiles), pixels=int(stats.pixels), n_eval=n_eval, n_contrib=n_contrib),
                    wall_s=wall)
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="pgs", choices=("pgs", "reference"))
    ap.add_argument("--workload", default="batch8_1600")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-tsdf", action="store_true", help="skip the TSDF fusion measurement")
    ap.add_argument("--no-tune", action="store_true", help="skip the launch-shape autotuner (16x16 tiles, batch 256)")
    ap.add_argument("--decode", default="bf16", choices=("bf16", "fp32"), help="decoder precision of the batched form")
    ap.add_argument("--cap-pairs", type=int, default=None, help="pair capacity (default 2^29)")
    ap.add_argument("--cap-rows", type=int, default=None, help="visible (view, anchor) row capacity")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3) if args.impl == "pgs" else args.warmup
    if args.impl == "reference":
        return run_reference(args)
    return run_pgs(args)


if __name__ == "__main__":
    sys.exit(main())
