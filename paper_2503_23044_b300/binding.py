"""ctypes binding of libpgs (include/pgs.h) with torch tensors as device memory.

Argument marshalling only: every step of the training step runs in the CUDA
library.  If ``libpgs.so`` is missing the first call fails loudly; there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os
from typing import Dict, List, Optional, Sequence

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
# PGS_LIB=checked selects the bounds-checked build (libpgs_checked.so); the default is the production library
LIB_PATH = os.path.join(_HERE, "libpgs_checked.so" if os.environ.get("PGS_LIB") == "checked" else "libpgs.so")

(PGS_OK, PGS_ERR_INVALID_ARG, PGS_ERR_CAPACITY, PGS_ERR_TIMEOUT, PGS_ERR_NONFINITE, PGS_ERR_CUDA, PGS_ERR_UNSUPPORTED,
 PGS_ERR_BOUNDS) = range(8)
MODE_EXPLICIT, MODE_ANCHOR = 0, 1
N_OFFSETS, FEAT_DIM, HIDDEN, OUT_DIM = 10, 32, 32, 110   # PGS_N_OFFSETS, PGS_FEAT_DIM, PGS_HIDDEN, PGS_OUT_DIM
DECODE_FP32, DECODE_BF16, DECODE_BF16_1PASS = 0, 1, 2
MAX_VIEWS = 32


class PGSError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"pgs status {status}: {msg}")
        self.status = status


class ArgumentError(PGSError, ValueError):
    """An argument the binding refuses before any device work (status PGS_ERR_INVALID_ARG): the
    C entry points see bare pointers, so sizes and element types are checked here."""

    def __init__(self, msg: str):
        super().__init__(PGS_ERR_INVALID_ARG, msg)


_lib = None


def lib() -> C.CDLL:
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library {LIB_PATH} is missing: build it with "
                               "`python -m paper_2503_23044_b300.build` (add --checked for the bounds-checked "
                               "build; no CPU fallback exists)")
        _lib = C.CDLL(LIB_PATH)
        _declare(_lib)
    return _lib


# ------------------------------------------------------------------ structs (mirror include/pgs.h)
class Camera(C.Structure):
    _fields_ = [("R", C.c_float * 9), ("t", C.c_float * 3), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("width", C.c_int32), ("height", C.c_int32)]


class RenderParams(C.Structure):
    _fields_ = [("near_plane", C.c_float), ("dilation", C.c_float), ("alpha_min", C.c_float),
                ("alpha_max", C.c_float), ("t_min", C.c_float), ("jclamp", C.c_float), ("tile_pad", C.c_float),
                ("lod_d0", C.c_float), ("n_levels", C.c_int32), ("bg", C.c_float), ("tile_w", C.c_int32),
                ("tile_h", C.c_int32), ("decode_precision", C.c_int32), ("in_dim", C.c_int32),
                ("blend_batch", C.c_int32)]


class SceneDesc(C.Structure):
    _fields_ = [("mode", C.c_int32), ("n_primitives", C.c_int64), ("max_views", C.c_int32),
                ("max_pixels", C.c_int64), ("capacity_rows", C.c_int64), ("capacity_pairs", C.c_int64),
                ("params", RenderParams)]


class ExplicitPtrs(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("means", "log_scales", "quats", "opacity_logits", "colors")]


class AnchorPtrs(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("x", "level", "log_l", "offsets", "feat")]


class MlpPtrs(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("W1", "b1", "W2", "b2")]


class ImagePtrs(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("rgb", "depth", "normal", "dist", "t_final", "last", "n_contrib", "n_eval")]


class ImageGradPtrs(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("rgb", "depth", "normal")]


class TargetPtrs(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("rgb", "prior", "mask")]


class LossParams(C.Structure):
    _fields_ = [("lambda_depth", C.c_float), ("lambda_normal", C.c_float)]


PARAM_GRAD_FIELDS = ("means", "log_scales", "quats", "opacity_logits", "colors",
                     "x", "log_l", "offsets", "feat", "W1", "b1", "W2", "b2")


class ParamGradPtrs(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in PARAM_GRAD_FIELDS]


class Stats(C.Structure):
    _fields_ = [("rows", C.c_int64), ("gaussian_views", C.c_int64), ("launches", C.c_int64), ("pairs", C.c_int64),
                ("tiles", C.c_int64), ("pixels", C.c_int64), ("flags", C.c_uint32)]


class PriorParams(C.Structure):
    _fields_ = [("tau_d", C.c_float), ("k_neighbors", C.c_int32)]


class NccParams(C.Structure):
    _fields_ = [("lambda_ncc", C.c_float), ("eps", C.c_float), ("geometric", C.c_int32)]


class TsdfVolume(C.Structure):
    _fields_ = [("origin", C.c_float * 3), ("voxel", C.c_float), ("dims", C.c_int32 * 3), ("trunc", C.c_float)]


class TuneEntry(C.Structure):
    _fields_ = [("tile_w", C.c_int32), ("tile_h", C.c_int32), ("blend_batch", C.c_int32), ("ms", C.c_float)]


ENTRY_POINTS = ("pgs_last_error", "pgs_status_string", "pgs_default_params", "pgs_scene_create", "pgs_scene_destroy",
                "pgs_scene_bind_explicit", "pgs_scene_bind_anchors", "pgs_decode_anchors", "pgs_render_batch",
                "pgs_loss_grad", "pgs_backward", "pgs_read_status", "pgs_get_stats", "pgs_set_profiling",
                "pgs_get_stage_times", "pgs_scene_buffer", "pgs_sort_scratch_bytes", "pgs_sort_pairs",
                "pgs_scan_scratch_bytes", "pgs_exclusive_scan_u32", "pgs_sort_pairs_noalloc", "pgs_autotune",
                "pgs_scene_get_params", "pgs_filter_depth_prior", "pgs_ncc_loss_grad", "pgs_tsdf_integrate",
                "pgs_scene_set_wait_limits", "pgs_checked_build")
STAGES = ("project", "depth_sort", "bin", "tile_sort", "blend_fwd", "loss", "blend_bwd", "project_bwd", "wgrad",
          "prior", "ncc", "tsdf")


def _declare(L: C.CDLL) -> None:
    vp, i32, i64, P = C.c_void_p, C.c_int, C.c_int64, C.POINTER
    for name in ENTRY_POINTS:
        getattr(L, name).restype = C.c_int
    L.pgs_last_error.restype = C.c_char_p
    L.pgs_last_error.argtypes = []
    L.pgs_status_string.restype = C.c_char_p
    L.pgs_status_string.argtypes = [i32]
    L.pgs_default_params.argtypes = [P(RenderParams)]
    L.pgs_default_params.restype = None
    L.pgs_scene_create.argtypes = [P(SceneDesc), P(vp)]
    L.pgs_scene_destroy.argtypes = [vp]
    L.pgs_scene_destroy.restype = None
    L.pgs_scene_bind_explicit.argtypes = [vp, P(ExplicitPtrs)]
    L.pgs_scene_bind_anchors.argtypes = [vp, P(AnchorPtrs), P(MlpPtrs)]
    L.pgs_decode_anchors.argtypes = [vp, P(Camera), i32, vp, vp, vp, vp, vp, vp, vp, vp]
    L.pgs_render_batch.argtypes = [vp, P(Camera), i32, P(ImagePtrs), vp]
    L.pgs_loss_grad.argtypes = [vp, P(Camera), i32, P(ImagePtrs), P(TargetPtrs), P(LossParams), vp,
                                P(ImageGradPtrs), vp]
    L.pgs_backward.argtypes = [vp, P(Camera), i32, P(ImagePtrs), P(ImageGradPtrs), P(ParamGradPtrs), vp]
    L.pgs_read_status.argtypes = [vp, vp]
    L.pgs_get_stats.argtypes = [vp, P(Stats), vp]
    L.pgs_set_profiling.argtypes = [vp, i32]
    L.pgs_checked_build.argtypes = []
    L.pgs_scene_set_wait_limits.argtypes = [vp, C.c_uint32, C.c_uint32]
    L.pgs_get_stage_times.argtypes = [vp, P(C.c_float), i32]
    L.pgs_scene_buffer.argtypes = [vp, i32, P(vp), P(i64)]
    L.pgs_sort_scratch_bytes.argtypes = [i64]
    L.pgs_sort_scratch_bytes.restype = C.c_size_t
    L.pgs_sort_pairs.argtypes = [vp, vp, vp, vp, vp, i64, i32, i32, vp, C.c_size_t, vp, vp]
    L.pgs_scan_scratch_bytes.argtypes = []
    L.pgs_scan_scratch_bytes.restype = C.c_size_t
    L.pgs_exclusive_scan_u32.argtypes = [vp, vp, vp, vp, vp, vp, C.c_size_t, vp]
    L.pgs_sort_pairs_noalloc.argtypes = [vp, vp, i64, i32, i32, vp, vp]
    L.pgs_autotune.argtypes = [vp, P(Camera), i32, P(ImagePtrs), P(ImageGradPtrs), P(ParamGradPtrs), i32,
                               P(TuneEntry), i32, P(i32), vp]
    L.pgs_scene_get_params.argtypes = [vp, P(RenderParams)]
    L.pgs_filter_depth_prior.argtypes = [vp, P(Camera), i32, vp, vp, i64, P(PriorParams), vp, vp, vp, vp, vp]
    L.pgs_ncc_loss_grad.argtypes = [vp, P(Camera), i32, P(ImagePtrs), vp, i64, P(NccParams), vp, vp,
                                    P(ImageGradPtrs), vp]
    L.pgs_tsdf_integrate.argtypes = [vp, P(Camera), i32, vp, vp, P(TsdfVolume), vp, vp, vp, vp]


def check(status: int) -> None:
    if status != PGS_OK:
        raise PGSError(status, lib().pgs_last_error().decode())


def _ptr(t: Optional[torch.Tensor]) -> Optional[int]:
    if t is None:
        return None
    if not t.is_cuda:
        raise ArgumentError("tensor must live on a CUDA device")
    if not t.is_contiguous():
        raise ArgumentError("tensor must be contiguous")
    return t.data_ptr()


def _stream(stream: Optional[torch.cuda.Stream]) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


# The C entry points receive bare device pointers and cannot see how large a
# buffer is: a tensor of the wrong length or element type would be read or
# written out of range on the device.  The binding therefore checks every
# tensor it passes against the size the call implies and raises ValueError
# before any device work.
def _expect(t: Optional[torch.Tensor], numel: int, name: str, dtype=torch.float32, optional: bool = False) -> None:
    if t is None:
        if optional:
            return
        raise ArgumentError(f"{name} is required")
    if t.dtype != dtype:
        raise ArgumentError(f"{name} must be {dtype} (got {t.dtype})")
    if t.numel() != numel:
        raise ArgumentError(f"{name} must have {numel} elements (got {t.numel()})")


def check_anchor_tensors(n_anchors: int, in_dim: int, x, level, log_l, offsets, feat, W1, b1, W2, b2) -> None:
    """Shapes of pgs_anchor_ptrs / pgs_mlp_ptrs for a scene of n_anchors anchors (include/pgs.h)."""
    N = n_anchors
    _expect(x, 3 * N, "x"); _expect(level, N, "level", torch.int32); _expect(log_l, 3 * N, "log_l")
    _expect(offsets, N * N_OFFSETS * 3, "offsets"); _expect(feat, N * FEAT_DIM, "feat")
    _expect(W1, HIDDEN * in_dim, "W1"); _expect(b1, HIDDEN, "b1")
    _expect(W2, OUT_DIM * HIDDEN, "W2"); _expect(b2, OUT_DIM, "b2")


def check_explicit_tensors(n: int, means, log_scales, quats, opacity_logits, colors) -> None:
    """Shapes of pgs_explicit_ptrs for a scene of n explicit Gaussians (include/pgs.h)."""
    _expect(means, 3 * n, "means"); _expect(log_scales, 3 * n, "log_scales"); _expect(quats, 4 * n, "quats")
    _expect(opacity_logits, n, "opacity_logits"); _expect(colors, 3 * n, "colors")


def default_params(**kw) -> RenderParams:
    p = RenderParams()
    lib().pgs_default_params(C.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def pack_cameras(cams) -> C.Array:
    """synth.Camera (or anything with R, t, fx, fy, cx, cy, width, height) -> pgs_camera[]."""
    arr = (Camera * len(cams))()
    for i, c in enumerate(cams):
        arr[i].R[:] = [float(v) for v in list(c.R.reshape(-1))]
        arr[i].t[:] = [float(v) for v in list(c.t.reshape(-1))]
        arr[i].fx, arr[i].fy, arr[i].cx, arr[i].cy = float(c.fx), float(c.fy), float(c.cx), float(c.cy)
        arr[i].width, arr[i].height = int(c.width), int(c.height)
    return arr


class _DevView:
    """__cuda_array_interface__ over a library-owned device buffer (read-only use)."""

    def __init__(self, ptr: int, n: int, typestr: str):
        self.__cuda_array_interface__ = dict(shape=(n,), typestr=typestr, data=(ptr, False), version=3)


# ------------------------------------------------------------------ images in the ragged arena
def arena_offsets(cams) -> List[int]:
    off, acc = [], 0
    for c in cams:
        off.append(acc)
        acc += int(c.width) * int(c.height)
    return off + [acc]


@dataclasses.dataclass
class Images:
    rgb: torch.Tensor
    depth: torch.Tensor
    normal: torch.Tensor
    dist: torch.Tensor
    t_final: torch.Tensor
    last: torch.Tensor
    n_contrib: Optional[torch.Tensor]   # diagnostic per-pixel counts; None skips them (faster forward)
    n_eval: Optional[torch.Tensor]
    offsets: List[int]
    shapes: List[tuple]

    @staticmethod
    def empty(cams, device="cuda", stats: bool = True) -> "Images":
        off = arena_offsets(cams)
        n = off[-1]
        f = lambda k: torch.zeros(k, device=device, dtype=torch.float32)
        i = lambda k: torch.zeros(k, device=device, dtype=torch.int32)
        return Images(f(3 * n), f(n), f(3 * n), f(n), f(n), i(n), i(n) if stats else None, i(n) if stats else None,
                      off, [(int(c.height), int(c.width)) for c in cams])

    def check(self, cams) -> None:
        """Raise ValueError unless these buffers are laid out for the arena of ``cams``."""
        if list(self.offsets) != arena_offsets(cams):
            raise ArgumentError("images were allocated for another set of views (arena offsets differ)")
        n = self.offsets[-1]
        for k, m in (("rgb", 3 * n), ("depth", n), ("normal", 3 * n), ("dist", n), ("t_final", n)):
            _expect(getattr(self, k), m, f"images.{k}")
        _expect(self.last, n, "images.last", torch.int32)
        _expect(self.n_contrib, n, "images.n_contrib", torch.int32, optional=True)
        _expect(self.n_eval, n, "images.n_eval", torch.int32, optional=True)

    def without_stats(self) -> "Images":
        """The same buffers with the diagnostic counts switched off."""
        return dataclasses.replace(self, n_contrib=None, n_eval=None)

    def ptrs(self) -> ImagePtrs:
        return ImagePtrs(_ptr(self.rgb), _ptr(self.depth), _ptr(self.normal), _ptr(self.dist), _ptr(self.t_final),
                         _ptr(self.last), _ptr(self.n_contrib), _ptr(self.n_eval))

    def view(self, v: int) -> Dict[str, torch.Tensor]:
        H, W = self.shapes[v]
        a, b = self.offsets[v], self.offsets[v + 1]
        out = dict(rgb=self.rgb[3 * a:3 * b].view(3, H, W), normal=self.normal[3 * a:3 * b].view(3, H, W))
        for k in ("depth", "dist", "t_final", "last", "n_contrib", "n_eval"):
            t = getattr(self, k)
            if t is not None:
                out[k] = t[a:b].view(H, W)
        return out


@dataclasses.dataclass
class ImageGrads:
    rgb: torch.Tensor
    depth: torch.Tensor
    normal: torch.Tensor

    @staticmethod
    def empty(n_pix: int, device="cuda") -> "ImageGrads":
        return ImageGrads(torch.zeros(3 * n_pix, device=device), torch.zeros(n_pix, device=device),
                          torch.zeros(3 * n_pix, device=device))

    @staticmethod
    def from_views(views: Sequence[dict], device="cuda") -> "ImageGrads":
        cat = lambda k: torch.cat([v[k].reshape(-1) for v in views]).to(device, torch.float32).contiguous()
        return ImageGrads(cat("rgb"), cat("depth"), cat("normal"))

    def check(self, n_pix: int) -> None:
        _expect(self.rgb, 3 * n_pix, "grads.rgb"); _expect(self.depth, n_pix, "grads.depth")
        _expect(self.normal, 3 * n_pix, "grads.normal")

    def ptrs(self) -> ImageGradPtrs:
        return ImageGradPtrs(_ptr(self.rgb), _ptr(self.depth), _ptr(self.normal))


@dataclasses.dataclass
class Targets:
    rgb: torch.Tensor
    prior: torch.Tensor
    mask: torch.Tensor

    @staticmethod
    def from_views(views: Sequence[dict], device="cuda") -> "Targets":
        cat = lambda k: torch.cat([v[k].reshape(-1) for v in views]).to(device, torch.float32).contiguous()
        return Targets(cat("rgb"), cat("prior"), cat("mask"))

    def check(self, n_pix: int) -> None:
        _expect(self.rgb, 3 * n_pix, "targets.rgb"); _expect(self.prior, n_pix, "targets.prior")
        _expect(self.mask, n_pix, "targets.mask")

    def ptrs(self) -> TargetPtrs:
        return TargetPtrs(_ptr(self.rgb), _ptr(self.prior), _ptr(self.mask))


# ------------------------------------------------------------------ scene
class Scene:
    """Owns a pgs_scene (workspace) and keeps references to the bound tensors."""

    def __init__(self, mode: int, n_primitives: int, max_views: int, max_pixels: int, capacity_pairs: int,
                 capacity_rows: int = 0, params: Optional[RenderParams] = None):
        self.desc = SceneDesc(mode=mode, n_primitives=n_primitives, max_views=max_views, max_pixels=max_pixels,
                              capacity_rows=capacity_rows, capacity_pairs=capacity_pairs,
                              params=params if params is not None else default_params())
        h = C.c_void_p()
        check(lib().pgs_scene_create(C.byref(self.desc), C.byref(h)))
        self.handle = h
        self._keep = []
        self._grad_numel: Dict[str, int] = {}

    def _param_grad_ptrs(self, param_grads: Dict[str, torch.Tensor]) -> ParamGradPtrs:
        """Gradient buffers are accumulated into: each one must match its bound parameter's size."""
        for n, t in param_grads.items():
            if t is None:
                continue
            if n not in self._grad_numel:
                raise ArgumentError(f"param_grads[{n!r}]: no such parameter is bound to this scene")
            _expect(t, self._grad_numel[n], f"param_grads[{n!r}]")
        return ParamGradPtrs(*[_ptr(param_grads.get(n)) for n in PARAM_GRAD_FIELDS])

    def close(self):
        if getattr(self, "handle", None):
            lib().pgs_scene_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def bind_explicit(self, means, log_scales, quats, opacity_logits, colors):
        check_explicit_tensors(self.desc.n_primitives, means, log_scales, quats, opacity_logits, colors)
        ts = [t.contiguous() for t in (means, log_scales, quats, opacity_logits, colors)]
        self._keep = ts
        self._grad_numel = dict(zip(("means", "log_scales", "quats", "opacity_logits", "colors"),
                                    (t.numel() for t in ts)))
        check(lib().pgs_scene_bind_explicit(self.handle, C.byref(ExplicitPtrs(*[_ptr(t) for t in ts]))))

    def bind_anchors(self, x, level, log_l, offsets, feat, W1, b1, W2, b2):
        check_anchor_tensors(self.desc.n_primitives, self.desc.params.in_dim, x, level, log_l, offsets, feat, W1, b1,
                             W2, b2)
        ts = [t.contiguous() for t in (x, level, log_l, offsets, feat, W1, b1, W2, b2)]
        self._keep = ts
        self._grad_numel = {n: t.numel() for n, t in zip(("x", "level", "log_l", "offsets", "feat", "W1", "b1", "W2",
                                                            "b2"), ts) if n != "level"}
        check(lib().pgs_scene_bind_anchors(self.handle, C.byref(AnchorPtrs(*[_ptr(t) for t in ts[:5]])),
                                           C.byref(MlpPtrs(*[_ptr(t) for t in ts[5:]]))))

    def render(self, cams, images: Optional[Images] = None, stream=None, packed=None) -> Images:
        images = images if images is not None else Images.empty(cams)
        images.check(cams)
        cc = packed if packed is not None else pack_cameras(cams)
        check(lib().pgs_render_batch(self.handle, cc, len(cams), C.byref(images.ptrs()), _stream(stream)))
        return images

    def loss_grad(self, cams, images: Images, targets: Targets, lambda_depth=1.0, lambda_normal=0.1,
                  loss: Optional[torch.Tensor] = None, grads: Optional[ImageGrads] = None, stream=None, packed=None):
        n = images.offsets[-1]
        loss = loss if loss is not None else torch.zeros(4, device=images.rgb.device)
        grads = grads if grads is not None else ImageGrads.empty(n, images.rgb.device)
        images.check(cams)
        targets.check(n)
        grads.check(n)
        if loss.dtype != torch.float32 or loss.numel() < 4:
            raise ArgumentError("loss must be float32 with at least 4 elements (total, rgb, depth, normal)")
        cc = packed if packed is not None else pack_cameras(cams)
        check(lib().pgs_loss_grad(self.handle, cc, len(cams), C.byref(images.ptrs()), C.byref(targets.ptrs()),
                                  C.byref(LossParams(lambda_depth, lambda_normal)), _ptr(loss), C.byref(grads.ptrs()),
                                  _stream(stream)))
        return loss, grads

    def backward(self, cams, images: Images, grads: ImageGrads, param_grads: Dict[str, torch.Tensor], stream=None,
                 packed=None):
        images.check(cams)
        grads.check(images.offsets[-1])
        pg = self._param_grad_ptrs(param_grads)
        cc = packed if packed is not None else pack_cameras(cams)
        check(lib().pgs_backward(self.handle, cc, len(cams), C.byref(images.ptrs()), C.byref(grads.ptrs()),
                                 C.byref(pg), _stream(stream)))

    def autotune(self, cams, images: Images, grads: ImageGrads, param_grads: Dict[str, torch.Tensor], reps: int = 3,
                 stream=None, packed=None) -> List[dict]:
        """Pick tile shape and forward shared-memory batch by timing (pgs_autotune); returns the
        timed combinations (one entry with ms = -1 when the choice came from the cache)."""
        images.check(cams)
        grads.check(images.offsets[-1])
        pg = self._param_grad_ptrs(param_grads)
        cc = packed if packed is not None else pack_cameras(cams)
        out = (TuneEntry * 16)()
        n = C.c_int(0)
        check(lib().pgs_autotune(self.handle, cc, len(cams), C.byref(images.ptrs()), C.byref(grads.ptrs()),
                                 C.byref(pg), reps, out, 16, C.byref(n), _stream(stream)))
        return [dict(tile_w=e.tile_w, tile_h=e.tile_h, blend_batch=e.blend_batch, ms=e.ms) for e in out[:n.value]]

    def filter_depth_prior(self, cams, pseudo: torch.Tensor, points: torch.Tensor, tau_d: float = 1.0,
                           k_neighbors: int = 2, with_error: bool = False, stream=None, packed=None,
                           out: Optional[dict] = None) -> dict:
        """Enhanced depth prior (pgs_filter_depth_prior): pseudo depth in the arena layout and world
        points [n, 3] -> dict(prior, mask, scale_shift [views, 2], err).  `out` may supply the
        prior / mask / scale_shift buffers (e.g. a Targets' prior and mask)."""
        n = arena_offsets(cams)[-1]
        _expect(pseudo, n, "pseudo")
        if points.dim() != 2 or points.shape[-1] != 3 or points.dtype != torch.float32:
            raise ArgumentError(f"points must be float32 [n, 3] (got {points.dtype} {tuple(points.shape)})")
        given = out or {}
        out = dict(prior=given.get("prior", None), mask=given.get("mask", None),
                   scale_shift=given.get("scale_shift", None), err=None)
        if out["prior"] is None:
            out["prior"] = torch.empty(n, device=pseudo.device)
        if out["mask"] is None:
            out["mask"] = torch.empty(n, device=pseudo.device)
        if out["scale_shift"] is None:
            out["scale_shift"] = torch.empty(len(cams), 2, device=pseudo.device)
        if with_error:
            out["err"] = torch.empty(n, device=pseudo.device)
        _expect(out["prior"], n, "out['prior']"); _expect(out["mask"], n, "out['mask']")
        _expect(out["scale_shift"], 2 * len(cams), "out['scale_shift']")
        cc = packed if packed is not None else pack_cameras(cams)
        pts = points.contiguous()
        pp = PriorParams(tau_d, k_neighbors)
        check(lib().pgs_filter_depth_prior(self.handle, cc, len(cams), _ptr(pseudo), _ptr(pts) if pts.numel() else None,
                                           pts.shape[0], C.byref(pp), _ptr(out["prior"]), _ptr(out["mask"]),
                                           _ptr(out["scale_shift"]), _ptr(out["err"]), _stream(stream)))
        return out

    def ncc_loss_grad(self, cams, images: "Images", centers: torch.Tensor, grads: "ImageGrads",
                      lambda_ncc: float = 0.2, eps: float = 1e-6, geometric: bool = True,
                      ncc_out: Optional[torch.Tensor] = None, loss: Optional[torch.Tensor] = None, stream=None,
                      packed=None) -> dict:
        """Batch geometric NCC loss (pgs_ncc_loss_grad, Eq. 10): centres int32/uint32 [B/2, N] local
        pixel indices of the reference views; gradients accumulated into `grads`.  Returns
        dict(ncc [B/2, N] (-2 = unused patch), loss [2] = (lambda * L, L))."""
        cc = packed if packed is not None else pack_cameras(cams)
        centers = centers.contiguous()
        n_pairs = len(cams) // 2
        n_per = centers.shape[-1] if centers.numel() else 0
        if ncc_out is None:
            ncc_out = torch.empty(max(1, n_pairs * n_per), device=images.rgb.device)
        if loss is None:
            loss = torch.zeros(2, device=images.rgb.device)
        images.check(cams)
        grads.check(images.offsets[-1])
        if centers.numel() and (centers.dtype not in (torch.int32, torch.uint32) or
                                centers.numel() != n_pairs * n_per):
            raise ArgumentError(f"centers must be int32/uint32 [{n_pairs}, N] (got {centers.dtype} "
                             f"{tuple(centers.shape)})")
        if ncc_out.dtype != torch.float32 or ncc_out.numel() < max(1, n_pairs * n_per):
            raise ArgumentError(f"ncc_out must be float32 with at least {max(1, n_pairs * n_per)} elements")
        if loss.dtype != torch.float32 or loss.numel() < 2:
            raise ArgumentError("loss must be float32 with at least 2 elements")
        npar = NccParams(lambda_ncc, eps, 1 if geometric else 0)
        check(lib().pgs_ncc_loss_grad(self.handle, cc, len(cams), C.byref(images.ptrs()),
                                      _ptr(centers) if centers.numel() else None, n_per, C.byref(npar),
                                      _ptr(ncc_out), _ptr(loss), C.byref(grads.ptrs()), _stream(stream)))
        return dict(ncc=ncc_out[:n_pairs * n_per].view(n_pairs, n_per), loss=loss)

    def tsdf_integrate(self, cams, depth: torch.Tensor, volume: dict, rgb: Optional[torch.Tensor] = None,
                       stream=None, packed=None) -> dict:
        """TSDF fusion (pgs_tsdf_integrate) of depth (and colour) maps in the arena layout into
        volume = dict(origin, voxel, dims, trunc, tsdf, weight[, color]) (state tensors updated in place)."""
        cc = packed if packed is not None else pack_cameras(cams)
        vol = TsdfVolume((C.c_float * 3)(*volume["origin"]), volume["voxel"], (C.c_int32 * 3)(*volume["dims"]),
                         volume["trunc"])
        color = volume.get("color") if rgb is not None else None
        n = arena_offsets(cams)[-1]
        nv = int(volume["dims"][0]) * int(volume["dims"][1]) * int(volume["dims"][2])
        _expect(depth, n, "depth"); _expect(rgb, 3 * n, "rgb", optional=True)
        _expect(volume["tsdf"], nv, "volume['tsdf']"); _expect(volume["weight"], nv, "volume['weight']")
        if rgb is not None:
            _expect(color, 3 * nv, "volume['color']")
        check(lib().pgs_tsdf_integrate(self.handle, cc, len(cams), _ptr(depth), _ptr(rgb), C.byref(vol),
                                       _ptr(volume["tsdf"]), _ptr(volume["weight"]), _ptr(color), _stream(stream)))
        return volume

    def params(self) -> dict:
        p = RenderParams()
        check(lib().pgs_scene_get_params(self.handle, C.byref(p)))
        return {k: getattr(p, k) for k, _ in RenderParams._fields_}

    def decode(self, cams, capacity_rows: int, stream=None):
        dev = "cuda"
        G = capacity_rows * 10
        rows = torch.zeros(capacity_rows, dtype=torch.int32, device=dev)
        out = dict(mu=torch.zeros(G, 3, device=dev), opacity=torch.zeros(G, device=dev),
                   color=torch.zeros(G, 3, device=dev), scale=torch.zeros(G, 3, device=dev),
                   quat=torch.zeros(G, 4, device=dev))
        n = torch.zeros(1, dtype=torch.int64, device=dev)
        check(lib().pgs_decode_anchors(self.handle, pack_cameras(cams), len(cams), _ptr(rows), _ptr(out["mu"]),
                                       _ptr(out["opacity"]), _ptr(out["color"]), _ptr(out["scale"]),
                                       _ptr(out["quat"]), _ptr(n), _stream(stream)))
        nr = int(n.item())
        out = {k: v[:nr * 10] for k, v in out.items()}
        out["rows"] = rows[:nr]
        return out

    def read_status(self, stream=None) -> None:
        check(lib().pgs_read_status(self.handle, _stream(stream)))

    def stats(self, stream=None) -> Stats:
        st = Stats()
        check(lib().pgs_get_stats(self.handle, C.byref(st), _stream(stream)))
        return st

    def set_wait_limits(self, spin_limit: int = 0, withhold_tile: Optional[int] = None) -> None:
        """pgs_scene_set_wait_limits: polls before a sort look-back gives up (0 = default) and the
        failure-path hook that withholds one onesweep tile's status (None = publish every tile)."""
        check(lib().pgs_scene_set_wait_limits(self.handle, spin_limit,
                                              NO_WITHHELD_TILE if withhold_tile is None else withhold_tile))

    def set_profiling(self, on: bool) -> None:
        check(lib().pgs_set_profiling(self.handle, 1 if on else 0))

    def stage_times(self) -> Dict[str, float]:
        ms = (C.c_float * len(STAGES))()
        check(lib().pgs_get_stage_times(self.handle, ms, len(STAGES)))
        return {k: float(v) for k, v in zip(STAGES, ms)}

    def buffer(self, which: int, n: int, typestr: str = "<i4") -> torch.Tensor:
        """Copy of the first n elements of a workspace buffer (see pgs_scene_buffer)."""
        p, cap = C.c_void_p(), C.c_int64()
        check(lib().pgs_scene_buffer(self.handle, which, C.byref(p), C.byref(cap)))
        n = max(0, min(n, cap.value))
        if n == 0:
            return torch.zeros(0, dtype=torch.int32 if typestr == "<i4" else torch.float32, device="cuda")
        return torch.as_tensor(_DevView(p.value, n, typestr), device="cuda").clone()


# ------------------------------------------------------------------ stand-alone stages
def _check_sort_operands(keys: torch.Tensor, vals: torch.Tensor) -> None:
    """The C entry points see only pointers and one count, so the binding
    checks what they cannot: equal element counts, 4-byte elements,
    contiguous CUDA tensors on the current device.  Raises ValueError."""
    if keys.numel() != vals.numel():
        raise ArgumentError(f"keys ({keys.numel()}) and values ({vals.numel()}) differ in length")
    if keys.element_size() != 4 or vals.element_size() != 4:
        raise ArgumentError(f"keys and values need 4-byte elements (got {keys.dtype}, {vals.dtype})")
    if not (keys.is_contiguous() and vals.is_contiguous()):
        raise ArgumentError("keys and values must be contiguous")
    if keys.device.type != "cuda" or vals.device.type != "cuda":
        raise ArgumentError(f"keys and values must be CUDA tensors (got {keys.device}, {vals.device})")
    cur = torch.cuda.current_device()
    if keys.device.index != cur or vals.device.index != cur:
        raise ArgumentError(f"keys ({keys.device}) and values ({vals.device}) must sit on the current device cuda:{cur}")


def sort_pairs(keys: torch.Tensor, vals: torch.Tensor, bit_lo: int = 0, bit_hi: int = 32):
    """Stable radix sort of int32-stored uint32 keys/values on device (in place)."""
    _check_sort_operands(keys, vals)
    n = keys.numel()
    if n == 0:                       # one-element buffers; the library sees n = 0
        keys = torch.zeros(1, dtype=keys.dtype, device=keys.device)
        vals = torch.zeros(1, dtype=vals.dtype, device=vals.device)
    alt_k, alt_v = torch.empty_like(keys), torch.empty_like(vals)
    nbytes = lib().pgs_sort_scratch_bytes(max(n, 1))
    scratch = torch.empty(nbytes, dtype=torch.uint8, device=keys.device)
    d_n = torch.tensor([n], dtype=torch.int64, device=keys.device)
    err = torch.zeros(1, dtype=torch.int32, device=keys.device)
    check(lib().pgs_sort_pairs(_ptr(keys), _ptr(vals), _ptr(alt_k), _ptr(alt_v), _ptr(d_n), max(n, 1), bit_lo, bit_hi,
                               _ptr(scratch), nbytes, _ptr(err), _stream(None)))
    return keys[:n], vals[:n], err


NOALLOC_MAX_N = 1 << 20
NO_WITHHELD_TILE = 0xFFFFFFFF


def sort_pairs_noalloc(keys: torch.Tensor, vals: torch.Tensor, bit_lo: int = 0, bit_hi: int = 32,
                       err: Optional[torch.Tensor] = None):
    """In-place stable radix sort through pgs_sort_pairs_noalloc: the library
    allocates nothing (its scratch is a fixed array in its device image), for
    callers that must not allocate device memory.  n <= NOALLOC_MAX_N.  The
    first call on a device may still load the library's device code (lazy
    loading): warm up once per device.  ``err`` (int32, one element) must be
    zero on entry."""
    _check_sort_operands(keys, vals)
    if keys.numel() == 0:
        return keys, vals
    check(lib().pgs_sort_pairs_noalloc(_ptr(keys), _ptr(vals), keys.numel(), bit_lo, bit_hi, _ptr(err),
                                       _stream(None)))
    return keys, vals


def exclusive_scan(x: torch.Tensor, index: Optional[torch.Tensor] = None):
    n = x.numel() if index is None else index.numel()
    if x.numel() == 0:
        x = torch.zeros(1, dtype=x.dtype, device=x.device)
    out = torch.empty(max(n, 1), dtype=torch.int32, device=x.device)
    total = torch.zeros(1, dtype=torch.int64, device=x.device)
    nbytes = lib().pgs_scan_scratch_bytes()
    scratch = torch.empty(nbytes, dtype=torch.uint8, device=x.device)
    d_n = torch.tensor([n], dtype=torch.int64, device=x.device)
    check(lib().pgs_exclusive_scan_u32(_ptr(x), _ptr(index), _ptr(out), _ptr(total), _ptr(d_n), _ptr(scratch), nbytes,
                                       _stream(None)))
    return out[:n], total


# ------------------------------------------------------------------ autograd
class RenderFunction(torch.autograd.Function):
    """forward = cull + decode + project + bin/sort + blend (pgs_render_batch);
    backward = pgs_backward (transmittance recomputed from t_final and last).
    The scene must already be bound to ``params`` (same tensors)."""

    @staticmethod
    def forward(ctx, scene: Scene, cams, names: tuple, *params):
        images = scene.render(cams)
        ctx.scene, ctx.cams, ctx.names, ctx.images = scene, cams, names, images
        ctx.shapes = [p.shape for p in params]
        return images.rgb, images.depth, images.normal

    @staticmethod
    def backward(ctx, g_rgb, g_depth, g_normal):
        imgs = ctx.images
        grads = ImageGrads(*(g.contiguous() if g is not None else torch.zeros_like(t)
                             for g, t in zip((g_rgb, g_depth, g_normal), (imgs.rgb, imgs.depth, imgs.normal))))
        pg = {n: torch.zeros(s, device=imgs.rgb.device) for n, s in zip(ctx.names, ctx.shapes) if n != "level"}
        ctx.scene.backward(ctx.cams, imgs, grads, pg)
        return (None, None, None) + tuple(pg.get(n) for n in ctx.names)
