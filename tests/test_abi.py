"""The C-ABI library loads and exports every entry point include/pgs.h
declares; the Python binding mirrors the header's structs (no GPU needed)."""
import ctypes
import os
import re

import pytest

from paper_2503_23044_b300 import binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(pgs_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def _lib():
    if not os.path.exists(B.LIB_PATH):
        from paper_2503_23044_b300 import build
        build.build()
    return B.lib()


def test_library_exports_every_declared_symbol():
    L = _lib()
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(B.ENTRY_POINTS)


def test_struct_sizes_match_header_layout():
    assert ctypes.sizeof(B.Camera) == 18 * 4
    assert ctypes.sizeof(B.RenderParams) == 15 * 4
    assert ctypes.sizeof(B.TuneEntry) == 4 * 4
    assert ctypes.sizeof(B.ImagePtrs) == 8 * 8
    assert ctypes.sizeof(B.ParamGradPtrs) == 13 * 8
    assert ctypes.sizeof(B.Stats) == 7 * 8
    assert ctypes.sizeof(B.PriorParams) == 2 * 4
    assert ctypes.sizeof(B.NccParams) == 3 * 4
    assert ctypes.sizeof(B.TsdfVolume) == 8 * 4


def test_default_params_and_argument_errors_without_gpu():
    _lib()
    p = B.default_params()
    assert abs(p.alpha_min - 1 / 255) < 1e-9 and p.alpha_max == pytest.approx(0.99) and p.t_min == pytest.approx(1e-4)
    assert p.tile_w == 16 and p.tile_h == 16 and p.in_dim == 35 and p.blend_batch == 256
    L = B.lib()
    h = ctypes.c_void_p()
    bad = B.SceneDesc(mode=7, n_primitives=10, max_views=1, max_pixels=100, capacity_rows=0, capacity_pairs=100,
                      params=p)
    assert L.pgs_scene_create(ctypes.byref(bad), ctypes.byref(h)) == B.PGS_ERR_INVALID_ARG
    assert b"mode" in L.pgs_last_error()
    bad.mode = 0
    bad.params.tile_w = 12
    assert L.pgs_scene_create(ctypes.byref(bad), ctypes.byref(h)) == B.PGS_ERR_INVALID_ARG
    assert b"tile shape" in L.pgs_last_error()
    bad.params.tile_w = 16
    bad.params.blend_batch = 100
    assert L.pgs_scene_create(ctypes.byref(bad), ctypes.byref(h)) == B.PGS_ERR_INVALID_ARG
    assert b"blend_batch" in L.pgs_last_error()
    bad.params.blend_batch = 256
    bad.capacity_pairs = 1 << 31
    assert L.pgs_scene_create(ctypes.byref(bad), ctypes.byref(h)) == B.PGS_ERR_INVALID_ARG
    assert L.pgs_status_string(B.PGS_ERR_TIMEOUT) == b"bounded wait timed out"


def test_stage_names_match_header_enum():
    src = open(os.path.join(ROOT, "include", "pgs.h")).read()
    stages = dict((m.group(1).lower(), int(m.group(2)))
                  for m in re.finditer(r"\bPGS_STAGE_([A-Z_0-9]+)\s*=\s*(\d+)", src))
    n = int(re.search(r"\bPGS_N_STAGES\s*=\s*(\d+)", src).group(1))
    assert len(B.STAGES) == n == len(stages)
    for i, name in enumerate(B.STAGES):
        assert stages[name] == i, name


def test_new_entry_points_reject_null_arguments_without_gpu():
    """The depth-prior, NCC and TSDF calls validate their arguments before any
    device work: a null scene or parameter block is an argument error."""
    L = _lib()
    pp = B.PriorParams(1.0, 2)
    assert L.pgs_filter_depth_prior(None, None, 2, None, None, 0, ctypes.byref(pp), None, None, None, None,
                                    None) == B.PGS_ERR_INVALID_ARG
    npar = B.NccParams(0.2, 1e-6, 1)
    img, grad = B.ImagePtrs(), B.ImageGradPtrs()
    assert L.pgs_ncc_loss_grad(None, None, 2, ctypes.byref(img), None, 16, ctypes.byref(npar), None, None,
                               ctypes.byref(grad), None) == B.PGS_ERR_INVALID_ARG
    vol = B.TsdfVolume((ctypes.c_float * 3)(0, 0, 0), 0.01, (ctypes.c_int32 * 3)(4, 4, 4), 0.04)
    assert L.pgs_tsdf_integrate(None, None, 1, None, None, ctypes.byref(vol), None, None, None,
                                None) == B.PGS_ERR_INVALID_ARG
    assert b"null" in L.pgs_last_error()


def test_sort_bindings_reject_operands_the_c_side_cannot_check():
    """The sort entry points receive pointers and one count: the binding must
    refuse mismatched lengths, element sizes other than 4 bytes and tensors
    not on the current CUDA device before any call into the library."""
    import torch
    k32 = torch.zeros(8, dtype=torch.int32)
    for fn in (B.sort_pairs, B.sort_pairs_noalloc):
        with pytest.raises(ValueError, match="differ in length"):
            fn(k32, torch.zeros(7, dtype=torch.int32))
        with pytest.raises(ValueError, match="4-byte"):
            fn(torch.zeros(8, dtype=torch.int16), torch.zeros(8, dtype=torch.int16))
        with pytest.raises(ValueError, match="4-byte"):
            fn(k32, torch.zeros(8, dtype=torch.int64))
        with pytest.raises(ValueError, match="CUDA"):
            fn(k32, torch.zeros(8, dtype=torch.int32))
