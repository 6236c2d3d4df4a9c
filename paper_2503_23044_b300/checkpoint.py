"""Checkpoint and resume of a training state.

One file holds the parameter tensors a scene is bound to (anchors and decoder
MLP, or explicit Gaussians), the render parameters (``pgs_render_params``),
the step count, and optionally an optimiser's ``state_dict`` and any extra
picklable entries.  Tensors are stored on the CPU and restored to the device
the caller names.  The file is written to a temporary name in the same folder
and renamed over the target, so a crash during the write leaves the previous
checkpoint intact.

This is bookkeeping around the training step, not part of it: the paper only
reports model storage sizes and describes no checkpoint mechanism.
"""
from __future__ import annotations

import os
import tempfile
from typing import Any, Dict, Optional, Union

import torch

from . import binding as B

FORMAT = 1


def render_params_dict(p: Union[B.RenderParams, Dict[str, Any]]) -> Dict[str, Any]:
    """The fields of a RenderParams struct as a plain dict (a dict is returned as a copy)."""
    if isinstance(p, dict):
        return dict(p)
    return {k: getattr(p, k) for k, _ in B.RenderParams._fields_}


def render_params_from_dict(d: Dict[str, Any]) -> B.RenderParams:
    """A RenderParams struct with the given fields (unknown keys are refused)."""
    p = B.RenderParams()
    names = {k for k, _ in B.RenderParams._fields_}
    for k, v in d.items():
        if k not in names:
            raise KeyError(f"not a render parameter: {k!r}")
        setattr(p, k, v)
    return p


def save(path: str, params: Dict[str, torch.Tensor], render_params: Union[B.RenderParams, Dict[str, Any]],
         step: int, optimizer_state: Optional[dict] = None, extra: Optional[dict] = None) -> None:
    """Write a checkpoint to ``path`` (atomically replaced)."""
    state = dict(format=FORMAT, step=int(step),
                 params={k: v.detach().to("cpu", copy=True) for k, v in params.items()},
                 render_params=render_params_dict(render_params),
                 optimizer_state=optimizer_state, extra=extra or {})
    folder = os.path.dirname(os.path.abspath(path))
    fd, tmp = tempfile.mkstemp(prefix=".ckpt-", dir=folder)
    try:
        with os.fdopen(fd, "wb") as f:
            torch.save(state, f)
            f.flush()
            os.fsync(f.fileno())
        os.replace(tmp, path)
    except BaseException:
        if os.path.exists(tmp):
            os.unlink(tmp)
        raise


def load(path: str, device: Union[str, torch.device] = "cuda") -> Dict[str, Any]:
    """Read a checkpoint: dict(step, params (on ``device``), render_params (dict),
    optimizer_state, extra).  Optimiser tensors stay on the CPU; the optimiser's
    ``load_state_dict`` moves them next to its parameters.  The file is read with
    torch's weights-only unpickler, so loading runs no code from the file; ``extra``
    must therefore hold plain values (numbers, strings, lists, tuples, dicts, tensors)."""
    state = torch.load(path, map_location="cpu", weights_only=True)
    if not isinstance(state, dict) or state.get("format") != FORMAT:
        raise ValueError(f"{path}: not a checkpoint of format {FORMAT}")
    state["params"] = {k: v.to(device) for k, v in state["params"].items()}
    return state
