"""Autotuning cache for uneven batches.

``ffeq_batch_autotune`` times launch shapes on the GPU and keeps the fastest in
the plan; this module stores the result in a JSON file keyed by the GPU name,
the batch configuration and the multiset of instance shapes, so that a later
process with the same batch skips the timing and restores the tuning with
``ffeq_batch_set_tuning``.  Only launch shapes are cached: pipeline depth and
CTA width give bit-identical results, lanes per row changes only the rounding
order of the solve.
"""
from __future__ import annotations

import hashlib
import json
import os

from . import ffeq

__all__ = ["batch_key", "default_cache_path", "autotune_cached"]


def default_cache_path() -> str:
    return os.environ.get("FFEQ_TUNING_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "ffeq", "tuning.json"))


def batch_key(batch: ffeq.Batch, device_name: str) -> str:
    c = batch.config
    shapes = sorted((i.B, i.U, i.C, i.n_sc, i.n_sym) for i in batch.instances)
    text = json.dumps([device_name, c.arch, c.precision, c.estimate, c.llr_bits, c.equalizer, c.lama_iters, shapes])
    return hashlib.sha256(text.encode()).hexdigest()[:32]


def _load(path: str) -> dict:
    try:
        with open(path) as f:
            data = json.load(f)
        return data if isinstance(data, dict) else {}
    except (OSError, ValueError):
        return {}


def autotune_cached(batch: ffeq.Batch, H, y, z, sigma2, llr=None, info=None, workspace=None,
                    workspace_bytes: int = 0, stream=None, reps: int = 5, path: str | None = None,
                    device_name: str | None = None) -> tuple[list, bool]:
    """Restore the cached tuning of this batch or autotune and store it.

    Returns ``(tuning, from_cache)``.  A cached entry that the plan rejects
    (a different library build) is replaced by a fresh autotune.
    """
    if device_name is None:
        import torch
        device_name = torch.cuda.get_device_name()
    path = path or default_cache_path()
    key = batch_key(batch, device_name)
    cache = _load(path)
    if key in cache:
        try:
            ffeq.ffeq_batch_set_tuning(batch, [tuple(t) for t in cache[key]])
            return ffeq.ffeq_batch_get_tuning(batch), True
        except ffeq.FfeqError:
            pass
    ffeq.ffeq_batch_autotune(batch, H, y, z, sigma2, llr, info, workspace, workspace_bytes, stream, reps)
    tuning = ffeq.ffeq_batch_get_tuning(batch)
    cache = _load(path)
    cache[key] = [list(t) for t in tuning]
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)
    return tuning, False
