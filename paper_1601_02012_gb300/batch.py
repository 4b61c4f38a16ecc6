"""Batches of lightcones behind rr_batch_* (one persistent launch per step),
with a JSON cache for the autotuner's choice."""
from __future__ import annotations

import hashlib
import json
import os

from . import _rr


def _cache_path():
    root = os.environ.get("RR_TUNE_CACHE") or os.path.join(os.path.expanduser("~"), ".cache", "rayramses_gb300")
    return os.path.join(root, "tuning.json")


class Batch:
    """Several bundles traced together; bundle i gets its own rr_ctx."""

    def __init__(self, bundles, fp64_dda: bool = False):
        _rr.load()
        self.descs = [_rr.bundle_desc(b, fp64_dda=fp64_dda) for b in bundles]
        self.handle = _rr.rr_batch_create(self.descs)
        self.n = len(self.descs)
        self.where = _rr.RR_AT_VERTICES if int(self.descs[0].interp) == _rr.RR_TRILINEAR else _rr.RR_AT_CENTRES

    def close(self):
        if getattr(self, "handle", None) is not None:
            _rr.rr_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def context(self, i):
        return _rr.rr_batch_context(self.handle, i)

    def reset(self, stream=None):
        _rr.rr_batch_reset(self.handle, stream)

    def clear(self, stream=None):
        _rr.rr_batch_clear(self.handle, stream)

    def stage(self, i, grid, rec, chi_a, chi_b, scale=1.0, a=1.0):
        _rr.rr_batch_set_step(self.handle, i, _rr.grid_desc(grid), rec, chi_a, chi_b, scale, a)

    def upload(self, stream=None):
        _rr.rr_batch_upload(self.handle, stream)

    def trace(self, stream=None):
        _rr.rr_batch_trace(self.handle, stream)

    def finalize(self, kappas, kborns=None, stream=None):
        _rr.rr_batch_finalize(self.handle, kappas, kborns, stream)

    def sync(self, stream=None):
        """(status code, total segments since reset)."""
        return _rr.rr_batch_sync_status(self.handle, stream)

    def set_tuning(self, wx, bwx, bwy, chunk=1, blocks_per_sm=0):
        _rr.rr_batch_set_tuning(self.handle, wx, bwx, bwy, chunk, blocks_per_sm)

    def tuning(self):
        return _rr.rr_batch_get_tuning(self.handle)

    def signature(self) -> str:
        import torch
        dev = torch.cuda.get_device_name()
        key = json.dumps([dev, [[d.nx, d.ny, d.interp, d.flags] for d in self.descs]])
        return hashlib.sha256(key.encode()).hexdigest()[:24]

    def autotune(self, reps: int = 3, stream=None, use_cache: bool = True):
        """Pick the launch shape with rr_batch_autotune (the step must be
        staged); remembered per device and bundle set in a JSON file."""
        path = _cache_path()
        sig = self.signature()
        cache = {}
        if use_cache and os.path.exists(path):
            try:
                with open(path) as f:
                    cache = json.load(f)
            except (OSError, ValueError):
                cache = {}
        if use_cache and sig in cache:
            t = cache[sig]["tuning"]
            self.set_tuning(*t)
            self.upload(stream)
            return tuple(t), cache[sig]["ms"], True
        ms = _rr.rr_batch_autotune(self.handle, reps, stream)
        t = self.tuning()
        cache[sig] = {"tuning": list(t), "ms": ms}
        try:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            with open(path + ".tmp", "w") as f:
                json.dump(cache, f, indent=1)
            os.replace(path + ".tmp", path)
        except OSError:
            pass
        return t, ms, False
