"""Persistent cache of tuned schedules: checkpoint and resume of the search.

nk_tune times candidate schedules on the GPU, and a search over a network's
layers times thousands of them.  This cache keeps each problem's result in
a JSON file, so that a later process -- or the same job after a restart --
reuses it instead of timing again.  tune_cached() is nk_tune behind the
cache.

An entry is tagged with a fingerprint of the library's sources (the CUDA
sources and public headers) and with the device (name, compute capability,
SM count).  A rebuild that changes a kernel or its schedule space, or a
different GPU, makes the entry stale, because the ranking of schedules may
no longer hold.  Before use, a stored schedule is checked again against
the problem's current schedule space.  For the cost-model search the key
also holds a digest of the model parameters.

Writes go to a temporary file in the same directory, which then replaces
the cache file.  Another process's entries are merged in rather than
overwritten.  A missing, corrupt or foreign file reads as an empty cache.
The file lives at $NK_CACHE_DIR/schedules.json, by default
~/.cache/nk/schedules.json.
"""
from __future__ import annotations

import hashlib
import json
import os
import tempfile

from . import nk_tune as nt

FORMAT = 1
_FIELDS = [f for f, _ in nt.nk_problem._fields_]


def source_fingerprint() -> str:
    """Digest of the sources that define the kernels and the schedule space."""
    pkg = os.path.dirname(os.path.abspath(__file__))
    h = hashlib.sha256()
    for d in (os.path.join(pkg, "csrc"), os.path.join(os.path.dirname(pkg), "include")):
        for name in sorted(os.listdir(d)):
            if name.endswith((".cu", ".cuh", ".h")):
                h.update(name.encode())
                with open(os.path.join(d, name), "rb") as f:
                    h.update(f.read())
    return h.hexdigest()[:16]


def device_id() -> str:
    """Name, compute capability and SM count of the current GPU."""
    import torch
    from . import nk
    sms, major, minor = nk.nk_device_info()
    return f"{torch.cuda.get_device_name()}|sm_{major}{minor}|{sms}"


def default_path() -> str:
    base = os.environ.get("NK_CACHE_DIR") or os.path.join(os.path.expanduser("~"), ".cache", "nk")
    return os.path.join(base, "schedules.json")


def _params_digest(params) -> str:
    if params is None:
        return ""
    data = params.detach().float().cpu().numpy().tobytes() if hasattr(params, "detach") else bytes(params)
    return hashlib.sha256(data).hexdigest()[:16]


class ScheduleCache:
    def __init__(self, path: str | None = None, device: str | None = None, fingerprint: str | None = None):
        self.path = path or default_path()
        self._device = device
        self._fingerprint = fingerprint
        self._entries = self._read()

    @property
    def device(self) -> str:
        if self._device is None:
            self._device = device_id()
        return self._device

    @property
    def fingerprint(self) -> str:
        if self._fingerprint is None:
            self._fingerprint = source_fingerprint()
        return self._fingerprint

    def _read(self) -> dict:
        try:
            with open(self.path) as f:
                doc = json.load(f)
        except (OSError, ValueError):
            return {}
        if not isinstance(doc, dict) or doc.get("format") != FORMAT or not isinstance(doc.get("entries"), dict):
            return {}
        return doc["entries"]

    @staticmethod
    def key(p, mode: int, topk: int, params=None) -> str:
        prob = ",".join(f"{f}={int(getattr(p, f))}" for f in _FIELDS)
        k = f"{prob}|mode={int(mode)}"
        if mode != nt.NK_TUNE_EXHAUSTIVE:
            k += f"|topk={int(topk)}"
        if mode == nt.NK_TUNE_MODEL_TOPK:
            k += f"|model={_params_digest(params)}"
        return k

    def get(self, p, mode: int = nt.NK_TUNE_EXHAUSTIVE, topk: int = 5, params=None):
        """The stored schedule for this problem and search, or None."""
        e = self._entries.get(self.key(p, mode, topk, params))
        if not isinstance(e, dict):
            return None
        if e.get("fingerprint") != self.fingerprint or e.get("device") != self.device:
            return None
        try:
            s = tuple(int(v) for v in e["schedule"])
        except (KeyError, TypeError, ValueError):
            return None
        if len(s) != 6 or s not in nt.nk_enumerate_schedules(p):
            return None
        return s

    def put(self, p, mode: int, topk: int, schedule, best_ms: float | None = None, params=None):
        self._entries[self.key(p, mode, topk, params)] = {
            "schedule": [int(v) for v in schedule], "best_ms": best_ms,
            "fingerprint": self.fingerprint, "device": self.device}
        self._write()

    def _write(self):
        merged = self._read()          # keep entries another process wrote meanwhile
        merged.update(self._entries)
        self._entries = merged
        d = os.path.dirname(os.path.abspath(self.path))
        os.makedirs(d, exist_ok=True)
        fd, tmp = tempfile.mkstemp(prefix=".schedules.", dir=d)
        try:
            with os.fdopen(fd, "w") as f:
                json.dump({"format": FORMAT, "entries": merged}, f, indent=1, sort_keys=True)
            os.replace(tmp, self.path)
        except BaseException:
            if os.path.exists(tmp):
                os.unlink(tmp)
            raise

    def __len__(self) -> int:
        return len(self._entries)


def tune_cached(p, mode: int = nt.NK_TUNE_EXHAUSTIVE, topk: int = 5, params=None, reps: int = 5,
                cache: ScheduleCache | None = None, stream=None):
    """nk_tune behind the cache: (schedule, report), report None on a hit."""
    cache = ScheduleCache() if cache is None else cache
    s = cache.get(p, mode, topk, params)
    if s is not None:
        return s, None
    best, rep = nt.nk_tune(p, mode, topk, params, reps, stream)
    cache.put(p, mode, topk, best, float(rep.best_ms), params)
    return best, rep
