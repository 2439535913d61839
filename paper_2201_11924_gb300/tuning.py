"""Persistent cache of the batched form's launch choices (host side only).

``SimSenseBatch.tune()`` times each size class's stages for every candidate
launch choice (cost-ring depth of the path kernel, selection blocks per SM),
then whole batches in the per-class form and in every schedule of the fused
launch (pair order, lag, path-volume store policy), with CUDA events, and
keeps the fastest.  The choices depend on the GPU and on the shapes, not on
the pixels, so they can be kept between runs: this module stores them in a
JSON file, the per-class choices keyed by (GPU name, W, H, D, census window,
paths) and the schedule by the GPU and the batch's classes with their pair
counts, and applies stored choices to a new batch, so a server or benchmark
tunes once per GPU model and shape.  Writes go to a temporary file that
replaces the cache in one step, so a reader never sees a half-written file.
"""
from __future__ import annotations

import json
import os
import tempfile

VERSION = 2
# the launch choices the native autotuner picks from
PREFETCH = (8, 12, 16)
SELECT_BLOCKS = (1, 2)
SCHEDULE_SETS = {"fused": (0, 1), "prefetch": (16,), "keep_paths": (0, 1), "lag": (1, 2), "order": (0, 1, 2)}


def _valid(t) -> bool:
    try:
        return int(t["prefetch"]) in PREFETCH and int(t["select_blocks"]) in SELECT_BLOCKS
    except (KeyError, TypeError, ValueError):
        return False


def _valid_schedule(sc) -> bool:
    try:
        return set(sc) == set(SCHEDULE_SETS) and all(int(sc[k]) in v for k, v in SCHEDULE_SETS.items())
    except (KeyError, TypeError, ValueError):
        return False


def class_key(gpu: str, prm: dict) -> str:
    """Key of one size class: GPU name and the parameters the launch choice
    depends on (prm: the class's pair parameters, as SimSenseBatch.class_info
    returns them)."""
    win = int(prm["census_win"])
    w, h = win & 0xff, (win >> 8) & 0xff
    h = h or w
    return f"{gpu}|{int(prm['W'])}x{int(prm['H'])}|D{int(prm['D'])}|census{w}x{h}|paths{int(prm['paths'])}"


def batch_key(gpu: str, batch) -> str:
    """Key of a batch's schedule: the GPU and its classes with their pair
    counts, in a canonical order."""
    parts = []
    for c in range(batch.num_classes()):
        prm, n = batch.class_info(c)
        parts.append(f"{class_key('', prm)[1:]}x{int(n)}")
    return f"{gpu}|batch|" + "+".join(sorted(parts))


class TuningCache:
    """A JSON file of {key: {"prefetch": p, "select_blocks": s}} per class and
    {key: schedule} per batch."""

    def __init__(self, path: str):
        self.path = path
        self.entries: dict[str, dict] = {}
        self.schedules: dict[str, dict] = {}
        # an unreadable file, another version or an entry outside the
        # autotuner's choices counts as absent (and is rewritten on save)
        try:
            with open(path) as fh:
                data = json.load(fh)
        except (OSError, ValueError):
            data = {}
        if isinstance(data, dict) and data.get("version") == VERSION and isinstance(data.get("entries"), dict):
            self.entries = {k: {"prefetch": int(v["prefetch"]), "select_blocks": int(v["select_blocks"])}
                            for k, v in data["entries"].items() if _valid(v)}
            sch = data.get("schedules")
            if isinstance(sch, dict):
                self.schedules = {k: {kk: int(v[kk]) for kk in SCHEDULE_SETS}
                                  for k, v in sch.items() if isinstance(v, dict) and _valid_schedule(v)}

    def get(self, key: str):
        return self.entries.get(key)

    def put(self, key: str, tuning: dict):
        if not _valid(tuning):
            raise ValueError(f"not a launch choice of the autotuner: {tuning}")
        self.entries[key] = {"prefetch": int(tuning["prefetch"]), "select_blocks": int(tuning["select_blocks"])}

    def get_schedule(self, key: str):
        return self.schedules.get(key)

    def put_schedule(self, key: str, schedule: dict):
        if not _valid_schedule(schedule):
            raise ValueError(f"not a schedule of the autotuner: {schedule}")
        self.schedules[key] = {k: int(schedule[k]) for k in SCHEDULE_SETS}

    def save(self):
        d = os.path.dirname(os.path.abspath(self.path))
        fd, tmp = tempfile.mkstemp(prefix=".tuning-", suffix=".json", dir=d)
        try:
            with os.fdopen(fd, "w") as fh:
                json.dump({"version": VERSION, "entries": self.entries, "schedules": self.schedules}, fh, indent=1,
                          sort_keys=True)
            os.replace(tmp, self.path)
        except BaseException:
            if os.path.exists(tmp):
                os.unlink(tmp)
            raise


def _gpu_name(batch, gpu):
    if gpu is not None:
        return gpu
    import torch
    return torch.cuda.get_device_name(batch.device)


def store(batch, cache: TuningCache, gpu: str | None = None) -> int:
    """Records the current launch choice of every class of ``batch`` and its
    schedule (after its tune()); returns the number of classes stored."""
    gpu = _gpu_name(batch, gpu)
    n = batch.num_classes()
    for c in range(n):
        prm, _ = batch.class_info(c)
        cache.put(class_key(gpu, prm), batch.get_tuning(c))
    cache.put_schedule(batch_key(gpu, batch), batch.get_schedule())
    return n


def apply(batch, cache: TuningCache, gpu: str | None = None) -> list[int]:
    """Sets the stored launch choice on every class of ``batch`` that has one,
    and the stored schedule of a batch of the same classes; returns the
    classes left untuned (candidates for tune())."""
    gpu = _gpu_name(batch, gpu)
    missing = []
    for c in range(batch.num_classes()):
        prm, _ = batch.class_info(c)
        t = cache.get(class_key(gpu, prm))
        if t is None:
            missing.append(c)
        else:
            batch.set_tuning(c, t["prefetch"], t["select_blocks"])
    sc = cache.get_schedule(batch_key(gpu, batch))
    if sc is not None:
        batch.set_schedule(**sc)
    return missing
