"""Autotuner for the library's execution parameters.

It times candidate launch shapes on the caller's workload and keeps the fastest.
Only parameters that leave every result unchanged are tuned: tiles per CTA of the
propagation kernel, from which level spacing on the random search runs as a
kernel of its own, from which spacing on the propagation runs one CTA per tile
(and with how many threads per candidate), and the launch layout: flows on one or
several streams, the kd trees of all flows in one launch chain, one persistent
launch per level. The tile edge T of the parallel
schedule is part of the method's definition and stays as given. The search is
coordinate-wise, one parameter at a time in the order of CANDIDATES. Choices are cached in a small JSON file
keyed by GPU name, image sizes and method parameters.
"""
from __future__ import annotations

import json
import os

import torch

from . import ffapi, synth

CANDIDATES = dict(wide_min_n=(0, 1, 2, 4, 8), split8_min_n=(0, 1, 2, 4, 8), split2_max_n=(0, 1, 2),
                  pass_warps=(1, 2, 4, 8), rs_min_n=(0, 1, 2, 4, 8), serial_flows=(0, 1),
                  kd_merge=(0, 1), persist_levels=(0, 1))
_CACHE = os.environ.get("FF_TUNE_CACHE",
                        os.path.join(os.path.expanduser("~"), ".cache", "flowfields_tune.json"))


def _key(sizes, params):
    gpu = torch.cuda.get_device_name() if torch.cuda.is_available() else "none"
    p = ffapi._params(params).as_dict()
    sz = ",".join(f"{w}x{h}" for w, h in sorted(set(map(tuple, sizes))))
    return f"{gpu}|{sz}|n{len(sizes)}|" + ",".join(f"{k}={p[k]}" for k in sorted(p))


def _load():
    try:
        with open(_CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(db):
    try:
        os.makedirs(os.path.dirname(_CACHE), exist_ok=True)
        with open(_CACHE + ".tmp", "w") as f:
            json.dump(db, f, indent=1, sort_keys=True)
        os.replace(_CACHE + ".tmp", _CACHE)
    except OSError:
        pass


def time_batch(batch, frames, reps=3):
    """Median device time (ms) of one batch run."""
    batch.run(frames)
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        batch.run(frames)
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return sorted(ts)[len(ts) // 2]


def tune(sizes, params=None, frames=None, reps=3, use_cache=True, seed=0):
    """Pick the fastest execution parameters for pairs of the given sizes.

    frames: optional list of (I1, I2) CUDA tensors; synthetic pairs otherwise.
    Returns dict(choice=..., timings={setting: ms}, cached=bool) and applies the
    choice with ffapi.set_exec_params.
    """
    key = _key(sizes, params)
    db = _load() if use_cache else {}
    if use_cache and key in db:
        ffapi.set_exec_params(**db[key]["choice"])
        return dict(db[key], cached=True)
    if frames is None:
        frames = []
        for i, (W, H) in enumerate(sizes):
            p = synth.pair_shift(seed + i, W=W, H=H,
                                 max_shift=(max(1, W // 8), max(1, H // 8)))
            frames.append((torch.from_numpy(p["I1"]).cuda(), torch.from_numpy(p["I2"]).cuda()))
    batch = ffapi.FlowFieldsBatch(sizes, params)
    before = ffapi.get_exec_params()
    timings = {}
    choice = dict(pass_warps=4, rs_min_n=0, wide_min_n=1, split8_min_n=0, serial_flows=0,
                  kd_merge=0, persist_levels=0, split2_max_n=0)
    best_t = None
    for name in CANDIDATES:  # one parameter at a time
        for v in CANDIDATES[name]:
            trial = dict(choice, **{name: v})
            tk = ",".join(f"{k}={trial[k]}" for k in sorted(trial))
            if tk not in timings:
                ffapi.set_exec_params(**trial)
                timings[tk] = time_batch(batch, frames, reps)
            if best_t is None or timings[tk] < best_t:
                choice, best_t = trial, timings[tk]
    ffapi.set_exec_params(**choice)
    rec = dict(choice=choice, timings=timings, before=before)
    if use_cache:
        db[key] = rec
        _store(db)
    return dict(rec, cached=False)
