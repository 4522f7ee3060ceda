"""Autotuner for the window size and the number of worker CTAs.

Runs a workload once per candidate (window, CTA slots), keeps the median
device time of a few repeats, and caches the best choice as JSON keyed by the
workload's description and the GPU name. The candidates are the ones the paper
varies (window 16 / 32, Sec. VI-D) widened to {8, 16, 32, 64}, and CTA-slot
counts in multiples of the SM count, capped at what can be co-resident.
"""
from __future__ import annotations

import hashlib
import json
import os
import statistics
from typing import Callable, Dict, Iterable, Optional

import torch

from . import acs, harness

DEFAULT_WINDOWS = (8, 16, 32, 64)
DEFAULT_SLOTS = (64, 148, 296, 444, 592, 740, 888, 1036, 1184)


def cache_path() -> str:
    base = os.environ.get("ACS_AUTOTUNE_CACHE")
    if base:
        return base
    root = os.environ.get("XDG_CACHE_HOME", os.path.join(os.path.expanduser("~"), ".cache"))
    return os.path.join(root, "acs", "autotune.json")


def cache_key(workload: str) -> str:
    gpu = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
    return hashlib.sha1(f"{workload}|{gpu}".encode()).hexdigest()[:16] + "|" + gpu


def load_cache(path: Optional[str] = None) -> Dict[str, dict]:
    path = path or cache_path()
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, json.JSONDecodeError):
        return {}


def save_cache(entries: Dict[str, dict], path: Optional[str] = None) -> None:
    path = path or cache_path()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(entries, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def max_worker_slots(window: int, n_streams: int) -> int:
    """Worker CTAs that fit beside n_streams scheduler CTAs (all co-resident)."""
    with harness.Context(window, n_streams=n_streams) as ctx:
        return ctx.stats()["cta_slots"]


def tune(workload: str, make_run: Callable[[harness.Context], Callable[[], int]], n_streams: int,
         windows: Iterable[int] = DEFAULT_WINDOWS, slots: Iterable[int] = DEFAULT_SLOTS, repeats: int = 5,
         warmup: int = 1, use_cache: bool = True, path: Optional[str] = None, capacity: int = 1 << 13) -> dict:
    """Pick (window, cta_slots) minimising the median device time of a run.

    ``make_run(ctx)`` prepares the workload on a context and returns a
    function that performs one complete run (flush + sync) and returns the
    number of tasks it ran. Returns {"window", "cta_slots", "ms", "table"}.
    """
    key = cache_key(workload)
    cache = load_cache(path) if use_cache else {}
    if use_cache and key in cache:
        return dict(cache[key], cached=True)
    table = []
    best = None
    for W in windows:
        cap = max_worker_slots(W, n_streams)
        for sl in sorted({min(s, cap) for s in slots}):
            with harness.Context(W, n_streams=n_streams, cta_slots=sl, timing=True, capacity=capacity) as ctx:
                run = make_run(ctx)
                for _ in range(warmup):
                    run()
                times = []
                for _ in range(repeats):
                    before = ctx.stats()["kernel_ms"]
                    tasks = run()
                    times.append(ctx.stats()["kernel_ms"] - before)
            ms = statistics.median(times)
            table.append({"window": W, "cta_slots": sl, "ms": ms, "tasks": tasks})
            if best is None or ms < best["ms"]:
                best = {"window": W, "cta_slots": sl, "ms": ms}
    out = dict(best, table=table, workload=workload)
    if use_cache:
        cache[key] = out
        save_cache(cache, path)
    return out
