"""Tile-shape autotuner (Section 3.3 sweeps threads per block x items per thread).

Each operator is compiled for a few tile shapes (``crys_tile_variants``).  ``tune`` times
every variant of an operator on a caller-supplied launch (CUDA events, warm-up first,
median of several runs) and selects the fastest with ``crys_set_tile``; ``save`` / ``load``
persist the choice per device name as JSON so later processes start with it.  The choice
is stored as the tile shape, not the variant's index, so a library whose variant list
changed still finds it (or ignores it when that shape is no longer compiled).
"""
from __future__ import annotations

import json
import os
import statistics

import torch

from . import OP_NAMES, crys_get_tile, crys_set_tile, crys_tile_variants

DEFAULT_PATH = os.path.join(os.path.expanduser("~"), ".cache", "crystal_gb300_tiles.json")


def time_variant(launch, reps: int = 5, warmup: int = 2, stream=None) -> float:
    stream = stream or torch.cuda.current_stream()
    for _ in range(warmup):
        launch()
    ms = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        launch()
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
    return statistics.median(ms)


def tune(op: int, launch, reps: int = 5, warmup: int = 2) -> dict:
    """Times every tile variant of `op` on `launch()`; selects and returns the best."""
    results = {}
    for v, (threads, items) in enumerate(crys_tile_variants(op)):
        crys_set_tile(op, v)
        results[v] = {"threads": threads, "items": items, "ms": time_variant(launch, reps, warmup)}
    best = min(results, key=lambda v: results[v]["ms"])
    crys_set_tile(op, best)
    return {"op": OP_NAMES[op], "best": best, "variants": results}


def _key() -> str:
    return torch.cuda.get_device_name()


def save(path: str = DEFAULT_PATH) -> None:
    data = {}
    if os.path.exists(path):
        with open(path) as f:
            data = json.load(f)
    data[_key()] = {OP_NAMES[op]: list(crys_tile_variants(op)[crys_get_tile(op)]) for op in range(len(OP_NAMES))}
    os.makedirs(os.path.dirname(path), exist_ok=True)
    with open(path, "w") as f:
        json.dump(data, f, indent=1)


def load(path: str = DEFAULT_PATH) -> bool:
    """Applies the persisted choice for this device, if any.  A stored shape that is not
    among an operator's variants (or an entry in another form) is ignored."""
    if not os.path.exists(path):
        return False
    with open(path) as f:
        data = json.load(f).get(_key())
    if not data:
        return False
    for op, name in enumerate(OP_NAMES):
        shape = data.get(name)
        if not isinstance(shape, list) or len(shape) != 2:
            continue
        variants = [list(v) for v in crys_tile_variants(op)]
        if shape in variants:
            crys_set_tile(op, variants.index(shape))
    return True
