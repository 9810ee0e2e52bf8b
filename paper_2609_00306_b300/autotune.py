"""Autotuner for batched decompositions.

Chooses, per basis-size class, the speculative block size b (the number of
ERI columns computed and updated together) and, for the stream batch, the
number of concurrent host workers/streams, by timing the library on
representative synthetic systems; :func:`tune_persistent` chooses b per class
for the one-launch persistent batch (b <= 64) the same way.  The result is
cached as JSON next to this file (`tuning.json`) and applied by
:func:`blocks_for`.
"""
from __future__ import annotations

import json
import os
import time
from typing import Dict, List, Sequence

HERE = os.path.dirname(os.path.abspath(__file__))
CACHE = os.path.join(HERE, "tuning.json")
CLASSES = [(0, 200), (200, 400), (400, 100000)]   # basis-size classes [lo, hi)
BLOCKS = (16, 32, 64, 128)
PERSISTENT_BLOCKS = (32, 48, 64)
WORKERS = (4, 8, 16)


def _cls(n: int) -> str:
    for lo, hi in CLASSES:
        if lo <= n < hi:
            return f"{lo}-{hi}"
    return f"{CLASSES[-1][0]}-{CLASSES[-1][1]}"


def load() -> Dict:
    try:
        with open(CACHE) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def blocks_for(systems: Sequence, table: Dict = None, key: str = "blocks") -> List[int]:
    """Block size per system from the tuning table (0 = library default);
    key "persistent_blocks" for the persistent batch."""
    table = table if table is not None else load()
    bl = table.get(key, {})
    return [int(bl.get(_cls(s.n_basis), 0)) for s in systems]


def tune_persistent(systems: Sequence, write: bool = True) -> Dict:
    """Block size b per basis-size class for cd_batch_persistent: each class's
    middle systems (up to 4) are run as one persistent batch per candidate b
    and the fastest b is kept."""
    import torch
    from . import cderi as cd
    table = load()
    table.setdefault("timings", {})
    table["persistent_blocks"] = {}
    by_cls: Dict[str, list] = {}
    for s in systems:
        by_cls.setdefault(_cls(s.n_basis), []).append(s)
    for c, group in by_cls.items():
        g = sorted(group, key=lambda s: s.n_basis)
        sample = g[max(0, len(g) // 2 - 2):len(g) // 2 + 2]
        best, best_t = 64, float("inf")
        for b in PERSISTENT_BLOCKS:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            cd.batch_persistent(sample, blocks=[b] * len(sample))
            torch.cuda.synchronize()
            t = time.perf_counter() - t0
            table["timings"][f"persistent/{c}/b{b}"] = t
            if t < best_t:
                best, best_t = b, t
        table["persistent_blocks"][c] = best
    if write:
        with open(CACHE, "w") as fh:
            json.dump(table, fh, indent=1)
    return table


def tune(systems: Sequence, repeats: int = 1, write: bool = True) -> Dict:
    """Time candidate block sizes per class and worker counts for the batch."""
    import torch
    from . import cderi as cd
    by_cls: Dict[str, list] = {}
    for s in systems:
        by_cls.setdefault(_cls(s.n_basis), []).append(s)
    table = {"blocks": {}, "timings": {}}
    for c, group in by_cls.items():
        sample = sorted(group, key=lambda s: s.n_basis)[len(group) // 2:len(group) // 2 + 2]
        best, best_t = 0, float("inf")
        for b in BLOCKS:
            t0 = time.perf_counter()
            for _ in range(repeats):
                for s in sample:
                    f = cd.cd_eri_factor(s.basis, s.tau, s.schwarz, block=b)
                    f.free()
            torch.cuda.synchronize()
            t = time.perf_counter() - t0
            table["timings"][f"{c}/b{b}"] = t
            if t < best_t:
                best, best_t = b, t
        table["blocks"][c] = best
    blocks = blocks_for(systems, table)
    best_w, best_t = 8, float("inf")
    sub = list(systems)[:16]
    for w in WORKERS:
        t0 = time.perf_counter()
        cd.batch_run(sub, workers=w, blocks=blocks[:len(sub)])
        t = time.perf_counter() - t0
        table["timings"][f"workers{w}"] = t
        if t < best_t:
            best_w, best_t = w, t
    table["workers"] = best_w
    if write:
        with open(CACHE, "w") as fh:
            json.dump(table, fh, indent=1)
    return table
