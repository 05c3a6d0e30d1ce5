"""Cache of autotuned sweep tile shapes, keyed by workload class.

The fastest tile shape (cells per thread, warps per block, rows per work item, row
pipeline) of a batch depends on the device, the storage type, the kernel variant
(pulsating bodies or not), how many cells the batch holds and how wide its domains are
(a warp covers vec x 32 columns of a row, so narrow domains waste lanes at their east
ends and favour narrower tiles). Timing all candidates costs a few hundred sweep
launches, so the chosen shape is kept per workload class and reused when a batch of the
same class is tuned again, in this process or, when the cache has a path, in later ones.

Workload class of a batch (`workload_key`):
- device name and SM count,
- storage type and whether a resident domain has pulsating bodies,
- cells class: log2 of the resident cells, rounded to half octaves,
- width classes: the octaves of the domain width (floor(log2 nx)) that hold at least a
  quarter of the resident cells, in increasing order.

The JSON file maps each key to {"tile": [vec, warps, rows, pipeline], "us": best time per
sweep launch}; it is written whole to a temporary file and renamed over the old one, so a
reader never sees a partial file (concurrent writers may drop each other's new entries,
which only costs a retune).
"""
from __future__ import annotations

import json
import math
import os
import tempfile


def workload_key(device: str, sms: int, storage: str, deform: bool, domains) -> str:
    """The class of a batch; `domains` is an iterable of (nx, ny) of its resident domains."""
    dims = [(int(nx), int(ny)) for nx, ny in domains]
    cells = sum(nx * ny for nx, ny in dims)
    if cells == 0:
        return f"{device}|{sms}|{storage}|{int(bool(deform))}|empty"
    per_octave = {}
    for nx, ny in dims:
        o = int(math.floor(math.log2(nx)))
        per_octave[o] = per_octave.get(o, 0) + nx * ny
    widths = sorted(o for o, c in per_octave.items() if 4 * c >= cells)
    cells_class = round(2.0 * math.log2(cells)) / 2.0
    return (f"{device}|{sms}|{storage}|{int(bool(deform))}|c{cells_class:g}|"
            f"w{'.'.join(str(o) for o in widths)}")


class TuneCache:
    """Tile shapes by workload key; in memory, and in a JSON file when `path` is given."""

    def __init__(self, path: str | None = None):
        self.path = path
        self.entries = {}
        self.hits = 0
        self.misses = 0
        if path and os.path.exists(path):
            with open(path) as f:
                data = json.load(f)
            for k, v in data.items():
                tile = v.get("tile")
                if isinstance(tile, list) and len(tile) == 4:
                    self.entries[k] = {"tile": [int(t) for t in tile], "us": float(v.get("us", 0.0))}

    def get(self, key: str):
        """(tile, us) for the key, or None."""
        e = self.entries.get(key)
        if e is None:
            self.misses += 1
            return None
        self.hits += 1
        return tuple(e["tile"]), e["us"]

    def put(self, key: str, tile, us: float):
        self.entries[key] = {"tile": [int(t) for t in tile], "us": float(us)}
        self.save()

    def save(self):
        if not self.path:
            return
        d = os.path.dirname(os.path.abspath(self.path))
        os.makedirs(d, exist_ok=True)
        fd, tmp = tempfile.mkstemp(prefix=".tune-", suffix=".json", dir=d)
        try:
            with os.fdopen(fd, "w") as f:
                json.dump(self.entries, f, indent=1, sort_keys=True)
            os.replace(tmp, self.path)
        except BaseException:
            if os.path.exists(tmp):
                os.unlink(tmp)
            raise


def cached_autotune(cache, key, tune, set_tile, get_tile) -> float:
    """Tune through the cache: a shape already stored for `key` is set by `set_tile`
    without timing and its stored time returned; otherwise `tune()` times the candidates
    (returning the best time) and the shape it kept (`get_tile()`) is stored."""
    hit = cache.get(key)
    if hit is not None:
        set_tile(*hit[0])
        return hit[1]
    us = tune()
    cache.put(key, get_tile(), us)
    return us
