"""Cache of measured stencil tile shapes (irls_plan_autotune results) in a JSON file.

One entry per (H, W, precision, system, GPU name): the chosen image rows per block of the CG
direction and update kernels and the times that chose them.  Plain file handling, no device
work: a missing or unreadable file is an empty cache, and entries that name a row count the
kernels are not built for are ignored.
"""
from __future__ import annotations

import json
import os
import tempfile

TILE_ROWS = (8, 16, 24, 32)


def tuning_key(H, W, precision, system, gpu):
    return f"{int(H)}x{int(W)}/prec{int(precision)}/sys{int(system)}/{gpu}"


def batch_key(shapes, precision, system, gpu):
    """Key of a batch: its image shapes in order (a digest), their count, precision, system, GPU."""
    import hashlib
    h = hashlib.sha1(";".join(f"{int(a)}x{int(b)}" for a, b in shapes).encode()).hexdigest()[:16]
    return f"batch{len(shapes)}-{h}/prec{int(precision)}/sys{int(system)}/{gpu}"


def _load(path):
    try:
        with open(path) as f:
            data = json.load(f)
    except (OSError, ValueError):
        return {}
    return data if isinstance(data, dict) else {}


def cache_get(path, key):
    """(dir_rows, upd_rows) stored under `key`, or None."""
    e = _load(path).get(key)
    if not isinstance(e, dict):
        return None
    tiles = e.get("tiles")
    if (not isinstance(tiles, list) or len(tiles) != 2
            or any(t not in TILE_ROWS for t in tiles)):
        return None
    return int(tiles[0]), int(tiles[1])


def cache_put(path, key, tiles, ms=None):
    """Stores `tiles` (and the timings that chose them) under `key`; the file is replaced
    atomically, other keys are kept."""
    if len(tiles) != 2 or any(int(t) not in TILE_ROWS for t in tiles):
        raise ValueError(f"tile rows must be two of {TILE_ROWS}")
    data = _load(path)
    entry = {"tiles": [int(t) for t in tiles]}
    if ms is not None:
        entry["ms"] = {"direction": [float(x) for x in ms[:4]],
                       "update": [float(x) for x in ms[4:8]], "rows": list(TILE_ROWS)}
    data[key] = entry
    d = os.path.dirname(os.path.abspath(path))
    os.makedirs(d, exist_ok=True)
    fd, tmp = tempfile.mkstemp(dir=d, suffix=".tmp")
    try:
        with os.fdopen(fd, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except BaseException:
        if os.path.exists(tmp):
            os.unlink(tmp)
        raise
