"""Multislice autotuning with a JSON cache.

``best_multislice_config(grid)`` returns how many snapshots one multislice
call should advance together on this GPU for this grid, and which variants of
the passes to use (tacaw_multislice flags: for 512-point rows two warps per
row or one, for 512-point columns the persistent TMA-staged pass or one block
per column block; on square grids also the work-queue multislice, all slices
in one persistent launch); candidates whose potentials would exceed MAX_TUNING_BYTES
are skipped.  On a cache miss it times every (batch, flags) pair with the
library's ``tacaw_tune_multislice`` (random slice potentials: the transform
cost does not depend on the values) and stores the result under the key
"<device name>|<nx>x<ny>x<n_slices>".  ``best_multislice_batch`` returns the
batch alone.

The cache file is ``$TACAW_TUNE_CACHE`` when set, else
``~/.cache/tacaw/tune.json``.  Entries hold the batch, the variant and the
measured milliseconds per snapshot of every candidate; entries written before
the variant was tuned are tuned again.
"""

from __future__ import annotations

import ctypes
import json
import os
import tempfile

import torch

from . import _lib as L

DEFAULT_CANDIDATES = (8, 16, 32, 64, 128, 256, 512)
MAX_TUNING_BYTES = 64 << 30         # potentials allocated for the largest candidate (HBM: 288 GB)


def cache_path() -> str:
    return os.environ.get("TACAW_TUNE_CACHE") or os.path.join(os.path.expanduser("~"), ".cache", "tacaw",
                                                               "tune.json")


def load_cache(path=None) -> dict:
    try:
        with open(path or cache_path()) as f:
            data = json.load(f)
        return data if isinstance(data, dict) else {}
    except (OSError, ValueError):
        return {}


def store_cache(entries: dict, path=None) -> None:
    """Merge entries into the cache file (written atomically)."""
    path = path or cache_path()
    data = load_cache(path)
    data.update(entries)
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    fd, tmp = tempfile.mkstemp(dir=os.path.dirname(os.path.abspath(path)), suffix=".tmp")
    with os.fdopen(fd, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def cache_key(grid, device_name: str) -> str:
    return f"{device_name}|{int(grid.nx)}x{int(grid.ny)}x{int(grid.n_slices)}"


CACHE_VERSION = 4


def multislice_variants(grid):
    """tacaw_multislice flags worth comparing for this grid: the variants of the
    per-slice passes, and on square grids the work-queue multislice."""
    rows = (0, L.TACAW_MS_WARP_ROWS) if int(grid.nx) == 512 else (0,)
    cols = (0, L.TACAW_MS_BLOCK_COLS) if int(grid.ny) == 512 else (0,)
    queue = (L.TACAW_MS_QUEUE,) if int(grid.nx) == int(grid.ny) else ()
    return tuple(r | c for r in rows for c in cols) + queue


def measure_multislice_batches(grid, candidates=DEFAULT_CANDIDATES, reps=3, device="cuda", flags=0):
    """Time every candidate batch on this device with the given tacaw_multislice
    flags: ({batch: ms per snapshot}, best batch)."""
    lib = L.load()
    dev = torch.device(device)
    per_snapshot = 4 * int(grid.n_slices) * int(grid.ny) * int(grid.nx)
    cap = max(1, MAX_TUNING_BYTES // per_snapshot)
    cand = sorted({int(c) for c in candidates if 1 <= int(c) <= cap}) or [min(int(c) for c in candidates)]
    top = max(cand)
    gen = torch.Generator(device=dev).manual_seed(0)
    V = torch.rand((top, grid.n_slices, grid.ny, grid.nx), generator=gen, device=dev) * 30.0
    psi = torch.empty((top, grid.ny, grid.nx), dtype=torch.complex64, device=dev)
    g = L.make_grid(grid)
    c_arr = (ctypes.c_int32 * len(cand))(*cand)
    ms = (ctypes.c_float * len(cand))()
    best = ctypes.c_int32(0)
    stream = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)

    def call(ws, nbytes):
        return lib.tacaw_tune_multislice(ctypes.byref(g), top, ctypes.c_void_p(V.data_ptr()),
                                         ctypes.c_void_p(psi.data_ptr()), c_arr, len(cand), int(reps), int(flags),
                                         ms, ctypes.byref(best), ws, nbytes, stream)

    nbytes = ctypes.c_size_t(0)
    L.check("tacaw_tune_multislice", call(ctypes.c_void_p(0), ctypes.byref(nbytes)))
    ws = torch.empty(max(nbytes.value, 256), dtype=torch.uint8, device=dev)
    nbytes = ctypes.c_size_t(ws.numel())
    L.check("tacaw_tune_multislice", call(ctypes.c_void_p(ws.data_ptr()), ctypes.byref(nbytes)))
    return {c: float(m) for c, m in zip(cand, ms)}, int(best.value)


def best_multislice_config(grid, candidates=DEFAULT_CANDIDATES, device="cuda", path=None, measure=None):
    """Cached best (batch, tacaw_multislice flags) for this grid on this device (tuned on a
    miss).  ``measure(grid, candidates, device=..., flags=...)`` replaces the
    timing function (tests)."""
    dev = torch.device(device)
    name = torch.cuda.get_device_name(dev) if measure is None else "test-device"
    key = cache_key(grid, name)
    entry = load_cache(path).get(key)
    if entry and int(entry.get("version", 0)) == CACHE_VERSION and int(entry.get("batch", 0)) >= 1:
        return int(entry["batch"]), int(entry.get("flags", 0))
    best = None
    timings = {}
    for flags in multislice_variants(grid):
        t, b = (measure or measure_multislice_batches)(grid, candidates, device=device, flags=flags)
        timings[str(flags)] = {str(k): v for k, v in t.items()}
        if best is None or t[b] < best[0]:
            best = (t[b], b, flags)
    _, batch, flags = best
    store_cache({key: {"version": CACHE_VERSION, "batch": int(batch), "flags": int(flags),
                       "ms_per_snapshot": timings}}, path)
    return int(batch), int(flags)


def best_multislice_batch(grid, candidates=DEFAULT_CANDIDATES, device="cuda", path=None, measure=None):
    """Cached best snapshot batch for this grid on this device (tuned on a miss)."""
    return best_multislice_config(grid, candidates, device=device, path=path, measure=measure)[0]
