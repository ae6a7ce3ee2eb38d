"""Autotuner of the collide+stream launch shape of a batch of runs.

A launch shape is (threads per block, register-budget variant minb, tile width
tx): the batched collide+stream launch has one block size and one register
variant for all runs, and a tile width per run.  Candidates are timed on one
representative run per (nx, storage) class with the library's timing call
(``Turret.time_collide``), normalised to microseconds per million cells, and
cached in a JSON file keyed by device name and class, so a later batch on the
same device skips the timing.  The batch-wide (threads, minb) minimises the
cell-weighted sum over runs of each run's best time; each run then takes its
best tile width at that (threads, minb).  Tile choice never changes results.
"""
import json
import os
from collections import namedtuple

RunInfo = namedtuple("RunInfo", "nx storage cells handle")
Choice = namedtuple("Choice", "threads minb tx predicted_us table")

CANDIDATES = tuple((th, tx, mb) for th in (128, 256) for tx in (32, 64, 128) if tx <= th for mb in (2, 3))
CACHE_VERSION = 2  # 2: collide+stream on plane pairs (new register budgets)


def class_key(nx, storage):
    return "k1/nx=%d/%s" % (int(nx), storage)


def cand_key(threads, tx, minb):
    return "%d/%d/%d" % (threads, tx, minb)


def _load(path):
    if not path or not os.path.exists(path):
        return {"version": CACHE_VERSION, "devices": {}}
    with open(path) as f:
        data = json.load(f)
    if data.get("version") != CACHE_VERSION or not isinstance(data.get("devices"), dict):
        return {"version": CACHE_VERSION, "devices": {}}
    return data


def _save(path, data):
    if not path:
        return
    tmp = path + ".tmp%d" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tune(runs, timer, cache_path=None, device_name="gpu", candidates=None):
    """runs: RunInfo per run of the batch; timer(handle, threads, tx, minb) -> us
    of one launch over that run's window.  Returns a Choice."""
    if not runs:
        raise ValueError("no runs to tune")
    cands = tuple(candidates) if candidates else CANDIDATES
    data = _load(cache_path)
    table = data["devices"].setdefault(device_name, {})
    reps = {}
    for r in runs:
        reps.setdefault(class_key(r.nx, r.storage), r)
    timed = False
    for key, rep in reps.items():
        entry = table.setdefault(key, {})
        for th, tx, mb in cands:
            ck = cand_key(th, tx, mb)
            if ck not in entry:
                entry[ck] = float(timer(rep.handle, th, tx, mb)) * 1e6 / rep.cells
                timed = True
    if timed:
        _save(cache_path, data)
    shapes = sorted({(th, mb) for th, _, mb in cands})
    best = None
    for th, mb in shapes:
        total, txs = 0.0, []
        for r in runs:
            entry = table[class_key(r.nx, r.storage)]
            opts = [(entry[cand_key(th, tx, mb)], tx) for t2, tx, m2 in cands if t2 == th and m2 == mb]
            us, tx = min(opts)
            total += us * r.cells * 1e-6
            txs.append(tx)
        if best is None or total < best[0]:
            best = (total, th, mb, txs)
    total, th, mb, txs = best
    return Choice(th, mb, txs, total, {k: dict(table[k]) for k in reps})
