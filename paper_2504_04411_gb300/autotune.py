"""Autotuner for the gather: picks the traversal (ppm_params.mapping) and the
grid cell factor by timing the candidates on the problem itself.

Results do not depend on either choice (the tests check that); only the
time does.  Timings are cached per size class -- hit points, photons per
iteration and initial radius, each on a log2 scale -- in a JSON file, so a
class is measured once per machine.

* ``tune`` times one problem (a context per candidate, a warm-up iteration,
  then the gather of the next ones, CUDA events on the current stream);
* ``tune_batch`` times every candidate on the whole batch (one persistent
  launch hides the small problems' latency behind the large ones, so
  per-problem timings would mislead), then the tile sizes of the persistent
  gather for the best one.
"""
from __future__ import annotations

import json
import math
import os

import torch

from . import ppm

# Cell factors 2/k (0.5, 2/3, 1) make a sphere of the largest radius span
# the same number of cells along each axis for nearly every hit point (2 r / h
# just above an integer), so the threads of a warp walk boxes of one size;
# 0.6 and 0.75 trade that for fewer or larger cells.
CANDIDATES = ((0, 0.5), (0, 0.6), (0, 2.0 / 3.0), (0, 0.75), (0, 1.0), (1, 0.5), (1, 1.0), (4, 0.5),
              (4, 1.0))
TILES = (64, 128, 256)       # batch tile sizes (hit points), tried for the best traversal
DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")


def supported(mapping: int, params) -> bool:
    """Traversal 3 tests one channel and traversal 4 gathers one flux
    channel (the library refuses the other combinations)."""
    if params is None:
        return True
    if mapping == 3 and params.rgb_test:
        return False
    if mapping == 4 and params.channels == 3:
        return False
    return True


def size_class(nh: int, J: int, r0: float) -> str:
    return f"h{round(math.log2(max(nh, 1)))}-j{round(math.log2(max(J, 2)))}-r{round(4 * math.log2(r0))}"


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(path, data):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def time_config(hp, batches, r0: float, mapping: int, cell_factor: float, params=None) -> float:
    """Mean gather time in ms over batches[1:] (batches[0] warms up)."""
    p = ppm.ppm_default_params() if params is None else params
    p.mapping, p.cell_factor = mapping, cell_factor
    est = ppm.Estimator(hp, r0, 0.75, p)
    est.step(batches[0])
    stream = torch.cuda.current_stream()
    times = []
    for ph in batches[1:]:
        ppm.ppm_build_grid(est.ctx, ph.pos, ph.flux, ph.pos.shape[0], nq=ph.nq,
                           rho=ph.rho if p.vcm else None, wq=ph.wq if p.vcm else None)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        est.it += 1
        a.record(stream)
        ppm.ppm_gather_test_update(est.ctx, est.it)
        b.record(stream)
        b.synchronize()
        times.append(a.elapsed_time(b))
    est.close()
    return sum(times) / len(times)


def tune(hp, batches, r0: float, key: str | None = None, cache: str | None = DEFAULT_CACHE,
         candidates=CANDIDATES, params=None) -> dict:
    """Best (mapping, cell_factor) for one problem; batches: >= 2 photon
    batches of the problem."""
    key = key or size_class(int(hp.pos.shape[0]), int(batches[0].pos.shape[0]), r0)
    data = _load(cache) if cache else {}
    ent = data.get(key)
    if ent is None:
        times = {f"{m},{cf}": time_config(hp, batches, r0, m, cf, params) for m, cf in candidates
                 if supported(m, params)}
        best = min(times, key=times.get)
        m, cf = best.split(",")
        ent = {"mapping": int(m), "cell_factor": float(cf), "ms": times}
        if cache:
            data = _load(cache)
            data[key] = ent
            _store(cache, data)
    return dict(ent, key=key)


def _time_batch(scenes, hps, photon_lists, mapping, cf, tile) -> float:
    p = ppm.ppm_default_params()
    p.mapping, p.tile = mapping, tile
    b = ppm.Batch(hps, [s.r0 for s in scenes], [s.J for s in scenes], params=p,
                  cell_factors=[cf] * len(scenes))
    b.step(photon_lists[0])
    ms = []
    for it in photon_lists[1:]:
        b.step(it)
        ms.append(b.stats()[0].gather_ms)
    b.close()
    return sum(ms) / len(ms)


def tune_batch(scenes, hps, photon_lists, cache: str | None = DEFAULT_CACHE,
               candidates=CANDIDATES, tiles=TILES) -> dict:
    """Traversal and cell factor of a batch, timed on the batch itself.

    In one persistent launch the small problems' latencies hide behind the
    large ones, so per-problem timings mislead: every candidate runs the
    whole batch (a warm-up iteration, then the gather of one more,
    measured by the events the batch records around its gather launch).
    scenes: objects with nh, J, r0; hps: their hit points; photon_lists:
    >= 2 iterations, each a list with one photon batch per problem.
    Returns {"mapping": m, "cell_factors": [...], "tile": t, "ms": {...},
    "key": ...}."""
    key = "batch-" + "-".join(size_class(s.nh, s.J, s.r0) for s in scenes[:4]) + f"-n{len(scenes)}"
    data = _load(cache) if cache else {}
    ent = data.get(key)
    if ent is None:
        times = {f"{m},{cf},{tiles[0]}": _time_batch(scenes, hps, photon_lists, m, cf, tiles[0])
                 for m, cf in candidates}
        best = min(times, key=times.get)
        m, cf, _ = best.split(",")
        for t in tiles[1:]:
            times[f"{m},{cf},{t}"] = _time_batch(scenes, hps, photon_lists, int(m), float(cf), t)
        best = min(times, key=times.get)
        m, cf, t = best.split(",")
        ent = {"mapping": int(m), "cell_factor": float(cf), "tile": int(t), "ms": times}
        if cache:
            data = _load(cache)
            data[key] = ent
            _store(cache, data)
    return {"mapping": ent["mapping"], "cell_factors": [ent["cell_factor"]] * len(scenes),
            "tile": ent.get("tile", 64), "ms": ent["ms"], "key": key}
