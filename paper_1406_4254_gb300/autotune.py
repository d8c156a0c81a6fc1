"""Autotuner for the launch shape of batched SCF (etics_scf_batch).

Times every candidate :class:`~paper_1406_4254_gb300.etics.BatchTuning`
(particles per coefficient tile, coefficient blocks per SM, field threads per
block, particles per field work item) on a given batch with CUDA events and
records the fastest in a JSON table keyed by the batch's largest n_max, largest
l_max and total-N bucket (log2).  :func:`lookup` reads the table back.

    python -m paper_1406_4254_gb300.autotune      # tunes the 256-system ensemble
"""
from __future__ import annotations

import itertools
import json
import math
import os
import statistics

import torch

from . import etics

TABLE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "autotune.json")

# tiles: 64 serves both precisions; mixed-precision plans also take 256 and
# 512 (FP64 plans reject tiles above 128, and the tuner skips those)
CANDIDATES = {
    "tile": [64, 256, 512],
    "blocks_per_sm": [1, 2, 3],
    "field_threads": [128, 256],
    "field_chunk": [1024, 4096],
}


def key_of(n_maxes, l_maxes, sizes) -> str:
    total = max(1, sum(int(n) for n in sizes))
    return f"n{max(n_maxes)}_l{max(l_maxes)}_N{int(math.log2(total))}"


def time_tuning(posm, sizes, n_maxes, l_maxes, tuning, reps=5) -> float:
    prec = etics.MIXED if posm.dtype == torch.float32 else etics.FP64
    plan = etics.BatchPlan(sizes, n_maxes, l_maxes, precision=prec, tuning=tuning,
                           device=posm.device)
    coeffs = torch.empty(max(plan.coeff_count, 1), dtype=torch.float64, device=posm.device)
    out = torch.empty_like(posm)
    for _ in range(2):
        etics.scf_batch(posm, plan, coeffs=coeffs, out=out)
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ts = []
    for _ in range(reps):
        t0.record()
        etics.scf_batch(posm, plan, coeffs=coeffs, out=out)
        t1.record()
        torch.cuda.synchronize()
        ts.append(t0.elapsed_time(t1))
    etics.check_error()
    return statistics.median(ts)


def tune(posm, sizes, n_maxes, l_maxes, reps=5, write=True):
    """Time all candidates; return (best tuning dict, all timings)."""
    results = []
    for vals in itertools.product(*CANDIDATES.values()):
        t = etics.BatchTuning(*vals)
        try:
            ms = time_tuning(posm, sizes, n_maxes, l_maxes, t, reps)
        except etics.EticsError:
            continue
        results.append((ms, t.as_dict()))
    results.sort(key=lambda x: x[0])
    best = results[0][1]
    if write:
        table = load_table()
        table[key_of(n_maxes, l_maxes, sizes)] = {"tuning": best, "ms": results[0][0],
                                                   "candidates": len(results)}
        with open(TABLE, "w") as f:
            json.dump(table, f, indent=1, sort_keys=True)
    return best, results


def load_table() -> dict:
    if os.path.exists(TABLE):
        with open(TABLE) as f:
            return json.load(f)
    return {}


def lookup(n_maxes, l_maxes, sizes):
    """The tuned BatchTuning for this batch shape, or None (library defaults)."""
    entry = load_table().get(key_of(n_maxes, l_maxes, sizes))
    if not entry:
        return None
    t = entry["tuning"]
    return etics.BatchTuning(t["tile"], t["blocks_per_sm"], t["field_threads"], t["field_chunk"])


def ensemble(seed: int = 0, ninst: int = 256):
    """The 256-system ensemble: N log-uniform in [2^12, 2^18], n_max in 6..14,
    l_max in 2..8, system i drawn with seed i (Hernquist spheres)."""
    import numpy as np
    from . import inputs
    rng = np.random.default_rng(seed)
    sizes = [int(round(2 ** rng.uniform(12, 18))) for _ in range(ninst)]
    n_maxes = [int(rng.integers(6, 15)) for _ in range(ninst)]
    l_maxes = [int(rng.integers(2, 9)) for _ in range(ninst)]
    parts = [inputs.hernquist(n, seed=i) for i, n in enumerate(sizes)]
    return np.concatenate(parts), sizes, n_maxes, l_maxes


if __name__ == "__main__":
    pm, sizes, nm, lm = ensemble()
    x = torch.tensor(pm, dtype=torch.float32, device="cuda")
    best, res = tune(x, sizes, nm, lm)
    print(json.dumps({"key": key_of(nm, lm, sizes), "best": best, "best_ms": res[0][0],
                      "worst_ms": res[-1][0], "candidates": len(res)}))
