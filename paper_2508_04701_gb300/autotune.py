"""Autotuner of the batched and single-query pipelines.

It times candidate settings on the device (CUDA events, after a warm-up) and keeps the
fastest.  The knobs are the join table's load factor (table size against probe-walk length),
the probe work unit of a batch (load balance against per-unit set-up and shared-memory flushes),
the probe kernel variant and its block shape.  Results are cached in a JSON file keyed by device
name and a size bucket of the workload (log2 of the fact rows, dim rows and query count), so
later runs of similar batches reuse them without timing.
"""
from __future__ import annotations

import json
import math
import os
import time
from typing import Dict, List, Optional, Sequence

import torch

from . import sirius as S

_DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")

BATCH_UNITS = (16_384, 65_536, 262_144, 1_048_576)
LOAD_FACTORS = (0.35, 0.5, 0.7)


def cache_path() -> str:
    return os.environ.get("SIRIUS_AUTOTUNE_CACHE", _DEFAULT_CACHE)


def _load() -> Dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except Exception:
        return {}


def _store(d: Dict):
    p = cache_path()
    os.makedirs(os.path.dirname(p), exist_ok=True)
    tmp = p + f".{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, p)


def _bucket(x: float) -> int:
    return int(math.log2(max(x, 1)))


def batch_key(descs: Sequence[S.PipelineDesc]) -> str:
    n = sum(d.n for d in descs)
    m = sum(d.m for d in descs)
    return f"{torch.cuda.get_device_name()}|batch|q{_bucket(len(descs))}|n{_bucket(n)}|m{_bucket(m)}"


def _time(fn, reps: int = 3) -> float:
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def tune_batch(plan: S.BatchPlan, descs: List[S.PipelineDesc], outputs, scratch: Optional[torch.Tensor] = None,
               use_graph: bool = True, units: Sequence[int] = BATCH_UNITS,
               load_factors: Sequence[float] = LOAD_FACTORS, use_cache: bool = True) -> Dict:
    """Best (rows_per_unit, load_factor) for this batch; updates descs' load factors in place."""
    key = batch_key(descs)
    cache = _load() if use_cache else {}
    if key in cache:
        best = cache[key]
        for d in descs:
            d.load_factor = best["load_factor"]
        return dict(best, cached=True)
    trials = []
    for lf in load_factors:
        for d in descs:
            d.load_factor = lf
        need = S.batch_scratch_bytes(descs)
        sc = scratch if scratch is not None and scratch.numel() >= need else \
            torch.empty(need, dtype=torch.uint8, device="cuda")
        for u in units:
            ms = _time(lambda: plan.run(descs, outputs, rows_per_unit=u, use_graph=use_graph, scratch=sc,
                                        sync=False))
            trials.append({"rows_per_unit": u, "load_factor": lf, "ms": ms})
    best = min(trials, key=lambda t: t["ms"])
    for d in descs:
        d.load_factor = best["load_factor"]
    rec = {"rows_per_unit": best["rows_per_unit"], "load_factor": best["load_factor"], "ms": best["ms"],
           "trials": len(trials), "when": time.strftime("%Y-%m-%dT%H:%M:%S")}
    if use_cache:
        cache[key] = rec
        _store(cache)
    return dict(rec, cached=False, all=trials)


def tune_pipeline(desc: S.PipelineDesc, outputs: S.PipelineOutputs,
                  load_factors: Sequence[float] = LOAD_FACTORS,
                  variants: Sequence[str] = ("single", "direct", "staged"),
                  block_threads: Sequence[int] = (256, 512)) -> Dict:
    """Best (load_factor, probe_variant, block_threads) for one query; sets them on desc.
    Variants: the single launch (every phase in one cooperative launch), the per-phase kernels
    with each block shape, and the staged probe (settings a query does not take are skipped)."""
    trials = []
    for lf in load_factors:
        desc.load_factor = lf
        sc = torch.empty(S.pipeline_scratch_bytes(desc), dtype=torch.uint8, device="cuda")
        for v in variants:
            desc.probe_variant = S.PROBE_VARIANTS[v]
            for bt in (block_threads if v == "direct" else (0,)):
                desc.block_threads = bt
                try:
                    ms = _time(lambda: S.sirius_run_pipeline(desc, outputs, sc, sync=False))
                except S.SiriusError:
                    continue
                trials.append({"load_factor": lf, "probe_variant": v, "block_threads": bt, "ms": ms})
    best = min(trials, key=lambda t: t["ms"])
    desc.load_factor = best["load_factor"]
    desc.probe_variant = S.PROBE_VARIANTS[best["probe_variant"]]
    desc.block_threads = best["block_threads"]
    return dict(best, all=trials)
