"""Full-size runs of the oracle on every host core: the fact table in row chunks, each chunk
generated and run through ``relational.pipeline`` in a worker process, the chunks' group
results merged.

TEST INFRASTRUCTURE ONLY (see the package docstring): the test suite, ``bench.py``'s CPU
baseline and its reference arm use it; the product path never does.

Why chunking is exact.  The filter, the join and the late materialisation act row by row on
the fact table (Sec. 3.2.2: stateless operators pushed over the rows), so the joined rows of
the whole table are the disjoint union of those of its chunks, and the four aggregates are
distributive: per group key, SUM and COUNT of the union are the sums of the chunks' SUMs and
COUNTs, MIN and MAX the extremes of the chunks' MINs and MAXs.  ``merge_sorted_partials`` is
that merge written with a stable sort and segmented reductions; it is pinned against the
dictionary merge ``relational.merge_partials`` and the chunked result against the whole-table
``pipeline`` (tests/test_oracle_pins.py).

Inputs come from the seeded host generator (``datagen``'s numpy functions: the input recipe,
none of the method's arithmetic), so no input or expected value here passes through a GPU.
Workers are started with the ``spawn`` method (safe after the parent has used CUDA).
"""
from __future__ import annotations

import multiprocessing as mp
import os
import time
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

from .relational import INT64_MAX, INT64_MIN, pipeline

COLS = ("key", "sum", "count", "min", "max")


def host_cores() -> int:
    """The cores this process may run on (sched_getaffinity)."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # not Linux
        return os.cpu_count() or 1


# ------------------------------------------------------------------------------- merge
def merge_sorted_partials(parts: Sequence[Dict[str, np.ndarray]]) -> Dict[str, np.ndarray]:
    """Combine group-by results of disjoint row chunks (any order of keys within a part):
    per key SUM and COUNT add, MIN and MAX take the extreme; groups sorted by key.

    A stable sort of the concatenated keys, then per run of equal keys np.add / np.minimum /
    np.maximum .reduceat.  Sums are exact: when the parts' SUMs could pass 2**63 in total they
    are added as Python integers, and a total that does not fit int64 raises OverflowError."""
    parts = [p for p in parts if np.asarray(p["key"]).shape[0] > 0]
    if not parts:
        z = np.zeros(0, np.int64)
        return {c: z.copy() for c in COLS}
    cat = {c: np.concatenate([np.asarray(p[c]) for p in parts]) for c in COLS}
    keys = cat["key"]
    if keys.dtype != np.uint64:
        keys = keys.astype(np.int64)
    order = np.argsort(keys, kind="stable")
    k = keys[order]
    uniq, start = np.unique(k, return_index=True)
    s = cat["sum"].astype(np.int64)[order]
    smax = max(abs(int(s.max())), abs(int(s.min())))
    if smax * s.size < (1 << 63):
        sums = np.add.reduceat(s, start)
    else:
        ends = np.append(start[1:], s.size)
        tot = [sum(int(x) for x in s[a:b]) for a, b in zip(start, ends)]
        if any(x < INT64_MIN or x > INT64_MAX for x in tot):
            raise OverflowError("a group's SUM does not fit int64")
        sums = np.array(tot, dtype=np.int64)
    return {"key": uniq,
            "sum": sums.astype(np.int64),
            "count": np.add.reduceat(cat["count"].astype(np.int64)[order], start),
            "min": np.minimum.reduceat(cat["min"].astype(np.int64)[order], start),
            "max": np.maximum.reduceat(cat["max"].astype(np.int64)[order], start)}


# ------------------------------------------------------------------------------- workers
_TABLES: Dict[object, tuple] = {}   # per worker process: spec -> (dim, zipf cdf, filter dims)


def _tables(spec):
    from paper_2508_04701_gb300 import datagen as dg
    ent = _TABLES.get(spec)
    if ent is None:
        if len(_TABLES) >= 4:
            _TABLES.clear()
        dim = dg.gen_dim_host(spec)
        cdf = dg.zipf_cdf(spec.m, spec.zipf_s) if spec.zipf_s > 0 else None
        semi = dg.gen_semi_dims_host(spec) if spec.semi else None
        ent = (dim, cdf, semi)
        _TABLES[spec] = ent
    return ent


def _fact(spec, i0: int, i1: int):
    from paper_2508_04701_gb300 import datagen as dg
    dim, cdf, _ = _tables(spec)
    return dg.gen_fact_host(spec, i0, i1, dim=dim, cdf=cdf)


def _run(spec, fact) -> Dict[str, np.ndarray]:
    """relational.pipeline on one chunk of the query's fact rows."""
    dim, _, semi_dims = _tables(spec)
    kw = {}
    if spec.dt:
        kw.update(dim_op="lt", dim_literal=spec.dt)
    if spec.semi:
        kw["semi"] = [{"fk": fact[f"sk{k}"], "dim": semi_dims[k], "op": "lt", "literal": spec.semi_t}
                      for k in range(spec.semi)]
    return pipeline(fact, dim, "lt", spec.t, **kw)


def _chunk_task(task):
    q, spec, i0, i1 = task
    return q, _run(spec, _fact(spec, i0, i1))


def _worker_init():
    os.environ.setdefault("OMP_NUM_THREADS", "1")


def chunk_plan(n: int, chunk_rows: int) -> List[Tuple[int, int]]:
    """[i0, i1) ranges covering 0..n-1 once each, in order."""
    chunk_rows = max(1, int(chunk_rows))
    return [(i0, min(n, i0 + chunk_rows)) for i0 in range(0, n, chunk_rows)]


def query_results(specs, chunk_rows: int = 10_000_000, workers: Optional[int] = None,
                  rows: Optional[int] = None) -> List[Dict[str, np.ndarray]]:
    """The oracle's result of every query in `specs` (datagen StarSpecs: fact and dim tables
    from the seeded host generator), computed over row chunks on `workers` processes (default:
    every host core) and merged.  rows: only the first `rows` fact rows of each query."""
    specs = list(specs)
    tasks = []
    for q, sp in enumerate(specs):
        n = sp.n if rows is None else min(rows, sp.n)
        tasks += [(q, sp, i0, i1) for i0, i1 in chunk_plan(n, chunk_rows)]
    tasks.sort(key=lambda t: t[3] - t[2], reverse=True)   # largest first: even finish
    parts: List[list] = [[] for _ in specs]
    workers = min(workers or host_cores(), max(1, len(tasks)))
    if workers <= 1:
        for t in tasks:
            q, r = _chunk_task(t)
            parts[q].append(r)
    else:
        ctx = mp.get_context("spawn")
        with ctx.Pool(workers, initializer=_worker_init) as pool:
            for q, r in pool.imap_unordered(_chunk_task, tasks):
                parts[q].append(r)
    out = []
    for q, sp in enumerate(specs):
        if not parts[q]:
            # no fact rows: the whole-table definition on an empty fact table
            out.append(_run(sp, _fact(sp, 0, 0)))
        else:
            out.append(merge_sorted_partials(parts[q]))
    return out


# ------------------------------------------------------------------------------- timed runs
def _hot_worker(conn, spec, ranges):
    """Generate this worker's chunks once, then on every "run" message run the oracle over
    them and send back (merged result, seconds)."""
    _worker_init()
    facts = [_fact(spec, i0, i1) for i0, i1 in ranges]
    conn.send("ready")
    while True:
        msg = conn.recv()
        if msg != "run":
            break
        t0 = time.perf_counter()
        res = merge_sorted_partials([_run(spec, f) for f in facts])
        conn.send((res, time.perf_counter() - t0))
    conn.close()


class HotOracle:
    """The oracle timed on resident inputs ("hot" runs, as the GPU is timed): `workers`
    processes each generate their share of the first `rows` fact rows once; every run() then
    runs relational.pipeline over all chunks in parallel and merges the results, timed from
    the start message to the last worker's reply plus the final merge."""

    def __init__(self, spec, rows: Optional[int] = None, workers: Optional[int] = None,
                 chunk_rows: int = 20_000_000):
        self.spec = spec
        self.rows = spec.n if rows is None else min(int(rows), spec.n)
        self.workers = max(1, min(workers or host_cores(), max(1, self.rows // 100_000)))
        plan = chunk_plan(self.rows, min(chunk_rows, max(1, -(-self.rows // self.workers))))
        shares = [plan[w::self.workers] for w in range(self.workers)]
        ctx = mp.get_context("spawn")
        self.conns, self.procs = [], []
        for w in range(self.workers):
            a, b = ctx.Pipe()
            p = ctx.Process(target=_hot_worker, args=(b, spec, shares[w]), daemon=True)
            p.start()
            self.conns.append(a)
            self.procs.append(p)
        for c in self.conns:
            if c.recv() != "ready":
                raise RuntimeError("oracle worker failed to start")

    def run(self) -> Tuple[Dict[str, np.ndarray], float]:
        t0 = time.perf_counter()
        for c in self.conns:
            c.send("run")
        parts = [c.recv() for c in self.conns]
        res = merge_sorted_partials([p[0] for p in parts])
        return res, time.perf_counter() - t0

    def close(self):
        for c in self.conns:
            try:
                c.send("stop")
                c.close()
            except Exception:
                pass
        for p in self.procs:
            p.join(timeout=10)
            if p.is_alive():
                p.kill()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


__all__ = ["host_cores", "merge_sorted_partials", "chunk_plan", "query_results", "HotOracle"]
