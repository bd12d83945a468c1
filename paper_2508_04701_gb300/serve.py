"""A9: served execution -- continuous batching of query requests over resident tables.

The buffer manager's two regions (Sec. 3.2.3) map onto this module: a *caching region* holds
the fact columns, dim columns and their built dim indexes (join + group tables) for the whole
run; a *processing region* holds the per-request scratch (aggregates) and result arrays of the
batches in flight, and is what admission control accounts for.  Requests (fact_id, t) arrive
over time; the loop keeps up to `slots` batches in flight, each on its own CUDA stream with
its own batch plan, scratch and pinned result arena.  Whenever a slot is free it takes every
request that has arrived (up to `max_batch`) and fits the memory budget, launches them as one
batched pipeline (sirius_batch_plan_run against the resident dim indexes) and copies the result
rows back on the same stream; completions are polled by CUDA event.  Requests that arrive while
other batches run are admitted as soon as a slot and memory are free, so their work overlaps on
the device.  Pipelines as tasks pulled from a queue follow Sec. 3.2.2.
"""
from __future__ import annotations

import dataclasses
import math
import time
from collections import deque
from typing import Dict, List, Optional

import numpy as np
import torch

from . import datagen as dg
from . import sirius as S

RESULT_COLS = ("key", "sum", "count", "min", "max")


@dataclasses.dataclass
class Request:
    rid: int
    fact_id: int
    t: int
    arrival: float                 # seconds since the start of the run
    start: float = math.nan        # launch time
    done: float = math.nan         # completion time (result rows on the host)
    groups: int = -1
    status: int = -1
    result: Optional[Dict[str, np.ndarray]] = None


class ResidentPool:
    """The caching region: fact tables, dim tables and their built dim indexes."""

    def __init__(self, n_facts: int, n_dims: int, seed: int = 0, device="cuda", n_hi=20_000_000,
                 m_hi=2_000_000, group_cap_hint: int = 1000):
        self.device = torch.device(device)
        self.hint = group_cap_hint
        self.dims, self.dim_index, self.facts, self.fact_dim = [], [], [], []
        self.fact_rows = []
        for d in range(n_dims):
            spec = dg.batch_query(d, seed=seed, n_hi=n_hi, m_hi=m_hi)
            spec = dataclasses.replace(spec, n=4)
            dim = dg.gen_dim_device(spec, self.device)
            self.dims.append((spec, dim))
        for f in range(n_facts):
            dspec, dim = self.dims[f % n_dims]
            fspec = dg.batch_query(10_000 + f, seed=seed, n_hi=n_hi, m_hi=m_hi)
            fspec = dataclasses.replace(fspec, m=dspec.m, fk_domain=dspec.m, dim_table=dspec.dim_table)
            fact = dg.gen_fact_device(fspec, dim, self.device)
            self.facts.append((fspec, fact))
            self.fact_dim.append(f % n_dims)
            self.fact_rows.append(fspec.n)
        for d, (dspec, dim) in enumerate(self.dims):
            fact0 = self.facts[d][1] if d < len(self.facts) else None
            desc = S.make_desc(fact0 if fact0 is not None else _empty_fact(self.device), dim, "lt", 50,
                               group_cap_hint=self.hint)
            self.dim_index.append(S.sirius_dim_index_build(desc, self.device))
        torch.cuda.synchronize(self.device)

    def bytes(self) -> int:
        tot = 0
        for _, cols in self.dims + self.facts:
            tot += sum(v.numel() * v.element_size() for v in cols.values())
        return tot + sum(ix.nbytes for ix in self.dim_index)

    def desc(self, fact_id: int, t: int) -> S.PipelineDesc:
        fspec, fact = self.facts[fact_id]
        _, dim = self.dims[self.fact_dim[fact_id]]
        return S.make_desc(fact, dim, "lt", t, group_cap_hint=self.hint)

    def index(self, fact_id: int) -> S.DimIndexBuffer:
        return self.dim_index[self.fact_dim[fact_id]]


def _empty_fact(device):
    z32 = torch.zeros(4, dtype=torch.int32, device=device)
    return {"fk": z32, "pred": z32.clone(), "val": torch.zeros(4, dtype=torch.int64, device=device)}


class Admission:
    """Byte accounting of the processing region against a device-memory budget."""

    def __init__(self, budget_bytes: int, resident_bytes: int):
        self.budget = budget_bytes
        self.resident = resident_bytes
        self.in_flight = 0
        self.rejected = 0

    def fits(self, nbytes: int) -> bool:
        return self.resident + self.in_flight + nbytes <= self.budget

    def take(self, nbytes: int):
        self.in_flight += nbytes

    def give(self, nbytes: int):
        self.in_flight -= nbytes


class _OutView:
    """Result arrays of request i of a slot: rows of the slot's contiguous output block."""

    def __init__(self, slot, i):
        self.slot, self.i = slot, i
        self.d_groups = slot.d_groups

    def result(self, sync: bool) -> S.Result:
        s, i = self.slot, self.i
        base = s.d_out.data_ptr() + i * s.row_bytes
        cb = s.out_cap * 8
        return S.Result(base, base + cb, base + 2 * cb, base + 3 * cb, base + 4 * cb, s.out_cap,
                        s.d_groups.data_ptr() + 8 * i, s.d_status.data_ptr() + 4 * i,
                        1 if sync else 0, 0, 0)


class _Slot:
    """One in-flight batch: stream, plan, scratch, one device output block for all its requests
    and its pinned host twin (the result rows come back in one copy per batch)."""

    def __init__(self, max_batch: int, out_cap: int, scratch_bytes: int, device):
        self.stream = torch.cuda.Stream(device)
        self.plan = S.BatchPlan(max_batch)
        self.out_cap = out_cap
        self.row_bytes = len(RESULT_COLS) * out_cap * 8
        self.scratch = torch.empty(scratch_bytes, dtype=torch.uint8, device=device)
        self.d_out = torch.empty((max_batch, len(RESULT_COLS), out_cap), dtype=torch.int64, device=device)
        self.d_groups = torch.zeros(max_batch, dtype=torch.int64, device=device)
        self.d_status = torch.zeros(max_batch, dtype=torch.int32, device=device)
        self.h_out = torch.empty((max_batch, len(RESULT_COLS), out_cap), dtype=torch.int64, pin_memory=True)
        self.h_groups = torch.empty(max_batch, dtype=torch.int64, pin_memory=True)
        self.h_status = torch.empty(max_batch, dtype=torch.int32, pin_memory=True)
        self.views = [_OutView(self, i) for i in range(max_batch)]
        # device-side span of the batch in flight: from the stream reaching the batch to its
        # result copies finishing (timing events, comparable across streams)
        self.start_event = torch.cuda.Event(enable_timing=True)
        self.event = torch.cuda.Event(enable_timing=True)
        self.reqs: List[Request] = []
        self.bytes = 0

    @property
    def busy(self) -> bool:
        return bool(self.reqs)


class Server:
    """Continuous-batching request loop over a ResidentPool."""

    def __init__(self, pool: ResidentPool, slots: int = 4, max_batch: int = 64,
                 budget_bytes: int = 150 * 10**9, rows_per_unit: int = 0, use_graph: bool = True):
        self.pool = pool
        self.max_batch = max_batch
        self.rows_per_unit = rows_per_unit
        self.use_graph = use_graph
        dev = pool.device
        self.out_cap = S.lib().sirius_groupby_capacity(pool.hint) + 1
        probe_bytes = pool.dim_index[0].probe_scratch_bytes(S.PipelineDesc())  # aggregates only
        # processing-region bytes of one request: its aggregates and its result arrays
        self.req_bytes = probe_bytes + len(RESULT_COLS) * 8 * self.out_cap
        self.slots = [_Slot(max_batch, self.out_cap, max_batch * probe_bytes + 4096, dev) for _ in range(slots)]
        self.admission = Admission(budget_bytes, pool.bytes())
        self.batches = 0
        # overlap and attribution of the last run(): device spans of its batches (ms from the
        # run's reference event), the most batches in flight on the device at once, the most
        # slots busy at once as the host loop saw them, and the host loop's own time
        self.spans: List[tuple] = []
        self.max_busy_device = 0
        self.max_busy_slots = 0
        self.host_launch_s = 0.0
        self.host_complete_s = 0.0
        self._ref = None
        # one descriptor per fact table; a request copies it and sets its threshold
        self._base_desc = [pool.desc(f, 50) for f in range(len(pool.facts))]
        self._keep = self._base_desc

    # -- one batch ---------------------------------------------------------------------------
    def _desc(self, r: Request) -> S.PipelineDesc:
        d = S.PipelineDesc.from_buffer_copy(self._base_desc[r.fact_id])
        d.literal = r.t
        return d

    def _launch(self, slot: _Slot, reqs: List[Request], now: float):
        nb = len(reqs)
        descs = [self._desc(r) for r in reqs]
        idx = [self.pool.index(r.fact_id) for r in reqs]
        with torch.cuda.stream(slot.stream):
            slot.start_event.record(slot.stream)
            slot.plan.run(descs, slot.views[:nb], indexes=idx, rows_per_unit=self.rows_per_unit,
                          use_graph=self.use_graph, scratch=slot.scratch, stream=slot.stream, sync=False)
            slot.h_out[:nb].copy_(slot.d_out[:nb], non_blocking=True)
            slot.h_groups[:nb].copy_(slot.d_groups[:nb], non_blocking=True)
            slot.h_status[:nb].copy_(slot.d_status[:nb], non_blocking=True)
            slot.event.record(slot.stream)
        self.batches += 1
        for r in reqs:
            r.start = now
        slot.reqs = reqs

    def _complete(self, slot: _Slot, now: float, keep_results: bool):
        self.spans.append((self._ref.elapsed_time(slot.start_event), self._ref.elapsed_time(slot.event)))
        for i, r in enumerate(slot.reqs):
            r.done = now
            r.groups = int(slot.h_groups[i])
            r.status = int(slot.h_status[i])
            if keep_results:
                g = max(min(r.groups, self.out_cap), 0)
                r.result = {c: slot.h_out[i, k, :g].numpy().copy() for k, c in enumerate(RESULT_COLS)}
        self.admission.give(slot.bytes)
        slot.bytes = 0
        slot.reqs = []

    # -- the loop ----------------------------------------------------------------------------
    def run(self, requests: List[Request], keep_results: bool = False, poll_sleep: float = 0.0):
        """Serve requests (sorted by arrival, times relative to the call); returns them filled."""
        pending = deque()
        todo = deque(sorted(requests, key=lambda r: r.arrival))
        self.spans, self.max_busy_slots = [], 0
        self.host_launch_s = self.host_complete_s = 0.0
        self._ref = torch.cuda.Event(enable_timing=True)
        self._ref.record(torch.cuda.current_stream(self.pool.device))
        t0 = time.perf_counter()
        finished = 0
        total = len(requests)
        while finished < total:
            now = time.perf_counter() - t0
            while todo and todo[0].arrival <= now:
                pending.append(todo.popleft())
            for slot in self.slots:
                if slot.busy and slot.event.query():
                    finished += len(slot.reqs)
                    h0 = time.perf_counter()
                    self._complete(slot, h0 - t0, keep_results)
                    self.host_complete_s += time.perf_counter() - h0
            for slot in self.slots:
                if slot.busy or not pending:
                    continue
                batch = []
                while pending and len(batch) < self.max_batch:
                    need = (len(batch) + 1) * self.req_bytes
                    if not self.admission.fits(need):
                        self.admission.rejected += 1
                        break
                    batch.append(pending.popleft())
                if batch:
                    slot.bytes = len(batch) * self.req_bytes
                    self.admission.take(slot.bytes)
                    h0 = time.perf_counter()
                    self._launch(slot, batch, h0 - t0)
                    self.host_launch_s += time.perf_counter() - h0
                    self.max_busy_slots = max(self.max_busy_slots, sum(1 for x in self.slots if x.busy))
            if poll_sleep:
                time.sleep(poll_sleep)
        self.max_busy_device = max_overlap(self.spans)
        return requests

    def device_busy_ms(self) -> float:
        """Time (ms) during which at least one batch of the last run was in flight on the device
        (the union of the batches' device spans)."""
        return union_length(self.spans)


def max_overlap(spans) -> int:
    """The largest number of (start, end) intervals that contain one instant."""
    ev = sorted([(a, 1) for a, b in spans] + [(b, -1) for a, b in spans], key=lambda x: (x[0], x[1]))
    cur = best = 0
    for _, d in ev:
        cur += d
        best = max(best, cur)
    return best


def union_length(spans) -> float:
    """Total length covered by at least one (start, end) interval."""
    tot, end = 0.0, None
    for a, b in sorted(spans):
        if end is None or a > end:
            tot += b - a
            end = b
        elif b > end:
            tot += b - end
            end = b
    return tot


def sequential_fifo(pool: ResidentPool, requests: List[Request], keep_results: bool = False):
    """The plain baseline on the same GPU: one request at a time in arrival order, each one
    sirius_run_probe call against the resident dim index, results copied back before the next."""
    dev = pool.device
    out_cap = S.lib().sirius_groupby_capacity(pool.hint) + 1
    outs = S.PipelineOutputs(out_cap, dev)
    scratch = torch.empty(pool.dim_index[0].probe_scratch_bytes(S.PipelineDesc()) + 4096, dtype=torch.uint8,
                          device=dev)
    t0 = time.perf_counter()
    for r in sorted(requests, key=lambda r: r.arrival):
        now = time.perf_counter() - t0
        if now < r.arrival:
            time.sleep(r.arrival - now)
        r.start = time.perf_counter() - t0
        g = S.sirius_run_probe(pool.desc(r.fact_id, r.t), pool.index(r.fact_id), outs, scratch)
        res = {c: outs.t[c][:g].cpu().numpy() for c in RESULT_COLS}
        r.done = time.perf_counter() - t0
        r.groups, r.status = g, 0
        if keep_results:
            r.result = res
    return requests


def poisson_requests(rate: float, duration: float, n_facts: int, seed: int = 0,
                     t_lo: int = 5, t_hi: int = 90) -> List[Request]:
    """Open-loop Poisson arrivals: exponential gaps of mean 1/rate, uniform fact and threshold."""
    n = int(rate * duration * 1.2) + 16
    r = dg.stream(seed, 0x7000, 0, 0, 3 * n).reshape(n, 3)
    u = (r[:, 0] >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    gaps = -np.log1p(-u) / rate
    arr = np.cumsum(gaps)
    facts = dg.bounded(r[:, 1], n_facts)
    ts = t_lo + dg.bounded(r[:, 2], t_hi - t_lo + 1)
    out = []
    for i in range(n):
        if arr[i] > duration:
            break
        out.append(Request(i, int(facts[i]), int(ts[i]), float(arr[i])))
    return out


def latency_stats(reqs: List[Request], warmup: float = 0.0) -> Dict[str, float]:
    done = [r for r in reqs if r.arrival >= warmup and not math.isnan(r.done)]
    lat = np.array([r.done - r.arrival for r in done]) * 1e3
    if lat.size == 0:
        return {"requests": 0}
    span = max(r.done for r in done) - min(r.arrival for r in done)
    return {"requests": int(lat.size), "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
            "max_ms": float(lat.max()), "throughput_qps": lat.size / span if span > 0 else 0.0}
