"""Parity at the full sizes of the measured workloads, in the launch configuration bench.py
times (default agg_mode / probe variant, the bench's group_cap_hint): every group of every
query compared with the oracle, column by column.

The oracle runs the whole-table definition over row chunks on every host core (oracle.chunked:
the operators act row by row and the four aggregates merge exactly), from the seeded host
generator, in worker processes started before the GPU work and running beside it.  The GPU
side takes its inputs from the generator's CUDA twin (bit-identical to the host generator,
tests/test_gpu_datagen.py).
"""
import concurrent.futures as cf
import dataclasses

import numpy as np
import pytest
import torch

import oracle as O
from paper_2508_04701_gb300 import datagen as dg

pytestmark = pytest.mark.gpu

COLS = ("key", "sum", "count", "min", "max")
FULL = {"plain_600M": dg.plain_scale(), "plain_600M_composite": dg.plain_scale(composite=True),
        "skewed_300M": dg.skewed()}
HINT = {"plain_600M": 100_000, "plain_600M_composite": 100_000, "skewed_300M": dg.skewed().m}
BATCH = [dg.batch_query(q) for q in range(512)]

_POOL = cf.ThreadPoolExecutor(max_workers=1)
_FUTURES = {}


def oracle_future(name, fn):
    """Start (once) an oracle computation in the background; the GPU tests run meanwhile."""
    if name not in _FUTURES:
        _FUTURES[name] = _POOL.submit(fn)
    return _FUTURES[name]


def full_results():
    return oracle_future("full", lambda: dict(zip(FULL, O.query_results(list(FULL.values()),
                                                                        chunk_rows=5_000_000))))


def batch_results():
    return oracle_future("batch", lambda: O.query_results(BATCH, chunk_rows=5_000_000))


@pytest.fixture(scope="module")
def S():
    full_results()      # the host oracle starts before the first GPU call
    batch_results()
    from paper_2508_04701_gb300 import build
    build.build()
    from paper_2508_04701_gb300 import sirius
    sirius.lib()
    return sirius


def host(d):
    return {k: v.cpu().numpy() for k, v in d.items()}


def assert_all_groups(got, want, aggs, where=""):
    got = O.sort_groups(got)
    assert want["key"].size > 0
    assert np.array_equal(got["key"], want["key"]), (where, "key")
    for c in ["count"] + [a for a in ("sum", "min", "max") if a in aggs]:
        assert np.array_equal(got[c], want[c]), (where, c)


def run_bench_config(S, name):
    spec, hint = FULL[name], HINT[name]
    dim = dg.gen_dim_device(spec)
    fact = dg.gen_fact_device(spec, dim)
    desc = S.make_desc(fact, dim, "lt", spec.t, spec.aggs, hint)
    outs = S.PipelineOutputs(hint + 1)
    scratch = torch.empty(S.pipeline_scratch_bytes(desc), dtype=torch.uint8, device="cuda")
    g = S.sirius_run_pipeline(desc, outs, scratch)
    got = {k: v.cpu().numpy() for k, v in outs.trimmed(g).items()}
    del fact, dim, scratch
    torch.cuda.empty_cache()
    return g, got


@pytest.mark.parametrize("name", list(FULL))
def test_full_size_every_group(S, name):
    """600M fact rows / 15M dim rows / 100 000 groups, pred < 30 (one- and two-column join
    keys); 300M Zipf(1.1) rows over 10M dim keys with (grp, flag) groups, pred < 50."""
    g, got = run_bench_config(S, name)
    want = full_results().result()[name]
    assert g == want["key"].size
    assert_all_groups(got, want, FULL[name].aggs, name)


def test_batch_512_every_query(S):
    """The 512-query batch as the bench runs it (one plan, CUDA graph): every query's groups
    against the oracle."""
    tabs = []
    for sp in BATCH:
        d = dg.gen_dim_device(sp)
        tabs.append((d, dg.gen_fact_device(sp, d)))
    descs = [S.make_desc(f, d, "lt", sp.t, "sum,count,min,max", 1000) for sp, (d, f) in zip(BATCH, tabs)]
    cap = S.lib().sirius_groupby_capacity(1000) + 1
    outs = [S.PipelineOutputs(cap) for _ in BATCH]
    plan = S.BatchPlan(512)
    scratch = torch.empty(S.batch_scratch_bytes(descs), dtype=torch.uint8, device="cuda")
    g = plan.run(descs, outs, scratch=scratch, use_graph=True)
    got = [{k: v.cpu().numpy() for k, v in outs[q].trimmed(g[q]).items()} for q in range(512)]
    plan.close()
    del tabs, descs, outs, scratch
    torch.cuda.empty_cache()
    want = batch_results().result()
    for q in range(512):
        assert g[q] == want[q]["key"].size, q
        assert_all_groups(got[q], want[q], "sum,count,min,max", f"query {q}")


def test_served_full_pool_alone_mix_and_oracle(S):
    """The served workload's full resident pool (512 fact tables, 64 dims with their resident
    indexes): a Poisson run with batches overlapping on the device; every request's result
    equals the same request run alone, and 64 requests equal the oracle."""
    from paper_2508_04701_gb300 import serve
    pool = serve.ResidentPool(n_facts=512, n_dims=64, seed=0)
    reqs = serve.poisson_requests(rate=8000, duration=0.25, n_facts=len(pool.facts), seed=21)
    assert len(reqs) > 1000
    srv = serve.Server(pool, slots=4, max_batch=64)
    srv.run(reqs, keep_results=True)
    assert all(r.status == 0 for r in reqs)
    assert srv.max_busy_device > 1          # batches ran on the device at the same time
    alone = serve.sequential_fifo(pool, [serve.Request(r.rid, r.fact_id, r.t, 0.0) for r in reqs],
                                  keep_results=True)
    by_rid = {a.rid: a for a in alone}
    for r in reqs:
        a = by_rid[r.rid]
        assert r.groups == a.groups, r.rid
        for c in COLS:
            x, y = O.sort_groups(r.result), O.sort_groups(a.result)
            assert np.array_equal(x[c], y[c]), (r.rid, c)
    # 64 requests (spread over the run) against the oracle on host-generated tables
    pick = reqs[:: max(1, len(reqs) // 64)][:64]
    specs = [dataclasses.replace(pool.facts[r.fact_id][0], t=r.t) for r in pick]
    want = O.query_results(specs, chunk_rows=5_000_000)
    for r, w in zip(pick, want):
        assert r.groups == w["key"].size, r.rid
        assert_all_groups(r.result, w, "sum,count,min,max", f"request {r.rid}")
