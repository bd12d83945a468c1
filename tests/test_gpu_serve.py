"""Served execution: continuous batching over resident tables gives each request exactly the
result it gets alone (and the oracle's), under overlap and under a tight memory budget (GPU)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2508_04701_gb300 import datagen as dg

pytestmark = pytest.mark.gpu
COLS = ("key", "sum", "count", "min", "max")


@pytest.fixture(scope="module")
def env():
    from paper_2508_04701_gb300 import build
    build.build()
    from paper_2508_04701_gb300 import serve
    pool = serve.ResidentPool(n_facts=6, n_dims=3, seed=7, n_hi=300_000, m_hi=20_000, group_cap_hint=1000)
    host = {}
    for f, (fspec, _) in enumerate(pool.facts):
        dspec, _ = pool.dims[pool.fact_dim[f]]
        host[f] = (dg.gen_fact_host(fspec), dg.gen_dim_host(dspec))
    return serve, pool, host


def oracle_of(host, r):
    fact, dim = host[r.fact_id]
    return O.pipeline(fact, dim, "lt", r.t)


def same(a, b):
    a, b = O.sort_groups(a), O.sort_groups(b)
    return all(np.array_equal(a[c], b[c]) for c in COLS)


def test_pool_tables_match_host_generator(env):
    serve, pool, host = env
    for f, (fspec, fact) in enumerate(pool.facts):
        for k, v in fact.items():
            assert np.array_equal(v.cpu().numpy(), host[f][0][k])


def test_served_results_equal_alone_and_oracle(env):
    serve, pool, host = env
    reqs = serve.poisson_requests(rate=4000, duration=0.05, n_facts=len(pool.facts), seed=3)
    assert len(reqs) > 100
    srv = serve.Server(pool, slots=3, max_batch=16)
    srv.run(reqs, keep_results=True)
    assert srv.batches < len(reqs)          # requests were batched
    alone = serve.sequential_fifo(pool, [serve.Request(r.rid, r.fact_id, r.t, 0.0) for r in reqs],
                                  keep_results=True)
    for r, a in zip(sorted(reqs, key=lambda x: x.rid), sorted(alone, key=lambda x: x.rid)):
        assert r.status == 0 and r.groups == a.groups
        assert same(r.result, a.result)
    for r in reqs[:12]:
        assert same(r.result, oracle_of(host, r))


def test_overlapping_batches_with_graphs_off(env):
    serve, pool, host = env
    reqs = serve.poisson_requests(rate=20000, duration=0.01, n_facts=len(pool.facts), seed=4)
    srv = serve.Server(pool, slots=4, max_batch=8, use_graph=False, rows_per_unit=16384)
    srv.run(reqs, keep_results=True)
    assert srv.max_busy_slots > 1             # batches were in flight together
    assert srv.max_busy_device >= 1 and len(srv.spans) == srv.batches
    for r in reqs[:10]:
        assert same(r.result, oracle_of(host, r))


def test_tight_memory_budget_defers_but_completes(env):
    serve, pool, host = env
    reqs = serve.poisson_requests(rate=50000, duration=0.004, n_facts=len(pool.facts), seed=5)
    srv = serve.Server(pool, slots=2, max_batch=32)
    srv.admission.budget = srv.admission.resident + 3 * srv.req_bytes   # at most 3 requests in flight
    srv.run(reqs, keep_results=True)
    assert srv.admission.rejected > 0
    assert srv.admission.in_flight == 0
    assert all(r.status == 0 for r in reqs)
    for r in reqs[:8]:
        assert same(r.result, oracle_of(host, r))


def test_latency_stats(env):
    serve, pool, _ = env
    reqs = serve.poisson_requests(rate=2000, duration=0.1, n_facts=len(pool.facts), seed=6)
    serve.Server(pool, slots=2, max_batch=32).run(reqs)
    st = serve.latency_stats(reqs)
    assert st["requests"] == len(reqs)
    assert 0 < st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]
