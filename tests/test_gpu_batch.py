"""Batched pipelines (one set of persistent launches, optionally one CUDA graph): every
query's result equals the CPU oracle and the same query run alone, bit-exact (GPU)."""
import dataclasses

import numpy as np
import pytest
import torch

import oracle as O
from paper_2508_04701_gb300 import datagen as dg

pytestmark = pytest.mark.gpu
COLS = ("key", "sum", "count", "min", "max")


@pytest.fixture(scope="module")
def S():
    from paper_2508_04701_gb300 import build
    build.build()
    from paper_2508_04701_gb300 import sirius
    sirius.lib()
    return sirius


def dev(d):
    return {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in d.items()}


def mixed_queries(nq, seed):
    """Uneven sizes, thresholds, operators, key kinds and group counts."""
    rng = np.random.default_rng(seed)
    specs = []
    for q in range(nq):
        kind = q % 6
        n = int(np.exp(rng.uniform(np.log(3), np.log(400_000))))
        m = int(np.exp(rng.uniform(np.log(1), np.log(30_000))))
        spec = dg.StarSpec(f"b{q}", n=n, m=m, fk_domain=max(1, int(m * rng.uniform(0.8, 1.5))),
                           grp_bound=int(rng.choice([1, 7, 300, 1000, 5000])), t=int(rng.integers(0, 101)),
                           composite=(kind == 3), group_flag=(kind == 4), seed=1000 * seed + q,
                           fact_table=dg.BATCH_TABLE0 + 2 * q, dim_table=dg.BATCH_TABLE0 + 2 * q + 1)
        op = O.OPS[int(rng.integers(0, 6))] if kind == 5 else "lt"
        specs.append((spec, op))
    return specs


def build_batch(S, specs, hint_of=None):
    tabs, descs, outs = [], [], []
    for spec, op in specs:
        dim, fact = dg.gen_dim_host(spec), dg.gen_fact_host(spec)
        if spec.m > 0 and spec.group_flag is False and spec.m % 5 == 0:
            dim["pk"][: spec.m // 5] = dim["pk"][spec.m // 5: 2 * (spec.m // 5)]   # duplicate keys
        hint = (hint_of(spec) if hint_of else (spec.m if spec.group_flag else min(spec.grp_bound, max(spec.m, 1))))
        df, dd = dev(fact), dev(dim)
        descs.append(S.make_desc(df, dd, op, spec.t, group_cap_hint=hint))
        outs.append(S.PipelineOutputs(S.lib().sirius_groupby_capacity(hint) + 1))
        tabs.append((fact, dim, op, spec.t))
    return tabs, descs, outs


def check_all(tabs, outs, groups):
    for (fact, dim, op, t), o, g in zip(tabs, outs, groups):
        got = O.sort_groups({k: v.cpu().numpy() for k, v in o.trimmed(g).items()})
        want = O.pipeline(fact, dim, op, t)
        for c in COLS:
            assert np.array_equal(got[c], want[c]), c


@pytest.mark.parametrize("use_graph", [False, True])
def test_batch_matches_oracle(S, use_graph):
    tabs, descs, outs = build_batch(S, mixed_queries(36, 1))
    plan = S.BatchPlan(64)
    g = plan.run(descs, outs, use_graph=use_graph, rows_per_unit=8192)
    check_all(tabs, outs, g)
    # the same plan again, with another batch of a different size (graph replay or recapture)
    tabs2, descs2, outs2 = build_batch(S, mixed_queries(20, 2))
    g2 = plan.run(descs2, outs2, use_graph=use_graph, rows_per_unit=4096)
    check_all(tabs2, outs2, g2)
    plan.close()


def test_graph_replay_reuses_capture(S):
    specs = [(dg.batch_query(q, n_hi=300_000, m_hi=20_000), "lt") for q in range(24)]
    tabs, descs, outs = build_batch(S, specs, hint_of=lambda s: 1000)
    plan = S.BatchPlan(32)
    l0 = S.launch_count()
    for _ in range(3):
        g = plan.run(descs, outs, use_graph=True)
        check_all(tabs, outs, g)
    # per replay: init, min/max, two clears, build, fallback, one probe class, finalize, publish
    assert S.launch_count() - l0 == 3 * 9
    plan.close()


def test_batch_equals_standalone(S):
    specs = mixed_queries(12, 3)
    tabs, descs, outs = build_batch(S, specs)
    g = S.sirius_run_pipeline_batch(descs, outs)
    for d, o, gi in zip(descs, outs, g):
        alone = S.PipelineOutputs(o.cap)
        ga = S.sirius_run_pipeline(d, alone)
        assert ga == gi
        a = O.sort_groups({k: v.cpu().numpy() for k, v in alone.trimmed(ga).items()})
        b = O.sort_groups({k: v.cpu().numpy() for k, v in o.trimmed(gi).items()})
        for c in COLS:
            assert np.array_equal(a[c], b[c])


def test_batch_with_resident_dim_indexes(S):
    """Many queries share two resident dim indexes (no build inside the batch)."""
    dims = []
    for j in range(2):
        spec = dg.StarSpec(f"d{j}", n=4, m=10_000 + j, fk_domain=11_000, grp_bound=800, seed=50 + j)
        dim = dg.gen_dim_host(spec)
        dd = dev(dim)
        fd = dev(dg.gen_fact_host(spec))
        idx = S.sirius_dim_index_build(S.make_desc(fd, dd, "lt", 50, group_cap_hint=800))
        dims.append((dim, dd, idx))
    tabs, descs, outs, indexes = [], [], [], []
    for q in range(10):
        dim, dd, idx = dims[q % 2]
        fs = dg.StarSpec(f"f{q}", n=50_000 + 977 * q, m=dim["pk"].size, fk_domain=11_000, grp_bound=800,
                         t=10 + 7 * q, seed=60 + q)
        fact = dg.gen_fact_host(fs)
        descs.append(S.make_desc(dev(fact), dd, "lt", fs.t, group_cap_hint=800))
        outs.append(S.PipelineOutputs(S.lib().sirius_groupby_capacity(800) + 1))
        indexes.append(idx)
        tabs.append((fact, dim, "lt", fs.t))
    plan = S.BatchPlan(16)
    for use_graph in (False, True):
        g = plan.run(descs, outs, indexes=indexes, use_graph=use_graph)
        check_all(tabs, outs, g)
    plan.close()


def test_batch_per_query_status(S):
    """One query's group table overflows (TABLE_FULL); the others finish normally."""
    specs = mixed_queries(6, 4)
    over = dg.skewed(n=50_000, m=20_000, seed=5)
    specs.insert(2, (over, "lt"))
    hint_of = lambda s: 1000 if s is over else (s.m if s.group_flag else min(s.grp_bound, max(s.m, 1)))  # noqa: E731
    tabs, descs, outs = build_batch(S, specs, hint_of=hint_of)
    plan = S.BatchPlan(8)
    with pytest.raises(S.SiriusError) as e:
        plan.run(descs, outs)
    assert e.value.status == S.ERR_TABLE_FULL
    assert plan.last_status[2] == S.ERR_TABLE_FULL
    assert all(s == 0 for i, s in enumerate(plan.last_status) if i != 2)
    plan.close()


@pytest.mark.parametrize("use_graph", [False, True])
def test_batch_with_dim_predicates(S, use_graph):
    """Queries with dim-side predicates (one- and two-column keys, different thresholds) in one
    batch with queries without."""
    tabs, descs, outs = [], [], []
    for q in range(10):
        spec = dg.plain_scale(n=50_000 + 7919 * q, m=3000 + 101 * q, composite=(q % 3 == 2),
                              dt=(10 * q if q % 4 else 0), seed=q)
        spec = dataclasses.replace(spec, grp_bound=300, fact_table=dg.BATCH_TABLE0 + 2 * q,
                                   dim_table=dg.BATCH_TABLE0 + 2 * q + 1)
        dim, fact = dg.gen_dim_host(spec), dg.gen_fact_host(spec)
        dop = "lt" if spec.dt else None
        descs.append(S.make_desc(dev(fact), dev(dim), "lt", spec.t, group_cap_hint=300, dim_op=dop,
                                 dim_literal=spec.dt))
        outs.append(S.PipelineOutputs(S.lib().sirius_groupby_capacity(300) + 1))
        tabs.append((fact, dim, spec.t, dop, spec.dt))
    plan = S.BatchPlan(16)
    g = plan.run(descs, outs, use_graph=use_graph)
    for (fact, dim, t, dop, dt), o, gq in zip(tabs, outs, g):
        got = O.sort_groups({k: v.cpu().numpy() for k, v in o.trimmed(gq).items()})
        want = O.pipeline(fact, dim, "lt", t, dim_op=dop, dim_literal=dt)
        for c in COLS:
            assert np.array_equal(got[c], want[c]), c
    plan.close()
