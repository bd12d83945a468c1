"""The single-launch pipeline (probe_variant 3: every phase in one cooperative launch, phases
separated by grid-wide barriers) against the CPU oracle, bit-exact after sorting groups by key,
beside the per-phase kernels (probe_variant 1) on the same inputs (GPU).

Each case takes a different route through the phases: direct array, direct array turned down
by a duplicate key (fallback into the hash table), sparse keys (hash table), two-column keys,
dim-side predicate with and without a Bloom filter, every aggregation mode the single launch
takes, ragged and empty inputs, unaligned columns, and the TABLE_FULL / CAPACITY errors."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2508_04701_gb300 import datagen as dg

pytestmark = pytest.mark.gpu

COLS = ("key", "sum", "count", "min", "max")
VARIANTS = ("single", "direct")


@pytest.fixture(scope="module")
def S():
    from paper_2508_04701_gb300 import build
    build.build()
    from paper_2508_04701_gb300 import sirius
    sirius.lib()
    return sirius


def dev(d):
    return {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in d.items()}


def check(S, fact, dim, op, t, hint, aggs="sum,count,min,max", dim_op=None, dim_literal=0, **kw):
    want = O.pipeline(fact, dim, op, t, dim_op=dim_op, dim_literal=dim_literal)
    df, dd = dev(fact), dev(dim)
    for variant in VARIANTS:
        got = S.run_pipeline(df, dd, op, t, aggs, hint, probe_variant=variant, dim_op=dim_op,
                             dim_literal=dim_literal, **kw)
        torch.cuda.synchronize()
        got = O.sort_groups({k: v.cpu().numpy() for k, v in got.items()})
        for c in ["key", "count"] + [a for a in ("sum", "min", "max") if a in aggs]:
            assert np.array_equal(got[c], want[c]), (variant, c)
    return want["key"].size


def rand_tables(seed, n, m, key_lo, key_hi, fk_lo, fk_hi, groups, vbound=10**9):
    rng = np.random.default_rng(seed)
    dim = {"pk": rng.integers(key_lo, key_hi, size=m).astype(np.int32),
           "grp": rng.integers(-groups // 4, groups - groups // 4, size=m).astype(np.int32)}
    fact = {"fk": rng.integers(fk_lo, fk_hi, size=n).astype(np.int32),
            "pred": rng.integers(0, 100, size=n).astype(np.int32),
            "val": rng.integers(-vbound, vbound, size=n)}
    return fact, dim


def test_one_million_row_query(S):
    """The 1M-row fact / 65 536-row dim / 1 000-group query at its full size."""
    spec = dg.plain_small()
    dim, fact = dg.gen_dim_host(spec), dg.gen_fact_host(spec)
    assert check(S, fact, dim, "lt", spec.t, hint=spec.grp_bound) == 1000


@pytest.mark.parametrize("mode", ["smem", "global", "hot"])
@pytest.mark.parametrize("n", [1, 3, 4, 5, 1023, 100_003])
def test_ragged_sizes_every_mode(S, mode, n):
    spec = dg.StarSpec("t", n=n, m=3001, fk_domain=3500, grp_bound=300, t=60, seed=n)
    dim, fact = dg.gen_dim_host(spec), dg.gen_fact_host(spec)
    check(S, fact, dim, "lt", spec.t, hint=300, agg_mode=mode)


@pytest.mark.parametrize("mode", ["smem", "global", "hot"])
def test_duplicate_keys_turn_the_direct_array_down(S, mode):
    """Dense keys with repeats: the build first takes the direct array, finds a duplicate,
    and every row then goes into the hash table (the fallback phase)."""
    fact, dim = rand_tables(5, 300_001, 3000, 0, 2000, -100, 2500, 40)
    check(S, fact, dim, "lt", 70, hint=40, agg_mode=mode)


@pytest.mark.parametrize("join_mode", ["auto", "hash"])
def test_sparse_keys_hash_table(S, join_mode):
    rng = np.random.default_rng(8)
    m = 20_000
    pk = rng.choice(2**31 - 1, size=m, replace=False).astype(np.int32) - 2**30
    dim = {"pk": pk, "grp": rng.integers(0, 900, size=m).astype(np.int32)}
    fk = pk[rng.integers(0, m, size=500_001)]
    fk[::3] = rng.integers(-2**31, 2**31 - 1, size=fk[::3].size)   # mostly absent keys
    fact = {"fk": fk, "pred": rng.integers(0, 100, size=fk.size).astype(np.int32),
            "val": rng.integers(-10**12, 10**12, size=fk.size)}
    check(S, fact, dim, "lt", 45, hint=900, join_mode=join_mode)


@pytest.mark.parametrize("mode", ["smem", "global", "hot"])
def test_two_column_keys(S, mode):
    spec = dg.plain_scale(n=700_001, m=30_000, composite=True)
    dim, fact = dg.gen_dim_host(spec), dg.gen_fact_host(spec)
    hint = 1000 if mode == "smem" else 100_000
    if mode == "smem":   # a group domain small enough for the per-block table (2049 slots)
        dim = dict(dim, grp=(dim["grp"] % 900).astype(np.int32))
    check(S, fact, dim, "lt", spec.t, hint=hint, agg_mode=mode)


def test_flag_group_keys(S):
    spec = dg.skewed(n=1_000_000, m=100_000)
    dim = dg.gen_dim_host(spec)
    fact = dg.gen_fact_host(spec, dim=dim)
    assert check(S, fact, dim, "lt", spec.t, aggs="sum,count", hint=spec.m) > 1000


@pytest.mark.parametrize("join_mode", ["auto", "hash"])
@pytest.mark.parametrize("bloom", ["off", "on"])
def test_dim_predicate(S, join_mode, bloom):
    spec = dg.plain_scale(n=1_000_003, m=60_000, dt=10)
    dim, fact = dg.gen_dim_host(spec), dg.gen_fact_host(spec)
    for dop, dt in (("lt", 10), ("ge", 50), ("lt", 0)):
        check(S, fact, dim, "lt", 30, 100_000, dim_op=dop, dim_literal=dt, join_mode=join_mode, bloom=bloom)


def test_empty_and_unmatched_inputs(S):
    spec = dg.StarSpec("t", n=1000, m=100, fk_domain=100, grp_bound=10, seed=6)
    dim, fact = dg.gen_dim_host(spec), dg.gen_fact_host(spec)
    assert check(S, fact, {k: v[:0] for k, v in dim.items()}, "lt", 50, 10) == 0
    assert check(S, {k: v[:0] for k, v in fact.items()}, dim, "lt", 50, 10) == 0
    assert check(S, fact, dict(dim, pk=dim["pk"] + 10_000), "lt", 50, 10) == 0
    assert check(S, fact, dim, "lt", 0, 10) == 0


def test_unaligned_columns(S):
    spec = dg.StarSpec("t", n=100_001, m=4000, fk_domain=4000, grp_bound=100, seed=7)
    dim, fact = dg.gen_dim_host(spec), dg.gen_fact_host(spec)
    d = dev(fact)
    shifted = {k: v[1:] for k, v in d.items()}   # 4-byte offsets: the scalar load path
    want = O.pipeline({k: v[1:] for k, v in fact.items()}, dim, "lt", 50)
    for variant in VARIANTS:
        got = S.run_pipeline(shifted, dev(dim), "lt", 50, group_cap_hint=100, probe_variant=variant)
        got = O.sort_groups({k: v.cpu().numpy() for k, v in got.items()})
        for c in COLS:
            assert np.array_equal(got[c], want[c]), (variant, c)


def test_group_table_full_and_output_capacity(S):
    spec = dg.skewed(n=200_000, m=40_000)
    dim = dg.gen_dim_host(spec)
    fact = dg.gen_fact_host(spec, dim=dim)
    df, dd = dev(fact), dev(dim)
    with pytest.raises(S.SiriusError) as e:
        S.run_pipeline(df, dd, "lt", 50, "sum,count", group_cap_hint=spec.m // 4, probe_variant="single")
    assert e.value.status == S.ERR_TABLE_FULL
    spec = dg.StarSpec("t", n=100_000, m=1000, fk_domain=1000, grp_bound=200, seed=8)
    dim, fact = dg.gen_dim_host(spec), dg.gen_fact_host(spec)
    with pytest.raises(S.SiriusError) as e:
        S.run_pipeline(dev(fact), dev(dim), "lt", 50, group_cap_hint=200, out_cap=10, probe_variant="single")
    assert e.value.status == S.ERR_CAPACITY and e.value.needed == 200


def test_default_takes_one_launch_and_large_queries_do_not(S):
    spec = dg.plain_small()
    dim, fact = dg.gen_dim_host(spec), dg.gen_fact_host(spec)
    df, dd = dev(fact), dev(dim)
    desc = S.make_desc(df, dd, "lt", spec.t, group_cap_hint=1000)
    outs = S.PipelineOutputs(1001)
    scratch = torch.empty(S.pipeline_scratch_bytes(desc), dtype=torch.uint8, device="cuda")
    S.sirius_run_pipeline(desc, outs, scratch)
    n0 = S.launch_count()
    g = S.sirius_run_pipeline(desc, outs, scratch)
    assert S.launch_count() - n0 == 1 and g == 1000
    desc = S.make_desc(df, dd, "lt", spec.t, group_cap_hint=1000, probe_variant="direct")
    n0 = S.launch_count()
    S.sirius_run_pipeline(desc, outs, scratch)
    assert S.launch_count() - n0 > 1


def test_replayed_from_a_cuda_graph(S):
    """Captured once (clear of the run header + the cooperative launch), replayed three times
    over inputs changed in place between replays: each replay equals the oracle."""
    spec = dg.StarSpec("t", n=300_001, m=20_000, fk_domain=21_000, grp_bound=700, t=40, seed=19)
    dim, fact = dg.gen_dim_host(spec), dg.gen_fact_host(spec)
    df, dd = dev(fact), dev(dim)
    desc = S.make_desc(df, dd, "lt", spec.t, group_cap_hint=700, probe_variant="single")
    outs = S.PipelineOutputs(1000)
    scratch = torch.empty(S.pipeline_scratch_bytes(desc), dtype=torch.uint8, device="cuda")
    cs = torch.cuda.Stream()
    cs.wait_stream(torch.cuda.current_stream())
    S.sirius_run_pipeline(desc, outs, scratch, cs, sync=False)
    cs.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=cs):
        S.sirius_run_pipeline(desc, outs, scratch, cs, sync=False)
    rng = np.random.default_rng(3)
    for rep in range(3):
        pred = rng.integers(0, 100, size=spec.n).astype(np.int32)
        df["pred"].copy_(torch.from_numpy(pred))
        torch.cuda.synchronize()
        graph.replay()
        torch.cuda.synchronize()
        assert int(outs.d_status.item()) == 0
        g = int(outs.d_groups.item())
        got = O.sort_groups({k: v.cpu().numpy() for k, v in outs.trimmed(g).items()})
        want = O.pipeline(dict(fact, pred=pred), dim, "lt", spec.t)
        for c in COLS:
            assert np.array_equal(got[c], want[c]), (rep, c)


@pytest.mark.parametrize("case", ["range_at_limit", "range_past_limit", "distinct_past_limit"])
def test_group_key_range_at_the_direct_slot_limit(S, case):
    """Group keys whose range spans exactly the group table's limit of distinct keys take
    direct slots (slot = key - min); a range one past it takes the hash table (same distinct
    count, one value skipped); one distinct key past the limit fails with TABLE_FULL on both
    paths, as it does through the hash table."""
    hint = 1000
    cap = int(S.lib().sirius_groupby_capacity(hint))
    limit = cap - cap // 8
    base = -12_345
    if case == "range_at_limit":
        keys = base + np.arange(limit)
    elif case == "range_past_limit":
        keys = base + np.concatenate([np.arange(limit - 1), [limit]])
    else:
        keys = base + np.arange(limit + 1)
    rng = np.random.default_rng(len(case))
    m = 4 * len(keys)
    dim = {"pk": rng.permutation(m).astype(np.int32), "grp": np.tile(keys, 4).astype(np.int32)}
    fact = {"fk": rng.integers(0, m, size=400_001).astype(np.int32),
            "pred": rng.integers(0, 100, size=400_001).astype(np.int32),
            "val": rng.integers(-10**9, 10**9, size=400_001)}
    if case == "distinct_past_limit":
        for variant in VARIANTS:
            with pytest.raises(S.SiriusError) as e:
                S.run_pipeline(dev(fact), dev(dim), "lt", 50, group_cap_hint=hint, out_cap=cap,
                               probe_variant=variant)
            assert e.value.status == S.ERR_TABLE_FULL, variant
        return
    assert check(S, fact, dim, "lt", 50, hint, out_cap=cap) == limit


def test_autotuner_weighs_the_single_launch(S):
    """tune_pipeline times the single launch beside the per-phase kernels and the staged probe;
    the settings it keeps give the oracle's result."""
    from paper_2508_04701_gb300 import autotune
    spec = dg.StarSpec("t", n=1_000_003, m=65_536, fk_domain=65_536, grp_bound=1000, t=50, seed=23)
    dim, fact = dg.gen_dim_host(spec), dg.gen_fact_host(spec)
    desc = S.make_desc(dev(fact), dev(dim), "lt", spec.t, group_cap_hint=1000)
    outs = S.PipelineOutputs(1001)
    best = autotune.tune_pipeline(desc, outs, load_factors=(0.5,))
    assert {t["probe_variant"] for t in best["all"]} == {"single", "direct", "staged"}
    assert desc.probe_variant == S.PROBE_VARIANTS[best["probe_variant"]]
    scratch = torch.empty(S.pipeline_scratch_bytes(desc), dtype=torch.uint8, device="cuda")
    g = S.sirius_run_pipeline(desc, outs, scratch)
    got = O.sort_groups({k: v.cpu().numpy() for k, v in outs.trimmed(g).items()})
    want = O.pipeline(fact, dim, "lt", spec.t)
    for c in COLS:
        assert np.array_equal(got[c], want[c]), c
