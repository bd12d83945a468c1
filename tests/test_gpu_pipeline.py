"""Parity of the fused pipeline (build -> filter/probe/aggregate -> finalize) with the CPU
oracle, bit-exact after sorting groups by key (GPU)."""
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


def run(S, fact, dim, op="lt", t=50, aggs="sum,count,min,max", hint=0, **kw):
    got = S.run_pipeline(dev(fact), dev(dim), op, t, aggs, hint, **kw)
    torch.cuda.synchronize()
    return O.sort_groups({k: v.cpu().numpy() for k, v in got.items()})


def check(S, fact, dim, op="lt", t=50, aggs="sum,count,min,max", hint=0, **kw):
    got = run(S, fact, dim, op, t, aggs, hint, **kw)
    want = O.pipeline(fact, dim, op, t)
    for c in ["key", "count"] + [a for a in ("sum", "min", "max") if a in aggs]:
        assert np.array_equal(got[c], want[c]), c
    return want["key"].size


def test_plain_small_full_size(S):
    """The 1M-row fact / 65 536-row dim / 1 000-group query at its full size."""
    spec = dg.plain_small()
    dim, fact = dg.gen_dim_host(spec), dg.gen_fact_host(spec)
    assert check(S, fact, dim, "lt", spec.t, hint=spec.grp_bound) == 1000


@pytest.mark.parametrize("mode", ["smem", "global"])
@pytest.mark.parametrize("n", [1, 3, 4, 5, 1023, 100_003])
def test_ragged_sizes_both_agg_modes(S, mode, n):
    spec = dg.StarSpec("t", n=n, m=3001, fk_domain=3500, grp_bound=300, t=60, seed=n)
    dim, fact = dg.gen_dim_host(spec), dg.gen_fact_host(spec)
    check(S, fact, dim, "lt", spec.t, hint=300, agg_mode=mode)


@pytest.mark.parametrize("t", [0, 1, 99, 100])
def test_selectivity_edges(S, t):
    spec = dg.StarSpec("t", n=200_001, m=5000, fk_domain=5000, grp_bound=50, t=t, seed=3)
    dim, fact = dg.gen_dim_host(spec), dg.gen_fact_host(spec)
    check(S, fact, dim, "lt", t, hint=50)


@pytest.mark.parametrize("op", O.OPS)
def test_comparison_ops(S, op):
    spec = dg.StarSpec("t", n=50_000, m=2000, fk_domain=2000, grp_bound=40, seed=4)
    dim, fact = dg.gen_dim_host(spec), dg.gen_fact_host(spec)
    check(S, fact, dim, op, 50, hint=40)


@pytest.mark.parametrize("lf", [0.3, 0.5, 0.8, 0.95])
def test_load_factors(S, lf):
    spec = dg.plain_scale(n=400_000, m=150_000)
    dim, fact = dg.gen_dim_host(spec), dg.gen_fact_host(spec)
    check(S, fact, dim, "lt", spec.t, hint=100_000, load_factor=lf)


def test_scale_shape_small(S):
    """The 600M-row query's distributions at 1/300 of its size (100 000 groups, global path)."""
    spec = dg.plain_scale(n=2_000_000, m=50_000)
    dim, fact = dg.gen_dim_host(spec), dg.gen_fact_host(spec)
    check(S, fact, dim, "lt", spec.t, hint=100_000)


def test_composite_keys(S):
    spec = dg.plain_scale(n=1_000_003, m=40_000, composite=True)
    dim, fact = dg.gen_dim_host(spec), dg.gen_fact_host(spec)
    check(S, fact, dim, "lt", spec.t, hint=100_000)


def test_skewed_flag_groups(S):
    spec = dg.skewed(n=1_000_000, m=100_000)
    dim = dg.gen_dim_host(spec)
    fact = dg.gen_fact_host(spec, dim=dim)
    g = check(S, fact, dim, "lt", spec.t, aggs="sum,count", hint=spec.m)
    assert g > 1000


def test_duplicate_dim_keys_and_misses(S):
    rng = np.random.default_rng(5)
    m = 3000
    dim = {"pk": rng.integers(0, 2000, size=m).astype(np.int32),
           "grp": rng.integers(-5, 30, size=m).astype(np.int32)}
    fact = {"fk": rng.integers(-100, 2500, size=300_001).astype(np.int32),
            "pred": rng.integers(0, 100, size=300_001).astype(np.int32),
            "val": rng.integers(-10**9, 10**9, size=300_001)}
    for mode in ("smem", "global"):
        check(S, fact, dim, "lt", 70, hint=35, agg_mode=mode)


def test_empty_inputs(S):
    spec = dg.StarSpec("t", n=1000, m=100, fk_domain=100, grp_bound=10, seed=6)
    dim, fact = dg.gen_dim_host(spec), dg.gen_fact_host(spec)
    empty_dim = {k: v[:0] for k, v in dim.items()}
    empty_fact = {k: v[:0] for k, v in fact.items()}
    assert run(S, fact, empty_dim, hint=10)["key"].size == 0
    assert run(S, empty_fact, dim, hint=10)["key"].size == 0
    miss = dict(dim, pk=dim["pk"] + 10_000)
    assert run(S, fact, miss, hint=10)["key"].size == 0


def test_unaligned_columns(S):
    spec = dg.StarSpec("t", n=100_001, m=4000, fk_domain=4000, grp_bound=100, seed=7)
    dim, fact = dg.gen_dim_host(spec), dg.gen_fact_host(spec)
    d = dev(fact)
    shifted = {k: v[1:] for k, v in d.items()}   # 4-byte offsets: the scalar load path
    got = S.run_pipeline(shifted, dev(dim), "lt", 50, group_cap_hint=100)
    got = O.sort_groups({k: v.cpu().numpy() for k, v in got.items()})
    want = O.pipeline({k: v[1:] for k, v in fact.items()}, dim, "lt", 50)
    for c in COLS:
        assert np.array_equal(got[c], want[c]), c


def test_group_table_full_then_retry(S):
    spec = dg.skewed(n=200_000, m=40_000)
    dim = dg.gen_dim_host(spec)
    fact = dg.gen_fact_host(spec, dim=dim)
    with pytest.raises(S.SiriusError) as e:
        S.run_pipeline(dev(fact), dev(dim), "lt", 50, "sum,count", group_cap_hint=spec.m // 4)
    assert e.value.status == S.ERR_TABLE_FULL
    check(S, fact, dim, "lt", 50, aggs="sum,count", hint=spec.m)


def test_group_table_full_fails_promptly(S):
    """2M dim rows with 2M distinct group keys against a table sized for a quarter of them:
    past the limit, further keys must stop walking (a walk over the full 2^20-slot table for
    each of ~1M keys would take hours)."""
    import time
    m = 2_000_000
    rng = np.random.default_rng(17)
    dim = {"pk": rng.permutation(m).astype(np.int32), "grp": rng.permutation(m).astype(np.int32)}
    fact = {"fk": rng.integers(0, m, size=1_000_000).astype(np.int32),
            "pred": rng.integers(0, 100, size=1_000_000).astype(np.int32),
            "val": rng.integers(0, 10**8, size=1_000_000)}
    d, f = dev(dim), dev(fact)
    t0 = time.perf_counter()
    with pytest.raises(S.SiriusError) as e:
        S.run_pipeline(f, d, "lt", 50, "sum,count", group_cap_hint=m // 4)
    assert e.value.status == S.ERR_TABLE_FULL
    assert time.perf_counter() - t0 < 30.0
    check(S, fact, dim, "lt", 50, aggs="sum,count", hint=m)


def test_output_capacity(S):
    spec = dg.StarSpec("t", n=100_000, m=1000, fk_domain=1000, grp_bound=200, seed=8)
    dim, fact = dg.gen_dim_host(spec), dg.gen_fact_host(spec)
    with pytest.raises(S.SiriusError) as e:
        S.run_pipeline(dev(fact), dev(dim), "lt", 50, group_cap_hint=200, out_cap=10)
    assert e.value.status == S.ERR_CAPACITY and e.value.needed == 200


@pytest.mark.parametrize("variant", ["direct", "staged"])
@pytest.mark.parametrize("n", [1, 3, 4, 511, 512, 513, 4099, 1_000_003])
def test_probe_variants(S, variant, n):
    spec = dg.StarSpec("t", n=n, m=7001, fk_domain=7500, grp_bound=900, t=41, seed=n + 17)
    dim, fact = dg.gen_dim_host(spec), dg.gen_fact_host(spec)
    check(S, fact, dim, "lt", spec.t, hint=900, agg_mode="global", probe_variant=variant)


@pytest.mark.parametrize("lf", [0.5, 0.95])
def test_staged_probe_duplicates_composite_overflow(S, lf):
    """Full home buckets (load factor 0.95) force walks past the gathered bucket."""
    rng = np.random.default_rng(21)
    m = 20_000
    dim = {"pk": rng.integers(0, 9000, size=m).astype(np.int32),
           "grp": rng.integers(0, 3000, size=m).astype(np.int32)}
    fact = {"fk": rng.integers(-50, 9100, size=600_001).astype(np.int32),
            "pred": rng.integers(0, 100, size=600_001).astype(np.int32),
            "val": rng.integers(-10**9, 10**9, size=600_001)}
    check(S, fact, dim, "lt", 60, hint=3000, load_factor=lf, agg_mode="global", probe_variant="staged")
    spec = dg.plain_scale(n=700_001, m=30_000, composite=True)
    dim, fact = dg.gen_dim_host(spec), dg.gen_fact_host(spec)
    check(S, fact, dim, "lt", spec.t, hint=100_000, load_factor=lf, probe_variant="staged")


def _keys_case(case, rng, m):
    if case == "offset":
        return (rng.permutation(m) + 1_000_000_000).astype(np.int32), "direct"
    if case == "negative":
        return (rng.permutation(m) - 2**31).astype(np.int32), "direct"
    if case == "gaps":        # range 1.9 m, unique
        return rng.choice(int(1.9 * m), size=m, replace=False).astype(np.int32), "direct"
    if case == "too_sparse":  # range 3 m
        return rng.choice(3 * m, size=m, replace=False).astype(np.int32), "hash"
    if case == "dups_dense":  # dense range with repeated keys: falls back to the hash table
        return rng.integers(0, m // 2, size=m).astype(np.int32), "hash"
    if case == "extremes":    # INT32_MIN .. INT32_MIN + m and INT32_MAX at the top: sparse
        k = (np.arange(m) - 2**31).astype(np.int32)
        k[-1] = 2**31 - 1
        return k, "hash"
    raise ValueError(case)


@pytest.mark.parametrize("case", ["offset", "negative", "gaps", "too_sparse", "dups_dense", "extremes"])
@pytest.mark.parametrize("join_mode", ["auto", "hash"])
def test_direct_array_decision(S, case, join_mode):
    rng = np.random.default_rng(31)
    m = 50_000
    pk, kind = _keys_case(case, rng, m)
    dim = {"pk": pk, "grp": rng.integers(0, 700, size=m).astype(np.int32)}
    lo, hi = int(pk.min()), int(pk.max())
    fk = rng.integers(lo, hi + 1, size=400_003, dtype=np.int64)
    fk[::5] = pk[rng.integers(0, m, size=fk[::5].size)]
    fact = {"fk": fk.astype(np.int32), "pred": rng.integers(0, 100, size=fk.size).astype(np.int32),
            "val": rng.integers(-10**9, 10**9, size=fk.size)}
    dd, df = dev(dim), dev(fact)
    desc = S.make_desc(df, dd, "lt", 55, group_cap_hint=700, join_mode=join_mode)
    index = S.sirius_dim_index_build(desc)
    assert index.join_kind() == (kind if join_mode == "auto" else "hash")
    outs = S.PipelineOutputs(S.lib().sirius_groupby_capacity(700) + 1)
    g = S.sirius_run_probe(desc, index, outs)
    got = O.sort_groups({k: v.cpu().numpy() for k, v in outs.trimmed(g).items()})
    want = O.pipeline(fact, dim, "lt", 55)
    for c in COLS:
        assert np.array_equal(got[c], want[c]), c
    for mode in ("smem", "global"):   # the fused call takes the same decision
        check(S, fact, dim, "lt", 55, hint=700, agg_mode=mode, join_mode=join_mode)


@pytest.mark.parametrize("n", [1, 5, 4095, 4097, 1_000_003])
@pytest.mark.parametrize("join_mode", ["auto", "hash"])
def test_partitioned_aggregation(S, n, join_mode):
    """100 000 groups (262 145 slots, 65 partitions): tuples per 4096-row tile, then
    per-partition shared-memory aggregation."""
    spec = dg.plain_scale(n=n, m=60_000, seed=n % 7)
    dim, fact = dg.gen_dim_host(spec), dg.gen_fact_host(spec)
    check(S, fact, dim, "lt", spec.t, hint=100_000, agg_mode="part", join_mode=join_mode)


def test_partitioned_duplicates_composite_and_limits(S):
    rng = np.random.default_rng(41)
    m = 30_000
    dim = {"pk": rng.integers(0, 12_000, size=m).astype(np.int32),          # duplicate keys
           "grp": rng.integers(-500_000, 500_000, size=m).astype(np.int32)}  # ~30 000 groups
    fact = {"fk": rng.integers(-100, 12_100, size=900_001).astype(np.int32),
            "pred": rng.integers(0, 100, size=900_001).astype(np.int32),
            "val": rng.integers(-10**12, 10**12, size=900_001)}
    for jm in ("auto", "hash"):
        check(S, fact, dim, "lt", 65, hint=m, agg_mode="part", join_mode=jm)
    spec = dg.plain_scale(n=800_001, m=40_000, composite=True)
    dim, fact = dg.gen_dim_host(spec), dg.gen_fact_host(spec)
    check(S, fact, dim, "lt", spec.t, hint=100_000, agg_mode="part")
    # the largest group table the partitioned mode takes (hint 250 000: 2^19 + 1 slots, 129
    # partitions of 4096; 2^20 + 1 slots would be one over 256 x 4096) and one beyond it
    # (hint 600 000: plain reductions): both must give the same exact result
    rng = np.random.default_rng(42)
    dim = {"pk": rng.permutation(600_000).astype(np.int32),
           "grp": rng.integers(0, 200_000, size=600_000).astype(np.int32)}  # ~190 000 groups
    fact = {"fk": rng.integers(0, 600_000, size=2_000_003).astype(np.int32),
            "pred": rng.integers(0, 100, size=2_000_003).astype(np.int32),
            "val": rng.integers(0, 10**8, size=2_000_003)}
    check(S, fact, dim, "lt", 50, hint=250_000, agg_mode="part")
    check(S, fact, dim, "lt", 50, hint=600_000, agg_mode="part")


@pytest.mark.parametrize("mode", ["hot", "global", "part"])
def test_skewed_keys_all_large_table_modes(S, mode):
    """Zipf(1.1) keys: the hot-group cache, plain reductions and partitioned aggregation give
    the oracle's exact result."""
    spec = dg.skewed(n=1_500_001, m=200_000)
    dim = dg.gen_dim_host(spec)
    fact = dg.gen_fact_host(spec, dim=dim)
    check(S, fact, dim, "lt", spec.t, aggs="sum,count", hint=spec.m, agg_mode=mode)
    check(S, fact, dim, "ge", 80, hint=spec.m, agg_mode=mode)


def test_resident_dim_index_serves_many_probes(S):
    spec = dg.StarSpec("t", n=300_001, m=20_000, fk_domain=22_000, grp_bound=500, seed=9)
    dim = dg.gen_dim_host(spec)
    ddim = dev(dim)
    desc0 = S.make_desc(dev(dg.gen_fact_host(spec)), ddim, "lt", 50, group_cap_hint=500)
    index = S.sirius_dim_index_build(desc0)
    for seed, op, t in ((9, "lt", 50), (10, "ge", 20), (11, "ne", 3)):
        fs = dg.StarSpec("t", n=200_000 + seed, m=20_000, fk_domain=22_000, grp_bound=500, seed=seed)
        fact = dg.gen_fact_host(fs)
        dfact = dev(fact)
        desc = S.make_desc(dfact, ddim, op, t, group_cap_hint=500)
        outs = S.PipelineOutputs(600)
        g = S.sirius_run_probe(desc, index, outs)
        got = O.sort_groups({k: v.cpu().numpy() for k, v in outs.trimmed(g).items()})
        want = O.pipeline(fact, dim, op, t)
        for c in COLS:
            assert np.array_equal(got[c], want[c]), (seed, c)


def test_host_columns_in_place_need_pinned_memory(S):
    spec = dg.StarSpec("t", n=10_000, m=500, fk_domain=500, grp_bound=30, seed=14)
    dim, fact = dg.gen_dim_host(spec), dg.gen_fact_host(spec)
    hf = {k: torch.from_numpy(v) for k, v in fact.items()}          # pageable
    hd = {k: torch.from_numpy(v) for k, v in dim.items()}
    desc = S.make_desc(hf, hd, "lt", spec.t, group_cap_hint=30, host=True)
    with pytest.raises(S.SiriusError) as e:
        S.sirius_run_pipeline_host(desc, S.HostOutputs(64), -1)
    assert e.value.status == S.ERR_INVALID and "pinned" in str(e.value)


@pytest.mark.parametrize("chunk", [0, 4096, 10_000, 77_777, -1])
def test_host_columns_streamed_in_chunks(S, chunk):
    spec = dg.StarSpec("t", n=250_003, m=9000, fk_domain=9500, grp_bound=300, t=45, seed=12)
    dim, fact = dg.gen_dim_host(spec), dg.gen_fact_host(spec)
    hf = {k: torch.from_numpy(v).pin_memory() for k, v in fact.items()}
    hd = {k: torch.from_numpy(v).pin_memory() for k, v in dim.items()}
    desc = S.make_desc(hf, hd, "lt", spec.t, group_cap_hint=300, host=True)
    outs = S.HostOutputs(400)
    g = S.sirius_run_pipeline_host(desc, outs, chunk)
    got = O.sort_groups({k: v.numpy() for k, v in outs.trimmed(g).items()})
    want = O.pipeline(fact, dim, "lt", spec.t)
    for c in COLS:
        assert np.array_equal(got[c], want[c]), c


def test_host_columns_composite_and_flag(S):
    spec = dg.StarSpec("t", n=120_001, m=5000, fk_domain=5000, t=60, composite=True, group_flag=True,
                       seed=13)
    dim, fact = dg.gen_dim_host(spec), dg.gen_fact_host(spec)
    hf = {k: torch.from_numpy(v) for k, v in fact.items()}       # pageable host memory works too
    hd = {k: torch.from_numpy(v) for k, v in dim.items()}
    desc = S.make_desc(hf, hd, "lt", spec.t, group_cap_hint=5000, host=True)
    outs = S.HostOutputs(5001)
    g = S.sirius_run_pipeline_host(desc, outs, 30_000)
    got = O.sort_groups({k: v.numpy() for k, v in outs.trimmed(g).items()})
    want = O.pipeline(fact, dim, "lt", spec.t)
    for c in COLS:
        assert np.array_equal(got[c], want[c]), c


def test_repeatable_across_block_shapes(S):
    spec = dg.plain_scale(n=500_000, m=20_000)
    dim, fact = dg.gen_dim_host(spec), dg.gen_fact_host(spec)
    ref = run(S, fact, dim, "lt", 30, hint=100_000)
    for bt, bps in ((64, 1), (128, 3), (512, 1), (256, 0)):
        got = run(S, fact, dim, "lt", 30, hint=100_000, block_threads=bt, blocks_per_sm=bps)
        for c in COLS:
            assert np.array_equal(got[c], ref[c])


# ----------------------------------------------------------------------------- dim-side predicate
def check_dim_pred(S, fact, dim, op, t, dop, dt, hint, **kw):
    got = run(S, fact, dim, op, t, hint=hint, dim_op=dop, dim_literal=dt, **kw)
    want = O.pipeline(fact, dim, op, t, dim_op=dop, dim_literal=dt)
    for c in COLS:
        assert np.array_equal(got[c], want[c]), (dop, dt, kw, c)
    return want["key"].size


@pytest.mark.parametrize("join_mode", ["auto", "hash"])
@pytest.mark.parametrize("bloom", ["auto", "off", "on"])
def test_dim_predicate(S, join_mode, bloom):
    """Predicate transfer: only dim rows with dattr < 10 take part (direct array and hash
    table, Bloom filter on and off); every operator once, and the edges none / all."""
    spec = dg.plain_scale(n=1_000_003, m=60_000, dt=10)
    dim, fact = dg.gen_dim_host(spec), dg.gen_fact_host(spec)
    assert check_dim_pred(S, fact, dim, "lt", 30, "lt", 10, 100_000, join_mode=join_mode, bloom=bloom) > 0
    for dop, dt in (("le", 3), ("gt", 90), ("ge", 50), ("eq", 7), ("ne", 7)):
        check_dim_pred(S, fact, dim, "lt", 30, dop, dt, 100_000, join_mode=join_mode, bloom=bloom)
    assert check_dim_pred(S, fact, dim, "lt", 30, "lt", 0, 100_000, join_mode=join_mode, bloom=bloom) == 0
    check_dim_pred(S, fact, dim, "lt", 30, "lt", 100, 100_000, join_mode=join_mode, bloom=bloom)


@pytest.mark.parametrize("bloom", ["off", "on"])
def test_dim_predicate_composite_duplicates_and_misses(S, bloom):
    """Two-column keys (hash table + filter), then duplicate keys and fact keys absent from the
    dim, both with a dim-side predicate."""
    spec = dg.plain_scale(n=700_001, m=30_000, composite=True, dt=25)
    dim, fact = dg.gen_dim_host(spec), dg.gen_fact_host(spec)
    check_dim_pred(S, fact, dim, "lt", 30, "lt", 25, 100_000, bloom=bloom)
    rng = np.random.default_rng(31)
    m = 20_000
    dim = {"pk": rng.integers(0, 12_000, size=m).astype(np.int32),        # duplicate keys
           "grp": rng.integers(0, 700, size=m).astype(np.int32),
           "dattr": rng.integers(0, 100, size=m).astype(np.int32)}
    fact = {"fk": rng.integers(-500, 15_000, size=900_001).astype(np.int32),  # many misses
            "pred": rng.integers(0, 100, size=900_001).astype(np.int32),
            "val": rng.integers(-10**12, 10**12, size=900_001)}
    for am in ("smem", "global", "hot"):
        check_dim_pred(S, fact, dim, "lt", 60, "ge", 40, 1000, bloom=bloom, agg_mode=am)


def test_dim_predicate_resident_index_and_host_columns(S):
    """A dim index built with a dim-side predicate (and its Bloom filter) serves several probe
    passes; the same query through pinned host columns."""
    spec = dg.plain_scale(n=400_003, m=25_000, composite=True, dt=15)
    dim, fact = dg.gen_dim_host(spec), dg.gen_fact_host(spec)
    ddim = dev(dim)
    desc0 = S.make_desc(dev(fact), ddim, "lt", 30, group_cap_hint=100_000, dim_op="lt", dim_literal=15)
    index = S.sirius_dim_index_build(desc0)
    assert index.struct.bloom_log2 > 0
    for op, t in (("lt", 30), ("ge", 80)):
        dfact = dev(fact)
        desc = S.make_desc(dfact, ddim, op, t, group_cap_hint=100_000, dim_op="lt", dim_literal=15)
        outs = S.PipelineOutputs(100_001)
        g = S.sirius_run_probe(desc, index, outs)
        got = O.sort_groups({k: v.cpu().numpy() for k, v in outs.trimmed(g).items()})
        want = O.pipeline(fact, dim, op, t, dim_op="lt", dim_literal=15)
        for c in COLS:
            assert np.array_equal(got[c], want[c]), (op, c)
    hf = {k: torch.from_numpy(v).pin_memory() for k, v in fact.items()}
    hd = {k: torch.from_numpy(v).pin_memory() for k, v in dim.items()}
    desc = S.make_desc(hf, hd, "lt", 30, group_cap_hint=100_000, host=True, dim_op="lt", dim_literal=15)
    outs = S.HostOutputs(100_001)
    g = S.sirius_run_pipeline_host(desc, outs, 100_000)
    got = O.sort_groups({k: v.numpy() for k, v in outs.trimmed(g).items()})
    want = O.pipeline(fact, dim, "lt", 30, dim_op="lt", dim_literal=15)
    for c in COLS:
        assert np.array_equal(got[c], want[c]), c


# ----------------------------------------------------------------------------- star queries
def star_check(S, fact, dim, semi, t=30, hint=100_000, **kw):
    dsemi = [dict(sj, fk=dev({"k": sj["fk"]})["k"], fk_hi=(dev({"k": sj["fk_hi"]})["k"] if sj.get("fk_hi") is not None else None),
                  dim=dev(sj["dim"])) for sj in semi]
    got = S.run_pipeline(dev(fact), dev(dim), "lt", t, "sum,count,min,max", hint, semi=dsemi, **kw)
    torch.cuda.synchronize()
    got = O.sort_groups({k: v.cpu().numpy() for k, v in got.items()})
    want = O.pipeline(fact, dim, "lt", t, dim_op=kw.get("dim_op"), dim_literal=kw.get("dim_literal", 0), semi=semi)
    for c in COLS:
        assert np.array_equal(got[c], want[c]), (kw, c)
    return want["key"].size


@pytest.mark.parametrize("nsemi", [1, 2, 3])
@pytest.mark.parametrize("agg_mode", ["auto", "smem", "global", "hot"])
def test_star_query(S, nsemi, agg_mode):
    """The fused pass with further dims joined as filters (bitmap membership: dense keys)."""
    groups = 1000 if agg_mode == "smem" else 100_000   # a 2049-slot table fits shared memory
    spec = dg.StarSpec("star", n=700_003, m=40_000, fk_domain=40_000, grp_bound=groups,
                       t=30, semi=nsemi, semi_m=25_000 + 1000 * nsemi, semi_t=60, seed=nsemi)
    dim, fact, sd = dg.gen_dim_host(spec), dg.gen_fact_host(spec), dg.gen_semi_dims_host(spec)
    assert star_check(S, fact, dim, dg.semi_args(spec, fact, sd), hint=groups, agg_mode=agg_mode) > 0


def test_star_query_hash_sets_composite_and_edges(S):
    """Filter dims whose keys need the hash set (sparse one-column keys, two-column keys, keys
    the fact never references, duplicates), no attr predicate, a predicate nothing passes, and
    a dim-side predicate with its Bloom filter on the main dim at the same time."""
    rng = np.random.default_rng(77)
    n, m = 500_003, 30_000
    fact = {"fk": rng.integers(0, m, size=n).astype(np.int32), "pred": rng.integers(0, 100, size=n).astype(np.int32),
            "val": rng.integers(-10**12, 10**12, size=n),
            "s0": rng.integers(-2**31, 2**31 - 1, size=n).astype(np.int32)}
    dim = {"pk": rng.permutation(m).astype(np.int32), "grp": rng.integers(0, 3000, size=m).astype(np.int32),
           "dattr": rng.integers(0, 100, size=m).astype(np.int32)}
    sparse = {"pk": np.concatenate([fact["s0"][:: 7][:20_000], rng.integers(-2**31, 2**31 - 1, size=5000)]).astype(np.int32),
              "attr": rng.integers(0, 100, size=25_000).astype(np.int32)}
    pool = rng.integers(-2**31, 2**31, size=(4000, 2)).astype(np.int64)
    fi = rng.integers(0, 6000, size=n) % 4000
    fact["w_lo"], fact["w_hi"] = pool[fi, 1].astype(np.int32), pool[fi, 0].astype(np.int32)
    wide = {"pk": pool[:2500, 1].astype(np.int32), "pk_hi": pool[:2500, 0].astype(np.int32),
            "attr": rng.integers(0, 100, size=2500).astype(np.int32)}
    wide_dups = {k: np.concatenate([v, v[:300]]) for k, v in wide.items()}
    s_sparse = {"fk": fact["s0"], "dim": sparse, "op": "lt", "literal": 70}
    s_wide = {"fk": fact["w_lo"], "fk_hi": fact["w_hi"], "dim": wide_dups, "op": "ge", "literal": 30}
    s_all = {"fk": fact["fk"], "dim": {"pk": dim["pk"]}, "op": "lt", "literal": 0}
    assert star_check(S, fact, dim, [s_sparse]) > 0
    assert star_check(S, fact, dim, [s_wide, s_sparse]) > 0
    assert star_check(S, fact, dim, [s_all, s_wide]) > 0
    none = {"fk": fact["fk"], "dim": {"pk": dim["pk"], "attr": dim["dattr"]}, "op": "lt", "literal": 0}
    assert star_check(S, fact, dim, [s_wide, none]) == 0
    for bloom in ("auto", "off"):
        star_check(S, fact, dim, [s_sparse], dim_op="lt", dim_literal=40, join_mode="hash", bloom=bloom)


def test_star_query_rejected_where_not_taken(S):
    spec = dg.star(n=10_000, m=2000)
    spec = dg.StarSpec(**{**spec.__dict__, "semi_m": 1000})
    dim, fact, sd = dg.gen_dim_host(spec), dg.gen_fact_host(spec), dg.gen_semi_dims_host(spec)
    semi = [dict(sj, fk=dev({"k": sj["fk"]})["k"], dim=dev(sj["dim"])) for sj in dg.semi_args(spec, fact, sd)]
    desc = S.make_desc(dev(fact), dev(dim), "lt", 30, group_cap_hint=100_000, semi=semi)
    outs = S.PipelineOutputs(100_001)
    plan = S.BatchPlan(1)
    with pytest.raises(S.SiriusError) as e:
        plan.run([desc], [outs])
    assert e.value.status == S.ERR_INVALID
    plan.close()
    index = S.sirius_dim_index_build(desc)
    with pytest.raises(S.SiriusError) as e:
        S.sirius_run_probe(desc, index, outs)
    assert e.value.status == S.ERR_INVALID
