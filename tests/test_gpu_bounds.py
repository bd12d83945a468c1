"""Parity of the bound filter (agg_mode 6: the hot-group cache plus, per group slot, shared-memory
bytes that bound MAX from below and MIN from above, so that rows which cannot move an extreme
skip its L2 reduction) with the CPU oracle, bit-exact after sorting groups by key (GPU).

The filter only decides which reductions are skipped, so the cases aim at the decisions: value
orders that move the bounds on every row (ascending, descending) or never (all equal), scales
the first rows misjudge (a narrow start, then values far outside it; int64's edges), group
tables larger than the filter (slots above it go unfiltered), each subset of MIN and MAX, skew
that lands in the hot-group cache, and the entry points and join forms that run the probe pass."""
import dataclasses

import numpy as np
import pytest
import torch

import oracle as O
from paper_2508_04701_gb300 import datagen as dg

pytestmark = pytest.mark.gpu

KW = dict(agg_mode="bounds", probe_variant="direct")   # per-phase kernels, bound filter


@pytest.fixture(scope="module")
def S():
    from paper_2508_04701_gb300 import build
    build.build()
    from paper_2508_04701_gb300 import sirius
    sirius.lib()
    return sirius


def dev(d):
    return {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in d.items()}


def compare(got, want, aggs="sum,count,min,max"):
    got = O.sort_groups({k: (v.cpu().numpy() if torch.is_tensor(v) else v) for k, v in got.items()})
    for c in ["key", "count"] + [a for a in ("sum", "min", "max") if a in aggs]:
        assert np.array_equal(got[c], want[c]), c


def check(S, fact, dim, op="lt", t=50, aggs="sum,count,min,max", hint=0, **kw):
    got = S.run_pipeline(dev(fact), dev(dim), op, t, aggs, hint, **{**KW, **kw})
    want = O.pipeline(fact, dim, op, t)
    compare(got, want, aggs)
    return want["key"].size


def star(m, n, groups, seed, vals=None):
    """A dim of m rows (pk a permutation, grp uniform over `groups`) and n fact rows."""
    rng = np.random.default_rng(seed)
    dim = {"pk": rng.permutation(m).astype(np.int32),
           "grp": rng.integers(0, groups, size=m).astype(np.int32)}
    fact = {"fk": rng.integers(0, m, size=n).astype(np.int32),
            "pred": rng.integers(0, 100, size=n).astype(np.int32),
            "val": rng.integers(0, 10**8, size=n) if vals is None else vals}
    return dim, fact


def test_mode_is_accepted_and_needs_no_scratch(S):
    """Mode 6 adds nothing to the scratch (its state lives in shared memory)."""
    spec = dg.plain_scale(n=1000, m=5000)
    f, d = dev(dg.gen_fact_host(spec)), dev(dg.gen_dim_host(spec))
    b = S.pipeline_scratch_bytes(S.make_desc(f, d, "lt", 30, group_cap_hint=100_000, **KW))
    h = S.pipeline_scratch_bytes(S.make_desc(f, d, "lt", 30, group_cap_hint=100_000, agg_mode="hot"))
    assert b == h


@pytest.mark.parametrize("n", [1, 3, 4, 5, 2047, 2048, 2049, 100_003, 1_000_003])
def test_ragged_sizes(S, n):
    spec = dg.plain_scale(n=n, m=150_000, seed=n % 5)
    dim, fact = dg.gen_dim_host(spec), dg.gen_fact_host(spec)
    check(S, fact, dim, "lt", spec.t, hint=100_000)


def test_many_blocks_against_chunked_oracle(S):
    """25M rows, 100 000 groups: every block's bounds tighten over ~20 rows per group."""
    spec = dg.plain_scale(n=25_000_001, m=2_000_000, seed=3)
    want = O.query_results([spec], chunk_rows=5_000_000)[0]
    d = dg.gen_dim_device(spec)
    f = dg.gen_fact_device(spec, d)
    got = S.run_pipeline(f, d, "lt", spec.t, "sum,count,min,max", 100_000, **KW)
    compare(got, want)


@pytest.mark.parametrize("order", ["ascending", "descending", "equal", "alternating"])
def test_value_orders(S, order):
    """Ascending values move every MAX bound, descending ones every MIN bound; equal values
    share one code (the first rows' range is 0); alternating extremes hit both ends."""
    n = 3_000_001
    base = np.arange(n, dtype=np.int64) * 37 - 50_000_000
    vals = {"ascending": base, "descending": base[::-1].copy(), "equal": np.full(n, -7, np.int64),
            "alternating": np.where(np.arange(n) % 2 == 0, base, -base)}[order]
    dim, fact = star(60_000, n, 20_000, seed=21, vals=vals)
    check(S, fact, dim, "lt", 60, hint=20_000)


def test_scale_misjudged_by_the_first_rows(S):
    """The rows every block reads first (its first 4 x 512 rows, for up to 320 blocks) hold values
    in [0, 10); the rest span int64's edges: the codes clamp at both ends and the filter must
    still let every new extreme through."""
    n = 4_000_003
    rng = np.random.default_rng(22)
    vals = rng.integers(-10**18, 10**18, size=n)
    vals[rng.random(n) < 0.001] = np.iinfo(np.int64).max
    vals[rng.random(n) < 0.001] = np.iinfo(np.int64).min
    head = np.arange(n) < 2048 * 320
    vals[head] = rng.integers(0, 10, size=int(head.sum()))
    dim, fact = star(80_000, n, 50_000, seed=22, vals=vals)
    check(S, fact, dim, "lt", 70, hint=50_000)
    check(S, fact, dim, "ge", 0, hint=50_000)


@pytest.mark.parametrize("aggs", ["sum,count", "min", "max", "min,max", "sum,count,min"])
def test_aggregate_subsets(S, aggs):
    dim, fact = star(70_000, 2_000_003, 40_000, seed=23)
    check(S, fact, dim, "lt", 55, aggs=aggs, hint=40_000)


def test_group_table_larger_than_the_filter(S):
    """300 000 groups: direct slots above the filter's 102 400 go without bounds."""
    dim, fact = star(400_000, 6_000_001, 300_000, seed=24)
    check(S, fact, dim, "lt", 65, hint=300_000)


def test_hashed_group_slots(S):
    """Group keys spread over a wide range (no direct group slots): hashed slots, part of them
    above the filter."""
    rng = np.random.default_rng(25)
    m = 90_000
    dim = {"pk": rng.permutation(m).astype(np.int32),
           "grp": (rng.integers(0, 60_000, size=m) * 30_011 - 900_000_000).astype(np.int32)}
    n = 3_000_001
    fact = {"fk": rng.integers(0, m, size=n).astype(np.int32),
            "pred": rng.integers(0, 100, size=n).astype(np.int32), "val": rng.integers(-10**9, 10**9, size=n)}
    check(S, fact, dim, "lt", 50, hint=60_000)


def test_skew_in_the_hot_cache(S):
    """Nine in ten dim rows share one group: the hot-group cache takes it, the bounds the rest."""
    rng = np.random.default_rng(26)
    m = 50_000
    grp = np.zeros(m, dtype=np.int32)
    other = rng.random(m) < 0.1
    grp[other] = rng.integers(1, 20_000, size=int(other.sum())).astype(np.int32)
    dim = {"pk": rng.permutation(m).astype(np.int32), "grp": grp}
    n = 5_000_003
    vals = rng.integers(-10**12, 10**12, size=n)
    vals[:3] = [np.iinfo(np.int64).max // 8, np.iinfo(np.int64).min // 8, 0]
    fact = {"fk": rng.integers(0, m, size=n).astype(np.int32),
            "pred": rng.integers(0, 100, size=n).astype(np.int32), "val": vals}
    check(S, fact, dim, "lt", 70, hint=20_000)


def test_zipf_query(S):
    """The skewed recipe (Zipf(1.1) foreign keys, two-column group key) at 3M rows, with MIN
    and MAX asked for; and with SUM and COUNT only, where the launch keeps the plain cache."""
    spec = dataclasses.replace(dg.skewed(n=3_000_001, m=200_000, seed=27), aggs="sum,count,min,max")
    dim, fact = dg.gen_dim_host(spec), dg.gen_fact_host(spec)
    check(S, fact, dim, "lt", spec.t, hint=spec.m)
    check(S, fact, dim, "lt", spec.t, aggs="sum,count", hint=spec.m)


def test_duplicate_build_keys(S):
    rng = np.random.default_rng(28)
    m = 40_000
    dim = {"pk": rng.integers(0, 15_000, size=m).astype(np.int32),
           "grp": rng.integers(0, 30_000, size=m).astype(np.int32)}
    fact = {"fk": rng.integers(-50, 15_050, size=1_200_001).astype(np.int32),
            "pred": rng.integers(0, 100, size=1_200_001).astype(np.int32),
            "val": rng.integers(0, 10**8, size=1_200_001)}
    for jm in ("auto", "hash"):
        check(S, fact, dim, "lt", 55, hint=m, join_mode=jm)


@pytest.mark.parametrize("join_mode", ["auto", "hash"])
def test_two_column_keys_and_hash_join(S, join_mode):
    spec = dg.plain_scale(n=2_000_003, m=120_000, composite=True, seed=8)
    dim, fact = dg.gen_dim_host(spec), dg.gen_fact_host(spec)
    check(S, fact, dim, "lt", spec.t, hint=100_000, join_mode=join_mode)
    spec = dg.plain_scale(n=2_000_003, m=120_000, seed=9)
    dim, fact = dg.gen_dim_host(spec), dg.gen_fact_host(spec)
    check(S, fact, dim, "lt", spec.t, hint=100_000, join_mode=join_mode)


def test_unaligned_columns(S):
    """Columns one element past a 16-byte boundary: the scalar loads."""
    spec = dg.plain_scale(n=1_000_004, m=80_000, seed=10)
    dim, fact = dg.gen_dim_host(spec), dg.gen_fact_host(spec)
    df = {k: torch.from_numpy(v).cuda()[1:] for k, v in fact.items()}
    got = S.run_pipeline(df, dev(dim), "lt", spec.t, "sum,count,min,max", 100_000, **KW)
    want = O.pipeline({k: v[1:] for k, v in fact.items()}, dim, "lt", spec.t)
    compare(got, want)


def test_dim_predicate_with_bloom_filter(S):
    spec = dg.plain_scale(n=1_500_001, m=100_000, seed=11, dt=20)
    dim, fact = dg.gen_dim_host(spec), dg.gen_fact_host(spec)
    want = O.pipeline(fact, dim, "lt", spec.t, dim_op="lt", dim_literal=20)
    for jm in ("auto", "hash"):
        got = S.run_pipeline(dev(fact), dev(dim), "lt", spec.t, "sum,count,min,max", 100_000,
                             dim_op="lt", dim_literal=20, join_mode=jm, **KW)
        compare(got, want)


def test_star_query_takes_the_hot_cache(S):
    """A star query asked for mode 6 runs the star kernel with the plain hot-group cache."""
    spec = dg.StarSpec("star", n=700_003, m=40_000, fk_domain=40_000, grp_bound=100_000,
                       t=30, semi=2, semi_m=27_000, semi_t=60, seed=2)
    dim, fact, sd = dg.gen_dim_host(spec), dg.gen_fact_host(spec), dg.gen_semi_dims_host(spec)
    semi = dg.semi_args(spec, fact, sd)
    dsemi = [dict(sj, fk=dev({"k": sj["fk"]})["k"], dim=dev(sj["dim"])) for sj in semi]
    got = S.run_pipeline(dev(fact), dev(dim), "lt", 30, "sum,count,min,max", 100_000, semi=dsemi, **KW)
    compare(got, O.pipeline(fact, dim, "lt", 30, semi=semi))


def test_resident_index_and_host_columns(S):
    """The probe pass behind sirius_run_probe (resident dim index) and behind
    sirius_run_pipeline_host (chunks of host columns)."""
    spec = dg.plain_scale(n=3_000_001, m=150_000, seed=12)
    dim, fact = dg.gen_dim_host(spec), dg.gen_fact_host(spec)
    want = O.pipeline(fact, dim, "lt", spec.t)
    ddim, dfact = dev(dim), dev(fact)
    desc = S.make_desc(dfact, ddim, "lt", spec.t, group_cap_hint=100_000, **KW)
    idx = S.sirius_dim_index_build(desc)
    outs = S.PipelineOutputs(S.lib().sirius_groupby_capacity(100_000) + 1)
    for _ in range(2):
        g = S.sirius_run_probe(desc, idx, outs)
        compare(outs.trimmed(g), want)
    hf = S.pinned_copy(dfact)
    hd = S.pinned_copy(ddim)
    hdesc = S.make_desc(hf, hd, "lt", spec.t, group_cap_hint=100_000, host=True, **KW)
    houts = S.HostOutputs(S.lib().sirius_groupby_capacity(100_000) + 1)
    for chunk in (1 << 20, 0, -1):   # staged chunks, the default chunk, in-place reads
        scratch = torch.empty(S.pipeline_host_scratch_bytes(hdesc, chunk, houts.cap), dtype=torch.uint8,
                              device="cuda")
        g = S.sirius_run_pipeline_host(hdesc, houts, chunk, scratch)
        compare({k: v[:g] for k, v in houts.t.items()}, want)


@pytest.mark.parametrize("bt,bps", [(256, 1), (512, 1), (128, 2)])
def test_launch_shapes(S, bt, bps):
    dim, fact = star(100_000, 2_000_003, 100_000, seed=30)
    check(S, fact, dim, "lt", 50, hint=100_000, block_threads=bt, blocks_per_sm=bps)
