"""Parity of the split probe pass with the CPU oracle, bit-exact after sorting groups by key (GPU).

Queries that ask for MIN or MAX can run their probe pass in two phases (split_probe "on" here;
by default only large queries with many rows per group slot do):
the first 1/16 of the rows aggregate in full, the extreme bounds are taken over the group table
(the smallest MAX and the largest MIN of the groups seen so far, and a bitmap of those groups),
and the remaining rows skip the MIN / MAX reductions the bounds rule out.  The cases aim at the
bounds' decisions: value orders that make them useless or decisive (ascending, descending,
alternating), groups that first appear after the split, a first phase that selects nothing,
each subset of MIN and MAX, skew that the hot-group cache takes, group slots beyond the bitmap,
two-column keys and the entry points that run the probe pass."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2508_04701_gb300 import datagen as dg

pytestmark = pytest.mark.gpu

N = 20_000_003
SPLIT = (N // 16) >> 2 << 2


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
    kw.setdefault("split_probe", "on")
    got = S.run_pipeline(dev(fact), dev(dim), op, t, aggs, hint, probe_variant="direct", **kw)
    want = O.pipeline(fact, dim, op, t)
    compare(got, want, aggs)
    return want["key"].size


def tables(m, groups, seed, vals=None, n=N):
    rng = np.random.default_rng(seed)
    dim = {"pk": rng.permutation(m).astype(np.int32),
           "grp": rng.integers(0, groups, size=m).astype(np.int32)}
    fact = {"fk": rng.integers(0, m, size=n).astype(np.int32),
            "pred": rng.integers(0, 100, size=n).astype(np.int32),
            "val": rng.integers(0, 10**8, size=n) if vals is None else vals}
    return dim, fact


@pytest.mark.parametrize("agg_mode", ["auto", "hot", "global"])
def test_uniform_groups(S, agg_mode):
    dim, fact = tables(1_000_000, 100_000, seed=1)
    check(S, fact, dim, "lt", 30, hint=100_000, agg_mode=agg_mode)


@pytest.mark.parametrize("order", ["ascending", "descending", "alternating"])
def test_value_orders(S, order):
    """Ascending values: every later row is above the first phase's MAX floor (no MAX skipped)
    and above its MIN ceiling (every MIN skipped); descending the reverse."""
    base = np.arange(N, dtype=np.int64) * 41 - 300_000_000
    vals = {"ascending": base, "descending": base[::-1].copy(),
            "alternating": np.where(np.arange(N) % 2 == 0, base, -base)}[order]
    dim, fact = tables(500_000, 50_000, seed=2, vals=vals)
    check(S, fact, dim, "lt", 40, hint=50_000)


def test_groups_first_seen_after_the_split(S):
    """Half the dim rows are referenced only after the split: their groups are not in the bitmap
    and keep every reduction, with values below the floor and above the ceiling."""
    rng = np.random.default_rng(3)
    m, groups = 400_000, 60_000
    dim = {"pk": rng.permutation(m).astype(np.int32),
           "grp": np.concatenate([rng.integers(0, groups // 2, size=m // 2),
                                  rng.integers(groups // 2, groups, size=m - m // 2)]).astype(np.int32)}
    early = np.flatnonzero(dim["grp"] < groups // 2)
    fk = np.empty(N, dtype=np.int32)
    fk[:SPLIT] = dim["pk"][rng.choice(early, size=SPLIT)]
    fk[SPLIT:] = dim["pk"][rng.choice(np.arange(m), size=N - SPLIT)]
    vals = rng.integers(-10**9, 10**9, size=N)
    vals[SPLIT:SPLIT + 1000] = rng.choice([-2 * 10**9, 2 * 10**9], size=1000)
    fact = {"fk": fk, "pred": rng.integers(0, 100, size=N).astype(np.int32), "val": vals}
    grp_of_pk = np.empty(m, dtype=np.int32)
    grp_of_pk[dim["pk"]] = dim["grp"]
    assert (grp_of_pk[fk[:SPLIT]] < groups // 2).all() and (grp_of_pk[fk[SPLIT:]] >= groups // 2).any()
    check(S, fact, dim, "lt", 60, hint=groups)


def test_first_phase_selects_nothing(S):
    dim, fact = tables(300_000, 30_000, seed=4)
    fact["pred"][:SPLIT + 5] = 99
    check(S, fact, dim, "lt", 50, hint=30_000)


@pytest.mark.parametrize("aggs", ["min", "max", "min,max", "sum,count,max"])
def test_aggregate_subsets(S, aggs):
    dim, fact = tables(600_000, 80_000, seed=5, vals=np.random.default_rng(55).integers(-10**15, 10**15, size=N))
    check(S, fact, dim, "lt", 35, aggs=aggs, hint=80_000)


def test_skew_in_the_hot_cache(S):
    """Nine in ten dim rows share one group: the hot-group cache takes it in both phases."""
    rng = np.random.default_rng(6)
    m = 200_000
    grp = np.zeros(m, dtype=np.int32)
    other = rng.random(m) < 0.1
    grp[other] = rng.integers(1, 20_000, size=int(other.sum())).astype(np.int32)
    dim = {"pk": rng.permutation(m).astype(np.int32), "grp": grp}
    vals = rng.integers(-10**10, 10**10, size=N)
    fact = {"fk": rng.integers(0, m, size=N).astype(np.int32),
            "pred": rng.integers(0, 100, size=N).astype(np.int32), "val": vals}
    check(S, fact, dim, "lt", 70, hint=20_000)


def test_zipf_recipe(S):
    spec = dg.skewed(n=N, m=2_000_000, seed=7)
    dim, fact = dg.gen_dim_host(spec), dg.gen_fact_host(spec)
    check(S, fact, dim, "lt", spec.t, hint=spec.m)


def test_slots_beyond_the_bitmap(S):
    """300 000 groups (direct slots up to 300 000): slots above 2^17 are not in the bitmap."""
    dim, fact = tables(2_000_000, 300_000, seed=8)
    check(S, fact, dim, "lt", 45, hint=300_000)


def test_hashed_group_slots_and_hash_join(S):
    rng = np.random.default_rng(9)
    m = 900_000
    dim = {"pk": (rng.permutation(m) * 7 + 3).astype(np.int32),          # sparse keys: hash table
           "grp": (rng.integers(0, 70_000, size=m) * 30_011 - 900_000_000).astype(np.int32)}
    fact = {"fk": dim["pk"][rng.integers(0, m, size=N)],
            "pred": rng.integers(0, 100, size=N).astype(np.int32), "val": rng.integers(-10**9, 10**9, size=N)}
    check(S, fact, dim, "lt", 50, hint=70_000)


def test_two_column_keys(S):
    spec = dg.plain_scale(n=N, m=1_000_000, composite=True, seed=10)
    dim, fact = dg.gen_dim_host(spec), dg.gen_fact_host(spec)
    check(S, fact, dim, "lt", spec.t, hint=100_000)


def test_dim_predicate_with_bloom_filter(S):
    spec = dg.plain_scale(n=N, m=1_000_000, seed=11, dt=20)
    dim, fact = dg.gen_dim_host(spec), dg.gen_fact_host(spec)
    want = O.pipeline(fact, dim, "lt", spec.t, dim_op="lt", dim_literal=20)
    for jm in ("auto", "hash"):
        got = S.run_pipeline(dev(fact), dev(dim), "lt", spec.t, "sum,count,min,max", 100_000,
                             dim_op="lt", dim_literal=20, join_mode=jm, probe_variant="direct",
                             split_probe="on")
        compare(got, want)


def test_resident_index_and_host_columns(S):
    spec = dg.plain_scale(n=N, m=1_500_000, seed=12)
    dim, fact = dg.gen_dim_host(spec), dg.gen_fact_host(spec)
    want = O.pipeline(fact, dim, "lt", spec.t)
    ddim, dfact = dev(dim), dev(fact)
    desc = S.make_desc(dfact, ddim, "lt", spec.t, group_cap_hint=100_000, split_probe="on")
    idx = S.sirius_dim_index_build(desc)
    outs = S.PipelineOutputs(S.lib().sirius_groupby_capacity(100_000) + 1)
    for _ in range(2):
        g = S.sirius_run_probe(desc, idx, outs)
        compare(outs.trimmed(g), want)
    hf = S.pinned_copy(dfact)
    hd = S.pinned_copy(ddim)
    hdesc = S.make_desc(hf, hd, "lt", spec.t, group_cap_hint=100_000, host=True, split_probe="on")
    houts = S.HostOutputs(S.lib().sirius_groupby_capacity(100_000) + 1)
    for chunk in (1 << 24, 0, -1):   # staged chunks, the default chunk, in-place reads
        scratch = torch.empty(S.pipeline_host_scratch_bytes(hdesc, chunk, houts.cap), dtype=torch.uint8,
                              device="cuda")
        g = S.sirius_run_pipeline_host(hdesc, houts, chunk, scratch)
        compare({k: v[:g] for k, v in houts.t.items()}, want)


def test_unaligned_columns(S):
    dim, fact = tables(500_000, 40_000, seed=13, n=N + 1)
    df = {k: torch.from_numpy(v).cuda()[1:] for k, v in fact.items()}
    got = S.run_pipeline(df, dev(dim), "lt", 50, "sum,count,min,max", 40_000, probe_variant="direct",
                         split_probe="on")
    compare(got, O.pipeline({k: v[1:] for k, v in fact.items()}, dim, "lt", 50))


@pytest.mark.parametrize("split", ["auto", "off", "on"])
def test_split_modes_agree_at_the_default_threshold(S, split):
    """At 2^26 + 5 rows and 1 000 groups (about 65 000 rows per slot) auto splits; every mode
    gives the oracle's result."""
    spec = dg.StarSpec("split_auto", n=(1 << 26) + 5, m=200_000, fk_domain=200_000, grp_bound=1000, t=40, seed=14)
    want = O.query_results([spec], chunk_rows=8_000_000)[0]
    d = dg.gen_dim_device(spec)
    f = dg.gen_fact_device(spec, d)
    got = S.run_pipeline(f, d, "lt", spec.t, "sum,count,min,max", 1000, probe_variant="direct", split_probe=split)
    compare(got, want)



def test_star_query_keeps_one_pass(S):
    """A star query asked for the split runs its probe in one pass (measured slower split: its
    pass is bound by the filter dims' dependent lookups); results as the oracle's."""
    spec = dg.StarSpec("star", n=N, m=1_000_000, fk_domain=1_000_000, grp_bound=100_000, t=30, semi=2,
                       semi_m=500_000, semi_t=50, seed=15)
    dim, fact, sd = dg.gen_dim_host(spec), dg.gen_fact_host(spec), dg.gen_semi_dims_host(spec)
    semi = dg.semi_args(spec, fact, sd)
    dsemi = [dict(sj, fk=dev({"k": sj["fk"]})["k"], dim=dev(sj["dim"])) for sj in semi]
    got = S.run_pipeline(dev(fact), dev(dim), "lt", 30, "sum,count,min,max", 100_000, semi=dsemi,
                         probe_variant="direct", split_probe="on")
    compare(got, O.pipeline(fact, dim, "lt", 30, semi=semi))
