"""Parity of the routed probe (agg_mode 5: group slots dealt out to the blocks of one
cooperative launch, joined rows sent to their owner through an exchange buffer, aggregated in
shared memory) with the CPU oracle, bit-exact after sorting groups by key (GPU).

Sizes span one partial round and several rounds of the exchange (a round covers 2048 rows per
tile x 16 tiles x every resident block, about 10M rows on GB300), ragged tails, a skew that
overflows the runs into the global reductions, duplicate build keys (the launch falls back to
global reductions), two-column keys, unaligned columns and the other entry points that run the
probe pass (resident dim index, host columns)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2508_04701_gb300 import datagen as dg

pytestmark = pytest.mark.gpu

COLS = ("key", "sum", "count", "min", "max")
KW = dict(agg_mode="routed", probe_variant="direct")   # per-phase kernels, routed probe


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


def test_routed_mode_is_taken(S):
    """The descriptor's mode 5 plans a routed run for a 100 000-group table: its scratch holds
    the exchange buffers (hundreds of MB beyond the hot-cache run's)."""
    spec = dg.plain_scale(n=1000, m=5000)
    f, d = dev(dg.gen_fact_host(spec)), dev(dg.gen_dim_host(spec))
    routed = S.pipeline_scratch_bytes(S.make_desc(f, d, "lt", 30, group_cap_hint=100_000, **KW))
    hot = S.pipeline_scratch_bytes(S.make_desc(f, d, "lt", 30, group_cap_hint=100_000, agg_mode="hot"))
    assert routed > hot + 100_000_000


@pytest.mark.parametrize("n", [1, 3, 4, 5, 2047, 2048, 2049, 100_003, 1_000_003])
def test_ragged_sizes(S, n):
    spec = dg.plain_scale(n=n, m=150_000, seed=n % 5)
    dim, fact = dg.gen_dim_host(spec), dg.gen_fact_host(spec)
    check(S, fact, dim, "lt", spec.t, hint=100_000)


def test_several_rounds_against_chunked_oracle(S):
    """25M rows: three rounds of the exchange, both buffers reused."""
    spec = dg.plain_scale(n=25_000_001, m=2_000_000, seed=3)
    want = O.query_results([spec], chunk_rows=5_000_000)[0]
    d = dg.gen_dim_device(spec)
    f = dg.gen_fact_device(spec, d)
    got = S.run_pipeline(f, d, "lt", spec.t, "sum,count,min,max", 100_000, **KW)
    compare(got, want)


@pytest.mark.parametrize("t", [0, 1, 100])
def test_selectivity_edges(S, t):
    spec = dg.plain_scale(n=700_001, m=60_000, seed=t)
    dim, fact = dg.gen_dim_host(spec), dg.gen_fact_host(spec)
    check(S, fact, dim, "lt", t, hint=100_000)


def test_skew_overflows_runs_into_global_reductions(S):
    """Nine in ten dim rows share one group: most joined rows go to one owner, whose runs fill
    up and send the rest to the global table; values of both signs at int64's edges."""
    rng = np.random.default_rng(5)
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
    check(S, fact, dim, "ge", 0, aggs="sum,count", hint=20_000)


def test_duplicate_build_keys_fall_back(S):
    rng = np.random.default_rng(6)
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


def test_resident_index_and_host_columns(S):
    """The probe pass behind sirius_run_probe (resident dim index) and behind
    sirius_run_pipeline_host (chunks of host columns: one routed launch per chunk)."""
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
