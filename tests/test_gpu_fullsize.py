"""Parity at the full sizes of the measured workloads, in the launch configuration bench.py
times (default agg_mode / probe variant, the bench's group_cap_hint).

The oracle cannot run the whole 600M-row query in a test's time, so each check is made
where it can compute exactly:
  * sampled groups -- the fact rows whose join key belongs to a sampled set of groups (hot
    and random ones) and whose predicate holds are selected on the host, and the oracle
    computes those groups from them: dropping rows of other groups, or rows the filter
    rejects, does not change the sampled groups' results;
  * totals over all groups -- every fk of these workloads matches a dim key, so
    sum(COUNT) = #(pred < t) and sum(SUM) = the total of val over those rows;
  * per-group invariants: COUNT * MIN <= SUM <= COUNT * MAX.
Inputs come from the seeded generator's CUDA twin (bit-identical to datagen's host
generator, tests/test_gpu_datagen.py) and are read back in chunks.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2508_04701_gb300 import datagen as dg

pytestmark = pytest.mark.gpu

CHUNK = 50_000_000
COLS = ("key", "sum", "count", "min", "max")


@pytest.fixture(scope="module")
def S():
    from paper_2508_04701_gb300 import build
    build.build()
    from paper_2508_04701_gb300 import sirius
    sirius.lib()
    return sirius


def host(d, lo=None, hi=None):
    return {k: (v[lo:hi] if lo is not None else v).cpu().numpy() for k, v in d.items()}


def run_bench_config(S, spec, fact, dim, hint):
    desc = S.make_desc(fact, dim, "lt", spec.t, spec.aggs, hint)
    outs = S.PipelineOutputs(hint + 1)
    scratch = torch.empty(S.pipeline_scratch_bytes(desc), dtype=torch.uint8, device="cuda")
    g = S.sirius_run_pipeline(desc, outs, scratch)
    got = {k: v.cpu().numpy() for k, v in outs.trimmed(g).items()}
    return g, got


def group_keys(dim):
    return O.pack_group(dim["grp"], dim.get("flag"))


def check_sampled_and_totals(S, spec, hint, sample_rows, packed_keys=False):
    dim_d = dg.gen_dim_device(spec)
    fact_d = dg.gen_fact_device(spec, dim_d)
    g, got = run_bench_config(S, spec, fact_d, dim_d, hint)
    dim = host(dim_d)
    gkey = group_keys(dim)
    sample = np.unique(gkey[sample_rows])
    sel = np.isin(gkey, sample)
    dim_sub = {k: v[sel] for k, v in dim.items()}
    if packed_keys:
        want_keys = np.sort(O.pack_composite(dim_sub["pk_hi"], dim_sub["pk"]))
    else:
        lut = np.zeros(spec.m, dtype=bool)   # dim pk is a permutation of [0, m)
        lut[dim_sub["pk"]] = True
    parts, n_sel, v_sel = [], 0, 0
    for lo in range(0, spec.n, CHUNK):
        f = host(fact_d, lo, min(spec.n, lo + CHUNK))
        m = f["pred"] < spec.t
        n_sel += int(m.sum())
        v_sel += int(f["val"][m].sum())
        if packed_keys:
            k = O.pack_composite(f["fk_hi"], f["fk"])
            pos = np.minimum(np.searchsorted(want_keys, k), want_keys.size - 1)
            keep = want_keys[pos] == k
        else:
            keep = lut[f["fk"]]
        parts.append({c: v[keep & m] for c, v in f.items()})
    del fact_d
    fact_sub = {c: np.concatenate([p[c] for p in parts]) for c in parts[0]}
    want = O.pipeline(fact_sub, dim_sub, "lt", spec.t)
    # sampled groups: exact
    idx = np.isin(got["key"], sample)
    mine = O.sort_groups({c: got[c][idx] for c in got})
    assert want["key"].size > 0
    for c in ["key", "count"] + [a for a in ("sum", "min", "max") if a in spec.aggs]:
        assert np.array_equal(mine[c], want[c]), c
    # totals over all groups
    assert int(got["count"].sum()) == n_sel
    if "sum" in spec.aggs:
        assert sum(int(x) for x in got["sum"]) == v_sel
    if "min" in spec.aggs:
        c, s = got["count"].astype(object), got["sum"].astype(object)
        assert all(c * got["min"].astype(object) <= s) and all(s <= c * got["max"].astype(object))
    assert len(np.unique(got["key"])) == g
    return g


def test_plain_600M(S):
    """600M fact rows / 15M dim rows / 100 000 groups, pred < 30 (the bench's main line)."""
    spec = dg.plain_scale()
    rng = np.random.default_rng(11)
    g = check_sampled_and_totals(S, spec, 100_000, rng.integers(0, spec.m, size=16))
    assert g == 100_000


def test_plain_600M_composite_keys(S):
    """The same query on two-column join keys (hash-table join at full size)."""
    spec = dg.plain_scale(composite=True)
    rng = np.random.default_rng(12)
    g = check_sampled_and_totals(S, spec, 100_000, rng.integers(0, spec.m, size=16), packed_keys=True)
    assert g == 100_000


def test_skewed_300M(S):
    """300M Zipf(1.1) fact rows over 10M dim keys, (grp, flag) groups: the four hottest dim
    rows' groups (a fifth of all rows) and twelve random ones."""
    spec = dg.skewed()
    rng = np.random.default_rng(13)
    rows = np.concatenate([np.arange(4), rng.integers(4, spec.m, size=12)])
    check_sampled_and_totals(S, spec, spec.m, rows)


def test_batch_512_sampled_queries(S):
    """The 512-query batch as the bench runs it (one plan, CUDA graph); the smallest, the
    largest and four random queries checked in full against the oracle."""
    specs = [dg.batch_query(q) for q in range(512)]
    tabs = []
    for sp in specs:
        d = dg.gen_dim_device(sp)
        tabs.append((d, dg.gen_fact_device(sp, d)))
    descs = [S.make_desc(f, d, "lt", sp.t, "sum,count,min,max", 1000) for sp, (d, f) in zip(specs, tabs)]
    cap = S.lib().sirius_groupby_capacity(1000) + 1
    outs = [S.PipelineOutputs(cap) for _ in specs]
    plan = S.BatchPlan(512)
    scratch = torch.empty(S.batch_scratch_bytes(descs), dtype=torch.uint8, device="cuda")
    g = plan.run(descs, outs, scratch=scratch, use_graph=True)
    sizes = np.array([sp.n for sp in specs])
    rng = np.random.default_rng(14)
    pick = {int(sizes.argmin()), int(sizes.argmax())} | set(int(x) for x in rng.integers(0, 512, size=4))
    for q in sorted(pick):
        d, f = tabs[q]
        got = O.sort_groups({k: v.cpu().numpy() for k, v in outs[q].trimmed(g[q]).items()})
        want = O.pipeline(host(f), host(d), "lt", specs[q].t)
        for c in COLS:
            assert np.array_equal(got[c], want[c]), (q, c)
    plan.close()
