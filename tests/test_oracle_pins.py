"""Pins of the CPU oracle to things other than itself (CPU only, no GPU).

* brute force: Python-loop filter / nested-loop join / dict group-by on tiny random inputs;
* closed forms: a fact table with fk = i mod M, pred = i mod 100, val = i joined to a dim with
  pk = j, grp = j mod G has arithmetic-series aggregates per group;
* invariants: |filter| = #{pred < t}; join cardinality = sum over keys of
  count_probe(k) * count_build(k); sum of COUNT = join cardinality; sum of SUM = the filtered
  matched total; COUNT*MIN <= SUM <= COUNT*MAX;
* special cases: empty tables, t = 0, no key in the dim, a single group (plain Python
  sum / min / max / len), composite keys against Python tuples;
* planted mistakes: each check is run against a deliberately broken copy of the oracle and must
  fail, so a dropped term, a flipped comparison or a swapped operand cannot pass unseen.
"""
import types
from collections import Counter

import numpy as np
import pytest

import oracle as O
from paper_2508_04701_gb300 import datagen as dg


# ----------------------------------------------------------------------------- checks
def check_filter_brute(o, seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(0, 400))
    col = rng.integers(-5, 6, size=n).astype(np.int32)
    lit = int(rng.integers(-6, 7))
    for op in O.OPS:
        assert np.array_equal(o.filter_rows(col, op, lit), O.filter_rows_loop(col, op, lit)), op


def check_filter_closed_form(o):
    for n in (0, 1, 99, 100, 101, 12345):
        pred = (np.arange(n) % 100).astype(np.int32)
        for t in (0, 1, 50, 99, 100):
            ids = o.filter_rows(pred, "lt", t)
            want = (n // 100) * t + min(n % 100, t)
            assert ids.size == want
            assert np.all(np.diff(ids.astype(np.int64)) > 0)
            assert np.all(pred[ids] < t)


def check_join_brute(o, seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(0, 2000))
    m = int(rng.integers(0, 300))
    dom = int(rng.integers(1, 60))
    pk = rng.integers(-dom // 2, dom, size=n).astype(np.int64)
    bk = rng.integers(-dom // 2, dom, size=m).astype(np.int64)
    p, b = o.join_sorted(pk, bk)
    card = sum(c * Counter(bk.tolist())[k] for k, c in Counter(pk.tolist()).items())
    assert p.size == b.size == card
    if card:
        assert int(p.max()) < n and int(b.max()) < m
    if n * m <= 60_000:
        lp, lb = O.join_loop(pk, bk)
        assert np.array_equal(p, lp) and np.array_equal(b, lb)
    assert np.all(pk[p.astype(np.int64)] == bk[b.astype(np.int64)])


def check_groupby_brute(o, seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(0, 3000))
    keys = rng.integers(-20, 40, size=n).astype(np.int64)
    vals = rng.integers(-10**12, 10**12, size=n).astype(np.int64)
    r = o.groupby_agg(keys, vals)
    w = O.groupby_loop(keys, vals)
    for c in ("key", "sum", "count", "min", "max"):
        assert np.array_equal(r[c], w[c]), c


def check_groupby_single_group(o):
    rng = np.random.default_rng(5)
    vals = rng.integers(0, 10**8, size=10_000).astype(np.int64)
    r = o.groupby_agg(np.full(vals.size, 7), vals)
    py = [int(v) for v in vals]
    assert r["key"].tolist() == [7]
    assert r["sum"].tolist() == [sum(py)]
    assert r["count"].tolist() == [len(py)]
    assert r["min"].tolist() == [min(py)] and r["max"].tolist() == [max(py)]


def closed_form_tables(B, M, G):
    """fact: fk = i mod M, pred = i mod 100, val = i (n = 100 B); dim: pk = j, grp = j mod G."""
    n = 100 * B
    i = np.arange(n)
    fact = {"fk": (i % M).astype(np.int32), "pred": (i % 100).astype(np.int32),
            "val": i.astype(np.int64)}
    j = np.arange(M)
    dim = {"pk": j.astype(np.int32), "grp": (j % G).astype(np.int32)}
    return fact, dim


def closed_form_result(B, G, t):
    """With G | M and G | 100: row i = 100 b + r is in group g iff r < t and r = g (mod G).
    Over b = 0..B-1: COUNT = B |R|, SUM = 100 |R| B(B-1)/2 + B sum(R), MIN = min R,
    MAX = 100 (B-1) + max R, where R = {r < t : r = g mod G}."""
    out = {"key": [], "sum": [], "count": [], "min": [], "max": []}
    for g in range(G):
        R = list(range(g, t, G))
        if not R or B == 0:
            continue
        out["key"].append(g)
        out["count"].append(B * len(R))
        out["sum"].append(100 * len(R) * B * (B - 1) // 2 + B * sum(R))
        out["min"].append(min(R))
        out["max"].append(100 * (B - 1) + max(R))
    return {k: np.array(v, dtype=np.int64) for k, v in out.items()}


def check_pipeline_closed_form(o):
    for B, M, G in ((1, 20, 4), (7, 20, 4), (30, 50, 10), (13, 100, 25), (5, 60, 1)):
        fact, dim = closed_form_tables(B, M, G)
        for t in (0, 1, 50, 100):
            r = o.pipeline(fact, dim, "lt", t)
            w = closed_form_result(B, G, t)
            for c in ("key", "sum", "count", "min", "max"):
                assert np.array_equal(r[c], w[c]), (B, M, G, t, c)


def check_pipeline_invariants(o, seed):
    rng = np.random.default_rng(seed)
    n, m = int(rng.integers(0, 20_000)), int(rng.integers(0, 500))
    dom = max(1, int(m * rng.uniform(0.5, 2.0)))
    fact = {"fk": rng.integers(0, dom, size=n).astype(np.int32),
            "pred": rng.integers(0, 100, size=n).astype(np.int32),
            "val": rng.integers(0, 10**8, size=n).astype(np.int64)}
    dim = {"pk": rng.integers(0, dom, size=m).astype(np.int32),   # duplicates allowed
           "grp": rng.integers(0, 17, size=m).astype(np.int32)}
    t = int(rng.integers(0, 101))
    r = o.pipeline(fact, dim, "lt", t)
    sel = fact["pred"] < t
    cb = Counter(dim["pk"].tolist())
    mult = np.array([cb.get(int(k), 0) for k in fact["fk"]], dtype=np.int64)
    card = int(np.sum(mult[sel]))
    assert int(r["count"].sum()) == card
    assert int(r["sum"].sum()) == int(np.sum(fact["val"][sel] * mult[sel]))
    assert np.all(r["count"] * r["min"] <= r["sum"]) and np.all(r["sum"] <= r["count"] * r["max"])
    assert set(r["key"].tolist()) <= set(dim["grp"].tolist())
    assert np.all(np.diff(r["key"]) > 0)
    # against the brute-force pipeline on a prefix small enough for the nested loop
    k = min(n, 600)
    small = {c: v[:k] for c, v in fact.items()}
    rs, wl = o.pipeline(small, dim, "lt", t), O.pipeline(small, dim, "lt", t, join="loop")
    for c in ("key", "sum", "count", "min", "max"):
        assert np.array_equal(rs[c], wl[c]), c


def check_special_cases(o):
    fact, dim = closed_form_tables(3, 20, 4)
    empty_dim = {"pk": np.zeros(0, np.int32), "grp": np.zeros(0, np.int32)}
    empty_fact = {c: v[:0] for c, v in fact.items()}
    assert o.pipeline(fact, empty_dim, "lt", 50)["key"].size == 0
    assert o.pipeline(empty_fact, dim, "lt", 50)["key"].size == 0
    assert o.pipeline(fact, dim, "lt", 0)["key"].size == 0
    miss = dict(dim, pk=dim["pk"] + 1000)
    assert o.pipeline(fact, miss, "lt", 50)["key"].size == 0


def check_composite_and_group_keys(o, seed):
    rng = np.random.default_rng(seed)
    n, m = 3000, 200
    pool = rng.integers(-2**31, 2**31, size=(40, 2)).astype(np.int64)
    pool[0] = (-1, -1)
    pool[1] = (-2**31, 0)
    pool[2] = (0, -2**31)
    pool[3] = (2**31 - 1, -1)
    fi = rng.integers(0, 40, size=n)
    bi = rng.integers(0, 40, size=m)
    fact = {"fk_hi": pool[fi, 0].astype(np.int32), "fk": pool[fi, 1].astype(np.int32),
            "pred": rng.integers(0, 100, size=n).astype(np.int32),
            "val": rng.integers(0, 10**8, size=n).astype(np.int64)}
    dim = {"pk_hi": pool[bi, 0].astype(np.int32), "pk": pool[bi, 1].astype(np.int32),
           "grp": rng.integers(-3, 3, size=m).astype(np.int32),
           "flag": rng.integers(-128, 128, size=m).astype(np.int8)}
    r = o.pipeline(fact, dim, "lt", 60)
    # brute force on Python tuples: join on (hi, lo), group on (grp, flag)
    acc = {}
    by_key = {}
    for j in range(m):
        by_key.setdefault((int(dim["pk_hi"][j]), int(dim["pk"][j])), []).append(j)
    for i in range(n):
        if fact["pred"][i] >= 60:
            continue
        for j in by_key.get((int(fact["fk_hi"][i]), int(fact["fk"][i])), []):
            g = (int(dim["grp"][j]), int(dim["flag"][j]))
            v = int(fact["val"][i])
            a = acc.setdefault(g, [0, 0, v, v])
            a[0] += v; a[1] += 1; a[2] = min(a[2], v); a[3] = max(a[3], v)
    assert r["key"].size == len(acc)
    # decode the packed group key: grp = floor(key / 256), flag = key mod 256 as a signed byte
    for k, s, c, mn, mx in zip(r["key"], r["sum"], r["count"], r["min"], r["max"]):
        k = int(k)
        g = (k >> 8, ((k & 0xFF) ^ 0x80) - 0x80)
        assert g in acc, g
        assert acc[g] == [int(s), int(c), int(mn), int(mx)], g


def check_dim_predicate_brute(o, seed):
    """The dim-side predicate (predicate transfer): a Python triple loop over tiny tables with
    duplicate keys, misses and every comparison operator on both sides."""
    rng = np.random.default_rng(seed)
    n, m = int(rng.integers(0, 300)), int(rng.integers(0, 60))
    fact = {"fk": rng.integers(0, 50, size=n).astype(np.int32),
            "pred": rng.integers(0, 10, size=n).astype(np.int32),
            "val": rng.integers(-10**6, 10**6, size=n).astype(np.int64)}
    dim = {"pk": rng.integers(0, 40, size=m).astype(np.int32),
           "grp": rng.integers(0, 6, size=m).astype(np.int32),
           "dattr": rng.integers(0, 10, size=m).astype(np.int32)}
    cmp = {"lt": lambda a, b: a < b, "le": lambda a, b: a <= b, "gt": lambda a, b: a > b,
           "ge": lambda a, b: a >= b, "eq": lambda a, b: a == b, "ne": lambda a, b: a != b}
    for dop in O.OPS:
        op, t, dt = O.OPS[int(rng.integers(0, 6))], int(rng.integers(0, 11)), int(rng.integers(0, 11))
        acc = {}
        for i in range(n):
            if not cmp[op](int(fact["pred"][i]), t):
                continue
            for j in range(m):
                if int(dim["pk"][j]) != int(fact["fk"][i]) or not cmp[dop](int(dim["dattr"][j]), dt):
                    continue
                g, v = int(dim["grp"][j]), int(fact["val"][i])
                a = acc.setdefault(g, [0, 0, v, v])
                a[0] += v; a[1] += 1; a[2] = min(a[2], v); a[3] = max(a[3], v)
        r = o.pipeline(fact, dim, op, t, dim_op=dop, dim_literal=dt)
        assert r["key"].tolist() == sorted(acc), (dop, dt)
        for k, s_, c, mn, mx in zip(r["key"], r["sum"], r["count"], r["min"], r["max"]):
            assert acc[int(k)] == [int(s_), int(c), int(mn), int(mx)], (dop, dt, int(k))
    # a predicate every dim row passes changes nothing; one none passes empties the result
    whole = o.pipeline(fact, dim, "lt", 5)
    same = o.pipeline(fact, dim, "lt", 5, dim_op="lt", dim_literal=10)
    none = o.pipeline(fact, dim, "lt", 5, dim_op="lt", dim_literal=0)
    for c in ("key", "sum", "count", "min", "max"):
        assert np.array_equal(whole[c], same[c])
    assert none["key"].size == 0


def check_semi_brute(o, seed):
    """Star query: one or two further dims joined as filters (duplicate keys, misses, a
    predicate on each or none, two-column keys for one of them), against Python loops."""
    rng = np.random.default_rng(seed)
    n, m = int(rng.integers(0, 300)), int(rng.integers(1, 40))
    fact = {"fk": rng.integers(0, 30, size=n).astype(np.int32),
            "pred": rng.integers(0, 10, size=n).astype(np.int32),
            "val": rng.integers(-10**6, 10**6, size=n).astype(np.int64)}
    dim = {"pk": rng.integers(0, 25, size=m).astype(np.int32), "grp": rng.integers(0, 5, size=m).astype(np.int32)}
    semi = []
    for s_ in range(int(rng.integers(1, 3))):
        ms = int(rng.integers(0, 30))
        wide = bool(rng.integers(0, 2)) and s_ == 1
        sd = {"pk": rng.integers(0, 20, size=ms).astype(np.int32), "attr": rng.integers(0, 10, size=ms).astype(np.int32)}
        sj = {"fk": rng.integers(0, 24, size=n).astype(np.int32), "dim": sd,
              "op": o.OPS[int(rng.integers(0, 6))], "literal": int(rng.integers(0, 11))}
        if wide:
            sd["pk_hi"] = rng.integers(-1, 2, size=ms).astype(np.int32)
            sj["fk_hi"] = rng.integers(-1, 2, size=n).astype(np.int32)
        if rng.integers(0, 4) == 0:
            del sd["attr"]
        semi.append(sj)
    cmp = {"lt": lambda a, b: a < b, "le": lambda a, b: a <= b, "gt": lambda a, b: a > b,
           "ge": lambda a, b: a >= b, "eq": lambda a, b: a == b, "ne": lambda a, b: a != b}

    def key(cols_lo, cols_hi, i):
        return (int(cols_hi[i]) if cols_hi is not None else 0, int(cols_lo[i]))
    acc = {}
    for i in range(n):
        if not int(fact["pred"][i]) < 7:
            continue
        ok = True
        for sj in semi:
            sd = sj["dim"]
            k = key(sj["fk"], sj.get("fk_hi"), i)
            ok = ok and any(key(sd["pk"], sd.get("pk_hi"), j) == k and
                            ("attr" not in sd or cmp[sj["op"]](int(sd["attr"][j]), sj["literal"]))
                            for j in range(sd["pk"].size))
        if not ok:
            continue
        for j in range(m):
            if int(dim["pk"][j]) == int(fact["fk"][i]):
                g, v = int(dim["grp"][j]), int(fact["val"][i])
                a = acc.setdefault(g, [0, 0, v, v])
                a[0] += v; a[1] += 1; a[2] = min(a[2], v); a[3] = max(a[3], v)
    r = o.pipeline(fact, dim, "lt", 7, semi=semi)
    assert r["key"].tolist() == sorted(acc)
    for k, s_, c, mn, mx in zip(r["key"], r["sum"], r["count"], r["min"], r["max"]):
        assert acc[int(k)] == [int(s_), int(c), int(mn), int(mx)], int(k)


def check_topn(o, seed):
    """Top N: against numpy's lexsort (a library routine) on inputs with many ties, and by its
    invariants: distinct positions, non-increasing order values with ties in ascending key
    order, nothing outside better than the last one taken."""
    rng = np.random.default_rng(seed)
    g = int(rng.integers(0, 400))
    keys = rng.permutation(np.arange(-200, 10_000, dtype=np.int64))[:g]
    order = rng.integers(-5, 6, size=g).astype(np.int64) * (10**17 if seed % 3 == 0 else 1)
    if g and seed % 4 == 0:
        order[0], keys[0] = np.iinfo(np.int64).min, np.iinfo(np.int64).max
    for desc in (True, False):
        n = int(rng.integers(1, 50)) if seed % 5 else g + 7
        got = o.topn(keys, order, n, desc)
        ref = np.lexsort((keys, -order.astype(object) if desc else order))[:n]
        assert got.tolist() == [int(x) for x in ref], (desc, n)
        assert len(set(got.tolist())) == got.size == min(n, g)
        vals = [int(order[i]) * (-1 if desc else 1) for i in got]
        assert all((vals[i], int(keys[got[i]])) < (vals[i + 1], int(keys[got[i + 1]])) for i in range(len(vals) - 1))
        if got.size and got.size < g:
            last = (vals[-1], int(keys[got[-1]]))
            rest = set(range(g)) - set(got.tolist())
            assert all((int(order[i]) * (-1 if desc else 1), int(keys[i])) > last for i in rest)


# ----------------------------------------------------------------------------- the pins
@pytest.mark.parametrize("seed", range(60))
def test_filter_brute(seed):
    check_filter_brute(O, seed)


def test_filter_closed_form():
    check_filter_closed_form(O)


@pytest.mark.parametrize("seed", range(220))
def test_join_brute(seed):
    check_join_brute(O, seed)


@pytest.mark.parametrize("seed", range(40))
def test_groupby_brute(seed):
    check_groupby_brute(O, seed)


def test_groupby_single_group():
    check_groupby_single_group(O)


def test_groupby_exact_large_sums():
    # sums beyond 2**53 (no float path) but inside int64
    v = np.full(1000, 9 * 10**15, dtype=np.int64)
    r = O.groupby_agg(np.zeros(1000, np.int64), v)
    assert int(r["sum"][0]) == 9 * 10**18
    with pytest.raises(OverflowError):
        O.groupby_agg(np.zeros(1100, np.int64), np.full(1100, 9 * 10**15, dtype=np.int64))


def test_pipeline_closed_form():
    check_pipeline_closed_form(O)


@pytest.mark.parametrize("seed", range(30))
def test_pipeline_invariants(seed):
    check_pipeline_invariants(O, seed)


def test_special_cases():
    check_special_cases(O)


@pytest.mark.parametrize("seed", range(5))
def test_composite_and_group_keys(seed):
    check_composite_and_group_keys(O, seed)


@pytest.mark.parametrize("seed", range(40))
def test_topn_against_lexsort(seed):
    check_topn(O, seed)


@pytest.mark.parametrize("seed", range(40))
def test_semi_join_brute(seed):
    check_semi_brute(O, seed)


@pytest.mark.parametrize("seed", range(40))
def test_dim_predicate_brute(seed):
    check_dim_predicate_brute(O, seed)


def test_merge_partials_equals_whole():
    rng = np.random.default_rng(3)
    keys = rng.integers(0, 50, size=5000)
    vals = rng.integers(0, 10**8, size=5000)
    parts = [O.groupby_agg(keys[a:a + 700], vals[a:a + 700]) for a in range(0, 5000, 700)]
    m = O.merge_partials(parts)
    w = O.groupby_agg(keys, vals)
    for c in ("key", "sum", "count", "min", "max"):
        assert np.array_equal(m[c], w[c])


def check_merge_sorted_brute(o, seed):
    """merge_sorted_partials against the dictionary merge and against the group-by of all rows
    at once (Python loop): keys include negatives and INT64_MIN, values both signs."""
    rng = np.random.default_rng(500 + seed)
    n = int(rng.integers(0, 400))
    keys = rng.integers(-6, 6, size=n).astype(np.int64)
    keys[rng.random(n) < 0.05] = O.relational.INT64_MIN
    vals = rng.integers(-10**12, 10**12, size=n).astype(np.int64)
    cuts = np.sort(rng.integers(0, n + 1, size=int(rng.integers(1, 6))))
    bounds = [0] + cuts.tolist() + [n]
    parts = [O.groupby_loop(keys[a:b], vals[a:b]) for a, b in zip(bounds[:-1], bounds[1:])]
    got = o.merge_sorted_partials(parts)
    for want in (O.merge_partials(parts), O.groupby_loop(keys, vals)):
        for c in ("key", "sum", "count", "min", "max"):
            assert np.array_equal(np.asarray(got[c]), np.asarray(want[c])), c


def check_chunk_plan(o):
    """Chunk ranges cover rows 0..n-1 once each, in order, whatever n and the chunk size."""
    for n in (0, 1, 2, 7, 100, 1001):
        for c in (1, 3, 100, 1000, 5000):
            r = o.chunk_plan(n, c)
            covered = [i for a, b in r for i in range(a, b)]
            assert covered == list(range(n)), (n, c)
            assert all(b - a <= c for a, b in r)


def check_chunked_equals_whole(o):
    """The chunked, multi-process oracle gives the whole-table oracle's result on every
    workload shape: one- and two-column keys, Zipf keys with (grp, flag) groups, a dim-side
    predicate, filter dims of a star query."""
    specs = [dg.plain_scale(n=230_001, m=20_000),
             dg.plain_scale(n=120_003, m=9_000, composite=True),
             dg.skewed(n=150_007, m=40_000),
             dg.plain_scale(n=100_000, m=8_000, dt=20),
             dg.star(n=90_001, m=7_000)]
    specs[4] = dg.StarSpec(**{**specs[4].__dict__, "semi_m": 5_000})
    got = o.query_results(specs, chunk_rows=40_000, workers=2)
    for sp, g in zip(specs, got):
        dim, fact = dg.gen_dim_host(sp), dg.gen_fact_host(sp)
        kw = {}
        if sp.dt:
            kw.update(dim_op="lt", dim_literal=sp.dt)
        if sp.semi:
            kw["semi"] = dg.semi_args(sp, fact, dg.gen_semi_dims_host(sp))
        want = O.pipeline(fact, dim, "lt", sp.t, **kw)
        assert want["key"].size > 0
        for c in ("key", "sum", "count", "min", "max"):
            assert np.array_equal(g[c], want[c]), (sp.name, c)
    # a prefix of the rows: the same as the whole-table oracle on that prefix
    sp = specs[0]
    g = o.query_results([sp], chunk_rows=30_000, workers=1, rows=70_000)[0]
    want = O.pipeline(dg.gen_fact_host(sp, 0, 70_000), dg.gen_dim_host(sp), "lt", sp.t)
    for c in ("key", "sum", "count", "min", "max"):
        assert np.array_equal(g[c], want[c]), c


@pytest.mark.parametrize("seed", range(40))
def test_merge_sorted_partials_brute(seed):
    check_merge_sorted_brute(O, seed)


def test_chunk_plan_covers_rows_once():
    check_chunk_plan(O)


def test_chunked_oracle_equals_whole_table():
    check_chunked_equals_whole(O)


def test_hot_oracle_equals_whole_table():
    sp = dg.plain_scale(n=300_000, m=15_000)
    with O.HotOracle(sp, rows=250_000, workers=2, chunk_rows=20_000) as h:
        assert h.workers == 2
        (a, _), (b, sec) = h.run(), h.run()
    want = O.pipeline(dg.gen_fact_host(sp, 0, 250_000), dg.gen_dim_host(sp), "lt", sp.t)
    for c in ("key", "sum", "count", "min", "max"):
        assert np.array_equal(a[c], want[c]) and np.array_equal(b[c], want[c]), c
    assert sec > 0


def test_restrict_dim_selects_groups():
    rng = np.random.default_rng(4)
    fact = {"fk": rng.integers(0, 300, size=20000).astype(np.int32),
            "pred": rng.integers(0, 100, size=20000).astype(np.int32),
            "val": rng.integers(0, 10**8, size=20000).astype(np.int64)}
    dim = {"pk": np.arange(300, dtype=np.int32), "grp": rng.integers(0, 40, size=300).astype(np.int32)}
    full = O.pipeline(fact, dim, "lt", 40)
    pick = [3, 17, 39]
    part = O.pipeline(fact, O.restrict_dim(dim, pick), "lt", 40)
    keep = np.isin(full["key"], pick)
    for c in ("key", "sum", "count", "min", "max"):
        assert np.array_equal(part[c], full[c][keep])


# ----------------------------------------------------------------------------- string keys
def _tiny_strcol(rng, n):
    """Strings of 0..4 bytes over a 3-letter alphabet: duplicates, prefixes, the empty string."""
    strs = [bytes(rng.choice(list(b"abz"), size=int(rng.integers(0, 5))).tolist()) for _ in range(n)]
    return strs


def check_dict_brute(m, seed):
    """Codes by the definition, O(n^2): code_i = the number of distinct strings among the rows
    before the first row holding s_i; the dictionary lists those first rows."""
    rng = np.random.default_rng(seed)
    strs = _tiny_strcol(rng, int(rng.integers(1, 40)))
    off, chars = dg.strcol_from_list(strs)
    if seed % 2:  # a slice of a longer column: offsets need not start at 0
        off, chars = (off + 3).astype(np.int32), np.concatenate([np.frombuffer(b"xyz", np.uint8), chars])
    codes, rows = m.dict_encode(off, chars)
    n = len(strs)
    first = [min(j for j in range(n) if strs[j] == strs[i]) for i in range(n)]
    want = [len({strs[j] for j in range(first[i])}) for i in range(n)]
    assert codes.tolist() == want
    assert rows.tolist() == sorted(set(first))


def check_groupby_string_vs_ints(m, seed):
    """Strings written from integer keys (decimal, so one string per key): the same groups and
    aggregates as the integer group-by, each group's row its key's first row."""
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(1, 300))
    k = rng.integers(-20, 20, size=n)
    v = rng.integers(-10**6, 10**6, size=n)
    off, chars = dg.strcol_from_list([str(int(x)).encode() for x in k])
    got = m.groupby_string(off, chars, v)
    want = O.groupby_agg(k, v)
    keys = k[got["row"]]
    order = np.argsort(keys)
    assert np.array_equal(keys[order], want["key"])
    for c in ("sum", "count", "min", "max"):
        assert np.array_equal(got[c][order], want[c]), c
    assert all(int(np.flatnonzero(k == k[r])[0]) == int(r) for r in got["row"])
    assert np.all(np.diff(got["row"]) > 0)


@pytest.mark.parametrize("seed", range(12))
def test_dict_encode_brute(seed):
    check_dict_brute(O, seed)


@pytest.mark.parametrize("seed", range(6))
def test_groupby_string_against_integer_keys(seed):
    check_groupby_string_vs_ints(O, seed)


def test_dict_encode_special_cases():
    codes, rows = O.dict_encode(np.zeros(1, np.int32), np.zeros(0, np.uint8))      # no rows
    assert codes.size == 0 and rows.size == 0
    codes, rows = O.dict_encode(np.zeros(6, np.int32), np.zeros(0, np.uint8))      # five empty strings
    assert codes.tolist() == [0] * 5 and rows.tolist() == [0]
    off, chars = dg.strcol_from_list([b"a\x00", b"a", b"a\x00", b"\xff", b"a"])     # bytes, not text
    codes, rows = O.dict_encode(off, chars)
    assert codes.tolist() == [0, 1, 0, 2, 1] and rows.tolist() == [0, 1, 3]


# ----------------------------------------------------------------------------- planted mistakes
def _mutant(**over):
    """A copy of the oracle's public functions with some replaced by broken versions."""
    ns = {name: getattr(O, name) for name in O.__all__}
    m = types.SimpleNamespace(**ns)
    for k, v in over.items():
        setattr(m, k, v)
    # pipeline must call the mutant's pieces, so rebuild it over the namespace
    def pipeline(fact, dim, op="lt", literal=50, join="sorted", dim_op=None, dim_literal=0, semi=None):
        if dim_op is not None:
            keep = m.filter_rows(dim["dattr"], dim_op, dim_literal).astype(np.int64)
            dim = {k: v[keep] for k, v in dim.items()}
        sel = m.filter_rows(fact["pred"], op, literal).astype(np.int64)
        for sj in semi or []:
            keys = O.join_key({"fk": sj["fk"], "fk_hi": sj.get("fk_hi")}, "fk", "fk_hi")[sel]
            sop = sj.get("op") if sj["dim"].get("attr") is not None else None
            sel = sel[m.semi_keep(keys, sj["dim"], sop, sj.get("literal", 0))]
        fk = O.join_key(fact, "fk", "fk_hi")[sel]
        pk = O.join_key(dim, "pk", "pk_hi")
        p, b = m.join_sorted(fk, pk)
        rows = sel[p.astype(np.int64)]
        gkey = m.pack_group(dim["grp"], dim.get("flag"))[b.astype(np.int64)]
        return m.groupby_agg(gkey, np.asarray(fact["val"], np.int64)[rows])
    if "pipeline" not in over:
        m.pipeline = pipeline
    return m


def _le_instead_of_lt(col, op, lit):
    return O.filter_rows(col, "le" if op == "lt" else op, lit)


def _swapped_join(pk, bk):
    return O.join_sorted(bk, pk)      # outputs (build ids, probe ids) in the wrong slots


def _first_match_only(pk, bk):
    p, b = O.join_sorted(pk, bk)
    keep = np.ones(p.size, bool)
    keep[1:] = p[1:] != p[:-1]
    return p[keep], b[keep]


def _sum_drops_last(keys, vals):
    r = O.groupby_agg(keys, vals)
    if len(keys):
        r = O.groupby_agg(keys[:-1], vals[:-1]) if len(keys) > 1 else r
    return r


def _min_is_first(keys, vals):
    r = O.groupby_agg(keys, vals)
    order = np.argsort(np.asarray(keys), kind="stable")
    k = np.asarray(keys)[order]
    _, start = np.unique(k, return_index=True)
    r["min"] = np.asarray(vals)[order][start]
    return r


def _flag_signed_shift(grp, flag=None):
    g = np.asarray(grp, dtype=np.int64)
    if flag is None:
        return g
    return g * 256 + np.asarray(flag, dtype=np.int64)   # sign-extended byte: (g, -1) == (g-1, 255)


def _ignores_dim_predicate(fact, dim, op="lt", literal=50, join="sorted", dim_op=None, dim_literal=0,
                           semi=None):
    return O.pipeline(fact, dim, op, literal, join, semi=semi)


def _ignores_semi_joins(fact, dim, op="lt", literal=50, join="sorted", dim_op=None, dim_literal=0, semi=None):
    return O.pipeline(fact, dim, op, literal, join, dim_op, dim_literal)


def _semi_ignores_predicate(fact_keys, dim, op, literal):
    return O.semi_keep(fact_keys, dim, None, literal)


def _topn_ascending(keys, order, n, descending=True):
    return O.topn(keys, order, n, not descending)


def _topn_ties_by_larger_key(keys, order, n, descending=True):
    sign = -1 if descending else 1
    idx = sorted(range(len(keys)), key=lambda i: (sign * int(order[i]), -int(keys[i])))
    return np.asarray(idx[:n], dtype=np.int64)


def _dict_last_occurrence(offsets, chars):
    strs = O.strings_of(offsets, chars)
    rev_codes, rev_rows = O.dict_encode(*dg.strcol_from_list(strs[::-1]))
    n = len(strs)
    return rev_codes[::-1].copy(), np.sort(n - 1 - rev_rows)


def _dict_prefix2(offsets, chars):
    strs = [s[:2] for s in O.strings_of(offsets, chars)]   # compares only two bytes
    return O.dict_encode(*dg.strcol_from_list(strs))


def _groupby_string_max_is_min(offsets, chars, vals):
    r = O.groupby_string(offsets, chars, vals)
    r["max"] = r["min"]
    return r


def _merge_min_of_first_part(parts):
    r = O.merge_sorted_partials(parts)
    first = {int(k): int(v) for k, v in zip(parts[0]["key"], parts[0]["min"])} if parts else {}
    r["min"] = np.array([first.get(int(k), int(v)) for k, v in zip(r["key"], r["min"])], dtype=np.int64)
    return r


def _merge_counts_parts(parts):
    r = O.merge_sorted_partials(parts)
    r["count"] = O.merge_sorted_partials([dict(p, count=np.ones_like(p["count"])) for p in parts])["count"]
    return r


def _chunk_plan_overlaps(n, c):
    return [(max(0, a - 1), b) for a, b in O.chunk_plan(n, c)]


def _chunk_plan_gap(n, c):
    return [(a, max(a, b - 1)) for a, b in O.chunk_plan(n, c)]


MUTANTS = [
    ("dictionary by last occurrence", dict(dict_encode=_dict_last_occurrence),
     lambda m: [check_dict_brute(m, s) for s in range(12)]),
    ("dictionary compares a prefix", dict(dict_encode=_dict_prefix2),
     lambda m: [check_dict_brute(m, s) for s in range(12)]),
    ("string group-by max is min", dict(groupby_string=_groupby_string_max_is_min),
     lambda m: [check_groupby_string_vs_ints(m, s) for s in range(6)]),
    ("topn ascending for descending", dict(topn=_topn_ascending), lambda m: [check_topn(m, s) for s in range(5)]),
    ("topn ties by larger key", dict(topn=_topn_ties_by_larger_key), lambda m: [check_topn(m, s) for s in range(5)]),
    ("semi-joins ignored", dict(pipeline=_ignores_semi_joins),
     lambda m: [check_semi_brute(m, s) for s in range(10)]),
    ("semi-join predicate ignored", dict(semi_keep=_semi_ignores_predicate),
     lambda m: [check_semi_brute(m, s) for s in range(10)]),
    ("dim predicate ignored", dict(pipeline=_ignores_dim_predicate),
     lambda m: [check_dim_predicate_brute(m, s) for s in range(10)]),
    ("filter le for lt (dim predicate)", dict(filter_rows=_le_instead_of_lt),
     lambda m: [check_dim_predicate_brute(m, s) for s in range(10)]),
    ("filter le for lt", dict(filter_rows=_le_instead_of_lt),
     lambda m: check_filter_closed_form(m)),
    ("filter le for lt (pipeline)", dict(filter_rows=_le_instead_of_lt),
     lambda m: check_pipeline_closed_form(m)),
    ("join operands swapped", dict(join_sorted=_swapped_join),
     lambda m: [check_join_brute(m, s) for s in range(20)]),
    ("join keeps first match only", dict(join_sorted=_first_match_only),
     lambda m: [check_join_brute(m, s) for s in range(20)]),
    ("groupby drops a row", dict(groupby_agg=_sum_drops_last),
     lambda m: check_groupby_single_group(m)),
    ("groupby drops a row (pipeline)", dict(groupby_agg=_sum_drops_last),
     lambda m: check_pipeline_closed_form(m)),
    ("min is first value", dict(groupby_agg=_min_is_first),
     lambda m: [check_groupby_brute(m, s) for s in range(5)]),
    ("min is first value (pipeline)", dict(groupby_agg=_min_is_first),
     lambda m: [check_pipeline_invariants(m, s) for s in range(5)]),
    ("merge takes MIN of the first part", dict(merge_sorted_partials=_merge_min_of_first_part),
     lambda m: [check_merge_sorted_brute(m, s) for s in range(10)]),
    ("merge counts parts, not rows", dict(merge_sorted_partials=_merge_counts_parts),
     lambda m: [check_merge_sorted_brute(m, s) for s in range(10)]),
    ("chunks overlap", dict(chunk_plan=_chunk_plan_overlaps), lambda m: check_chunk_plan(m)),
    ("chunks leave gaps", dict(chunk_plan=_chunk_plan_gap), lambda m: check_chunk_plan(m)),
    ("group flag sign-extended", dict(pack_group=_flag_signed_shift),
     lambda m: [check_composite_and_group_keys(m, s) for s in range(3)]),
]


@pytest.mark.parametrize("name,over,check", MUTANTS, ids=[x[0] for x in MUTANTS])
def test_planted_mistake_is_caught(name, over, check):
    with pytest.raises(AssertionError):
        check(_mutant(**over))
