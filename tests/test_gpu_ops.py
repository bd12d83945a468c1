"""Parity of each CUDA operator with the CPU oracle, through the C-ABI (GPU).

Integer work, so the bar is bit-exact: filter output in order, join pairs and groups after a
canonical sort.  Sizes span several tiles plus a ragged tail; edge cases cover empty inputs,
selectivity 0 % / 100 %, duplicate and sentinel-valued keys, misses, unaligned columns."""
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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def u32(t):
    return t.cpu().numpy().view(np.uint32)


# ------------------------------------------------------------------------- filter
@pytest.mark.parametrize("n", [1, 5, 4095, 4096, 4097, 12289, 32767, 32768, 32769, 65537, 98305, 100_003,
                               1_048_577, 3_000_001, 40_000_003])
def test_filter_sizes(S, n):
    col = np.random.default_rng(n).integers(0, 100, size=n).astype(np.int32)
    for t in (0, 37, 100):
        got = u32(S.sirius_filter(dev(col), "lt", t))
        assert np.array_equal(got, O.filter_rows(col, "lt", t))


@pytest.mark.parametrize("op", O.OPS)
def test_filter_ops(S, op):
    col = np.random.default_rng(1).integers(-50, 50, size=50_001).astype(np.int32)
    col[:10] = [np.iinfo(np.int32).min, np.iinfo(np.int32).max, 0, -1, 1, 7, 7, 7, -7, 0]
    for lit in (np.iinfo(np.int32).min, -1, 0, 7, np.iinfo(np.int32).max):
        got = u32(S.sirius_filter(dev(col), op, int(lit)))
        assert np.array_equal(got, O.filter_rows(col, op, int(lit))), (op, lit)


def test_filter_empty_and_unaligned(S):
    assert S.sirius_filter(torch.zeros(0, dtype=torch.int32, device="cuda"), "lt", 5).numel() == 0
    col = np.random.default_rng(2).integers(0, 100, size=20_001).astype(np.int32)
    d = dev(col)
    got = u32(S.sirius_filter(d[1:], "ge", 42))   # 4-byte offset: scalar path
    assert np.array_equal(got, O.filter_rows(col[1:], "ge", 42))
    col = np.random.default_rng(4).integers(0, 100, size=1_000_003).astype(np.int32)
    got = u32(S.sirius_filter(dev(col)[3:], "lt", 61))   # scalar path over 31 tiles and a ragged one
    assert np.array_equal(got, O.filter_rows(col[3:], "lt", 61))


def test_filter_async_count(S):
    col = np.random.default_rng(3).integers(0, 100, size=777_777).astype(np.int32)
    out, d_count = S.sirius_filter(dev(col), "lt", 30, sync=False)
    torch.cuda.synchronize()
    want = O.filter_rows(col, "lt", 30)
    assert int(d_count.item()) == want.size
    assert np.array_equal(u32(out[:want.size]), want)


# ------------------------------------------------------------------------- join
def check_join(S, probe, build, sel=None, probe_hi=None, build_hi=None, lf=0.5, variant=0):
    tab = S.HashJoinTable(build.size, 8 if build_hi is not None else 4, lf, probe_variant=variant)
    tab = S.sirius_hash_join_build(dev(build), dev(build_hi) if build_hi is not None else None, lf, table=tab)
    p, b = S.sirius_hash_join_probe(tab, dev(probe), dev(probe_hi) if probe_hi is not None else None,
                                    dev(sel.view(np.int32)) if sel is not None else None)
    got = O.sort_pairs(u32(p), u32(b))
    pk = O.pack_composite(probe_hi, probe) if probe_hi is not None else probe.astype(np.int64)
    bk = O.pack_composite(build_hi, build) if build_hi is not None else build.astype(np.int64)
    rows = sel.astype(np.int64) if sel is not None else np.arange(probe.size)
    wp, wb = O.join_sorted(pk[rows], bk)
    want = O.sort_pairs(rows[wp.astype(np.int64)], wb)
    assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])
    has_dup = np.unique(bk).size < bk.size
    assert tab.has_dups == has_dup
    return want[0].size


@pytest.mark.parametrize("lf", [0.25, 0.5, 0.9])
def test_join_unique_keys(S, lf):
    m = 65_536
    build = np.random.default_rng(4).permutation(m).astype(np.int32)
    probe = np.random.default_rng(5).integers(0, 2 * m, size=300_007).astype(np.int32)
    assert check_join(S, probe, build, lf=lf) > 0


def test_join_with_selection_vector(S):
    m = 10_000
    build = np.random.default_rng(6).permutation(m).astype(np.int32)
    probe = np.random.default_rng(7).integers(0, m, size=200_000).astype(np.int32)
    pred = np.random.default_rng(8).integers(0, 100, size=200_000).astype(np.int32)
    sel = O.filter_rows(pred, "lt", 30)
    check_join(S, probe, build, sel=sel)


def test_join_duplicates_and_sentinel_values(S):
    rng = np.random.default_rng(9)
    special = np.array([-1, np.iinfo(np.int32).min, 0, np.iinfo(np.int32).max], dtype=np.int32)
    build = np.concatenate([rng.integers(-20, 20, size=3000).astype(np.int32), special, special])
    probe = np.concatenate([rng.integers(-25, 25, size=5001).astype(np.int32), special])
    assert check_join(S, probe, build) > 5001


def test_join_all_miss_and_empty(S):
    build = np.arange(1000, dtype=np.int32)
    assert check_join(S, build + 5000, build) == 0
    assert check_join(S, np.zeros(0, np.int32), build) == 0
    assert check_join(S, build, np.zeros(0, np.int32)) == 0


def test_join_composite_keys(S):
    rng = np.random.default_rng(10)
    pool = rng.integers(-2**31, 2**31, size=(500, 2)).astype(np.int64)
    pool[0] = (-1, -1)
    pool[1] = (0, -1)
    pool[2] = (-1, 0)
    bi = np.concatenate([np.arange(500), rng.integers(0, 500, size=100)])
    pi = rng.integers(0, 700, size=40_001) % 600
    pool_ext = np.concatenate([pool, rng.integers(-2**31, 2**31, size=(100, 2))])
    b_hi, b_lo = pool[bi % 500, 0].astype(np.int32), pool[bi % 500, 1].astype(np.int32)
    p_hi, p_lo = pool_ext[pi, 0].astype(np.int32), pool_ext[pi, 1].astype(np.int32)
    check_join(S, p_lo, b_lo, probe_hi=p_hi, build_hi=b_hi)


@pytest.mark.parametrize("variant", [1, 2])
@pytest.mark.parametrize("lf", [0.5, 0.95])
def test_join_probe_variants(S, variant, lf):
    """Four rows per thread (1) and four lanes per key (2): unique keys at two load factors (long
    walks at 0.95), a selection vector starting off a 16-byte boundary, ragged counts, two-column
    keys, and a table with duplicates (walked one row per lane by either)."""
    rng = np.random.default_rng(20 + variant)
    m = 50_001
    build = rng.permutation(3 * m)[:m].astype(np.int32) - m
    probe = rng.integers(-m - 100, 2 * m + 100, size=400_003).astype(np.int32)
    assert check_join(S, probe, build, lf=lf, variant=variant) > 0
    sel = O.filter_rows(rng.integers(0, 100, size=probe.size).astype(np.int32), "lt", 37)
    check_join(S, probe, build, sel=sel[1:], lf=lf, variant=variant)
    for n in (1, 3, 5, 33):
        check_join(S, probe[:n], build, lf=lf, variant=variant)
    pool = rng.integers(-2**31, 2**31, size=(20_000, 2)).astype(np.int64)
    bi = rng.permutation(20_000)[:15_000]
    pi = rng.integers(0, 20_000, size=100_001)
    check_join(S, pool[pi, 1].astype(np.int32), pool[bi, 1].astype(np.int32), probe_hi=pool[pi, 0].astype(np.int32),
               build_hi=pool[bi, 0].astype(np.int32), lf=lf, variant=variant)
    dups = np.concatenate([build[:5000], build[:3000]])
    check_join(S, probe, dups, lf=lf, variant=variant)


def test_join_capacity_retry(S):
    build = np.concatenate([np.arange(100, dtype=np.int32)] * 4)
    probe = np.arange(100, dtype=np.int32)
    tab = S.sirius_hash_join_build(dev(build))
    p, b = S.sirius_hash_join_probe(tab, dev(probe), out_cap=10)
    assert p.numel() == 400


# ------------------------------------------------------------------------- gather
def test_gather(S):
    rng = np.random.default_rng(11)
    src64 = rng.integers(-2**62, 2**62, size=100_000)
    src32 = rng.integers(-2**31, 2**31, size=100_000).astype(np.int32)
    idx = rng.integers(0, 100_000, size=333_333).astype(np.uint32)
    assert np.array_equal(S.sirius_gather(dev(src64), dev(idx.view(np.int32))).cpu().numpy(), src64[idx])
    assert np.array_equal(S.sirius_gather(dev(src32), dev(idx.view(np.int32))).cpu().numpy(), src32[idx])
    for n, off in ((1, 0), (3, 1), (7, 1), (1001, 2)):   # ragged counts, indexes off 16-byte boundaries
        di = dev(idx.view(np.int32))[off:off + n]
        assert np.array_equal(S.sirius_gather(dev(src64), di).cpu().numpy(), src64[idx[off:off + n]])
        assert np.array_equal(S.sirius_gather(dev(src32), di).cpu().numpy(), src32[idx[off:off + n]])
    grp = rng.integers(-1000, 1000, size=100_000).astype(np.int32)
    flag = rng.integers(-128, 128, size=100_000).astype(np.int8)
    got = S.sirius_gather_group_key(dev(grp), dev(flag), dev(idx.view(np.int32))).cpu().numpy()
    assert np.array_equal(got, O.pack_group(grp, flag)[idx])


# ------------------------------------------------------------------------- group-by
def check_groupby(S, keys, vals, hint, aggs="sum,count,min,max"):
    got = S.sirius_groupby_agg(dev(keys), dev(vals), aggs, group_cap_hint=hint)
    got = O.sort_groups({k: v.cpu().numpy() for k, v in got.items()})
    want = O.groupby_agg(keys, vals)
    cols = ["key", "count"] + [a for a in ("sum", "min", "max") if a in aggs]
    for c in cols:
        assert np.array_equal(got[c], want[c]), c
    return want["key"].size


@pytest.mark.parametrize("n,dom,hint", [(1, 1, 1), (1000, 10, 16), (300_001, 1000, 1000),
                                        (300_001, 100_000, 100_000), (2_000_003, 5, 8)])
def test_groupby_int32(S, n, dom, hint):
    rng = np.random.default_rng(n + dom)
    keys = rng.integers(-dom // 2, dom - dom // 2, size=n).astype(np.int32)
    vals = rng.integers(-10**10, 10**10, size=n)
    check_groupby(S, keys, vals, hint)


def test_groupby_int64_with_sentinel_key(S):
    rng = np.random.default_rng(12)
    keys = rng.integers(-2**63, 2**63 - 1, size=50_000, dtype=np.int64) % 3000
    keys[::7] = np.iinfo(np.int64).min
    keys[::11] = np.iinfo(np.int64).max
    vals = rng.integers(0, 10**8, size=50_000)
    for hint in (4000, 1_000_000):   # shared-memory and global paths
        check_groupby(S, keys, vals, hint)


def test_groupby_subsets_and_single_group(S):
    rng = np.random.default_rng(13)
    vals = rng.integers(0, 10**8, size=123_457)
    check_groupby(S, np.zeros(vals.size, np.int32), vals, 1, "sum,count")
    check_groupby(S, rng.integers(0, 50, size=vals.size).astype(np.int32), vals, 64, "min")


@pytest.mark.parametrize("offset", [0, 1])
@pytest.mark.parametrize("n,dom", [(5, 3), (3_000_003, 1_000_000), (2_000_001, 4000), (6_000_001, 4_000_000)])
def test_groupby_direct_slots_large_tables(S, n, dom, offset):
    """Dense keys of a table too large for shared memory: direct slots (key - min) behind the
    hot-group cache, 16-byte loads (offset 0) or scalar loads (columns one element off); a range of
    4M slots is aggregated in three passes over L2-sized windows of the table."""
    rng = np.random.default_rng(n + dom + offset)
    keys = (rng.integers(0, dom, size=n + offset) - dom // 3).astype(np.int32)
    vals = rng.integers(-10**12, 10**12, size=n + offset)
    dk, dvals = dev(keys)[offset:], dev(vals)[offset:]
    got = S.sirius_groupby_agg(dk, dvals, group_cap_hint=max(dom, 3000))
    got = O.sort_groups({k: v.cpu().numpy() for k, v in got.items()})
    want = O.groupby_agg(keys[offset:], vals[offset:])
    for c in COLS:
        assert np.array_equal(got[c], want[c]), c


def test_groupby_direct_slots_int64_edges(S):
    """Dense int64 keys far from zero, at INT64_MIN and at INT64_MAX; a range of exactly the
    table's limit (direct) and one past it with two keys (hashed)."""
    rng = np.random.default_rng(14)
    vals = rng.integers(-10**8, 10**8, size=400_003)
    for base in (1 << 40, np.iinfo(np.int64).min, np.iinfo(np.int64).max - 4999):
        keys = (np.int64(base) + rng.integers(0, 5000, size=vals.size)).astype(np.int64)
        check_groupby(S, keys, vals, 5000)
    cap = S.lib().sirius_groupby_capacity(3000)
    limit = cap - cap // 8
    keys = np.arange(limit, dtype=np.int64).repeat(3)
    check_groupby(S, keys, np.arange(keys.size, dtype=np.int64), 3000)
    keys = np.array([0, limit] * 5000, dtype=np.int64)
    check_groupby(S, keys, np.arange(keys.size, dtype=np.int64), 3000)


def test_groupby_direct_slots_skewed(S):
    """Zipf(1.1) ranks over 1e6 dense keys: hot groups aggregate in the per-block cache."""
    rng = np.random.default_rng(15)
    keys = np.minimum(rng.zipf(1.1, size=2_000_003), 1_000_000).astype(np.int32) - 1
    vals = rng.integers(0, 10**8, size=keys.size)
    check_groupby(S, keys, vals, 1_000_000)


SPLIT_N = 20_000_003   # at least 2^24 rows and 256 per group slot (hint 30 000: 65 537 slots)


@pytest.mark.parametrize("order", ["uniform", "ascending", "descending"])
@pytest.mark.parametrize("key_dtype", [np.int32, np.int64])
def test_groupby_split_pass(S, order, key_dtype):
    """Inputs with many rows per direct slot take the split pass (the first 1/16 of the rows in
    full, then the rest behind the extreme bounds of the groups seen): value orders that make
    the bounds decisive or useless, int32 and int64 keys far from zero."""
    rng = np.random.default_rng(40 + (key_dtype == np.int64))
    keys = rng.integers(0, 30_000, size=SPLIT_N).astype(key_dtype)
    if key_dtype == np.int64:
        keys = keys + np.int64(10**15)
    vals = {"uniform": rng.integers(-10**12, 10**12, size=SPLIT_N),
            "ascending": np.arange(SPLIT_N, dtype=np.int64) * 7 - 10**8,
            "descending": 10**8 - np.arange(SPLIT_N, dtype=np.int64) * 7}[order]
    check_groupby(S, keys, vals, 30_000)


def test_groupby_split_pass_late_keys_subsets_and_unaligned(S):
    """Half the keys appear only after the split (no bound applies to them; values beyond the
    first phase's extremes), each subset of MIN and MAX, and columns one element off (scalar
    loads)."""
    rng = np.random.default_rng(43)
    n0 = ((SPLIT_N // 16) >> 2) << 2
    keys = rng.integers(0, 30_000, size=SPLIT_N).astype(np.int32)
    keys[:n0] = rng.integers(0, 15_000, size=n0)
    vals = rng.integers(-10**9, 10**9, size=SPLIT_N)
    vals[n0:n0 + 2000] = rng.choice([-3 * 10**9, 3 * 10**9], size=2000)
    check_groupby(S, keys, vals, 30_000)
    for aggs in ("min", "max", "min,max", "sum,count"):
        check_groupby(S, keys, vals, 30_000, aggs)
    keys1 = np.concatenate([[7], keys]).astype(np.int32)
    vals1 = np.concatenate([[5], vals]).astype(np.int64)
    got = S.sirius_groupby_agg(dev(keys1)[1:], dev(vals1)[1:], group_cap_hint=30_000)
    got = O.sort_groups({k: v.cpu().numpy() for k, v in got.items()})
    want = O.groupby_agg(keys, vals)
    for c in COLS:
        assert np.array_equal(got[c], want[c]), c


def test_groupby_table_full_then_retry(S):
    keys = np.arange(10_000, dtype=np.int64)
    vals = np.ones(10_000, dtype=np.int64)
    with pytest.raises(S.SiriusError) as e:
        S.sirius_groupby_agg(dev(keys), dev(vals), group_cap_hint=1000)
    assert e.value.status == S.ERR_TABLE_FULL
    assert check_groupby(S, keys, vals, 10_000) == 10_000


def test_groupby_capacity(S):
    keys = np.arange(1000, dtype=np.int32)
    vals = np.ones(1000, dtype=np.int64)
    with pytest.raises(S.SiriusError) as e:
        S.sirius_groupby_agg(dev(keys), dev(vals), group_cap_hint=1000, out_cap=10)
    assert e.value.status == S.ERR_CAPACITY and e.value.needed == 1000


# ----------------------------------------------------------------------------- top N groups
@pytest.mark.parametrize("g", [0, 1, 5, 1000, 100_003, 1_000_000])
@pytest.mark.parametrize("n_top", [1, 10, 100, 8192])
def test_topn(S, g, n_top):
    rng = np.random.default_rng(g + n_top)
    keys = rng.permutation(np.arange(-g, 4 * g + 1, dtype=np.int64))[:g]
    order = rng.integers(-50, 50, size=g).astype(np.int64) * (10**15 if g % 2 else 1)  # many ties
    if g > 2:
        order[:2] = [np.iinfo(np.int64).min, np.iinfo(np.int64).max]
    dk, do = torch.from_numpy(keys).cuda(), torch.from_numpy(order).cuda()
    for desc in (True, False):
        got = S.sirius_topn_groups(dk, do, n_top, desc).cpu().numpy().astype(np.int64)
        want = O.topn(keys, order, n_top, desc)
        assert np.array_equal(got, want), desc


def test_topn_of_pipeline_and_errors(S):
    """ORDER BY SUM DESC, key LIMIT 100 after the fused pipeline, the columns gathered."""
    spec = dg.plain_scale(n=2_000_000, m=50_000)
    dim, fact = dg.gen_dim_host(spec), dg.gen_fact_host(spec)
    res = S.run_pipeline({k: torch.from_numpy(v).cuda() for k, v in fact.items()},
                         {k: torch.from_numpy(v).cuda() for k, v in dim.items()}, "lt", spec.t,
                         group_cap_hint=100_000)
    pos = S.sirius_topn_groups(res["key"], res["sum"], 100, True)
    got = {c: S.sirius_gather(res[c], pos).cpu().numpy() for c in res}
    want = O.pipeline(fact, dim, "lt", spec.t)
    top = O.topn(want["key"], want["sum"], 100, True)
    for c in ("key", "sum", "count", "min", "max"):
        assert np.array_equal(got[c], want[c][top]), c
    k = torch.arange(10, dtype=torch.int64, device="cuda")
    for bad in (0, 8193):
        with pytest.raises(S.SiriusError) as e:
            S.sirius_topn_groups(k, k, bad)
        assert e.value.status == S.ERR_INVALID


# ----------------------------------------------------------------------------- sort-based group-by
@pytest.mark.parametrize("n", [0, 1, 2, 2047, 2048, 2049, 100_003, 3_000_001])
@pytest.mark.parametrize("dom", [1, 7, 1000, 100_000, None])
def test_groupby_sort(S, n, dom):
    """Same results as the definition, groups in ascending key order: int32 keys with
    negatives, int64 keys with the extreme values, every key distinct (dom None)."""
    rng = np.random.default_rng(n * 7 + (dom or 3))
    if dom is None:
        k32 = rng.permutation(np.arange(-(n // 2), n - n // 2, dtype=np.int64)).astype(np.int32)
    else:
        k32 = rng.integers(-dom // 2, dom - dom // 2 + 1, size=n).astype(np.int32)
    vals = rng.integers(-10**12, 10**12, size=n)
    for keys in (k32, k32.astype(np.int64) * 1_000_003 + (np.iinfo(np.int64).min // 2 if dom == 7 else 0)):
        if keys.dtype == np.int64 and n > 2:
            keys[:2] = [np.iinfo(np.int64).min, np.iinfo(np.int64).max]
        got = S.sirius_groupby_sort(torch.from_numpy(keys).cuda(), torch.from_numpy(vals).cuda())
        got = {c: v.cpu().numpy() for c, v in got.items()}
        want = O.groupby_agg(keys, vals)
        for c in ("key", "sum", "count", "min", "max"):
            assert np.array_equal(got[c], want[c]), (keys.dtype, c)


def test_groupby_sort_int64_keys_spanning_all_digits(S):
    """int64 keys whose every byte varies (eight passes), with duplicates, against the oracle."""
    rng = np.random.default_rng(9)
    distinct = rng.integers(np.iinfo(np.int64).min, np.iinfo(np.int64).max, size=20_000, dtype=np.int64)
    keys = distinct[rng.integers(0, distinct.size, size=700_001)]
    vals = rng.integers(-10**15, 10**15, size=keys.size)
    got = S.sirius_groupby_sort(torch.from_numpy(keys).cuda(), torch.from_numpy(vals).cuda())
    want = O.groupby_agg(keys, vals)
    for c in ("key", "sum", "count", "min", "max"):
        assert np.array_equal(got[c].cpu().numpy(), want[c]), c


def test_groupby_sort_skipped_digits_subsets_and_capacity(S):
    rng = np.random.default_rng(3)
    keys = (rng.integers(0, 50, size=500_000).astype(np.int64) << 40) | 0x1234  # only high digits vary
    vals = rng.integers(0, 10**9, size=500_000)
    dk, dv = torch.from_numpy(keys).cuda(), torch.from_numpy(vals).cuda()
    want = O.groupby_agg(keys, vals)
    for aggs in ("sum,count", "count,min", "count,max", "sum,count,min,max"):
        got = S.sirius_groupby_sort(dk, dv, aggs)
        for c in ["key", "count"] + [a for a in ("sum", "min", "max") if a in aggs]:
            assert np.array_equal(got[c].cpu().numpy(), want[c]), (aggs, c)
    same = S.sirius_groupby_sort(torch.full((10_000,), 42, dtype=torch.int32, device="cuda"),
                                 torch.ones(10_000, dtype=torch.int64, device="cuda"))
    assert same["key"].tolist() == [42] and same["count"].tolist() == [10_000] and same["sum"].tolist() == [10_000]
    with pytest.raises(S.SiriusError) as e:
        S.sirius_groupby_sort(dk, dv, out_cap=10)
    assert e.value.status == S.ERR_CAPACITY and e.value.needed == want["key"].size
    # values that start off a 16-byte boundary (no bulk copy for the first pass): same groups
    sub = S.sirius_groupby_sort(dk[1:], dv[1:])
    want_sub = O.groupby_agg(keys[1:], vals[1:])
    for c in ("key", "sum", "count", "min", "max"):
        assert np.array_equal(sub[c].cpu().numpy(), want_sub[c]), c
    assert dv[1:].data_ptr() % 16 == 8
    # the hash group-by on the same input gives the same groups
    h = S.sirius_groupby_agg(dk, dv, group_cap_hint=100)
    order = torch.argsort(h["key"]).cpu().numpy()
    for c in ("key", "sum", "count", "min", "max"):
        assert np.array_equal(h[c].cpu().numpy()[order], want[c]), c
