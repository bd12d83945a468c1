"""The seeded input generator: pinned to the published SplitMix64 sequence and to exact
integer arithmetic (CPU only; the CUDA twin is checked against it in test_gpu_datagen.py)."""
import os

import numpy as np
import pytest

from paper_2508_04701_gb300 import datagen as dg

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "splitmix64_seed1234567.txt")


def _golden():
    vals, seed = [], None
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line.startswith("seed"):
            seed = int(line.split()[1])
        else:
            vals.append(int(line))
    return seed, vals


def test_splitmix64_published_sequence():
    seed, vals = _golden()
    got = dg.stream_from_state(seed, 0, len(vals))
    assert [int(x) for x in got] == vals
    # the scalar twin used for stream bases
    z, out = seed, []
    for _ in vals:
        out.append(dg.splitmix64_int(z))
        z = (z + dg.GAMMA) & dg.MASK64
    assert out == vals


def test_stream_chunks_are_consistent():
    full = dg.stream(7, dg.FACT, dg.C_VAL, 0, 1000)
    parts = np.concatenate([dg.stream(7, dg.FACT, dg.C_VAL, a, a + 137) for a in range(0, 1000, 137)])
    assert np.array_equal(full, parts[:1000])


@pytest.mark.parametrize("n", [1, 2, 3, 100, 1000, 65536, 15_000_000, 100_000_000, (1 << 32) - 1])
def test_bounded_is_exact_mulhi(n):
    rng = np.random.default_rng(n)
    r = rng.integers(0, 1 << 64, size=2000, dtype=np.uint64, endpoint=False)
    r = np.concatenate([r, np.array([0, 1, (1 << 64) - 1, 1 << 63, (1 << 32) - 1], dtype=np.uint64)])
    got = dg.bounded(r, n)
    want = np.array([(int(x) * n) >> 64 for x in r], dtype=np.int64)
    assert np.array_equal(got, want)
    assert got.min() >= 0 and got.max() < n


def test_permutation_is_a_permutation():
    p = dg.permutation(0, dg.DIM, dg.C_PK_TAG, 65536)
    assert np.array_equal(np.sort(p), np.arange(65536))
    assert not np.array_equal(p, np.arange(65536))


def test_zipf_cdf_and_sampling():
    m, s = 1000, 1.1
    cdf = dg.zipf_cdf(m, s)
    assert cdf[-1] == 1.0 and np.all(np.diff(cdf) > 0)
    w = np.arange(1, m + 1, dtype=np.float64) ** -s
    assert abs(cdf[0] - w[0] / w.sum()) < 1e-15
    # u = 0 -> rank 1; u just below 1 -> rank m
    r = np.array([0, (1 << 64) - 1], dtype=np.uint64)
    assert list(dg.zipf_rank0(r, cdf)) == [0, m - 1]
    # frequency of rank 1 within 3 sigma of its probability
    x = dg.zipf_rank0(dg.stream(0, 9, 0, 0, 200_000), cdf)
    p0 = cdf[0]
    f0 = np.mean(x == 0)
    assert abs(f0 - p0) < 3 * np.sqrt(p0 * (1 - p0) / x.size)


def test_plain_small_tables():
    spec = dg.plain_small()
    dim = dg.gen_dim_host(spec)
    assert np.array_equal(np.sort(dim["pk"]), np.arange(65536, dtype=np.int32))
    assert dim["grp"].min() >= 0 and dim["grp"].max() < 1000
    f = dg.gen_fact_host(spec, 0, 10_000)
    assert f["fk"].dtype == np.int32 and f["pred"].dtype == np.int32 and f["val"].dtype == np.int64
    assert f["fk"].min() >= 0 and f["fk"].max() < 65536
    assert f["pred"].min() >= 0 and f["pred"].max() < 100
    assert f["val"].min() >= 0 and f["val"].max() < 100_000_000
    # selectivity of pred < 50 near one half
    assert abs(np.mean(f["pred"] < 50) - 0.5) < 0.03


def test_composite_keys_unique_and_match():
    spec = dg.plain_scale(n=20_000, m=5_000, composite=True)
    dim = dg.gen_dim_host(spec)
    pk64 = (dim["pk_hi"].view(np.uint32).astype(np.uint64) << np.uint64(32)) | dim["pk"].view(np.uint32)
    assert np.unique(pk64).size == spec.m
    f = dg.gen_fact_host(spec)
    fk64 = (f["fk_hi"].view(np.uint32).astype(np.uint64) << np.uint64(32)) | f["fk"].view(np.uint32)
    assert np.isin(fk64, pk64).all()


def test_skewed_tables():
    spec = dg.skewed(n=50_000, m=20_000)
    dim = dg.gen_dim_host(spec)
    gk = dim["grp"].astype(np.int64) * 2 + dim["flag"]
    assert np.array_equal(np.sort(gk), np.arange(spec.m))
    f = dg.gen_fact_host(spec, dim=dim)
    assert np.isin(f["fk"], dim["pk"]).all()
    # the hottest key takes about cdf[0] of the rows
    _, c = np.unique(f["fk"], return_counts=True)
    p0 = dg.zipf_cdf(spec.m, 1.1)[0]
    assert abs(c.max() / spec.n - p0) < 0.01


def test_batch_query_sizes():
    qs = [dg.batch_query(q) for q in range(512)]
    ns = np.array([q.n for q in qs]); ms = np.array([q.m for q in qs]); ts = np.array([q.t for q in qs])
    assert ns.min() >= 10_000 and ns.max() < 20_000_000
    assert ms.min() >= 1_000 and ms.max() < 2_000_000
    assert ts.min() >= 5 and ts.max() <= 90
    # log-uniform: mean of N = 1e4 * 1999 / ln 2000 ~ 2.63M (loose, 512 draws)
    assert 1.5e6 < ns.mean() < 4e6


def test_string_dictionary_format_and_distinct():
    import re
    sp = dg.StringSpec(n=10, d=20_000, seed=5)
    off, chars = dg.string_dict_host(sp)
    strs = [bytes(chars[off[i]:off[i + 1]]) for i in range(sp.d)]
    assert len(set(strs)) == sp.d
    pat = re.compile(rb"^[a-z]{0,12}#(\d+)$")
    for k, s in enumerate(strs):
        m = pat.match(s)
        assert m and int(m.group(1)) == k


def test_string_rows_follow_ids():
    sp = dg.StringSpec(n=5_000, d=300, seed=2)
    r = dg.gen_strings_host(sp)
    off, chars = dg.string_dict_host(sp)
    dstr = [bytes(chars[off[i]:off[i + 1]]) for i in range(sp.d)]
    o, c = r["offsets"], r["chars"]
    assert o.dtype == np.int32 and c.dtype == np.uint8 and o[0] == 0 and o[-1] == c.size
    assert [bytes(c[o[i]:o[i + 1]]) for i in range(sp.n)] == [dstr[k] for k in r["ids"]]
    assert r["ids"].min() >= 0 and r["ids"].max() < sp.d and r["vals"].max() < sp.val_bound
    assert np.array_equal(r["ids"], dg.bounded(dg.stream(sp.seed, dg.STR_TABLE, dg.C_SID, 0, sp.n), sp.d))
