"""String keys on the GPU against the oracle: dictionary codes and dictionary rows are compared
exactly (the codes are unique: order of first occurrence), the string group-by's aggregates
exactly.  Collisions are forced with the 8-bit test hash; bad offsets, an undersized table and
an undersized output give their errors."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2508_04701_gb300 import datagen as dg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    from paper_2508_04701_gb300 import build
    build.build()
    from paper_2508_04701_gb300 import sirius
    sirius.lib()
    return sirius


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def encode(S, off, chars, **kw):
    codes, rows = S.sirius_dict_encode(dev(off), dev(chars), **kw)
    return codes.cpu().numpy(), rows.cpu().numpy()


# the 8-bit test hash forces collisions: every distinct string shares its hash with ~d/256
# others, so the weak-hash cases stop at sizes where those chains stay short
GENERATED = [(n, d, False) for n, d in [(1, 1), (1000, 7), (4099, 4099), (100_003, 5000), (300_000, 200_000)]] + \
            [(n, d, True) for n, d in [(1, 1), (1000, 7), (4099, 4099), (100_003, 5000)]]


@pytest.mark.parametrize("n,d,weak", GENERATED)
def test_dict_encode_generated(S, n, d, weak):
    col = dg.gen_strings_host(dg.StringSpec(n=n, d=d, seed=n % 97))
    want_codes, want_rows = O.dict_encode(col["offsets"], col["chars"])
    codes, rows = encode(S, col["offsets"], col["chars"], distinct_hint=d, weak_hash=weak)
    assert np.array_equal(codes, want_codes)
    assert np.array_equal(rows, want_rows)


EDGE_COLUMNS = {
    "empty strings": [b""] * 50,
    "prefix chains": [b"abcdefghijklmnopq"[:k] for k in range(18)] * 3,
    "last byte differs": [b"x" * 40 + bytes([c]) for c in range(256)] * 2,
    "long strings": [bytes([(7 * i + j) % 251 for j in range(300 + i % 5)]) for i in range(40)] * 2,
    "binary bytes": [b"\x00", b"\x00\x00", b"", b"\xff", b"\x00\xff", b"\xff\x00"] * 7,
    "eight-byte boundaries": [b"12345678", b"123456789", b"1234567", b"12345678\x00"] * 5,
}


@pytest.mark.parametrize("name", list(EDGE_COLUMNS))
@pytest.mark.parametrize("weak", [False, True])
def test_dict_encode_edge_columns(S, name, weak):
    strs = EDGE_COLUMNS[name]
    rng = np.random.default_rng(len(strs))
    strs = [strs[i] for i in rng.permutation(len(strs))]
    off, chars = dg.strcol_from_list(strs)
    want = O.dict_encode(off, chars)
    got = encode(S, off, chars, distinct_hint=600, weak_hash=weak)
    assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])


def test_dict_encode_no_rows_and_sliced_offsets(S):
    codes, rows = encode(S, np.zeros(1, np.int32), np.zeros(1, np.uint8))
    assert codes.size == 0 and rows.size == 0
    col = dg.gen_strings_host(dg.StringSpec(n=2000, d=300, seed=4))
    off = col["offsets"][500:1201]          # rows 500..1199 of the column: offsets start mid-buffer
    want = O.dict_encode(off, col["chars"])
    got = encode(S, off, col["chars"], distinct_hint=300)
    assert off[0] > 0 and np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])
    # chars that start at an odd address (a slice of a larger buffer)
    big = dev(np.concatenate([np.frombuffer(b"abc", np.uint8), col["chars"]]))
    chars = big[3:]
    assert chars.data_ptr() % 8 != 0
    codes, rows = S.sirius_dict_encode(dev(col["offsets"]), chars, distinct_hint=300)
    want = O.dict_encode(col["offsets"], col["chars"])
    assert np.array_equal(codes.cpu().numpy(), want[0]) and np.array_equal(rows.cpu().numpy(), want[1])


def test_dict_encode_errors(S):
    col = dg.gen_strings_host(dg.StringSpec(n=20_000, d=5000, seed=8))
    off, chars = dev(col["offsets"]), dev(col["chars"])
    with pytest.raises(S.SiriusError) as e:          # more distinct strings than the table takes
        S.sirius_dict_encode(off, chars, distinct_hint=100)
    assert e.value.status == S.ERR_TABLE_FULL
    d = int(O.dict_encode(col["offsets"], col["chars"])[1].size)
    with pytest.raises(S.SiriusError) as e:          # more than the output holds
        S.sirius_dict_encode(off, chars, distinct_hint=5000, dict_cap=d - 1)
    assert e.value.status == S.ERR_CAPACITY and e.value.needed == d
    bad = col["offsets"].copy()
    bad[7], bad[8] = bad[8] + 1, bad[7]              # a decreasing pair
    with pytest.raises(S.SiriusError) as e:
        S.sirius_dict_encode(dev(bad), chars, distinct_hint=5000)
    assert e.value.status == S.ERR_INVALID
    past = col["offsets"].copy()
    past[-1] = chars.numel() + 5                     # past the end of the chars
    with pytest.raises(S.SiriusError) as e:
        S.sirius_dict_encode(dev(past), chars, distinct_hint=5000)
    assert e.value.status == S.ERR_INVALID


@pytest.mark.parametrize("n,d", [(1, 1), (5000, 3), (200_003, 1000), (400_000, 150_000)])
def test_groupby_string(S, n, d):
    col = dg.gen_strings_host(dg.StringSpec(n=n, d=d, seed=d))
    want = O.groupby_string(col["offsets"], col["chars"], col["vals"])
    got = S.sirius_groupby_string(dev(col["offsets"]), dev(col["chars"]), dev(col["vals"]), distinct_hint=d)
    for c in ("row", "sum", "count", "min", "max"):
        assert np.array_equal(got[c].cpu().numpy(), want[c]), c


def test_groupby_string_weak_hash_subsets_and_capacity(S):
    col = dg.gen_strings_host(dg.StringSpec(n=30_000, d=2000, seed=6))
    want = O.groupby_string(col["offsets"], col["chars"], col["vals"])
    args = (dev(col["offsets"]), dev(col["chars"]), dev(col["vals"]))
    for aggs in ("count", "sum,count", "count,min,max"):
        got = S.sirius_groupby_string(*args, aggs=aggs, distinct_hint=2000, weak_hash=True)
        for c in ["row", "count"] + [a for a in ("sum", "min", "max") if a in aggs]:
            assert np.array_equal(got[c].cpu().numpy(), want[c]), (aggs, c)
    with pytest.raises(S.SiriusError) as e:
        S.sirius_groupby_string(*args, distinct_hint=2000, out_cap=10)
    assert e.value.status == S.ERR_CAPACITY and e.value.needed == want["row"].size


def test_groupby_string_hot_string_and_extreme_values(S):
    """One string holds 60 % of the rows (every row of it reduces into one slot); values near
    +-2^62 so that MIN / MAX and exact sums are exercised at the ends of int64."""
    rng = np.random.default_rng(21)
    n = 300_000
    base = dg.gen_strings_host(dg.StringSpec(n=n, d=5000, seed=21))
    strs = O.strings_of(base["offsets"], base["chars"])
    hot = rng.random(n) < 0.6
    strs = [b"the-hot-string" if h else s for h, s in zip(hot, strs)]
    off, chars = dg.strcol_from_list(strs)
    vals = rng.integers(-(1 << 62) // n, (1 << 62) // n, size=n)
    vals[rng.integers(0, n, size=4)] = [(1 << 62), -(1 << 62), (1 << 62) - 1, -(1 << 62) + 1]
    want = O.groupby_string(off, chars, vals)
    got = S.sirius_groupby_string(dev(off), dev(chars), dev(vals), distinct_hint=6000)
    for c in ("row", "sum", "count", "min", "max"):
        assert np.array_equal(got[c].cpu().numpy(), want[c]), c
    codes, rows = S.sirius_dict_encode(dev(off), dev(chars), distinct_hint=6000)
    wc, wr = O.dict_encode(off, chars)
    assert np.array_equal(codes.cpu().numpy(), wc) and np.array_equal(rows.cpu().numpy(), wr)
