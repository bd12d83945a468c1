"""The rule behind the split pass, checked on the host against the oracle (no GPU).

The fused probe and the group-by may aggregate the first rows in full, take over the groups
seen so far the smallest MAX (`floor`) and the largest MIN (`ceil`), and then skip, for a later
row of a seen group, the MAX update when its value is below `floor` and the MIN update when it
is above `ceil`.  Because a group's MAX only grows and its MIN only shrinks, a skipped value can
never be the group's final extreme.  This file replays that rule in numpy on inputs chosen to
stress it (value orders, negative and int64-edge values, groups first seen after the split) and
requires the oracle's results exactly; a variant that also skips for groups not yet seen must
fail, which shows that the seen-bitmap is needed."""
import numpy as np
import pytest

import oracle as O


def split_rule(keys, vals, n0, skip_unseen=False):
    """SUM / COUNT / MIN / MAX per key with the split rule; returns oracle-shaped arrays."""
    keys = np.asarray(keys, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.int64)
    uniq, inv = np.unique(keys, return_inverse=True)
    g = uniq.size
    s = np.zeros(g, dtype=object)
    c = np.zeros(g, dtype=np.int64)
    mn = np.full(g, np.iinfo(np.int64).max, dtype=np.int64)
    mx = np.full(g, np.iinfo(np.int64).min, dtype=np.int64)
    for i in range(n0):                      # first phase: every update
        j = inv[i]
        s[j] += int(vals[i])
        c[j] += 1
        mn[j] = min(mn[j], vals[i])
        mx[j] = max(mx[j], vals[i])
    seen = c > 0
    floor = mx[seen].min() if seen.any() else np.iinfo(np.int64).max
    ceil = mn[seen].max() if seen.any() else np.iinfo(np.int64).min
    for i in range(n0, keys.size):           # second phase: MIN / MAX behind the bounds
        j = inv[i]
        v = vals[i]
        s[j] += int(v)
        c[j] += 1
        bounded = seen[j] or skip_unseen
        if not (bounded and v < floor):
            mx[j] = max(mx[j], v)
        if not (bounded and v > ceil):
            mn[j] = min(mn[j], v)
    return {"key": uniq, "sum": np.array([int(x) for x in s], dtype=np.int64), "count": c, "min": mn, "max": mx}


def check(keys, vals, n0):
    got = split_rule(keys, vals, n0)
    want = O.groupby_agg(np.asarray(keys, dtype=np.int64), np.asarray(vals, dtype=np.int64))
    for col in ("key", "sum", "count", "min", "max"):
        assert np.array_equal(got[col], want[col]), col


@pytest.mark.parametrize("order", ["uniform", "ascending", "descending", "alternating", "equal"])
def test_rule_is_exact_for_value_orders(order):
    rng = np.random.default_rng(1)
    n = 6000
    keys = rng.integers(0, 40, size=n)
    base = np.arange(n, dtype=np.int64) * 13 - 30_000
    vals = {"uniform": rng.integers(-10**6, 10**6, size=n), "ascending": base, "descending": base[::-1].copy(),
            "alternating": np.where(np.arange(n) % 2 == 0, base, -base), "equal": np.full(n, 5, np.int64)}[order]
    for n0 in (0, 1, n // 16, n // 2, n):
        check(keys, vals, n0)


def test_rule_is_exact_at_int64_edges_and_for_late_groups():
    rng = np.random.default_rng(2)
    n = 5000
    n0 = n // 16
    keys = rng.integers(0, 30, size=n)
    keys[:n0] = rng.integers(0, 15, size=n0)          # groups 15..29 first appear after the split
    vals = rng.integers(-1000, 1000, size=n)
    vals[n0:n0 + 40] = np.iinfo(np.int64).min // 64    # below every floor (sums stay in int64)
    vals[n0 + 40:n0 + 80] = np.iinfo(np.int64).max // 64
    check(keys, vals, n0)


def test_skipping_unseen_groups_would_be_wrong():
    """A group first seen after the split whose only values lie below the floor: the rule that
    skips for every group loses its MAX (the bitmap of seen groups is what keeps it exact)."""
    keys = np.array([0, 0, 0, 0, 1, 1], dtype=np.int64)
    vals = np.array([100, 200, 150, 120, 5, 7], dtype=np.int64)
    n0 = 4                                             # group 1 unseen; floor = 200
    want = O.groupby_agg(keys, vals)
    good = split_rule(keys, vals, n0)
    bad = split_rule(keys, vals, n0, skip_unseen=True)
    assert np.array_equal(good["max"], want["max"]) and np.array_equal(good["min"], want["min"])
    assert not np.array_equal(bad["max"], want["max"])
