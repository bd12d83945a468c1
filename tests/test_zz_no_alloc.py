"""sirius_filter_static, the filter for callers that cannot allocate device memory: through the
C ABI, its output equals the oracle's and sirius_filter's (exact: row ids are integers) on two
calls in a row and at its size limit, the calls after the first leave the device's free memory
unchanged, and sizes beyond its static scratch are refused before any device work (GPU).

Collected last on purpose (file name), so a run that stops at the first failure has already run
every other test; it also passes on its own in a fresh process, where its first call performs
the per-device set-up."""
import ctypes

import numpy as np
import pytest
import torch

import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    from paper_2508_04701_gb300 import build
    build.build()
    from paper_2508_04701_gb300 import sirius
    sirius.lib()
    return sirius


def filter_static(S, col, op, lit, stream):
    n = col.numel()
    out = torch.full((max(n, 1),), -7, dtype=torch.int32, device=col.device)
    d_count = torch.full((1,), -7, dtype=torch.int64, device=col.device)
    h = ctypes.c_int64(-1)
    st = S.lib().sirius_filter_static(col.data_ptr(), n, S.OPS[op], int(lit), out.data_ptr(),
                                      d_count.data_ptr(), ctypes.byref(h), stream.cuda_stream)
    assert st == S.OK, S.last_error()
    assert int(d_count.item()) == h.value
    return out[:h.value]


def test_static_filter_matches_filter_twice_in_a_row(S):
    stream = torch.cuda.current_stream()
    rng = np.random.default_rng(77)
    cases = [(rng.integers(0, 100, size=3_000_017).astype(np.int32), "lt", 30),
             (rng.integers(-1000, 1000, size=123_457).astype(np.int32), "ge", 17)]
    for col_np, op, lit in cases:   # the second call reuses the array the first one filled
        col = torch.from_numpy(col_np).cuda()
        got = filter_static(S, col, op, lit, stream)
        want = S.sirius_filter(col, op, lit)
        torch.cuda.synchronize()
        assert got.numel() == want.numel()
        assert torch.equal(got, want)
        assert np.array_equal(got.cpu().numpy().view(np.uint32), O.filter_rows(col_np, op, lit))


def test_static_filter_allocates_nothing(S):
    """After a first call (which looks up the array's address), further calls leave the
    device's free memory exactly as it was."""
    stream = torch.cuda.current_stream()
    col_np = np.random.default_rng(78).integers(0, 100, size=2_000_003).astype(np.int32)
    col = torch.from_numpy(col_np).cuda()
    out = torch.empty(col.numel(), dtype=torch.int32, device="cuda")
    d_count = torch.empty(1, dtype=torch.int64, device="cuda")
    h = ctypes.c_int64(-1)

    def call(lit):
        st = S.lib().sirius_filter_static(col.data_ptr(), col.numel(), S.OPS["lt"], lit, out.data_ptr(),
                                          d_count.data_ptr(), ctypes.byref(h), stream.cuda_stream)
        assert st == S.OK, S.last_error()
        return h.value

    call(50)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for lit in (10, 90):
        n = call(lit)
        assert np.array_equal(out[:n].cpu().numpy().view(np.uint32), O.filter_rows(col_np, "lt", lit))
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_static_filter_at_its_size_limit(S):
    """Exactly sirius_filter_static_max_rows() rows: every tile status word of the array in use."""
    stream = torch.cuda.current_stream()
    n = S.lib().sirius_filter_static_max_rows()
    col_np = np.random.default_rng(79).integers(0, 100, size=n, dtype=np.int32)
    col = torch.from_numpy(col_np).cuda()
    got = filter_static(S, col, "lt", 37, stream)
    want = O.filter_rows(col_np, "lt", 37)
    assert np.array_equal(got.cpu().numpy().view(np.uint32), want)
    ref = S.sirius_filter(col, "lt", 37)
    torch.cuda.synchronize()
    assert torch.equal(got, ref)


def test_static_filter_refuses_sizes_beyond_its_limit(S):
    limit = S.lib().sirius_filter_static_max_rows()
    assert limit == 1 << 28
    st = S.lib().sirius_filter_static(None, limit + 1, 0, 0, None, None, None, None)
    assert st == S.ERR_INVALID
    assert "limit" in S.last_error()
