"""Bounded device waits made to run out on purpose (GPU): the filter's decoupled look-back waits
on a tile that never publishes, and the single-launch pipeline's grid barrier waits for an
arrival that never comes.  Each wait must give up, record SIRIUS_ERR_TIMEOUT for the host to
read, and leave the context usable -- a query afterwards still matches the oracle.  Nothing here
faults: the awaited flags are ones that nothing sets, and every wait has its bound."""
import ctypes
import time

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


def query_still_matches_the_oracle(S):
    spec = dg.StarSpec("t", n=200_003, m=5000, fk_domain=5200, grp_bound=300, t=45, seed=29)
    dim, fact = dg.gen_dim_host(spec), dg.gen_fact_host(spec)
    dev = lambda d: {k: torch.from_numpy(v).cuda() for k, v in d.items()}  # noqa: E731
    for variant in ("single", "direct"):
        got = S.run_pipeline(dev(fact), dev(dim), "lt", spec.t, group_cap_hint=300, probe_variant=variant)
        got = O.sort_groups({k: v.cpu().numpy() for k, v in got.items()})
        want = O.pipeline(fact, dim, "lt", spec.t)
        for c in ("key", "sum", "count", "min", "max"):
            assert np.array_equal(got[c], want[c]), (variant, c)


def test_lookback_wait_runs_out_and_reports_timeout(S):
    mem = torch.zeros(256, dtype=torch.uint8, device="cuda")
    st = ctypes.c_int32(-1)
    t0 = time.perf_counter()
    rc = S.lib().sirius_selftest_lookback_timeout(mem.data_ptr(), mem.numel(), ctypes.byref(st),
                                                  torch.cuda.current_stream().cuda_stream)
    assert rc == S.OK, S.last_error()
    assert st.value == S.ERR_TIMEOUT
    assert time.perf_counter() - t0 < 30.0
    query_still_matches_the_oracle(S)


def test_grid_barrier_passes_with_every_arrival_and_times_out_without_one(S):
    mem = torch.zeros(256, dtype=torch.uint8, device="cuda")
    blocks = min(8, int(S.lib().sirius_device_sm_count()))
    stream = torch.cuda.current_stream().cuda_stream
    for missing, spins, want_status, want_passed in ((0, 1 << 20, S.OK, blocks),
                                                     (1, 1 << 14, S.ERR_TIMEOUT, 0),
                                                     (0, 1 << 20, S.OK, blocks)):
        st, passed = ctypes.c_int32(-1), ctypes.c_int32(-1)
        rc = S.lib().sirius_selftest_grid_barrier(blocks, missing, spins, mem.data_ptr(), mem.numel(),
                                                  ctypes.byref(st), ctypes.byref(passed), stream)
        assert rc == S.OK, S.last_error()
        assert (st.value, passed.value) == (want_status, want_passed), missing
    query_still_matches_the_oracle(S)
