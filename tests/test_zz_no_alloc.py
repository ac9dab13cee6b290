"""mpt_validate_noalloc: validation for callers that cannot allocate device
memory (their memory is reserved up front by their own manager, or they
must not wait on the driver's allocator).  It must give exactly what
mpt_validate gives, on consecutive calls that share its fixed scratch array.

Kept in a file of its own that pytest collects last."""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2301_06399_gb300 import scenes as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mpt():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2301_06399_gb300 import mpt as m

    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    return m


def _call_noalloc(mpt, ds, cands, sols, paths, stream):
    ep = ds.endpoints()
    cs = cands.struct()
    ss = sols.struct()
    ps = paths.struct()
    return mpt.lib().mpt_validate_noalloc(ds.ctx.h, ds.h, C.byref(ep), C.byref(cs), C.byref(ss),
                                          C.c_double(mpt.TAU), C.byref(ps), C.c_void_p(paths.count.data_ptr()),
                                          C.c_void_p(stream.cuda_stream))


def test_noalloc_validation_matches_validate_on_consecutive_calls(mpt):
    ctx = mpt.Context(0)
    stream = torch.cuda.current_stream()
    # two calls in a row: a larger input, then a smaller one that runs over
    # what the first call left in the shared array
    for sc, spec in ((S.urban_block(4), S.CONFIG_SPECS["urban_block"]),
                     (S.street_canyon(), S.CONFIG_SPECS["street_canyon"])):
        ds = mpt.DeviceScene(ctx, sc)
        cands = mpt.enumerate_candidates(ds, 2, spec)
        sols = mpt.solve(ds, cands, mpt.FP32_FP64REFINE)
        want = mpt.validate(ds, cands, sols, capacity=cands.capacity)
        got = mpt.alloc_paths(cands.capacity, ds.tx.device)
        got.cand.fill_(-7)
        assert _call_noalloc(mpt, ds, cands, sols, got, stream) == mpt.MPT_OK
        torch.cuda.synchronize()
        n = want.n()
        assert n > 0 and got.n() == n
        assert torch.equal(got.cand[:n], want.cand[:n])
        assert torch.allclose(got.X[:, :n], want.X[:, :n], rtol=0, atol=1e-12)
        assert torch.allclose(got.length[:n], want.length[:n], rtol=0, atol=1e-12)
        assert torch.equal(got.cost[:n], want.cost[:n])
        assert ctx.check() == mpt.MPT_OK


def test_noalloc_rejects_more_candidates_than_its_array_serves(mpt):
    ctx = mpt.Context(0)
    sc = S.street_canyon()
    ds = mpt.DeviceScene(ctx, sc)
    spec = S.CONFIG_SPECS["street_canyon"]
    cands = mpt.enumerate_candidates(ds, 2, spec)
    sols = mpt.solve(ds, cands, mpt.FP32_FP64REFINE)
    paths = mpt.alloc_paths(16, ds.tx.device)
    big = (1 << 24) + 1
    # sizes only: the call must refuse before touching any buffer
    cands.capacity = big
    sols.capacity = big
    rc = _call_noalloc(mpt, ds, cands, sols, paths, torch.cuda.current_stream())
    assert rc == mpt.MPT_ERR_CAPACITY
    assert "CAPACITY" in mpt.status_string(rc)


def test_noalloc_groups_beyond_its_list_match_validate(mpt):
    # FP64-plain solutions mark every candidate as final, so the converged
    # ones (about 400k of 602k here) exceed the fixed list of 2^18 entries:
    # the groups that do not fit are tested in full by the overflow kernel
    ctx = mpt.Context(0)
    stream = torch.cuda.current_stream()
    sc = S.urban_block(8)
    ds = mpt.DeviceScene(ctx, sc)
    cands = mpt.enumerate_candidates(ds, 2, S.CONFIG_SPECS["urban_block"])
    sols = mpt.solve(ds, cands, mpt.FP64_PLAIN)
    listed = int(((sols.status.to(torch.int32) & mpt.PATH_REFINED) != 0).logical_and(sols.cost < mpt.TAU).sum())
    assert listed > (1 << 18)
    want = mpt.validate(ds, cands, sols, capacity=cands.capacity)
    got = mpt.alloc_paths(cands.capacity, ds.tx.device)
    assert _call_noalloc(mpt, ds, cands, sols, got, stream) == mpt.MPT_OK
    torch.cuda.synchronize()
    n = want.n()
    assert n > 0 and got.n() == n
    assert torch.equal(got.cand[:n], want.cand[:n])
    assert torch.equal(got.X[:, :n], want.X[:, :n])
    assert torch.equal(got.length[:n], want.length[:n])
    assert ctx.check() == mpt.MPT_OK
