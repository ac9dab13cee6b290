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
    # FP64-plain solutions mark every candidate as final, so with every
    # candidate iterated (the solver's exclusion pass off) the converged ones
    # (about 400k of 602k here) exceed the fixed list of 2^18 entries: the
    # groups that do not fit are tested in full by the overflow kernel
    ctx = mpt.Context(0)
    stream = torch.cuda.current_stream()
    sc = S.urban_block(8)
    ds = mpt.DeviceScene(ctx, sc)
    cands = mpt.enumerate_candidates(ds, 2, S.CONFIG_SPECS["urban_block"])
    sols = mpt.solve(ds, cands, mpt.FP64_PLAIN, mpt.schedule_struct(exclude=2))
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


def test_noalloc_call_leaves_free_device_memory_unchanged(mpt):
    """The property the entry point exists for.  A fresh context (its own
    validation scratch never grown) takes a small warm-up call (the first call
    on a device looks up the array's address), then calls on a thousand times
    more candidates: an allocation sized by the input would have to grow
    there, yet the device's free memory is the same before and after."""
    ctx = mpt.Context(0)
    stream = torch.cuda.current_stream()
    small = S.street_canyon()
    ds_s = mpt.DeviceScene(ctx, small)
    c_s = mpt.enumerate_candidates(ds_s, 2, S.CONFIG_SPECS["street_canyon"])
    s_s = mpt.solve(ds_s, c_s, mpt.FP32_FP64REFINE)
    p_s = mpt.alloc_paths(c_s.capacity, ds_s.tx.device)
    big = S.urban_block(8)
    ds_b = mpt.DeviceScene(ctx, big)
    c_b = mpt.enumerate_candidates(ds_b, 2, S.CONFIG_SPECS["urban_block"])
    s_b = mpt.solve(ds_b, c_b, mpt.FP32_FP64REFINE)
    p_b = mpt.alloc_paths(c_b.capacity, ds_b.tx.device)
    assert _call_noalloc(mpt, ds_s, c_s, s_s, p_s, stream) == mpt.MPT_OK
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        assert _call_noalloc(mpt, ds_b, c_b, s_b, p_b, stream) == mpt.MPT_OK
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 == free0, (free0, free1)
    assert p_b.n() > 1000 and ctx.check() == mpt.MPT_OK
    # for contrast (reported): the allocating entry point grows the fresh
    # context's scratch for the same input
    mpt.validate(ds_b, c_b, s_b, out=p_b)
    torch.cuda.synchronize()
    print(f"free device memory: {free0} before and {free1} after three no-allocation calls; "
          f"{torch.cuda.mem_get_info()[0]} after one mpt_validate")


@pytest.mark.parametrize("which", ["mpt_validate", "mpt_validate_noalloc"])
def test_zero_capacity_candidate_list_writes_a_zero_count(mpt, which):
    ctx = mpt.Context(0)
    sc = S.street_canyon()
    ds = mpt.DeviceScene(ctx, sc)
    cands = mpt.enumerate_candidates(ds, 2, S.CONFIG_SPECS["street_canyon"])
    sols = mpt.solve(ds, cands, mpt.FP32_FP64REFINE)
    paths = mpt.alloc_paths(4, ds.tx.device)
    paths.count.fill_(77)
    torch.cuda.synchronize()
    cands.capacity = 0  # an empty candidate buffer
    ep, cs, ss, ps = ds.endpoints(), cands.struct(), sols.struct(), paths.struct()
    fn = getattr(mpt.lib(), which)
    stream = torch.cuda.current_stream()
    rc = fn(ds.ctx.h, ds.h, C.byref(ep), C.byref(cs), C.byref(ss), C.c_double(mpt.TAU), C.byref(ps),
            C.c_void_p(paths.count.data_ptr()), C.c_void_p(stream.cuda_stream))
    torch.cuda.synchronize()
    assert rc == mpt.MPT_OK
    assert int(paths.count.item()) == 0
