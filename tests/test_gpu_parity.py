"""GPU path (through the C ABI) against the FP64 CPU oracle.

Bar: bit-exact candidate records; identical valid-path sets on every
candidate the oracle does not flag as ambiguous (tolerance bands of the
acceptance rules); interaction points within 1e-6 m of the oracle's.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2301_06399_gb300 import scenes as S

pytestmark = pytest.mark.gpu

POINT_TOL = 1e-6  # metres, FP64-refined points vs the oracle


@pytest.fixture(scope="module")
def mpt():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2301_06399_gb300 import mpt as m

    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    return m


@pytest.fixture(scope="module")
def ctx(mpt):
    return mpt.Context(0)


def expand_oracle(table, n_pairs):
    E = len(table)
    pair = np.tile(np.arange(n_pairs), E)
    ids = np.repeat(table.ids, n_pairs, axis=0)
    order = np.repeat(table.order, n_pairs)
    start = np.repeat(table.start, n_pairs)
    return pair, ids, order, start


def gpu_trace(mpt, ctx, sc, max_order, spec, precision=None, schedule=None, keep_fp32=False, path_cap=None):
    ds = mpt.DeviceScene(ctx, sc)
    prec = mpt.FP32_FP64REFINE if precision is None else precision
    cands = mpt.enumerate_candidates(ds, max_order, spec)
    sols = mpt.solve(ds, cands, prec, schedule, keep_fp32=keep_fp32)
    cap = path_cap if path_cap is not None else cands.capacity
    paths = mpt.validate(ds, cands, sols, capacity=cap)
    torch.cuda.synchronize()
    assert ctx.check() == 0
    return ds, cands, sols, paths


def compare_entries(sc, table, paths, entries, n_pairs):
    """Oracle on whole entries (one object sequence x every pair) vs GPU."""
    n = paths.n()
    gcand = paths.cand[:n].cpu().numpy()
    gX = paths.X[:, :n].cpu().numpy().T
    gpos = {int(c): i for i, c in enumerate(gcand)}
    n_valid = n_amb = 0
    max_err = 0.0
    for e in entries:
        b, en = int(e) * n_pairs, (int(e) + 1) * n_pairs
        sol, ver = oracle.candidate_range(sc, table, b, en)
        for i in range(en - b):
            c = b + i
            if ver.ambiguous[i]:
                n_amb += 1
                continue
            want = bool(ver.valid[i])
            got = c in gpos
            assert want == got, f"candidate {c} (entry {e}, ids {table.ids[e]}): oracle {want}, gpu {got}, " \
                                f"oracle cost {sol.cost[i]:.3e}"
            if want:
                n_valid += 1
                k = 3 * int(table.order[e])
                err = np.abs(gX[gpos[c], :k] - sol.X[i, :k]).max()
                max_err = max(max_err, err)
    assert max_err < POINT_TOL, max_err
    return n_valid, n_amb, max_err


# ------------------------------------------------------------ enumeration --
@pytest.mark.parametrize("name,max_order", [("street_canyon", 2), ("mixed_order", 4), ("curved", 3)])
def test_enumeration_bit_exact(mpt, ctx, name, max_order):
    sc = S.config_scene(name)
    spec = S.CONFIG_SPECS[name]
    ds = mpt.DeviceScene(ctx, sc)
    cands = mpt.enumerate_candidates(ds, max_order, spec)
    torch.cuda.synchronize()
    table = oracle.enumerate_sequences(sc, max_order, spec)
    n = int(cands.count.item())
    assert n == len(table) * sc.n_pairs == cands.capacity
    pair, ids, order, start = mpt.decode_candidates(cands, n)
    p2, i2, o2, s2 = expand_oracle(table, sc.n_pairs)
    assert np.array_equal(pair, p2) and np.array_equal(ids, i2)
    assert np.array_equal(order, o2) and np.array_equal(start, s2)
    ob = cands.order_begin.cpu().numpy()
    for k in range(1, 5):
        first = np.nonzero(o2 >= k)[0]
        assert ob[k - 1] == (first[0] if len(first) else n)
    assert ob[4] == n


def test_enumeration_urban_block_entries(mpt, ctx):
    sc = S.urban_block(4)
    spec = S.CONFIG_SPECS["urban_block"]
    ds = mpt.DeviceScene(ctx, sc)
    cands = mpt.enumerate_candidates(ds, 2, spec)
    torch.cuda.synchronize()
    table = oracle.enumerate_sequences(sc, 2, spec)
    pair, ids, order, start = mpt.decode_candidates(cands)
    p2, i2, o2, s2 = expand_oracle(table, sc.n_pairs)
    assert np.array_equal(ids, i2) and np.array_equal(pair, p2) and np.array_equal(order, o2)


def test_enumeration_adjacency_mask(mpt, ctx):
    sc = S.urban_block(2)
    rng = np.random.default_rng(3)
    adj = (rng.uniform(size=(sc.n_obj, sc.n_obj)) < 0.3).astype(np.uint8)
    spec = S.SequenceSpec(quota=(-1, -1, 0, 0))
    ds = mpt.DeviceScene(ctx, sc)
    cap = mpt.candidate_count(ds, 2, spec)
    cands = mpt.enumerate_candidates(ds, 2, spec, adj=torch.as_tensor(adj).cuda(), capacity=cap)
    torch.cuda.synchronize()
    table = oracle.enumerate_sequences(sc, 2, spec, adj=adj)
    n = int(cands.count.item())
    assert n == len(table) * sc.n_pairs
    pair, ids, order, start = mpt.decode_candidates(cands, n)
    p2, i2, o2, s2 = expand_oracle(table, sc.n_pairs)
    assert np.array_equal(ids, i2) and np.array_equal(pair, p2)


def test_enumeration_capacity_error(mpt, ctx):
    sc = S.street_canyon()
    ds = mpt.DeviceScene(ctx, sc)
    with pytest.raises(RuntimeError, match="CAPACITY"):
        mpt.enumerate_candidates(ds, 2, S.CONFIG_SPECS["street_canyon"], capacity=100)


# ------------------------------------------------------------------ Fig. 4 --
@pytest.mark.parametrize("prec", ["FP64_PLAIN", "FP32_FP64REFINE"])
def test_fig4_gpu_path(mpt, ctx, prec):
    sc = S.fig4_scene()
    spec = S.SequenceSpec(quota=(-1, -1, 0, 0))
    ds, cands, sols, paths = gpu_trace(mpt, ctx, sc, 2, spec, getattr(mpt, prec))
    assert paths.n() == 1
    _, ids, _, _ = mpt.decode_candidates(cands)
    c = int(paths.cand[0].item())
    assert list(ids[c][:2]) == [0, 1]
    X = paths.X[:6, 0].cpu().numpy()
    assert np.allclose(X, [20 / 7, 20 / 7, 0, 5, 10 / 3, 0], atol=1e-9)
    assert abs(paths.length[0].item() - np.sqrt(85.0)) < 1e-9


# ---------------------------------------------------------- street canyon --
@pytest.mark.parametrize("prec", ["FP64_PLAIN", "FP32_FP64REFINE"])
def test_street_canyon_parity(mpt, ctx, prec):
    sc = S.street_canyon()
    spec = S.CONFIG_SPECS["street_canyon"]
    ds, cands, sols, paths = gpu_trace(mpt, ctx, sc, 2, spec, getattr(mpt, prec))
    table = oracle.enumerate_sequences(sc, 2, spec)
    n_valid, n_amb, err = compare_entries(sc, table, paths, range(len(table)), sc.n_pairs)
    assert n_valid == paths.n() and n_valid > 300
    print(f"canyon {prec}: {n_valid} valid, {n_amb} ambiguous, max err {err:.2e} m")


def test_street_canyon_ragged_pairs(mpt, ctx):
    """37 RX: tiles and warps straddle sequence boundaries."""
    sc = S.street_canyon()
    rng = np.random.default_rng(9)
    sc.rx = np.ascontiguousarray(np.c_[rng.uniform(-40, 40, 37), rng.uniform(-8, 8, 37), np.full(37, 1.5)])
    spec = S.CONFIG_SPECS["street_canyon"]
    ds, cands, sols, paths = gpu_trace(mpt, ctx, sc, 2, spec)
    table = oracle.enumerate_sequences(sc, 2, spec)
    compare_entries(sc, table, paths, range(len(table)), sc.n_pairs)


# ------------------------------------------------------------- urban block --
def test_urban_block_small_all_candidates(mpt, ctx):
    sc = S.urban_block(4)
    spec = S.CONFIG_SPECS["urban_block"]
    ds, cands, sols, paths = gpu_trace(mpt, ctx, sc, 2, spec, keep_fp32=True)
    table = oracle.enumerate_sequences(sc, 2, spec)
    n_valid, n_amb, err = compare_entries(sc, table, paths, range(len(table)), sc.n_pairs)
    assert n_valid == paths.n() - 0 or n_amb > 0
    print(f"urban 4x4: {n_valid} valid, {n_amb} ambiguous, max err {err:.2e} m")


def test_urban_block_full_size_sampled(mpt, ctx):
    """9,634,816 candidates in the launch configuration the benchmark times;
    the oracle checks every order-1 entry and 24 random order-2 entries."""
    sc = S.urban_block(32)
    spec = S.CONFIG_SPECS["urban_block"]
    ds, cands, sols, paths = gpu_trace(mpt, ctx, sc, 2, spec, path_cap=1 << 20)
    table = oracle.enumerate_sequences(sc, 2, spec)
    assert int(cands.count.item()) == 9634816
    rng = np.random.default_rng(2024)
    entries = list(range(97)) + sorted(rng.choice(np.arange(97, len(table)), 24, replace=False).tolist())
    n_valid, n_amb, err = compare_entries(sc, table, paths, entries, sc.n_pairs)
    print(f"urban full (sampled {len(entries)} entries): {n_valid} valid, {n_amb} ambiguous, max err {err:.2e} m,"
          f" total valid {paths.n()}")
