"""Whole-workload parity of the GPU path with the FP64 oracle, at the full
sizes of every workload, in the launch configurations the benchmark times.

Bar (Algorithm 1, "C < threshold and X is valid"): the GPU's valid set equals
the oracle's on every candidate the oracle does not flag as ambiguous, and
interaction points agree within 1e-6 m.  For curved sequences solved from
several starts (Sec. III-B) the bar is per (TX/RX pair, object sequence): the
sets of distinct valid roots over all starts are identical.  Each test also
prints the FP32-only point error against the oracle (the same solver without
the refinement, accepted at a looser cost), reported, not a pass criterion.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2301_06399_gb300 import scenes as S
import fullset as F

pytestmark = pytest.mark.gpu

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


def _trace(mpt, ds, max_order, spec, precision, schedule=None):
    cands = mpt.enumerate_candidates(ds, max_order, spec)
    sols = mpt.solve(ds, cands, precision, schedule, keep_fp32=True)
    paths = mpt.validate(ds, cands, sols, capacity=1 << 22)
    torch.cuda.synchronize()
    assert paths.n() < paths.capacity
    return cands, sols, paths


def _check_full_set(mpt, ctx, sc, spec, max_order, label, schedule=None):
    ds = mpt.DeviceScene(ctx, sc)
    cands, sols, paths = _trace(mpt, ds, max_order, spec, mpt.FP32_FP64REFINE, schedule)
    assert ctx.check() == 0
    table = oracle.enumerate_sequences(sc, max_order, spec)
    assert int(cands.count.item()) == len(table) * sc.n_pairs
    gpu = F.gpu_side(paths, sols)
    rep = F.compare_workload(sc, table, gpu, keep_sets=True)
    err32 = F.fp32_point_error(sc, table, rep, sols.T32.cpu().numpy())
    print(f"\nPER-CONFIG {label}: {rep.summary()}; FP32-only max point error {err32:.2e} m")
    assert rep.ok(), rep.summary()
    return ds, cands, sols, paths, table, rep


def test_urban_block_every_candidate(mpt, ctx):
    """The benchmark workload: 9,634,816 candidates, every one compared."""
    sc = S.urban_block(32)
    _check_full_set(mpt, ctx, sc, S.CONFIG_SPECS["urban_block"], 2, "urban_block_32x32rx_order2")


SCHEDULES = {"per_order": {}, "single_launch": {"mixed_orders": 1}, "warp_per_path": {"warp_orders": 15}}


@pytest.mark.parametrize("sched", list(SCHEDULES))
def test_mixed_orders_every_candidate(mpt, ctx, sched):
    """Orders 1-4 mixed (2,097,152 candidates, consecutive edge diffractions
    included) under three schedules: per-order launches, the single
    persistent launch over every order, and one candidate per warp for every
    order; each compared with the oracle candidate by candidate."""
    sc = S.mixed_order_city()
    _check_full_set(mpt, ctx, sc, S.CONFIG_SPECS["mixed_order"], 4, f"mixed_orders_{sched}",
                    mpt.schedule_struct(**SCHEDULES[sched]))


@pytest.mark.parametrize("warp_orders", [0, 7])
def test_curved_root_sets_at_full_size(mpt, ctx, warp_orders):
    """Paraboloids, arcs and posed rectangles, 4,096 TX/RX pairs, orders 1-3,
    8 starts for curved sequences: for every (pair, sequence) the sets of
    distinct valid roots of the GPU and of the oracle are identical; with
    one candidate per lane (the default) and one per warp for every order."""
    sc = S.curved_scene(n_pairs=4096)
    spec = S.CONFIG_SPECS["curved"]
    ds = mpt.DeviceScene(ctx, sc)
    cands, sols, paths = _trace(mpt, ds, 3, spec, mpt.FP32_FP64REFINE,
                                mpt.schedule_struct(warp_orders=warp_orders) if warp_orders else None)
    table = oracle.enumerate_sequences(sc, 3, spec)
    gpu = F.gpu_side(paths, sols)
    rep = F.compare_workload(sc, table, gpu, keep_sets=True)
    n_groups, diffs = F.root_set_differences(sc, table, gpu, rep)
    # FP32-only error over the candidates whose start reaches the oracle's root
    same = np.intersect1d(rep.valid_idx, gpu.cand)
    keep = np.isin(rep.valid_idx, same)
    sub = F.Report(valid_idx=rep.valid_idx[keep], valid_X=rep.valid_X[keep])
    err32 = F.fp32_point_error(sc, table, sub, sols.T32.cpu().numpy())
    print(f"\nPER-CONFIG curved_4096pairs_order3{'_warp_per_path' if warp_orders else ''}: {rep.summary()}; "
          f"root-set groups {n_groups}, differing "
          f"{len(diffs)}; FP32-only max point error {err32:.2e} m")
    for d in diffs[:20]:
        print("  root-set difference:", d)
    assert not diffs


def test_curved_root_sets_plain_fp64(mpt, ctx):
    """The curved workload with the plain FP64 GPU method (FP64 throughout,
    the same starts): for every (pair, sequence) the sets of distinct valid
    roots equal the oracle's, and the FP64 point error against the oracle is
    reported beside the FP32-only and FP32 + refinement errors of the test
    above."""
    sc = S.curved_scene(n_pairs=4096)
    spec = S.CONFIG_SPECS["curved"]
    ds = mpt.DeviceScene(ctx, sc)
    cands, sols, paths = _trace(mpt, ds, 3, spec, mpt.FP64_PLAIN)
    table = oracle.enumerate_sequences(sc, 3, spec)
    gpu = F.gpu_side(paths, sols)
    rep = F.compare_workload(sc, table, gpu, keep_sets=True)
    n_groups, diffs = F.root_set_differences(sc, table, gpu, rep)
    print(f"\nPER-CONFIG curved_4096pairs_order3_fp64_plain: {rep.summary()}; root-set groups {n_groups}, "
          f"differing {len(diffs)}")
    for d in diffs[:20]:
        print("  root-set difference:", d)
    assert not diffs


def test_differentiable_block_every_candidate_and_adjoint(mpt, ctx):
    """The urban block with 64x64 RX (38,539,264 candidates): valid set
    against the oracle, then the adjoint of the valid paths (length and point
    weights) against the oracle's implicit-function-theorem gradient
    evaluated at the GPU's converged parameters, summed per TX, RX and plane."""
    sc = S.urban_block(64)
    ds, cands, sols, paths, table, rep = _check_full_set(mpt, ctx, sc, S.CONFIG_SPECS["differentiable"], 2,
                                                         "differentiable_64x64rx_order2")
    n = paths.n()
    rng = np.random.default_rng(4)
    g_len = torch.as_tensor(rng.uniform(0.5, 1.5, paths.capacity)).cuda()
    g_pts = torch.as_tensor(rng.normal(size=(12, paths.capacity)) * 0.1).cuda()
    cand = paths.cand[:n].cpu().numpy()
    T = oracle.pack_params(sc, table, cand, paths.T[:, :n].cpu().numpy().T)
    for with_pts in (False, True):
        gtx, grx, gobj = mpt.grad(ds, cands, paths, g_len, g_pts if with_pts else None)
        torch.cuda.synchronize()
        wtx, wrx, wobj = oracle.grad_sums(sc, table, cand, T, g_len[:n].cpu().numpy(),
                                          g_pts[:, :n].cpu().numpy().T if with_pts else None)
        planes = sc.obj_kind == 0
        e_tx = np.abs(gtx.cpu().numpy() - wtx).max() / max(1.0, np.abs(wtx).max())
        e_rx = np.abs(grx.cpu().numpy() - wrx).max() / max(1.0, np.abs(wrx).max())
        e_obj = np.abs(gobj.cpu().numpy()[planes] - wobj[planes]).max() / max(1.0, np.abs(wobj).max())
        print(f"adjoint over {n} paths ({'length and point' if with_pts else 'length'} weights): relative error "
              f"TX {e_tx:.1e}, RX {e_rx:.1e}, plane offsets {e_obj:.1e}")
        assert e_tx < 1e-6 and e_rx < 1e-6 and e_obj < 1e-6


def _planes_only(sc):
    """The scene's planes alone (edges dropped, occluders kept): every
    candidate sequence is reflection-only."""
    keep = np.nonzero(sc.obj_kind == S.PLANE)[0]
    return S.Scene(sc.name + "_planes", sc.scale, sc.obj_kind[keep], sc.obj_param[keep], sc.occ_kind, sc.occ_param,
                   sc.tx, sc.rx, sc.pair_mode, sc.meta).contiguous()


@pytest.mark.parametrize("name", ["street_canyon", "urban_block_planes"])
def test_image_method_matches_oracle_and_minimiser(mpt, ctx, name):
    """The image method on the GPU (Sec. III-A, Eqs. 5-6) over every
    reflection-only candidate: its valid set (after mpt_validate's bounds and
    visibility) equals the FP64 oracle's and the minimiser's, points within
    1e-6 m of the oracle's."""
    sc = S.street_canyon() if name == "street_canyon" else _planes_only(S.urban_block(32))
    spec = S.SequenceSpec(quota=(-1, -1, 0, 0))
    ds = mpt.DeviceScene(ctx, sc)
    cands = mpt.enumerate_candidates(ds, 2, spec)
    im = mpt.image_method(ds, cands)
    p_im = mpt.validate(ds, cands, im, capacity=1 << 21)
    sols = mpt.solve(ds, cands, mpt.FP32_FP64REFINE)
    p_mpt = mpt.validate(ds, cands, sols, capacity=1 << 21)
    torch.cuda.synchronize()
    table = oracle.enumerate_sequences(sc, 2, spec)
    rep = F.compare_workload(sc, table, F.gpu_side(p_im), keep_sets=True)
    a = p_im.cand[:p_im.n()].cpu().numpy()
    b = p_mpt.cand[:p_mpt.n()].cpu().numpy()
    print(f"\nPER-CONFIG image_method_{name}: {rep.summary()}; minimiser valid {len(b)}, equal sets {np.array_equal(a, b)}")
    assert rep.ok(), rep.summary()
    assert np.array_equal(a, b)
    assert (p_im.X[:, :len(a)] - p_mpt.X[:, :len(b)]).abs().max().item() < 1e-6


def test_autotuned_schedule_keeps_the_oracle_valid_set(mpt, ctx):
    """mpt_autotune on the mixed-order city (orders 1-4, 2,097,152
    candidates): the schedule it picks gives exactly the oracle's valid set,
    and a second call on the same workload returns the cached choice."""
    import time

    sc = S.mixed_order_city()
    spec = S.CONFIG_SPECS["mixed_order"]
    ds = mpt.DeviceScene(ctx, sc)
    cands = mpt.enumerate_candidates(ds, 4, spec)
    t0 = time.perf_counter()
    best, ms = mpt.autotune(ds, cands)
    t1 = time.perf_counter()
    again, ms2 = mpt.autotune(ds, cands)
    t2 = time.perf_counter()
    print(f"\nautotune mixed orders: {mpt.schedule_dict(best)}, {ms:.3f} ms per solve; search {t1 - t0:.2f} s, "
          f"cached call {1e3 * (t2 - t1):.2f} ms")
    assert mpt.schedule_dict(again) == mpt.schedule_dict(best) and ms2 == ms
    assert t2 - t1 < 0.05 < t1 - t0
    _check_full_set(mpt, ctx, sc, spec, 4, "mixed_orders_autotuned", best)
